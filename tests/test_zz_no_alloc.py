"""The allocation-free totals entry point, lbm_mass_momentum_noalloc.

It exists for callers that cannot allocate device memory when they need the mass and momentum
totals (under a runtime that owns all device memory, or on a host that forbids allocation after
start-up).  Its scratch is a fixed device array inside the library.
These tests compare it, through the C-ABI, with the regular lbm_reduce_mass_momentum on the same
state, on two calls in a row so that a second call sees the array the first one left behind, and
with FP64 sums on the host where obstacle cells (NaN) must be skipped and counted.
"""
import numpy as np
import pytest

from paper_1508_07982_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1508_07982_gb300 import build, lbm as mod
    build.build()
    return mod


def _state(lbm, precision, case=None, steps=3):
    case = case or inputs.periodic_case(n=64, B=16, collision="trt", omega=1.7)
    f = lbm.Forest(case, precision=precision)
    f.init_fields(inputs.taylor_green_field(case["root"][0] * case["B"]))
    f.step_coarse(steps)
    # the same state written back: the regular reduction then sums the stored values, as the
    # allocation-free entry point does, instead of the moments the last step recorded
    f.set_pdfs(0, f.get_pdfs(0))
    return f


def _storage(lbm, pd, precision, u_shift=(0.0, 0.0, 0.0), rho0=1.0):
    """The storage layout of `precision` from FP64 f on the device: f itself, or f - f^eq(rho0,
    u_shift) in FP32 / FP16 (the shift in FP64, as the forest's own storage is formed)."""
    import torch
    if precision == "fp64":
        return pd
    e, w, opp = lbm.lbm_lattice()
    u = np.asarray(u_shift, dtype=np.float64)
    eu = e @ u
    sh = w * rho0 * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * (u @ u))
    shifted = pd - torch.tensor(sh, dtype=torch.float64, device=pd.device)[:, None]
    return shifted.to(torch.float32 if precision == "fp32s" else torch.float16).contiguous()


def _call(lbm, arr, precision, n, u_shift=None):
    import torch
    out = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
    lbm.lbm_mass_momentum_noalloc(arr, precision, n, 1.0, out, u_shift=u_shift)
    return out.cpu().numpy()


@pytest.mark.parametrize("precision", ["fp64", "fp32s", "fp16s"])
def test_noalloc_totals_match_the_regular_reduction_twice(lbm, precision):
    import torch
    f = _state(lbm, precision)
    ref = f.reduce_mass_momentum()
    n = f.n_cells(0)
    pd = torch.empty((19, n), dtype=torch.float64, device="cuda")
    f.get_pdfs(0, pd, on_device=True)
    arr = _storage(lbm, pd, precision)
    for _ in range(2):
        got = _call(lbm, arr, precision, n)
        assert abs(got[0] - ref[0]) <= 1e-12 * abs(ref[0])
        assert np.abs(got[1:4] - ref[1:]).max() <= 1e-12 * abs(ref[0])
        assert got[4] == 0.0
    f.close()


@pytest.mark.parametrize("precision", ["fp32s", "fp16s"])
def test_noalloc_totals_with_a_storage_shift(lbm, precision):
    """A forest stored relative to f^eq(rho0, u_shift) with u_shift != 0 (as the bench channel is):
    given the shift, the entry point adds rho0 u_shift per cell back and agrees with the regular
    reduction; without it the momentum is short by exactly that much."""
    import torch
    case = inputs.periodic_case(n=64, B=16, collision="trt", omega=1.7)
    us = (0.04, -0.01, 0.005)
    case["u_shift"] = us
    f = _state(lbm, precision, case)
    ref = f.reduce_mass_momentum()
    n = f.n_cells(0)
    pd = torch.empty((19, n), dtype=torch.float64, device="cuda")
    f.get_pdfs(0, pd, on_device=True)
    arr = _storage(lbm, pd, precision, us)
    # the values the forest holds are f - f^eq(rho0, u_shift) rounded to the storage type, and
    # get_pdfs adds the shift back in FP64: re-forming them here reproduces the stored values up to
    # the rounding of that FP64 addition, far below the tolerance
    for _ in range(2):
        got = _call(lbm, arr, precision, n, u_shift=us)
        assert abs(got[0] - ref[0]) <= 1e-9 * abs(ref[0])
        assert np.abs(got[1:4] - ref[1:]).max() <= 1e-9 * abs(ref[0])
    plain = _call(lbm, arr, precision, n)
    assert np.abs((ref[1:] - plain[1:4]) - n * np.asarray(us)).max() <= 1e-9 * abs(ref[0])
    f.close()


def test_noalloc_skips_and_counts_obstacle_cells(lbm):
    """A periodic box with a sphere: obstacle cells come back from lbm_get_pdfs as NaN; the entry
    point sums the finite cells only (checked against an FP64 sum on the host) and counts the
    others.  A smaller call after a larger one reads only the partial sums it wrote itself."""
    import torch
    case = inputs.periodic_case(n=64, B=16, collision="trt", omega=1.7)
    case["spheres"] = [(32.0, 32.0, 32.0, 9.0)]
    f = _state(lbm, "fp64", case)
    n = f.n_cells(0)
    pd = torch.empty((19, n), dtype=torch.float64, device="cuda")
    f.get_pdfs(0, pd, on_device=True)
    h = pd.cpu().numpy()
    e, w, opp = lbm.lbm_lattice()
    finite = np.isfinite(h.sum(axis=0))
    n_obst = int((~finite).sum())
    assert n_obst > 1000
    ref = np.concatenate([[h[:, finite].sum()], (e.T.astype(np.float64) @ h[:, finite]).sum(axis=1)])
    got = _call(lbm, pd, "fp64", n)
    assert abs(got[0] - ref[0]) <= 1e-12 * abs(ref[0])
    assert np.abs(got[1:4] - ref[1:]).max() <= 1e-12 * abs(ref[0])
    assert got[4] == n_obst
    # a smaller call after the larger one: three 16^3 bricks, the middle one holding the sphere's
    # centre (brick (2, 2, 2) of the 4^3, index 42 in x-fastest brick order)
    m = 4096 * 3
    hs = h[:, 41 * 4096:44 * 4096]
    sub = pd[:, 41 * 4096:44 * 4096].contiguous()
    fin = np.isfinite(hs.sum(axis=0))
    assert (~fin).sum() > 500
    ref = np.concatenate([[hs[:, fin].sum()], (e.T.astype(np.float64) @ hs[:, fin]).sum(axis=1)])
    for _ in range(2):
        got = _call(lbm, sub, "fp64", m)
        assert abs(got[0] - ref[0]) <= 1e-12 * abs(ref[0])
        assert np.abs(got[1:4] - ref[1:]).max() <= 1e-12 * abs(ref[0])
        assert got[4] == int((~fin).sum())
    f.close()


def test_noalloc_rejects_counts_beyond_its_fixed_array(lbm):
    import torch
    buf = torch.zeros(5, dtype=torch.float64, device="cuda")
    with pytest.raises(lbm.LBMError) as ei:
        lbm.lbm_mass_momentum_noalloc(buf, "fp64", lbm.NOALLOC_MAX_CELLS + 1, 1.0, buf)
    assert ei.value.status == lbm.LBM_EINVAL
    assert "exceeds the maximum" in str(ei.value)
