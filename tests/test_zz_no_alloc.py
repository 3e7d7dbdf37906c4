"""The allocation-free totals entry point, lbm_mass_momentum_noalloc.

It exists for callers that cannot allocate device memory when they need the mass and momentum
totals (during CUDA stream capture, under a runtime that owns all device memory, or on a host
that forbids allocation after start-up).  Its scratch is a fixed device array inside the library.
These tests compare it, through the C-ABI, with the regular lbm_reduce_mass_momentum on the same
state, on two calls in a row so that a second call sees the array the first one left behind.
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


def _state(lbm, precision):
    case = inputs.periodic_case(n=64, B=16, collision="trt", omega=1.7)
    f = lbm.Forest(case, precision=precision)
    f.init_fields(inputs.taylor_green_field(64))
    f.step_coarse(3)
    # the same state written back (bit-exact): the regular reduction then sums the stored values,
    # as the allocation-free entry point does, instead of the moments the last step recorded
    f.set_pdfs(0, f.get_pdfs(0))
    return f


@pytest.mark.parametrize("precision", ["fp64", "fp32s", "fp16s"])
def test_noalloc_totals_match_the_regular_reduction_twice(lbm, precision):
    import torch
    f = _state(lbm, precision)
    ref = f.reduce_mass_momentum()
    n = f.n_cells(0)
    pd = torch.empty((19, n), dtype=torch.float64, device="cuda")
    f.get_pdfs(0, pd, on_device=True)
    if precision == "fp64":
        arr = pd
    else:
        # the shifted storage layout: f - w rho0 in the storage type (exact for these values)
        e, w, opp = lbm.lbm_lattice()
        shifted = pd - torch.tensor(w, dtype=torch.float64, device="cuda")[:, None]
        arr = shifted.to(torch.float32 if precision == "fp32s" else torch.float16).contiguous()
    for _ in range(2):
        out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
        lbm.lbm_mass_momentum_noalloc(arr, precision, n, 1.0, out)
        got = out.cpu().numpy()
        assert abs(got[0] - ref[0]) <= 1e-12 * abs(ref[0])
        assert np.abs(got[1:] - ref[1:]).max() <= 1e-12 * abs(ref[0])
    f.close()


def test_noalloc_rejects_counts_beyond_its_fixed_array(lbm):
    import torch
    buf = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(lbm.LBMError) as ei:
        lbm.lbm_mass_momentum_noalloc(buf, "fp64", lbm.NOALLOC_MAX_CELLS + 1, 1.0, buf)
    assert ei.value.status == lbm.LBM_EINVAL
    assert "exceeds the maximum" in str(ei.value)
