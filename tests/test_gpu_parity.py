"""GPU parity: the CUDA path (through the C-ABI) against the CPU oracle, element by element.

The kernels store the post-collision state, so the GPU PDFs after n coarse steps are compared
with the oracle's state after n coarse steps plus one more collision (orc_get_f with
post_collision).  FP64 tolerance: relative max-norm 1e-12 over owned fluid cells of all levels
(FMA and summation order differ from the oracle; no bitwise equality is claimed).  Integer
results (block tables, which cells are fluid) must agree exactly.
"""
import numpy as np
import pytest

from paper_1508_07982_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1508_07982_gb300 import build, lbm as mod
    build.build()
    return mod


def _compare(f, o, post_collision=True):
    """max |f_gpu - f_oracle| / max |f_oracle| over owned fluid cells; also checks that exactly the
    oracle's non-fluid owned cells come back as NaN."""
    num, den = 0.0, 0.0
    for L in range(f.nlev):
        g = f.get_pdfs(L)
        X, Y, Z = f.cell_coords(L)
        if X.size == 0:
            continue
        idx = o.lookup(L, X, Y, Z)
        cls, flg = o.classes(L)
        fluid = (cls[idx] == 1) & (flg[idx] == 0)
        assert (cls[idx] == 1).all()
        ref = o.get_f(L, post_collision=post_collision)[idx].T
        gnan = np.isnan(g).any(axis=0)
        assert (gnan == ~fluid).all(), "NaN pattern differs from the oracle's fluid mask on level %d" % L
        num = max(num, float(np.abs(g[:, fluid] - ref[:, fluid]).max()))
        den = max(den, float(np.abs(ref[:, fluid]).max()))
    return num / den


def _pair(lbm, oracle_mod, case, precision="fp64", field=None, refine=None, flag=None):
    f = lbm.Forest(case, precision=precision, refine=refine, flag=flag)
    o = oracle_mod.Oracle(case, refine=refine, flag=flag)
    field = field or inputs.uniform_field(u=case.get("u_init", (0.0, 0.0, 0.0)))
    f.init_fields(field)
    o.init_fields(field)
    return f, o


def test_block_tables_match_the_oracle(lbm, oracle_mod):
    case = inputs.sphere_channel_case(H=32, B=8, radii=(20.0, 12.0, 6.5), inlet_outlet=True)
    f = lbm.Forest(case)
    o = oracle_mod.Oracle(case)
    assert f.nlev == o.nlev == 4
    for L in range(4):
        a, b = f.block_table(L), o.leaves(L)
        assert a.shape == b.shape
        assert (a[np.lexsort((a[:, 0], a[:, 1], a[:, 2]))] == b[np.lexsort((b[:, 0], b[:, 1], b[:, 2]))]).all()
    assert f.cell_updates_per_coarse_step() == o.cell_updates_per_coarse_step()


def test_cavity_fp64_matches_the_oracle_after_100_coarse_steps(lbm, oracle_mod):
    """Two-level lid-driven cavity (32^3 coarse, centre refined), TRT, 100 coarse steps."""
    f, o = _pair(lbm, oracle_mod, inputs.cavity_case())
    f.step_coarse(100)
    o.step(100)
    assert _compare(f, o) < TOL64


@pytest.mark.parametrize("cfg", [(0, 2), (1, 4), (3, 3)])
def test_cavity_matches_the_oracle_in_every_launch_configuration(lbm, oracle_mod, cfg):
    """The cavity (coupled cells along the whole level-0/1 interface, which run in their own CTAs
    at the head of each launch) in other launch configurations: cells per thread 1, 2, 8 and 2-4
    CTAs per SM; 30 coarse steps."""
    f, o = _pair(lbm, oracle_mod, inputs.cavity_case())
    f.set_kernel_config(*cfg)
    f.step_coarse(30)
    o.step(30)
    assert _compare(f, o) < TOL64


def test_uniform_periodic_fp64_matches_the_oracle(lbm, oracle_mod):
    """Uniform periodic 64^3, SRT omega = 1.9, Taylor-Green modes + density noise, 200 steps."""
    case = inputs.periodic_case(n=64, B=16, collision="srt", omega=1.9)
    f, o = _pair(lbm, oracle_mod, case, field=inputs.taylor_green_field(64))
    f.step_coarse(200)
    o.step(200)
    assert _compare(f, o) < TOL64


@pytest.mark.parametrize("B", [8, 16])
def test_three_level_periodic_fp64_matches_the_oracle(lbm, oracle_mod, B):
    """Three levels from a ball region; interface faces, edges and corners; block size 8 and 16
    on the same geometry (the oracle is block-free, so both must match it)."""
    case = inputs.periodic_case(n=64, B=B, collision="trt", omega=1.7,
                                regions=[("box", 1, (16, 16, 0), (48, 48, 64)), ("box", 2, (24, 24, 16), (40, 40, 48))],
                                lmax=2)
    f, o = _pair(lbm, oracle_mod, case, field=inputs.taylor_green_field(64))
    assert f.nlev == 3
    f.step_coarse(12)
    o.step(12)
    assert _compare(f, o) < TOL64


def test_sphere_channel_fp64_matches_the_oracle(lbm, oracle_mod):
    """The sphere-channel workload at H = 32 with B = 8: four levels, velocity inlet/outlet,
    periodic sides, a no-slip sphere on the finest level, uniform plug start."""
    case = inputs.sphere_channel_case(H=32, B=8, radii=(20.0, 12.0, 6.5), inlet_outlet=True)
    f, o = _pair(lbm, oracle_mod, case)
    assert f.nlev == 4
    f.step_coarse(6)
    o.step(6)
    assert _compare(f, o) < TOL64


def test_lid_scaling_workload_fp64_matches_the_oracle(lbm, oracle_mod):
    """The cavity of the performance benchmark (Sec. 5.2): the two lid edges across the lid motion
    refined three times (4 levels, 7 / 12 / 24 / 64 blocks) on 3 x 1 x 3 roots of 8^3 cells,
    velocity lid, TRT, 100 coarse steps."""
    case = inputs.lid_scaling_case(roots=(3, 1, 3), B=8)
    f, o = _pair(lbm, oracle_mod, case)
    assert f.nlev == 4
    f.step_coarse(100)
    o.step(100)
    assert _compare(f, o) < TOL64


def test_pipe_with_wall_refinement_fp64_matches_the_oracle(lbm, oracle_mod):
    """Pipe Poiseuille (Sec. 5.1) refined towards the pipe wall to level 2: a staircase obstacle
    whose surface lies in the finest band, coarser levels towards the axis, body force."""
    case, refine, flag, _ = inputs.pipe_poiseuille_case(lmax=2, where="wall")
    f, o = _pair(lbm, oracle_mod, case, refine=refine, flag=flag)
    assert f.nlev == 3
    f.step_coarse(20)
    o.step(20)
    assert _compare(f, o) < TOL64


def _golden_pipe():
    import os
    rows = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "pipe_poiseuille_table.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            p = line.split()
            rows[(p[0], int(p[1]))] = [float(v) for v in p[2:]]
    return rows


def _pipe_steady_errors(lbm, where, lmax, steps=3000):
    """Flow-rate error and L1 / L2 / Linf of |u - u_exact| / u_max (cell-volume weights, the pipe
    scaled to [0,1]) after `steps` coarse steps from the analytic profile, FP64."""
    import math
    D, B = 60, 8
    case, refine, flag, (c, R) = inputs.pipe_poiseuille_case(D=D, B=B, lmax=lmax, where=where)
    nu0 = (1 / case["lambda_e0"] - 0.5) / 3
    umax = case["accel"][0] * R * R / (4 * nu0)

    def field(L, X, Y, Z):
        s = 2.0 ** -L
        y, z = (Y + 0.5) * s - c, (Z + 0.5) * s - c
        u = np.maximum(umax * (1 - (y * y + z * z) / R ** 2), 0.0)
        return 1.0, (u, 0 * u, 0 * u)

    f = lbm.Forest(case, precision="fp64", refine=refine, flag=flag)
    f.init_fields(field)
    f.step_coarse(steps)
    Q, l1, l2, linf = 0.0, 0.0, 0.0, 0.0
    for L in range(f.nlev):
        X, Y, Z = f.cell_coords(L)
        if X.size == 0:
            continue
        rho, u = f.get_macroscopic(L)
        ok = np.isfinite(rho)
        s = 2.0 ** -L
        y, z = (Y + 0.5) * s - c, (Z + 0.5) * s - c
        ue = 1 - (y * y + z * z) / R ** 2
        du = np.sqrt((u[0] / umax - ue) ** 2 + (u[1] / umax) ** 2 + (u[2] / umax) ** 2)[ok]
        w = (1.0 / D) ** 3 * (D / B) * 8.0 ** -L         # cell volume, the B-cell section scaled to length 1
        l1 += (w * du).sum()
        l2 += (w * du * du).sum()
        linf = max(linf, float(du.max()))
        plane = (X == 0)[ok]                              # the first cell layer of the section
        Q += (u[0][ok][plane] / umax).sum() * (1.0 / D) ** 2 * 4.0 ** -L
    f.close()
    return [abs(Q - math.pi / 8) / (math.pi / 8), l1, math.sqrt(l2), linf]


@pytest.mark.parametrize("lmax", [0, 1, 2])
def test_pipe_poiseuille_global_refinement_matches_the_paper_table(lbm, lmax):
    """The printed pipe-Poiseuille table (Sec. 5.1), global refinement: the whole pipe on level
    lmax, with the relaxation rate and force scaled to that level (Eqs. omega_scaling,
    force_scaling).  Every column within 2 % (the table prints two or three digits; measured:
    0.3 % or better on levels 0-1, 1.2 % on the level-2 L1 column, 0.76e-3 against 0.77e-3)."""
    got = _pipe_steady_errors(lbm, "global", lmax)
    want = _golden_pipe()[("global", lmax)]
    for g, p in zip(got, want):
        assert abs(g - p) / p < 0.02, (got, want)


def test_pipe_poiseuille_wall_refinement_against_the_paper_table(lbm):
    """Wall refinement (Sec. 5.1): the finest level only along the pipe wall, coarser towards the
    axis.  Linf, set by the wall cells, matches the printed table within 2 % on levels 1-3; each
    level lowers every error.  The integral errors exceed the table's (by 1.2x, 1.4x and 1.7x for
    levels 1-3): with 8^3 blocks the refined band is thinner than the paper's 10^3 blocks make
    it, and the homogeneous explosion with averaging coalescence adds interface error that the
    paper's numbers (close to its global-refinement ones) do not show; so only a factor-2 band is
    asserted for them."""
    table = _golden_pipe()
    prev = _pipe_steady_errors(lbm, "global", 0)
    for lmax in (1, 2, 3):
        got = _pipe_steady_errors(lbm, "wall", lmax)
        want = table[("wall", lmax)]
        assert abs(got[3] - want[3]) / want[3] < 0.02, (lmax, got, want)
        for g, p in zip(got[:3], want[:3]):
            assert p <= g < 2 * p, (lmax, got, want)
        assert all(g < q for g, q in zip(got, prev)), (lmax, got, prev)
        prev = got


def _freeslip_case():
    return inputs.freeslip_box_case(lid=0.02, spheres=[(8.0, 1.0, 16.0, 4.0), (16.0, 16.0, 16.0, 2.5)])


def test_free_slip_box_fp64_matches_the_oracle(lbm, oracle_mod):
    """Free-slip y and z- faces, a velocity lid on z+ (its corners with the free-slip faces take
    the lid), a sphere cut by the y- face (mirrored cells inside it bounce back instead), a
    refined centre holding a second sphere; Taylor-Green start, 50 coarse steps."""
    f, o = _pair(lbm, oracle_mod, _freeslip_case(), field=inputs.taylor_green_field(32))
    assert f.nlev == 2
    f.step_coarse(50)
    o.step(50)
    assert _compare(f, o) < TOL64


@pytest.mark.parametrize("precision", ["fp32s", "fp16s"])
def test_free_slip_reflection_with_a_storage_shift_keeps_uniform_flow(lbm, precision):
    """Shifted storage with u_shift normal to the free-slip faces: a reflected value moves between
    directions whose shifts differ, and the kernel adds the difference.  A uniform flow along the
    walls is an exact steady state, so it must stay uniform to storage rounding; a wrong term at
    the walls would show as a velocity change of order 1e-3."""
    u = 0.03
    case = dict(inputs.freeslip_box_case(), u_shift=(0.02, 0.01, -0.01))
    g = lbm.Forest(case, precision=precision)
    g.init_uniform((u, 0.0, 0.0))
    g.step_coarse(50)
    tol = 1e-6 if precision == "fp32s" else 1e-3
    for L in range(g.nlev):
        rho, v = g.get_macroscopic(L)
        ok = np.isfinite(rho)
        assert np.abs(v[0, ok] - u).max() < tol * u and np.abs(v[1:, ok]).max() < tol * u
    g.close()


def test_free_slip_reflection_with_a_storage_shift(lbm):
    """FP32S storage shifted by f^eq(rho0, u_shift) with u_shift normal to free-slip faces, on the
    Taylor-Green start: after 50 coarse steps the velocity agrees with FP64 within 5e-6 of the
    largest velocity, shifted or not (the shift here does not match the flow, so its stored
    deviations, and their rounding, are larger than without it)."""
    errs = []
    for shift in ((0.0, 0.0, 0.0), (0.02, 0.01, -0.01)):
        case = dict(_freeslip_case(), u_shift=shift)
        ref = lbm.Forest(case, precision="fp64")
        g = lbm.Forest(case, precision="fp32s")
        for h in (ref, g):
            h.init_fields(inputs.taylor_green_field(32))
            h.step_coarse(50)
        du = umax = 0.0
        for L in range(ref.nlev):
            ra, ua = g.get_macroscopic(L)
            rb, ub = ref.get_macroscopic(L)
            ok = np.isfinite(rb)
            du = max(du, float(np.abs(ua[:, ok] - ub[:, ok]).max()))
            umax = max(umax, float(np.abs(ub[:, ok]).max()))
        errs.append(du / umax)
        ref.close()
        g.close()
    assert max(errs) < 5e-6, errs


def _freeslip_interface_case(B=8, levels=2, lid=0.02):
    """Free-slip y and z- faces, a velocity lid on z+, periodic x; refinement in the corner x in
    [0, n], y, z in [0, n/2] (level 2: [0, n/4]), so that level interfaces meet the free-slip faces
    y- and z-; a sphere cut by the y- face straddles the level-1 interface at z = n/2."""
    n = 32 if B == 8 else 64
    k = n / 32
    c = inputs.freeslip_box_case(n=n, B=B, lid=lid, spheres=[(8.0 * k, 1.0 * k, 16.0 * k, 4.0 * k)])
    c["regions"] = [("box", 1, (0, 0, 0), (n, n / 2, n / 2)), ("box", 2, (0, 0, 0), (n, n / 4, n / 4))][:levels]
    c["lmax"] = levels
    return c, n


@pytest.mark.parametrize("B,levels", [(8, 1), (8, 2), (16, 1)])
def test_free_slip_faces_met_by_level_interfaces_match_the_oracle(lbm, oracle_mod, B, levels):
    """Level interfaces meeting free-slip faces (Sec. 4.1: the boundary treatment reaches into the
    innermost ghost layers): ghost cells next to the faces take the reflection, from mirrored
    neighbours that are owned cells or ghost cells (exploded in sub-step 1 and in layer 3,
    streamed otherwise).  FP64, Taylor-Green start, 30 coarse steps, against the oracle."""
    case, n = _freeslip_interface_case(B, levels)
    f, o = _pair(lbm, oracle_mod, case, field=inputs.taylor_green_field(n))
    assert f.nlev == levels + 1
    f.step_coarse(30)
    o.step(30)
    assert _compare(f, o) < TOL64


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32s", 3e-6), ("fp16s", 1e-3)])
def test_uniform_flow_along_free_slip_faces_met_by_interfaces_stays_uniform(lbm, precision, tol):
    """The paired walk's coupled cells and the ghost stream take the reflection in FP32 with the
    storage-shift correction; a uniform flow along the faces is an exact steady state on every
    level (free-slip faces only, so no lid).  FP64 keeps it to round-off; the shifted layouts keep
    it to their storage rounding, accumulated over the 200 finest-level steps of 50 coarse steps
    (the shift (0.02, 0.01, -0.01) does not match the flow, so the stored deviations are of order
    0.01 and their FP32 rounding of order 1e-9 per step)."""
    u = 0.03
    case, n = _freeslip_interface_case(8, 2, lid=None)
    case = dict(case, spheres=[], u_shift=(0.02, 0.01, -0.01))
    g = lbm.Forest(case, precision=precision)
    g.init_uniform((u, 0.0, 0.0))
    g.step_coarse(50)
    for L in range(g.nlev):
        rho, v = g.get_macroscopic(L)
        ok = np.isfinite(rho)
        assert np.abs(v[0, ok] - u).max() < tol * u and np.abs(v[1:, ok]).max() < tol * u
    g.close()


def test_obstacle_across_an_interface_and_forced_flow(lbm, oracle_mod):
    """A sphere that straddles a level interface (ghost cells take the coarse flag), no-slip
    walls, body force, refinement touching a wall."""
    case = dict(root=(4, 2, 2), B=8, lmax=1, collision="trt", rho0=1.0,
                bc=["periodic", "periodic", "noslip", "noslip", "noslip", "noslip"],
                bc_u=[(0, 0, 0)] * 6, spheres=[(16.0, 8.0, 8.0, 5.0)],
                regions=[("box", 1, (0, 0, 0), (15, 16, 16))], lambda_e0=1.3, magic=3 / 16,
                accel=(2e-5, 0.0, 0.0))
    f, o = _pair(lbm, oracle_mod, case)
    f.step_coarse(30)
    o.step(30)
    assert _compare(f, o) < TOL64


def test_macroscopic_fields_match_the_oracle(lbm, oracle_mod):
    case = dict(inputs.plane_poiseuille_case(B=8, ny_roots=2, where="bottom"))
    f, o = _pair(lbm, oracle_mod, case)
    f.step_coarse(40)
    o.step(40)
    for L in range(f.nlev):
        rho, u = f.get_macroscopic(L)
        X, Y, Z = f.cell_coords(L)
        idx = o.lookup(L, X, Y, Z)
        orho, ou = o.macro(L)
        assert np.abs(rho - orho[idx]).max() < 1e-13
        for k in range(3):
            assert np.abs(u[k] - ou[k][idx]).max() < 1e-15


def test_mass_and_momentum_totals(lbm, oracle_mod):
    case = inputs.periodic_case(n=32, B=8, collision="trt", omega=1.6,
                                regions=[("box", 1, (8, 8, 8), (24, 24, 24))], lmax=1)
    f, o = _pair(lbm, oracle_mod, case, field=inputs.taylor_green_field(32))
    m0 = f.reduce_mass_momentum()
    assert np.abs(m0 - o.mass_momentum()).max() < 1e-11
    f.step_coarse(50)
    m1 = f.reduce_mass_momentum()
    assert abs(m1[0] - m0[0]) / m0[0] < 1e-13
    assert np.abs(m1[1:] - m0[1:]).max() < 1e-12 * m0[0]


def test_stepping_one_at_a_time_equals_stepping_in_one_call(lbm):
    case = inputs.cavity_case()
    a = lbm.Forest(case)
    b = lbm.Forest(case)
    a.init_uniform()
    b.init_uniform()
    for _ in range(7):
        a.step_coarse(1)
    b.step_coarse(7)
    for L in range(2):
        assert np.array_equal(a.get_pdfs(L), b.get_pdfs(L), equal_nan=True)


@pytest.mark.parametrize("precision", ["fp64", "fp32s", "fp16s"])
@pytest.mark.parametrize("shift", [False, True])
def test_checkpoint_resume_is_bit_exact(lbm, precision, shift):
    """lbm_get_pdfs / lbm_set_pdfs round trip, then 4 more coarse steps on both forests.  FP64,
    and the shifted layouts with the f - w rho0 shift, resume bit for bit.  With a storage shift
    by f^eq(rho0, u0) an FP32 stored value below about 2e-9 can lose low bits in the FP64 f it is
    read out as (f = v + f^eq then needs more than 53 bits): the resumed run then agrees to a few
    FP32 units in the last place, 1e-7 (FP16 values are never that small: exact)."""
    case = inputs.sphere_channel_case(H=32, B=8, radii=(20.0, 12.0, 6.5), inlet_outlet=True, shift=shift)
    a = lbm.Forest(case, precision=precision)
    a.init_uniform(case["u_init"])
    a.step_coarse(3)
    saved = [a.get_pdfs(L) for L in range(a.nlev)]
    b = lbm.Forest(case, precision=precision)
    for L in range(b.nlev):
        b.set_pdfs(L, saved[L])
    a.step_coarse(4)
    b.step_coarse(4)
    for L in range(a.nlev):
        pa, pb = a.get_pdfs(L), b.get_pdfs(L)
        if shift and precision == "fp32s":
            assert (np.isnan(pa) == np.isnan(pb)).all()
            assert np.nanmax(np.abs(pa - pb)) <= 1e-7
        else:
            assert np.array_equal(pa, pb, equal_nan=True)


def test_reduced_precision_errors_against_the_fp64_oracle(lbm, oracle_mod):
    """Shifted FP32 and FP16 storage with FP32 collide on the two-level cavity: the velocity error
    relative to the lid speed, against the FP64 oracle after 100 coarse steps."""
    case = inputs.cavity_case()
    o = oracle_mod.Oracle(case)
    o.init_fields(inputs.uniform_field())
    o.step(100)
    errs = {}
    for prec in ("fp32s", "fp16s"):
        f = lbm.Forest(case, precision=prec)
        f.init_uniform()
        f.step_coarse(100)
        e = 0.0
        for L in range(2):
            rho, u = f.get_macroscopic(L)
            X, Y, Z = f.cell_coords(L)
            idx = o.lookup(L, X, Y, Z)
            orho, ou = o.macro(L)
            e = max(e, max(float(np.abs(u[k] - ou[k][idx]).max()) for k in range(3)) / 0.05)
        errs[prec] = e
    assert errs["fp32s"] < 1e-5
    assert errs["fp16s"] < 2e-3


def test_timing_api_reports_every_launch(lbm):
    case = inputs.cavity_case()
    f = lbm.Forest(case)
    f.init_uniform()
    f.step_coarse(2)
    f.timing_begin(5)
    f.step_coarse(5)
    ms, cnt, ems, ecnt = f.timing_end(explode=True)
    assert cnt.tolist() == [5, 10]           # level 1 takes two sub-steps per coarse step
    assert ecnt.tolist() == [0, 5]           # one explosion per visit of level 1
    assert (ms > 0).all() and ems[1] > 0
    assert f.launches_per_coarse_step() == 4


def test_thread_mapping_does_not_change_results(lbm):
    """Every (cells per thread, CTAs per SM) variant of the step kernel computes each cell the same
    way, so the PDFs agree bit for bit."""
    case = inputs.sphere_channel_case(H=32, B=16, radii=(20.0, 12.0, 6.5))
    ref = None
    for lzc, minb in ((0, 3), (2, 3), (4, 2), (1, 2)):
        f = lbm.Forest(case, precision="fp32s")
        f.set_kernel_config(lzc, minb)
        f.init_uniform(case["u_init"])
        f.step_coarse(3)
        out = [f.get_pdfs(L) for L in range(f.nlev)]
        if ref is None:
            ref = out
        else:
            for L in range(f.nlev):
                assert np.array_equal(out[L], ref[L], equal_nan=True)


def test_periodic_sphere_channel_matches_the_oracle(lbm, oracle_mod):
    """The benchmark workload's geometry and boundaries (periodic faces, plug start) at H = 32."""
    case = inputs.sphere_channel_case(H=32, B=8, radii=(20.0, 12.0, 6.5))
    f, o = _pair(lbm, oracle_mod, case)
    assert f.nlev == 4
    f.step_coarse(8)
    o.step(8)
    assert _compare(f, o) < TOL64


def _mirror_gap(f, level, axis, n0=(256, 64, 64)):
    """max |u(p) - M u(M p)| over owned fluid cells for the mirror M that flips `axis` (1 = y,
    2 = z) about the centre of the domain of n0 level-0 cells (the sphere channel's by default,
    whose sphere centre lies on it)."""
    rho, u = f.get_macroscopic(level)
    X, Y, Z = f.cell_coords(level)
    n = [n0[0] << level, n0[1] << level, n0[2] << level]
    key = (Z.astype(np.int64) * n[1] + Y) * n[0] + X
    c = [X.copy(), Y.copy(), Z.copy()]
    c[axis] = n[axis] - 1 - c[axis]
    mkey = (c[2].astype(np.int64) * n[1] + c[1]) * n[0] + c[0]
    order = np.argsort(key)
    j = order[np.searchsorted(key[order], mkey)]
    assert (key[j] == mkey).all()
    ok = np.isfinite(rho)
    um = u.copy()
    um[axis] = -um[axis]
    return float(np.abs(u[:, ok] - um[:, j][:, ok]).max())


def test_recorded_totals_with_obstacle_warps_and_a_new_launch_configuration(lbm):
    """The bench workload (FP32S): on the finest level whole warps lie inside the sphere (they
    record zero moments), and a new launch configuration changes the number and layout of the
    warp entries.  The recorded totals (moments the last collisions started from) and the stored
    state's totals agree to FP32 rounding; a stale or missing warp entry would add or drop tens of
    cells."""
    case = inputs.sphere_channel_case()
    f = lbm.Forest(case, precision="fp32s")
    f.init_uniform(case["u_init"])
    lzc, minb = f.kernel_config()
    for cfg in ((lzc, minb), (lzc - 1, minb), (lzc, minb)):
        f.set_kernel_config(*cfg)
        f.step_coarse(5)
        rec = f.reduce_mass_momentum()
        f.set_kernel_config(*cfg)                 # drops the recorded moments: sum the stored PDFs
        sto = f.reduce_mass_momentum()
        assert abs(rec[0] - sto[0]) <= 1e-9 * sto[0], (cfg, rec, sto)
        assert np.abs(rec[1:] - sto[1:]).max() <= 1e-9 * sto[0], (cfg, rec, sto)
    f.close()


def test_full_size_lid_scaling_workload_conserves_mass_and_symmetry(lbm):
    """The benchmark cavity at the size bench.py times (3^3 roots of 32^3 cells, 10.5M cells,
    4 levels) in FP64: the flow stays mirror-symmetric about the y mid-plane (lid motion along
    x) and carries no y momentum.  Mass: where a wall meets a level interface, a fine ghost
    cell's wall links reach the coarse level through coalescence only in the coalescing
    directions, without their partners, so the scheme as read is not exactly conservative there
    (the oracle drifts alike, by about 1e-7 over 20 coarse steps, and by about 3e-8 with every
    wall at rest and a flow started inside); the bound here is a sanity bound, not conservation."""
    case = inputs.lid_scaling_case()
    f = lbm.Forest(case, precision="fp64")
    f.init_uniform()
    m0 = f.reduce_mass_momentum()
    f.step_coarse(20)
    m1 = f.reduce_mass_momentum()
    assert abs(m1[0] - m0[0]) / m0[0] < 1e-6
    assert abs(m1[2]) < 1e-12 * m0[0]
    n0 = tuple(r * case["B"] for r in case["root"])
    for L in range(f.nlev):
        assert _mirror_gap(f, L, 1, n0) < 1e-12
    rho, u = f.get_macroscopic(3)
    assert np.abs(u[0]).max() > 1e-3          # the lid has set the finest level in motion
    f.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32s", "fp16s"])
def test_recorded_totals_are_the_moments_of_the_streamed_state(lbm, precision):
    """After a coarse step the totals are the moments the step's collisions started from, recorded
    by the step kernel.  On a fully periodic single-level grid streaming permutes each direction's
    values among the cells, so they equal the totals of the state before the step, summed here in
    FP64 from its exact stored values.  The kernel sums each cell's 19 values, then the cells of a
    warp (at most 32 per thread, then a 5-level shuffle tree), in the compute type (FP64, or FP32
    from the shifted values f - w rho0), and the warps in FP64.  Recursive-summation bounds:
    gamma_18 sum_q |f_q| per cell, gamma_40 of the same sums for the warp, gamma_64 (FP64) of the
    cell totals for the rest."""
    case = inputs.periodic_case(n=64, B=16, collision="trt", omega=1.7)
    f = lbm.Forest(case, precision=precision)
    f.init_fields(inputs.taylor_green_field(64))
    f.step_coarse(2)
    pd = f.get_pdfs(0)
    e, w, _ = lbm.lbm_lattice()
    rho0 = case["rho0"]
    s = pd if precision == "fp64" else pd - w[:, None] * rho0       # exact: the stored values
    f.step_coarse(1)
    got = f.reduce_mass_momentum()
    u = 2.0 ** -53 if precision == "fp64" else 2.0 ** -24
    gamma = lambda k, u: k * u / (1 - k * u)

    def check(got, pd, s):
        ref = np.concatenate([[pd.sum()], (e.T.astype(float) @ pd).sum(axis=1)])
        bound = (gamma(18, u) + gamma(40, u)) * np.abs(s).sum() + gamma(64, 2.0 ** -53) * np.abs(pd.sum(axis=0)).sum()
        assert abs(got[0] - ref[0]) <= bound, (got[0] - ref[0], bound)
        assert np.abs(got[1:] - ref[1:]).max() <= bound, (got[1:] - ref[1:], bound)
        assert bound < 0.5          # a missing cell (rho near 1) would fail

    check(got, pd, s)
    # a new launch configuration drops the recorded moments: the totals are then summed from the
    # stored state (no body force here, so j needs no correction)
    lzc, minb = f.kernel_config()
    f.set_kernel_config(lzc - 1, minb)
    pd = f.get_pdfs(0)
    check(f.reduce_mass_momentum(), pd, pd if precision == "fp64" else pd - w[:, None] * rho0)
    f.close()


def test_full_size_bench_workload_conserves_mass_and_symmetry(lbm):
    """Bench workload at full size (8.39M cells, 4 levels, 32^3 blocks) in FP64, in the launch
    configuration bench.py times: total mass is conserved to round-off and the flow stays
    mirror-symmetric about the y and z mid-planes; FP32 storage conserves mass to 1e-6."""
    case = inputs.sphere_channel_case()
    f = lbm.Forest(case, precision="fp64")
    f.init_uniform(case["u_init"])
    m0 = f.reduce_mass_momentum()
    f.step_coarse(40)
    m1 = f.reduce_mass_momentum()
    assert abs(m1[0] - m0[0]) / m0[0] < 1e-12
    assert _mirror_gap(f, 1, 1) < 1e-12 and _mirror_gap(f, 1, 2) < 1e-12
    f.close()
    g = lbm.Forest(case, precision="fp32s")
    g.init_uniform(case["u_init"])
    m0 = g.reduce_mass_momentum()
    g.step_coarse(40)
    m1 = g.reduce_mass_momentum()
    assert abs(m1[0] - m0[0]) / m0[0] < 1e-6


# --------------------------------------------------------------------------- B = 32

def _macro_errors(f, o):
    """Velocity error (L-inf over owned fluid cells of every level, relative to the oracle's max |u|)
    and density error (L-inf) of forest f against the oracle's state."""
    du, dr, umax = 0.0, 0.0, 0.0
    for L in range(f.nlev):
        rho, u = f.get_macroscopic(L)
        X, Y, Z = f.cell_coords(L)
        idx = o.lookup(L, X, Y, Z)
        orho, ou = o.macro(L)
        ok = np.isfinite(orho[idx])
        assert (np.isfinite(rho) == ok).all()
        du = max(du, max(float(np.abs(u[k][ok] - ou[k][idx][ok]).max()) for k in range(3)))
        dr = max(dr, float(np.abs(rho[ok] - orho[idx][ok]).max()))
        umax = max(umax, max(float(np.abs(ou[k][idx][ok]).max()) for k in range(3)))
    return du / umax, dr


def test_b32_refined_box_with_a_sphere_on_the_interface_matches_the_oracle(lbm, oracle_mod):
    """32^3-cell blocks (the block size every bench workload uses): a periodic 64^3 box of 2^3 roots,
    one corner root refined, a sphere cut by the level interface, Taylor-Green flow; FP64 element by
    element after 20 coarse steps, in the default launch configuration and with one cell per thread
    on 2 CTAs per SM."""
    case = inputs.periodic_case(n=64, B=32, collision="trt", omega=1.7,
                                regions=[("box", 1, (0, 0, 0), (16, 16, 16))], lmax=1)
    case["spheres"] = [(16.0, 16.0, 16.0, 6.0)]
    field = inputs.taylor_green_field(64)
    o = oracle_mod.Oracle(case)
    o.init_fields(field)
    o.step(20)
    for cfg in (None, (0, 2)):
        f = lbm.Forest(case, precision="fp64")
        assert f.nlev == 2
        if cfg:
            f.set_kernel_config(*cfg)
        f.init_fields(field)
        f.step_coarse(20)
        assert _compare(f, o) < TOL64
        f.close()


def test_full_size_bench_workload_matches_the_oracle(lbm, oracle_mod):
    """The bench workload itself (sphere channel, 8.39M cells, 4 levels, 32^3 blocks, periodic,
    plug start) in the launch configuration bench.py times: FP64 equals the oracle element by
    element to 1e-12 after 4 coarse steps (60 level launches, 28 explosions).  The FP32S and FP16S
    storage (shifted by f^eq(rho0, plug)) against the same oracle state: velocity error relative to
    the largest oracle speed, and density error."""
    case = inputs.sphere_channel_case()
    steps = 4
    o = oracle_mod.Oracle(case)
    o.init_fields(inputs.uniform_field(u=case["u_init"]))
    o.step(steps)
    f = lbm.Forest(case, precision="fp64")
    assert f.nlev == 4 and [len(f.block_table(L)) for L in range(4)] == [16, 120, 56, 64]
    f.init_uniform(case["u_init"])
    f.step_coarse(steps)
    assert _compare(f, o) < TOL64
    f.close()
    errs = {}
    for prec in ("fp32s", "fp16s"):
        g = lbm.Forest(case, precision=prec)
        g.init_uniform(case["u_init"])
        g.step_coarse(steps)
        errs[prec] = _macro_errors(g, o)
        g.close()
    print("B=32 bench workload, %d coarse steps: (u L-inf / u_max, rho L-inf) fp32s %.3e %.3e, fp16s %.3e %.3e"
          % ((steps,) + errs["fp32s"] + errs["fp16s"]))
    assert errs["fp32s"][0] < 1e-5 and errs["fp32s"][1] < 1e-6
    assert errs["fp16s"][0] < 1e-3 and errs["fp16s"][1] < 1e-4


def test_macroscopic_fields_of_all_levels_in_one_call(lbm):
    """level = -1 returns every level in one array, level 0 first: the same values as the per-level
    calls, on the host and on the device."""
    import torch
    case = inputs.sphere_channel_case(H=32, B=8, radii=(20.0, 12.0, 6.5))
    f = lbm.Forest(case, precision="fp32s")
    f.init_uniform(case["u_init"])
    f.step_coarse(3)
    per = [f.get_macroscopic(L) for L in range(f.nlev)]
    rho, u = f.get_macroscopic(-1)
    assert np.array_equal(rho, np.concatenate([r for r, _ in per]), equal_nan=True)
    assert np.array_equal(u, np.concatenate([v for _, v in per], axis=1), equal_nan=True)
    n = rho.size
    dr = torch.empty(n, dtype=torch.float64, device="cuda")
    du = torch.empty((3, n), dtype=torch.float64, device="cuda")
    f.get_macroscopic(-1, dr, du, on_device=True)
    assert np.array_equal(dr.cpu().numpy(), rho, equal_nan=True)
    assert np.array_equal(du.cpu().numpy(), u, equal_nan=True)
    f.close()


def test_timing_api_reports_the_side_kernels_apart(lbm):
    """FP32S storage: the coupled cells and ghost work of each sub-step run in their own side kernel
    (on a graph branch beside the column walk); the timing mode runs them in series and reports
    them per level apart from the walk."""
    f = lbm.Forest(inputs.cavity_case(), precision="fp32s")
    f.init_uniform()
    f.step_coarse(2)
    f.timing_begin(3)
    f.step_coarse(3)
    ms, cnt, ems, ecnt, sms, scnt = f.timing_end(explode=True, side=True)
    assert cnt.tolist() == [3, 6] and ecnt.tolist() == [0, 3]
    assert scnt[0] == 3 and scnt[1] > 0          # level 0 has coupled cells, level 1 ghost work
    assert (sms[scnt > 0] > 0).all() and (ms > 0).all()
    assert f.launches_per_coarse_step() == 4 + int(scnt.sum()) // 3
    f.close()


def test_a_non_finite_value_is_reported_by_the_totals(lbm):
    """Failure detection on the host: a NaN written into one fluid cell through lbm_set_pdfs (as a
    diverged run would leave) makes lbm_reduce_mass_momentum return LBM_ENONFINITE after a step,
    in every storage precision; obstacle cells, which hold NaN by design, do not."""
    case = inputs.sphere_channel_case(H=32, B=8, radii=(20.0, 12.0, 6.5))
    for prec in ("fp64", "fp32s", "fp16s"):
        f = lbm.Forest(case, precision=prec)
        f.init_uniform(case["u_init"])
        f.step_coarse(1)
        f.reduce_mass_momentum()                      # obstacle NaNs are not counted
        pd = f.get_pdfs(0)
        fluid = np.flatnonzero(np.isfinite(pd).all(axis=0))
        pd[5, fluid[len(fluid) // 2]] = np.nan
        f.set_pdfs(0, pd)
        with pytest.raises(lbm.LBMError) as ei:
            f.reduce_mass_momentum()
        assert ei.value.status == lbm.LBM_ENONFINITE
        f.step_coarse(1)                              # the NaN spreads to its neighbours
        with pytest.raises(lbm.LBMError) as ei:
            f.reduce_mass_momentum()
        assert ei.value.status == lbm.LBM_ENONFINITE
        f.close()


def test_fp64_probe_measures_a_plausible_rate(lbm):
    """The FP64 FMA probe that the bench uses as the FP64 walk's roofline: positive and below the
    nominal FP64 rate of the part with a margin (1.25 TFLOP/s = 625 G FMA/s nominal)."""
    g = lbm.lbm_probe_fp64_fma(5)
    assert 50.0 < g < 2000.0
