"""Batches of forests (lbm_batch_*) and the thread-mapping autotuner (lbm_autotune).

A batch steps independent forests together, one launch per phase of Alg. 1 over all members.
Each member must compute exactly what it computes when stepped alone, so the GPU tests compare
batched and single stepping bit for bit (same kernels, same arithmetic), and one batched member
against the oracle.  The CPU tests check the batched workload's seeded case generator against
the library's forest planner.
"""
import ctypes

import numpy as np
import pytest

from paper_1508_07982_gb300 import inputs


def _rows(a):
    """Rows of a block list in lexicographic (z, y, x) order, to compare sets of blocks."""
    return a[np.lexsort((a[:, 0], a[:, 1], a[:, 2]))] if len(a) else a


def _same(a, b):
    """Bitwise equality of two PDF arrays, NaN positions included."""
    return a.shape == b.shape and np.array_equal(a.view(np.uint64), b.view(np.uint64))


# ---------------------------------------------------------------- host only

@pytest.fixture(scope="module")
def lbm_host():
    from paper_1508_07982_gb300 import build, lbm as mod
    build.build()
    return mod


def test_batch_cases_are_seeded_balanced_and_in_range(lbm_host):
    cases = inputs.batch_cases()
    again = inputs.batch_cases()
    assert len(cases) == 256 and cases == again
    levels = {c["lmax"] + 1 for c in cases}
    assert levels == {2, 3}
    for c in cases:
        assert 8 <= c["leaves"] <= 64 and c["B"] == 16
        assert all(1 <= r <= 4 for r in c["root"])
        assert 1.5 <= c["lambda_e0"] <= 1.9 and 0.02 <= c["bc_u"][5][0] <= 0.08
    # the generator's leaf count (boxes drawn 2:1-balanced) is what the planner builds: the
    # balance step adds no split
    for c in cases[:64]:
        p = lbm_host.Plan(c)
        assert p.nlev == c["lmax"] + 1
        assert sum(p.counts(L)["blocks"] for L in range(p.nlev)) == c["leaves"]


def test_block_size_tuner_rejects_a_refine_callback_before_any_cuda_call(lbm_host):
    """A refine callback takes block coordinates, which change with the block size, so the tuner
    refuses it (LBM_EINVAL) before it creates a forest."""
    case = inputs.periodic_case(n=64, B=16, regions=[("box", 1, (16, 16, 16), (48, 48, 48))], lmax=1)
    d = lbm_host.make_desc(case, "fp32s")
    cb = lbm_host.REFINE_FN(lambda L, x, y, z, u: 0)
    b = ctypes.c_int32()
    st = lbm_host.library().lbm_autotune_block_size(ctypes.byref(d), cb, lbm_host.FLAG_FN(), None, 1.6,
                                                    3 / 16, None, None, None, 2, ctypes.byref(b), None)
    assert st == lbm_host.LBM_EINVAL and "refine callback" in lbm_host.library().lbm_last_error().decode()


def test_batch_cases_match_the_oracle_forest(lbm_host, oracle_mod):
    for c in inputs.batch_cases(n=6, seed=11):
        p = lbm_host.Plan(c)
        o = oracle_mod.Oracle(c)
        assert p.nlev == o.nlev
        for L in range(p.nlev):
            a, b = p.leaves(L), o.leaves(L)
            assert a.shape == b.shape and (_rows(a) == _rows(b)).all()


# ---------------------------------------------------------------- GPU

@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1508_07982_gb300 import build, lbm as mod
    build.build()
    return mod


def _forests(lbm, cases, precision):
    fs = []
    for c in cases:
        f = lbm.Forest(c, precision=precision)
        f.init_uniform()
        fs.append(f)
    return fs


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "fp32s"])
def test_batch_steps_each_member_as_a_single_forest_would(lbm, precision):
    cases = inputs.batch_cases(n=10, seed=3)
    assert {c["lmax"] for c in cases} == {1, 2}
    alone = _forests(lbm, cases, precision)
    together = _forests(lbm, cases, precision)
    for f in alone:
        f.step_coarse(7)
    b = lbm.Batch(together)
    b.step(3)
    b.step(4)               # odd and even level-0 parities, graph per parity
    for fa, fb in zip(alone, together):
        for L in range(fa.nlev):
            assert _same(fa.get_pdfs(L), fb.get_pdfs(L)), "member differs on level %d" % L
    assert b.cell_updates_per_coarse_step() == sum(f.cell_updates_per_coarse_step() for f in together)
    # one launch per phase: level 0, and per level L >= 1 its explosions and sub-steps; with FP32/FP16
    # storage each sub-step's coupled cells and ghost work take a launch of their own before it
    assert b.launches_per_coarse_step() <= (1 + 3 + 6) * (1 if precision == "fp64" else 2)
    # members still step on their own afterwards, and the batch picks up where they are
    for f in together:
        f.step_coarse(1)
    for f in alone:
        f.step_coarse(2)
    b.step(1)
    for fa, fb in zip(alone, together):
        assert _same(fa.get_pdfs(fa.nlev - 1), fb.get_pdfs(fb.nlev - 1))
    b.close()


@pytest.mark.gpu
def test_batch_member_matches_the_oracle(lbm, oracle_mod):
    cases = inputs.batch_cases(n=8, seed=5)
    deep = next(i for i, c in enumerate(cases) if c["lmax"] == 2)
    fs = _forests(lbm, cases, "fp64")
    o = oracle_mod.Oracle(cases[deep])
    o.init_fields(inputs.uniform_field())
    b = lbm.Batch(fs)
    b.step(6)
    o.step(6)
    f = fs[deep]
    num = den = 0.0
    for L in range(f.nlev):
        g = f.get_pdfs(L)
        X, Y, Z = f.cell_coords(L)
        idx = o.lookup(L, X, Y, Z)
        ref = o.get_f(L, post_collision=True)[idx].T
        ok = np.isfinite(ref).all(axis=0)
        num = max(num, float(np.abs(g[:, ok] - ref[:, ok]).max()))
        den = max(den, float(np.abs(ref[:, ok]).max()))
    assert num / den <= 1e-12
    b.close()


@pytest.mark.gpu
def test_fp32s_batch_member_error_against_the_oracle(lbm, oracle_mod):
    """The batched workload runs in FP32S storage; its error against the FP64 oracle is stated: a
    3-level member, 20 coarse steps from rest, velocity within 1e-5 of the lid speed and density
    within 1e-6 on every owned fluid cell (FP32 rounding of the stored deviations, of order 1e-7
    relative, accumulated over 80 finest steps)."""
    cases = inputs.batch_cases(n=8, seed=5)
    deep = next(i for i, c in enumerate(cases) if c["lmax"] == 2)
    fs = _forests(lbm, cases, "fp32s")
    o = oracle_mod.Oracle(cases[deep])
    o.init_fields(inputs.uniform_field())
    b = lbm.Batch(fs)
    b.step(20)
    o.step(20)
    f = fs[deep]
    lid = cases[deep]["bc_u"][5][0]
    du = dr = 0.0
    for L in range(f.nlev):
        rho, u = f.get_macroscopic(L)
        X, Y, Z = f.cell_coords(L)
        idx = o.lookup(L, X, Y, Z)
        rr, ur = o.macro(L)
        ok = np.isfinite(rho)
        for k in range(3):
            du = max(du, float(np.abs(u[k][ok] - ur[k][idx][ok]).max()))
        dr = max(dr, float(np.abs(rho[ok] - rr[idx][ok]).max()))
    print("FP32S batch member against the oracle: u L-inf / lid %.3e, rho L-inf %.3e" % (du / lid, dr))
    assert du / lid < 1e-5 and dr < 1e-6
    b.close()


@pytest.mark.gpu
def test_autotune_leaves_the_state_and_results_unchanged(lbm):
    case = inputs.sphere_channel_case(H=32, B=16, radii=(20.0, 12.0, 6.5))
    f = lbm.Forest(case, precision="fp32s")
    g = lbm.Forest(case, precision="fp32s")
    for h in (f, g):
        h.init_uniform(case["u_init"])
        h.step_coarse(3)
    before = [f.get_pdfs(L) for L in range(f.nlev)]
    lzc, minb, ms = f.autotune(2)
    assert 0 <= lzc <= 4 and minb in (1, 2, 3, 4) and ms > 0
    assert f.kernel_config() == (lzc, minb)
    for L in range(f.nlev):
        assert _same(before[L], f.get_pdfs(L))
    f.step_coarse(3)
    g.step_coarse(3)
    for L in range(f.nlev):
        assert _same(f.get_pdfs(L), g.get_pdfs(L))


@pytest.mark.gpu
def test_batch_autotune_keeps_members_in_step(lbm):
    cases = inputs.batch_cases(n=6, seed=9)
    fs = _forests(lbm, cases, "fp32s")
    ref = _forests(lbm, cases, "fp32s")
    b = lbm.Batch(fs)
    lzc, minb, ms = b.autotune(2)
    assert 0 <= lzc <= 4 and minb in (1, 2, 3, 4) and ms > 0
    b.step(5)
    for f in ref:
        f.step_coarse(5)
    for fa, fb in zip(fs, ref):
        for L in range(fa.nlev):
            assert _same(fa.get_pdfs(L), fb.get_pdfs(L))
    b.close()


@pytest.mark.gpu
def test_block_size_tuner_times_every_candidate_and_keeps_the_fastest(lbm):
    """The block-size tuner builds the case with 8^3, 16^3 and 32^3 blocks (the same 64^3 domain and
    refined box), tunes and times each, and returns the fastest; the case itself is unchanged."""
    case = inputs.periodic_case(n=64, B=16, collision="trt", omega=1.7,
                                regions=[("box", 1, (16, 16, 16), (48, 48, 48))], lmax=1)
    B, ms = lbm.autotune_block_size(case, "fp32s", n_steps=3)
    assert set(ms) == {8, 16, 32} and all(v > 0 for v in ms.values()), ms
    assert B in (8, 16, 32) and ms[B] == min(ms.values())
    # a domain that 32 does not divide leaves that candidate out
    case48 = inputs.periodic_case(n=48, B=16, collision="trt", omega=1.7)
    B48, ms48 = lbm.autotune_block_size(case48, "fp32s", n_steps=2)
    assert ms48[32] == -1 and ms48[8] > 0 and ms48[16] > 0 and B48 in (8, 16)


@pytest.mark.gpu
def test_batch_rejects_mismatched_members(lbm):
    a = lbm.Forest(inputs.cavity_case(), precision="fp32s")
    c = lbm.Forest(inputs.cavity_case(), precision="fp64")
    with pytest.raises(lbm.LBMError) as ei:
        lbm.Batch([a, c])
    assert ei.value.status == lbm.LBM_EINVAL
    a.init_uniform()
    d = lbm.Forest(inputs.cavity_case(), precision="fp32s")
    d.init_uniform()
    d.step_coarse(1)        # one coarse step ahead: the level-0 parities differ
    b = lbm.Batch([a, d])
    with pytest.raises(lbm.LBMError) as ei:
        b.step(1)
    assert "parity" in str(ei.value)
    b.close()
