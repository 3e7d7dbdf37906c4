"""Warm-start data movement (lbm_warmstart_*) and the steady-state residual (lbm_velocity_residual).

The pins are closed forms:
- the residual equals its definition recomputed from two macroscopic snapshots;
- trilinear sampling reproduces a constant field, and a field linear in x, exactly at every cell
  centre away from walls;
- targets -> fields returns the refined solution.
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


def _case():
    c = inputs.warm_cases(1, seed=3, H=32, B=8)[0]
    return c


def test_velocity_residual_matches_its_definition(lbm):
    case = inputs.cavity_case()
    f = lbm.Forest(case, precision="fp64")
    f.init_uniform()
    f.step_coarse(5)
    assert f.velocity_residual() == float("inf")
    u0 = [f.get_macroscopic(L)[1] for L in range(f.nlev)]
    f.step_coarse(10)
    r = f.velocity_residual()
    num = den = 0.0
    for L in range(f.nlev):
        u1 = f.get_macroscopic(L)[1]
        ok = np.isfinite(u1).all(axis=0)
        w = 8.0 ** -L
        num += w * ((u1 - u0[L])[:, ok] ** 2).sum()
        den += w * (u1[:, ok] ** 2).sum()
    assert abs(r - np.sqrt(num / den)) <= 1e-12 * r


def test_features_reproduce_constant_and_linear_coarse_fields(lbm):
    import torch
    from paper_1508_07982_gb300 import warmstart as ws
    with_spheres = _case()
    # no obstacles (their cells drop out of the interpolation) and no body force (the macroscopic
    # velocity of a forced state includes a/2)
    case = dict(with_spheres, spheres=[], accel=(0.0, 0.0, 0.0))
    coarse = lbm.Forest(ws.coarse_case(case), precision="fp64")
    fine = lbm.Forest(case, precision="fp64")
    n0 = coarse.n_cells(0)
    X, Y, Z = coarse.cell_coords(0)
    rho = np.ones(n0)
    a, b = 0.01, 2e-4
    u = np.zeros((3, n0))
    u[0] = a + b * (X + 0.5)          # linear in the cell-centre coordinate
    u[1] = 0.02
    coarse.init_equilibrium(0, rho, u)
    crho, cu, nb = ws._coarse_fields(coarse)
    H0 = nb[0] * case["B"]
    for L in range(1, fine.nlev):
        bt = fine.block_table(L)
        blocks = torch.tensor(bt, dtype=torch.int32, device="cuda")
        x, skip = lbm.warmstart_features(crho, cu, nb, case["B"], ws.periodic_mask(case), L, 2, blocks,
                                         ws._spheres(with_spheres), ws.RHO_SCALE, ws.u_scale(case))
        s = skip.cpu().numpy()
        xf = x.float().cpu().numpy()
        D = case["B"] + 4
        r = np.arange(D) - 2
        gx = bt[:, 0, None, None, None] * case["B"] + r[None, None, None, :]
        px = (gx + 0.5) / 2 ** L
        inside = (px > 0.5) & (px < H0 - 0.5)                       # away from the clamped x walls
        inside = np.broadcast_to(inside, s.shape[:-1])
        ref_ux = (a + b * np.broadcast_to(px, s.shape[:-1])) * ws.u_scale(case)
        assert np.abs(s[..., 1][inside] - ref_ux[inside]).max() <= 2e-6 * np.abs(ref_ux).max()
        assert np.abs(s[..., 2] - 0.02 * ws.u_scale(case)).max() <= 1e-6
        assert np.abs(s[..., 0]).max() <= 1e-6 and np.abs(s[..., 3]).max() <= 1e-6
        assert np.all(xf[..., 5] == L * 0.5) and not xf[..., 6:].any()
        solid = xf[..., 4] > 0
        assert solid.any() and (~solid).any()
    coarse.close()
    fine.close()


def test_targets_then_fields_return_the_refined_solution(lbm):
    import torch
    from paper_1508_07982_gb300 import warmstart as ws
    case = _case()
    fine = lbm.Forest(case, precision="fp64")
    fine.init_uniform((0.01, 0.0, 0.0))
    fine.step_coarse(3)
    for L in range(1, fine.nlev):
        nbk = len(fine.block_table(L))
        n = fine.n_cells(L)
        rho = torch.empty(n, dtype=torch.float64, device="cuda")
        u = torch.empty((3, n), dtype=torch.float64, device="cuda")
        fine.get_macroscopic(L, rho, u, on_device=True)
        t, w = lbm.warmstart_targets(rho, u, case["B"], 5, nbk, ws.RHO_SCALE, ws.u_scale(case))
        r2, u2 = lbm.warmstart_fields(t, case["B"], 5, nbk, ws.RHO_SCALE, ws.u_scale(case))
        ok = torch.isfinite(rho)
        assert torch.allclose(r2[ok], rho[ok], rtol=0, atol=1e-8)
        assert torch.allclose(u2[:, ok], u[:, ok], rtol=0, atol=1e-8)
        assert int(w.sum().item()) == int(ok.sum().item())
    fine.close()


def test_the_trained_net_predicts_a_held_out_refined_solution_better_than_the_coarse_one(lbm):
    """What the learned part of the warm start gains where it acts: trained on four 32^3 channels
    (targets: each refined solution, converged from the coarse-only start), the net's prediction
    of a fifth, held-out channel's refined levels is closer to its converged refined solution than
    the sampled coarse solution alone (the skip term the net corrects).  The loss is the training
    objective (weighted mean squared error of scaled rho and u on the fluid voxels)."""
    from paper_1508_07982_gb300 import warmstart as ws
    g = ws.heldout_gain(n_train=4, H=32, B=8, max_steps=40000, epochs=10)
    print("warm-start net, training-set loss %s, held-out loss %s" % (g["train_set"], g["heldout"]))
    assert g["train_set"]["net"] < g["train_set"]["coarse_only"]
    assert g["heldout"]["net"] < g["heldout"]["coarse_only"]
