"""Learned warm start of the refined levels: the workflow around lbm_net_* and lbm_warmstart_*.

A warm start replaces the rest state f^eq(1, 0) of the refined forest by f^eq(rho^, u^), where
(rho^, u^) on each refined block is the net's prediction from the coarse-only steady solution
sampled onto the block and its halo; level 0 takes the coarse solution itself.  The LBM then runs
unmodified to the steady state.  Every step runs in the library's kernels; this module only
orders the calls and holds the device tensors (PyTorch provides memory and the stream).
"""
import time

import numpy as np

from . import lbm

RHO_SCALE = 100.0      # density deviations of order 1e-2 -> order 1
HALO = 5               # voxels of context around each refined block


def u_scale(case):
    u = case.get("u_in") or max(abs(float(v)) for w in case["bc_u"] for v in w) or 0.04
    return 1.0 / u


def coarse_case(case):
    """The same domain and obstacles on level 0 only."""
    c = dict(case)
    c["lmax"] = 0
    c["regions"] = []
    return c


def periodic_mask(case):
    return sum(1 << a for a in range(3) if case["bc"][2 * a] == "periodic")


THRESHOLDS = (1e-3, 1e-4, 1e-5, 1e-6)


def steady(f, max_steps, tol=1e-6, every=10):
    """Coarse steps until the residual of lbm_velocity_residual, taken every `every` steps, falls
    below tol; returns {steps, seconds, residual, first step below each of THRESHOLDS (or None)}."""
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    f.velocity_residual()
    steps, r = 0, float("inf")
    reached = {t: None for t in THRESHOLDS}
    while steps < max_steps:
        f.step_coarse(every)
        steps += every
        r = f.velocity_residual()
        for t in THRESHOLDS:
            if reached[t] is None and r < t:
                reached[t] = steps
        if r < tol:
            break
    torch.cuda.synchronize()
    return {"steps": steps, "seconds": round(time.perf_counter() - t0, 3), "residual": r,
            "steps_to": {"%g" % t: reached[t] for t in THRESHOLDS}}


def _coarse_fields(coarse):
    import torch
    n = coarse.n_cells(0)
    rho = torch.empty(n, dtype=torch.float64, device="cuda")
    u = torch.empty((3, n), dtype=torch.float64, device="cuda")
    coarse.get_macroscopic(0, rho, u, on_device=True)
    nb = coarse.block_table(0).max(axis=0) + 1
    return rho, u, nb


def _spheres(case):
    import torch
    if not case["spheres"]:
        return None
    return torch.tensor(np.asarray(case["spheres"], np.float64), device="cuda")


def features(coarse, fine, case, level, halo=HALO):
    """Net inputs (and the skip term) for the blocks of one refined level of `fine`."""
    import torch
    rho, u, nb = _coarse_fields(coarse)
    blocks = torch.tensor(fine.block_table(level), dtype=torch.int32, device="cuda")
    return lbm.warmstart_features(rho, u, nb, case["B"], periodic_mask(case), level, halo, blocks, _spheres(case),
                                  RHO_SCALE, u_scale(case))


def samples(coarse, fine, case, halo=HALO, max_blocks=None, seed=0):
    """Training volumes of every refined level: (x, skip, target, weight) on the device; with
    max_blocks, a seeded random subset of each level's blocks."""
    import torch
    rng = np.random.default_rng(seed)
    xs, ss, ts, ws = [], [], [], []
    rho0, u0, nb0 = _coarse_fields(coarse)
    B = case["B"]
    for L in range(1, fine.nlev):
        table = fine.block_table(L)
        nbk = len(table)
        if nbk == 0:
            continue
        pick = np.arange(nbk)
        if max_blocks is not None and nbk > max_blocks:
            pick = np.sort(rng.choice(nbk, max_blocks, replace=False))
        blocks = torch.tensor(table[pick], dtype=torch.int32, device="cuda")
        x, skip = lbm.warmstart_features(rho0, u0, nb0, B, periodic_mask(case), L, halo, blocks, _spheres(case),
                                         RHO_SCALE, u_scale(case))
        n = fine.n_cells(L)
        rho = torch.empty(n, dtype=torch.float64, device="cuda")
        u = torch.empty((3, n), dtype=torch.float64, device="cuda")
        fine.get_macroscopic(L, rho, u, on_device=True)
        sel = torch.tensor(pick, device="cuda")
        rho = rho.view(nbk, B ** 3)[sel].reshape(-1).contiguous()
        u = u.view(3, nbk, B ** 3)[:, sel].reshape(3, -1).contiguous()
        t, w = lbm.warmstart_targets(rho, u, B, halo, len(pick), RHO_SCALE, u_scale(case))
        xs.append(x)
        ss.append(skip)
        ts.append(t)
        ws.append(w)
    return torch.cat(xs), torch.cat(ss), torch.cat(ts), torch.cat(ws)


def train(net, data, epochs, lr=2e-3, batch=32, seed=0):
    """Adam on mini-batches of volumes; returns the mean loss of each epoch."""
    import torch
    x, skip, target, weight = data
    n = x.shape[0]
    g = torch.Generator(device="cpu").manual_seed(seed)
    losses = []
    for _ in range(epochs):
        perm = torch.randperm(n, generator=g).cuda()
        tot, cnt = 0.0, 0
        for i in range(0, n, batch):
            idx = perm[i:i + batch]
            if weight[idx].sum() == 0:
                continue
            tot += net.train_step(x[idx].contiguous(), target[idx].contiguous(), skip[idx].contiguous(),
                                  weight[idx].contiguous(), lr=lr)
            cnt += 1
        losses.append(tot / max(cnt, 1))
    return losses


def mean_loss(net, data, batch=32):
    """The net's loss (the training objective) averaged over the mini-batches of `data`, without
    updating it."""
    x, skip, target, weight = data
    tot, cnt = 0.0, 0
    for i in range(0, x.shape[0], batch):
        sl = slice(i, i + batch)
        if weight[sl].sum() == 0:
            continue
        net.predict(x[sl].contiguous(), skip[sl].contiguous())
        tot += net.gradient(target[sl].contiguous(), skip[sl].contiguous(), weight[sl].contiguous())
        cnt += 1
    return tot / max(cnt, 1)


def zero_net(like):
    """A net of the same shape with every parameter zero: its prediction is the skip term, the
    sampled coarse solution itself."""
    z = lbm.Net(like.layers, like.in_channels, like.out_channels)
    z.set_params(np.zeros(z.num_params(), np.float32))
    return z


def init_warm(net, coarse, fine, case, halo=HALO, use_net=True):
    """Starts every level of `fine` from f^eq of the coarse solution (level 0) or of the net's
    prediction on its blocks (refined levels); with use_net=False the refined levels take the
    sampled coarse solution alone.  Returns the seconds spent."""
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for L in range(fine.nlev):
        nbk = len(fine.block_table(L))
        if nbk == 0:
            fine.init_equilibrium(L)
            continue
        h = halo if L > 0 else 0
        x, skip = features(coarse, fine, case, L, h)
        pred = net.predict(x, skip) if (use_net and L > 0) else skip
        rho, u = lbm.warmstart_fields(pred, case["B"], h, nbk, RHO_SCALE, u_scale(case))
        fine.init_equilibrium(L, rho, u, on_device=True)
    torch.cuda.synchronize()
    return time.perf_counter() - t0


def level_fields(f):
    """(rho, u) of every level of f as device tensors, obstacle cells set to (1, 0)."""
    import torch
    out = []
    for L in range(f.nlev):
        n = f.n_cells(L)
        rho = torch.empty(n, dtype=torch.float64, device="cuda")
        u = torch.empty((3, n), dtype=torch.float64, device="cuda")
        if n:
            f.get_macroscopic(L, rho, u, on_device=True)
        out.append((torch.nan_to_num(rho, nan=1.0), torch.nan_to_num(u, nan=0.0)))
    return out


def init_ideal(coarse, fine, case, fields):
    """The bound of every predictor of the refined levels: level 0 from the coarse solution as in
    init_warm, every refined level from `fields`, the converged refined solution itself."""
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for L in range(fine.nlev):
        if L == 0:
            x, skip = features(coarse, fine, case, 0, 0)
            rho, u = lbm.warmstart_fields(skip, case["B"], 0, len(fine.block_table(0)), RHO_SCALE, u_scale(case))
            fine.init_equilibrium(0, rho, u, on_device=True)
        elif fine.n_cells(L):
            fine.init_equilibrium(L, fields[L][0], fields[L][1], on_device=True)
        else:
            fine.init_equilibrium(L)
    torch.cuda.synchronize()
    return time.perf_counter() - t0


def experiment(n_train=16, n_test=4, H=64, B=8, max_steps=6000, epochs=20, max_blocks=384, seed=20150827,
               precision="fp32s", log=print):
    """Trains the net on n_train cases of inputs.warm_cases and compares, on n_test held-out
    cases, the refined solve from rest (cold), from the sampled coarse solution alone, and from
    the net's prediction (warm); the coarse-only solve and the net's time count for the last two.
    A fourth start (ideal) takes level 0 from the coarse solution and every refined level from the
    cold run's converged solution: no predictor of the refined levels can start closer."""
    import torch
    from . import inputs
    cases = inputs.warm_cases(n_train + n_test, seed=seed, H=H, B=B)
    net = lbm.Net(5, 6, 4, seed=seed)
    data, gen = [], []
    for i, c in enumerate(cases[:n_train]):
        coarse = lbm.Forest(coarse_case(c), precision=precision)
        coarse.init_uniform()
        sc = steady(coarse, max_steps)
        fine = lbm.Forest(c, precision=precision)
        init_warm(net, coarse, fine, c, use_net=False)
        sf = steady(fine, max_steps)
        data.append(samples(coarse, fine, c, max_blocks=max_blocks, seed=i))
        gen.append({"coarse": sc, "fine": sf})
        log("train case %d: coarse %s fine %s" % (i, sc["steps"], sf["steps"]))
        coarse.close()
        fine.close()
    data = tuple(torch.cat([d[k] for d in data]) for k in range(4))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = train(net, data, epochs)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    zero = zero_net(net)
    fit = {"net": mean_loss(net, data), "coarse_only": mean_loss(zero, data)}
    log("losses %s; training-set loss %s" % (["%.4g" % v for v in losses], fit))
    tests = []
    for c in cases[n_train:]:
        row = {"spheres": len(c["spheres"]), "re": round(c["re"], 2)}
        coarse = lbm.Forest(coarse_case(c), precision=precision)
        coarse.init_uniform()
        row["coarse"] = steady(coarse, max_steps)
        converged = None
        for mode in ("cold", "coarse_only", "warm", "ideal"):
            fine = lbm.Forest(c, precision=precision)
            t_init = 0.0
            if mode == "cold":
                fine.init_uniform()
            elif mode == "ideal":
                t_init = init_ideal(coarse, fine, c, converged)
            else:
                t_init = init_warm(net, coarse, fine, c, use_net=(mode == "warm"))
            row[mode] = steady(fine, max_steps)
            row[mode]["init_seconds"] = round(t_init, 4)
            if mode == "cold":
                converged = level_fields(fine)
                held = samples(coarse, fine, c, max_blocks=max_blocks, seed=1000)
                row["heldout_loss"] = {"net": mean_loss(net, held), "coarse_only": mean_loss(zero, held)}
                del held
            fine.close()
        coarse.close()
        tests.append(row)
        log("test case: %s" % row)
    return {"config": {"H": H, "B": B, "levels": 3, "train_cases": n_train, "test_cases": n_test,
                       "max_steps": max_steps, "epochs": epochs, "blocks_per_level_sampled": max_blocks,
                       "halo": HALO, "precision": precision, "net": "5 x conv3d 3x3x3, width 16, BF16"},
            "train_seconds": round(t_train, 2), "train_loss": [round(v, 6) for v in losses],
            "train_set_loss": fit,
            "voxels_trained": int(data[0].shape[0] * data[0].shape[1] * data[0].shape[2] * data[0].shape[3]),
            "generation": gen, "tests": tests}


def heldout_gain(n_train=4, H=32, B=8, max_steps=40000, epochs=10, max_blocks=256, seed=20150827,
                 precision="fp32s"):
    """The net's gain where it acts, on one held-out case: trains on n_train cases of
    inputs.warm_cases (targets: each case's refined solution from the coarse-only start), then
    compares on case n_train the loss of the net's prediction with that of the sampled coarse
    solution alone (the skip term), both against the converged refined solution."""
    from . import inputs
    cases = inputs.warm_cases(n_train + 1, seed=seed, H=H, B=B)
    net = lbm.Net(5, 6, 4, seed=seed)
    zero = zero_net(net)
    sets = []
    for i, c in enumerate(cases):
        coarse = lbm.Forest(coarse_case(c), precision=precision)
        coarse.init_uniform()
        steady(coarse, max_steps)
        fine = lbm.Forest(c, precision=precision)
        init_warm(net, coarse, fine, c, use_net=False)
        steady(fine, max_steps)
        sets.append(samples(coarse, fine, c, max_blocks=max_blocks, seed=i))
        coarse.close()
        fine.close()
    import torch
    data = tuple(torch.cat([d[k] for d in sets[:n_train]]) for k in range(4))
    losses = train(net, data, epochs)
    held = sets[n_train]
    return {"train_loss": losses, "train_set": {"net": mean_loss(net, data), "coarse_only": mean_loss(zero, data)},
            "heldout": {"net": mean_loss(net, held), "coarse_only": mean_loss(zero, held)}}


if __name__ == "__main__":
    import argparse
    import json
    p = argparse.ArgumentParser(description="Train the warm-start net and compare warm and cold starts")
    p.add_argument("--train", type=int, default=16)
    p.add_argument("--test", type=int, default=4)
    p.add_argument("--H", type=int, default=64)
    p.add_argument("--B", type=int, default=8)
    p.add_argument("--max-steps", type=int, default=6000)
    p.add_argument("--epochs", type=int, default=20)
    p.add_argument("--max-blocks", type=int, default=384)
    a = p.parse_args()
    from . import build
    build.build()
    out = experiment(a.train, a.test, a.H, a.B, a.max_steps, a.epochs, a.max_blocks)
    print(json.dumps(out), flush=True)
