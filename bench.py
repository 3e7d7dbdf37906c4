#!/usr/bin/env python
"""Refined-grid D3Q19 benchmark: GLUPS and % of the HBM roofline, FP16/FP32 vs FP64.

Workload: the refined channel past a sphere (4 levels, 2:1-balanced blocks of 32^3
cells, 8.39M cells, 28.0M cell updates per coarse step, periodic faces, started from
the plug flow 0.04, Re 100 on the sphere diameter, TRT with Lambda = 3/16).  One timed step is one coarse time
step: the whole recursive level schedule (15 fused level kernels), replayed as a CUDA
graph, with the inputs resident in HBM.  GLUPS = sum_L (owned fluid cells of level L)
x 2^L / time per coarse step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs an independent replica on its own GPU (the method has no
cross-replica exchange); rank 0 prints one JSON line.  `--impl reference` times the
plain CPU oracle on the host cores (rank 0 only), one full coarse step per timed step.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "refined-grid D3Q19 GLUPS & % HBM roofline, FP16/FP32 vs FP64; ms/coarse step"
UNIT = "GLUPS"
BYTES_PER_VALUE = {"fp64": 8, "fp32s": 4, "fp16s": 2}
DTYPE = {"fp64": "f64", "fp32s": "f32", "fp16s": "f32 compute / f16 storage"}
WORKLOAD = "sphere_channel_4lvl_32cube_8.39Mcells"


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1000)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--precision", default="fp32s", choices=["fp64", "fp32s", "fp16s"])
    p.add_argument("--no-variants", action="store_true", help="skip the FP64/FP16 side measurements")
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline leg")
    p.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg")
    p.add_argument("--no-batch", action="store_true", help="skip the batched small-forest leg")
    p.add_argument("--no-net", action="store_true", help="skip the warm-start net leg")
    p.add_argument("--no-lid", action="store_true", help="skip the paper's lid-driven benchmark leg")
    p.add_argument("--no-uniform", action="store_true", help="skip the uniform 512^3 stream-collide leg")
    return p.parse_args()


def _config(case, f=None):
    cfg = {"workload": WORKLOAD, "domain_cells_level0": [case["root"][a] * case["B"] for a in range(3)],
           "block_cells": case["B"], "levels": case["lmax"] + 1, "collision": "trt", "magic": 3.0 / 16.0,
           "lambda_e0": round(case["lambda_e0"], 6), "refine_radii": [r[3] for r in case["regions"]],
           "boundaries": "periodic", "start": "plug u=(0.04,0,0), rho=1",
           "l2": "inputs larger than L2 (PDF grids exceed the 129 MB L2 several times over)"}
    if f is not None:
        cfg["cell_updates_per_coarse_step"] = f.cell_updates_per_coarse_step()
        cfg["leaf_blocks_per_level"] = [len(f.block_table(L)) for L in range(f.nlev)]
    return cfg


def _measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region (read-only queries)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _kernel_hash(read=None):
    """Hash of the step-kernel sources with comments and blank lines removed (a comment edit does
    not change the kernel the counters were taken on)."""
    h = hashlib.sha256()
    for name in ("step_kernel.cuh", "kernels_impl.cuh", "kernels_f32.cu", "kernels_f64.cu", "kernels_f16.cu", "kernels.h"):
        if read is None:
            with open(os.path.join(ROOT, "paper_1508_07982_gb300", "csrc", name)) as fh:
                text = fh.read()
        else:
            text = read(name)
        for line in text.splitlines():
            code = line.split("//", 1)[0].rstrip()
            if code:
                h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def _ncu_traffic(precision):
    """DRAM bytes per launch of the dominant kernel from the committed ncu summary, if it was
    taken on the kernel source that is built now; otherwise None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            t = json.load(fh)
    except (OSError, ValueError):
        return None
    e = t.get(precision)
    if not e or e.get("kernel_hash") != _kernel_hash():
        return None
    return e.get("dram_bytes_per_launch")


def _max_over_ranks(ms, dist, device):
    """The slowest rank's time of the timed region (every rank gets it)."""
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _job_value(world, updates_per_step, steps, ms):
    """Whole-job GLUPS: every rank runs its own replica of the workload (weak scaling), so the job
    updates world x updates_per_step cells per coarse step in the slowest rank's time ms."""
    return world * updates_per_step * steps / (ms / 1e3) / 1e9


def _timed_graph(f, torch, steps):
    """K coarse steps of graph replay on the current stream, timed with CUDA events."""
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    f.step_coarse(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def _timed_kernels(f, torch, steps):
    """The same K coarse steps with a CUDA event between every pair of kernels (the launches are
    enqueued directly and in series in this mode); returns (total ms, per-level kernel times and
    counts of the column walk, the explosions and the side kernels)."""
    f.timing_begin(steps)
    ms = _timed_graph(f, torch, steps)
    return ms, f.timing_end(explode=True, side=True)


def _run_timed(lbm, torch, case, precision, steps, warmup):
    f = lbm.Forest(case, precision=precision)
    f.init_uniform(case["u_init"])
    f.step_coarse(warmup)
    torch.cuda.synchronize()
    ms = _timed_graph(f, torch, steps)
    f.init_uniform(case["u_init"])
    f.step_coarse(warmup)
    _, lev = _timed_kernels(f, torch, steps)
    return f, ms, lev


def _roofline(f, lev, precision, peaks, peak_kind):
    ms_l, cnt_l, ems_l, ecnt_l, sms_l, scnt_l = lev

    L = int(np.argmax(ms_l))
    counts = _fluid_counts(f)
    bytes_per_launch = counts[L] * 2 * 19 * BYTES_PER_VALUE[precision]
    avg_s = ms_l[L] / cnt_l[L] / 1e3
    achieved = bytes_per_launch / avg_s / 1e9
    peak = float(peaks["hbm_gbs"])
    traffic = _ncu_traffic(precision)
    total = ms_l.sum() + ems_l.sum() + sms_l.sum()
    share = ms_l / total
    per_level = [{"level": i, "launches": int(cnt_l[i]), "ms_total": round(float(ms_l[i]), 4),
                  "share": round(float(share[i]), 4), "explode_launches": int(ecnt_l[i]),
                  "explode_ms_total": round(float(ems_l[i]), 4), "side_launches": int(scnt_l[i]),
                  "side_ms_total": round(float(sms_l[i]), 4),
                  "GBps_algorithmic": round(counts[i] * 2 * 19 * BYTES_PER_VALUE[precision] / (ms_l[i] / cnt_l[i] / 1e3) / 1e9, 1)
                  if cnt_l[i] else None} for i in range(f.nlev)]
    return {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": traffic,
            "kernel": "step_kernel level %d fused stream-collide (column walk; its side kernel timed apart)" % L,
            "bytes_per_launch_algorithmic": int(bytes_per_launch),
            "peak_source": "%s hbm_gbs (MEASURED_PEAKS.json)" % peak_kind if peak_kind == "measured" else "fallback 6.8 TB/s",
            "per_level": per_level}


# FP64 arithmetic of the FP64 step kernel: FP64 thread instructions per cell update, an ncu count
# (sm__sass_thread_inst_executed_op_fp64_pred_on) of the level-3 launch of this workload divided by
# its fluid cells.  The peak is measured on the device by lbm_probe_fp64_fma (independent FMA chains
# on every SM), once per run.
FP64_INST_PER_UPDATE = 161
NOMINAL_HBM_GBS = 7900.0   # GB300 HBM3e, nominal (the measured copy bandwidth is the roofline)
_FP64_PEAK = {}


def _fp64_peak(lbm):
    if "g" not in _FP64_PEAK:
        _FP64_PEAK["g"] = lbm.lbm_probe_fp64_fma(20)
    return _FP64_PEAK["g"]


def _fp64_alu_roofline(r, peak_g):
    """The FP64 kernel against its arithmetic bound, from the same launch timing as r."""
    ach = r["achieved"] / (2 * 19 * 8) * FP64_INST_PER_UPDATE      # GB/s -> G updates/s -> G inst/s
    return {"bound": "alu", "achieved": round(ach, 1), "peak": round(peak_g, 1), "unit": "G FP64 inst/s",
            "frac": round(ach / peak_g, 4), "instructions_per_update": FP64_INST_PER_UPDATE,
            "peak_source": "measured: lbm_probe_fp64_fma (FP64 FMA chains on every SM, CUDA events)"}


_COUNTS = {}


def _fluid_counts(f):
    key = repr(sorted(f.case.items()))
    if key not in _COUNTS:
        from paper_1508_07982_gb300 import lbm
        p = lbm.Plan(f.case)
        _COUNTS[key] = [p.counts(L)["fluid"] for L in range(p.nlev)]
    return _COUNTS[key]


def _e2e(lbm, torch, case, precision, steps):
    """Same metric through the public API with host buffers: init from pinned host (rho, u) of every
    level, `steps` coarse steps each followed by the FP64 mass/momentum totals read back to the
    host, then the macroscopic fields of every level read back."""
    f = lbm.Forest(case, precision=precision)
    host_in = []
    for L in range(f.nlev):
        n = f.n_cells(L)
        rho = torch.ones(n, dtype=torch.float64).pin_memory()
        u = torch.zeros(3, n, dtype=torch.float64).pin_memory()
        u[0] = case["u_init"][0]
        host_in.append((rho, u))
    host_out = [(torch.empty(f.n_cells(L), dtype=torch.float64).pin_memory(),
                 torch.empty(3, f.n_cells(L), dtype=torch.float64).pin_memory()) for L in range(f.nlev)]
    h2d = sum(r.numel() * 8 + u.numel() * 8 for r, u in host_in)
    d2h_end = sum(r.numel() * 8 + u.numel() * 8 for r, u in host_out)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for L, (rho, u) in enumerate(host_in):
        f.init_equilibrium(L, rho, u, on_device=False)
    for _ in range(steps):
        f.step_coarse(1)
        f.reduce_mass_momentum()
    for L, (rho, u) in enumerate(host_out):
        f.get_macroscopic(L, rho, u, on_device=False)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    upd = f.cell_updates_per_coarse_step() * steps
    f.close()
    return {"value": round(upd / dt / 1e9, 4), "unit": UNIT, "h2d_bytes_per_step": int(h2d // steps),
            "d2h_bytes_per_step": int((d2h_end + 32 * steps) // steps),
            "note": "lbm_init_equilibrium from pinned host (rho,u) of all levels, %d x (lbm_step_coarse(1) + "
                    "lbm_reduce_mass_momentum to host), lbm_get_macroscopic of all levels to pinned host" % steps}


def _precision_error(fa, fb):
    """Velocity and density error of forest fa against forest fb (FP64) over owned fluid cells."""
    du, dr, umax = 0.0, 0.0, 0.0
    for L in range(fa.nlev):
        ra, ua = fa.get_macroscopic(L)
        rb, ub = fb.get_macroscopic(L)
        ok = np.isfinite(rb)
        du = max(du, float(np.abs(ua[:, ok] - ub[:, ok]).max()))
        dr = max(dr, float(np.abs(ra[ok] - rb[ok]).max()))
        umax = max(umax, float(np.abs(ub[:, ok]).max()))
    return {"u_linf_rel_to_umax": du / umax, "rho_linf": dr}


def _cpu_baseline(case, steps=2):
    from oracle import oracle
    oracle.build()
    t0 = time.perf_counter()
    o = oracle.Oracle(case)
    o.init_fields(_uniform(case))
    setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    upd = o.cell_updates_per_coarse_step() * steps
    return {"value": round(upd / dt / 1e9, 6), "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": "%d full coarse steps of the same 8.39M-cell forest in FP64 (%.1f s; setup %.1f s excluded)"
                      % (steps, dt, setup)}


def _uniform(case):
    from paper_1508_07982_gb300 import inputs
    return inputs.uniform_field(u=case["u_init"])


def _batch(lbm, torch, steps=500, warmup=5, serial_steps=50):
    """The batched workload: 256 small lid-driven cavities (2-3 levels, 16^3 blocks, 8-64 leaves
    each) stepped together, one launch per phase, after autotuning the batch's thread mapping;
    beside it the same members stepped one forest after another."""
    from paper_1508_07982_gb300 import inputs
    cases = inputs.batch_cases()
    fs = []
    for c in cases:
        f = lbm.Forest(c, precision="fp32s")
        f.init_uniform()
        fs.append(f)
    b = lbm.Batch(fs)
    lzc, minb, _ = b.autotune(4)
    b.step(warmup)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    upd = b.cell_updates_per_coarse_step()
    launches = b.launches_per_coarse_step()
    for f in fs:
        f.step_coarse(1)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(serial_steps):
        for f in fs:
            f.step_coarse(1)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_serial = e0.elapsed_time(e1)
    cells = sum(c["leaves"] for c in cases) * 16 ** 3
    out = {"workload": "256 lid-driven cavities, 2-3 levels, 16^3 blocks, 8-64 leaves each (%d leaves, %.1fM cells)"
                       % (sum(c["leaves"] for c in cases), cells / 1e6),
           "value": round(upd * steps / (ms / 1e3) / 1e9, 4), "unit": UNIT, "precision": "fp32s",
           "steps": steps, "warmup": warmup, "ms_per_step": round(ms / steps, 5),
           "cell_updates_per_coarse_step": int(upd), "gpu_launches_per_coarse_step": int(launches),
           "kernel_config": {"cells_per_thread_log2": lzc, "ctas_per_sm": minb},
           "one_forest_at_a_time": {"value": round(upd * serial_steps / (ms_serial / 1e3) / 1e9, 4), "unit": UNIT,
                                    "ms_per_step": round(ms_serial / serial_steps, 5), "steps": serial_steps}}
    b.close()
    for f in fs:
        f.close()
    out["fp32s_error_vs_fp64"] = _batch_error(lbm, torch, cases[::16], steps)
    return out


def _batch_error(lbm, torch, cases, steps):
    """FP32S error of batched cases against FP64, per case: the same cases stepped `steps` coarse
    steps from rest as an FP32S batch and as an FP64 batch (whose members match the oracle to 1e-12
    in the batch tests), compared on every level's owned fluid cells: velocity L-inf over the lid
    speed, density L-inf."""
    fa = [lbm.Forest(c, precision="fp32s") for c in cases]
    fb = [lbm.Forest(c, precision="fp64") for c in cases]
    for f in fa + fb:
        f.init_uniform()
    ba, bb = lbm.Batch(fa), lbm.Batch(fb)
    ba.step(steps)
    bb.step(steps)
    torch.cuda.synchronize()
    du, dr = [], []
    for c, x, y in zip(cases, fa, fb):
        ra, ua = x.get_macroscopic(-1)
        rb, ub = y.get_macroscopic(-1)
        ok = np.isfinite(rb)
        du.append(float(np.abs(ua[:, ok] - ub[:, ok]).max()) / float(c["bc_u"][5][0]))
        dr.append(float(np.abs(ra[ok] - rb[ok]).max()))
    ba.close()
    bb.close()
    for f in fa + fb:
        f.close()
    return {"cases": len(cases), "steps": steps, "u_linf_rel_to_lid_max": max(du), "u_linf_rel_to_lid_median": float(np.median(du)),
            "rho_linf_max": max(dr), "sample": "every 16th case of the 256, stepped from rest"}


# The paper's strong-scaling figure for its lid-driven benchmark (Sec. 5.2, SuperMUC table): 8.56M
# cells, 32,768 cores, MPI + 4 OpenMP threads per process, FP64.  Context only: other machine,
# other size.
PAPER_LID_FINEST_STEPS_PER_S = 1113.97
PAPER_LID_CELLS = 8.56e6


def _lid(lbm, torch, peaks, peak_kind, steps=100, steps64=20):
    """The paper's own benchmark cavity (Sec. 5.2): lid edges across the lid motion refined three
    times, 3^3 roots of 32^3 cells (10.5M cells, 21 / 36 / 72 / 192 blocks on levels 0-3).  Per
    precision: ms per coarse step, GLUPS, finest-level steps per second, the finest kernel's
    roofline and each level's share of kernel time beside the table's workload shares."""
    from paper_1508_07982_gb300 import inputs
    case = inputs.lid_scaling_case()
    out = {"workload": "lid-driven benchmark cavity of Sec. 5.2, 3^3 roots of 32^3 cells, lid edges across the "
                       "lid motion refined 3x (4 levels, 21/36/72/192 blocks, %.2fM cells), rest start, TRT"
                       % (sum(_fluid_counts_case(case)) / 1e6),
           "paper_context": {"finest_steps_per_s": PAPER_LID_FINEST_STEPS_PER_S, "cells": PAPER_LID_CELLS,
                             "machine": "SuperMUC, 32,768 cores, FP64 (strong scaling, Sec. 5.2)"},
           "table_workload_share": [0.0110, 0.0376, 0.1502, 0.8013]}
    for prec, k in (("fp32s", steps), ("fp16s", steps), ("fp64", steps64)):
        f = lbm.Forest(case, precision=prec)
        f.init_uniform()
        f.step_coarse(3)
        torch.cuda.synchronize()
        ms = _timed_graph(f, torch, k)
        _, lev = _timed_kernels(f, torch, k)
        upd = f.cell_updates_per_coarse_step()
        r = _roofline(f, lev, prec, peaks, peak_kind)
        out[prec] = {"value": round(upd * k / (ms / 1e3) / 1e9, 4), "unit": UNIT, "ms_per_step": round(ms / k, 5),
                     "steps": k, "finest_steps_per_s": round(8 * k / (ms / 1e3), 1),
                     "roofline": {kk: r[kk] for kk in ("bound", "achieved", "peak", "unit", "frac", "kernel")},
                     "kernel_time_share": [lv["share"] for lv in r["per_level"]]}
        f.close()
    return out


def _taylor_green_on_device(f, torch, N, umax=0.02, sigma=1e-4, seed=None):
    """The periodic workload's start on the device: the seeded Taylor-Green modes of
    inputs.taylor_green_modes evaluated at every cell centre and scaled to max |u| = umax, and
    rho = 1 + N(0, sigma^2) from a seeded torch generator (the parity tests use the counter-based
    host generator at 64^3; at 512^3 the host would need minutes)."""
    from paper_1508_07982_gb300 import inputs
    seed = inputs.SEED if seed is None else seed
    modes = inputs.taylor_green_modes(seed)
    bt = torch.as_tensor(f.block_table(0), device="cuda", dtype=torch.float64)
    B = f.B
    r = torch.arange(B, device="cuda", dtype=torch.float64) + 0.5
    lz, ly, lx = torch.meshgrid(r, r, r, indexing="ij")
    X = (bt[:, 0:1] * B + lx.reshape(1, -1)).reshape(-1) * (2.0 * np.pi / N)
    Y = (bt[:, 1:2] * B + ly.reshape(1, -1)).reshape(-1) * (2.0 * np.pi / N)
    Z = (bt[:, 2:3] * B + lz.reshape(1, -1)).reshape(-1) * (2.0 * np.pi / N)
    u = torch.zeros((3, X.numel()), dtype=torch.float64, device="cuda")
    for k, a in modes:
        sx, cx = torch.sin(k[0] * X), torch.cos(k[0] * X)
        sy, cy = torch.sin(k[1] * Y), torch.cos(k[1] * Y)
        sz, cz = torch.sin(k[2] * Z), torch.cos(k[2] * Z)
        u[0] += a[0] * cx * sy * sz
        u[1] += a[1] * sx * cy * sz
        u[2] += a[2] * sx * sy * cz
    del X, Y, Z
    u *= umax / float(torch.sqrt((u * u).sum(0)).max())
    g = torch.Generator(device="cuda").manual_seed(seed)
    rho = 1.0 + sigma * torch.randn(u.shape[1], dtype=torch.float64, device="cuda", generator=g)
    f.init_equilibrium(0, rho, u, on_device=True)
    torch.cuda.synchronize()


def _uniform_grid_leg(lbm, torch, peaks, peak_kind, n=512, steps=200):
    """The pure stream-collide case of the periodic workload: a uniform periodic n^3 grid (one level,
    32^3 blocks), SRT omega = 1.9, from the seeded Taylor-Green start with density noise, `steps`
    steps per precision (FP32S, FP16S and FP64).  No interfaces and no walls: the column walk
    alone."""
    from paper_1508_07982_gb300 import inputs
    case = inputs.periodic_case(n=n, B=32, collision="srt", omega=1.9)
    out = {"workload": "uniform periodic %d^3 (one level, 32^3 blocks), SRT omega 1.9, Taylor-Green modes "
                       "k <= 4 scaled to max |u| 0.02 plus N(0, 1e-4) density noise, %d steps" % (n, steps)}
    for prec in ("fp32s", "fp16s", "fp64"):
        f = lbm.Forest(case, precision=prec)
        _taylor_green_on_device(f, torch, n)
        torch.cuda.synchronize()
        ms = _timed_graph(f, torch, steps)
        _taylor_green_on_device(f, torch, n)
        _, lev = _timed_kernels(f, torch, steps)
        upd = f.cell_updates_per_coarse_step()
        r = _roofline(f, lev, prec, peaks, peak_kind)
        entry = {"value": round(upd * steps / (ms / 1e3) / 1e9, 4), "unit": UNIT, "ms_per_step": round(ms / steps, 5),
                 "steps": steps,
                 "roofline": dict({kk: r[kk] for kk in ("bound", "achieved", "peak", "unit", "frac")}, traffic=None,
                                  kernel="step_kernel level 0 (the only level)")}
        if prec == "fp64":
            entry["roofline_alu"] = _fp64_alu_roofline(r, _fp64_peak(lbm))
        out[prec] = entry
        f.close()
    # the FP32S figures at the top level, as before
    out.update({k: out["fp32s"][k] for k in ("value", "unit", "ms_per_step", "steps", "roofline")})
    return out


def _fluid_counts_case(case):
    from paper_1508_07982_gb300 import lbm
    p = lbm.Plan(case)
    return [p.counts(L)["fluid"] for L in range(p.nlev)]


def _net(lbm, torch, peaks, peak_kind, reps=10):
    """The warm-start net on 512 volumes of 18^3 voxels (8^3 blocks with a halo of 5): forward
    passes and training steps, each on the tcgen05 and the mma.sync tensor-core paths.  FLOPs count
    the 27 x 16 x 16 multiply-adds per voxel and layer that the kernels issue."""
    shape = (512, 18, 18, 18)
    n = int(np.prod(shape))
    x = torch.zeros(shape + (16,), dtype=torch.bfloat16, device="cuda")
    g = torch.Generator(device="cuda").manual_seed(20150827)
    x[..., :6] = torch.randn(shape + (6,), device="cuda", generator=g).to(torch.bfloat16)
    target = torch.randn(shape + (4,), device="cuda", generator=g) * 0.1
    out = {"workload": "512 volumes of 18^3 voxels x 16 channels, 5 layers of 3^3 convolutions, width 16"}
    stream = torch.cuda.current_stream()
    for backend in ("tcgen05", "mma.sync"):
        net = lbm.Net(5, 6, 4, seed=1)
        net.set_backend(backend)
        res = {}
        for kind, fn, flop_layers in (("forward", lambda: net.forward(x), 5),
                                      ("train_step", lambda: net.train_step(x, target, lr=1e-4), 5 + 4 + 5)):
            for _ in range(3):
                fn()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            flops = flop_layers * 2 * 27 * 16 * 16 * n
            res[kind] = {"ms": round(ms, 4), "TFLOPs": round(flops / ms / 1e9, 1)}
        net.close()
        out[backend] = res
    peak = float(peaks["bf16_tflops"])
    ach = out["tcgen05"]["forward"]["TFLOPs"]
    out["roofline"] = {"bound": "tensor", "kernel": "conv_tc_kernel (net forward, 5 layers)", "achieved": ach,
                       "peak": peak, "unit": "TFLOP/s", "frac": round(ach / peak, 4),
                       "peak_source": "%s bf16_tflops (MEASURED_PEAKS.json)" % peak_kind}
    return out


REFERENCE_BUDGET_S = 90.0   # timed seconds of the reference arm at most


def run_reference(args, case):
    """The plain CPU oracle as the reference arm.  A timed step is one full coarse step of the
    workload; the run times the requested steps, or as many as fit in about REFERENCE_BUDGET_S
    seconds (estimated from one untimed warm-up step), so that it ends within a few minutes."""
    from oracle import oracle
    oracle.build()
    o = oracle.Oracle(case)
    o.init_fields(_uniform(case))
    t0 = time.perf_counter()
    o.step(1)
    t_one = time.perf_counter() - t0
    n = max(1, min(args.steps, int(REFERENCE_BUDGET_S / max(t_one, 1e-3))))
    t0 = time.perf_counter()
    o.step(n)
    dt = time.perf_counter() - t0
    upd = o.cell_updates_per_coarse_step() * n
    v = upd / dt / 1e9
    sample = "%d full coarse steps of the workload in FP64 on the host cores (%d requested; bounded to about %.0f s)" % (
        n, args.steps, REFERENCE_BUDGET_S)
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 6), "unit": UNIT, "n_gpus": args.gpus,
            "steps": n, "requested_steps": args.steps, "warmup": 1, "ms_per_step": round(dt * 1e3 / n, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _config(case),
            "cpu_baseline": {"value": round(v, 6), "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(v, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = _args()
    from paper_1508_07982_gb300 import inputs
    case = inputs.sphere_channel_case()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            run_reference(args, case)
        return
    import torch
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    from paper_1508_07982_gb300 import build, lbm
    if rank == 0 or world == 1:
        build.build()
    if dist:
        dist.barrier()
    build.build()
    peaks, peak_kind = _measured_peaks()

    # ---- timed region: K coarse steps of the resident workload, CUDA-graph replay
    f = lbm.Forest(case, precision=args.precision)
    f.init_uniform(case["u_init"])
    f.step_coarse(max(args.warmup, 3))
    torch.cuda.synchronize()
    launches = f.launches_per_coarse_step()
    sampler = ClockSampler(local_rank)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    ms = _timed_graph(f, torch, args.steps)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    # per-kernel durations: a second timed pass of the same K steps, from the same start, with
    # events between kernels
    f.init_uniform(case["u_init"])
    f.step_coarse(max(args.warmup, 3))
    ms_k, lev = _timed_kernels(f, torch, args.steps)
    if dist:
        ms = _max_over_ranks(ms, dist, "cuda")
    upd = f.cell_updates_per_coarse_step()
    value = _job_value(world, upd, args.steps, ms)
    roof = _roofline(f, lev, args.precision, peaks, peak_kind)
    roof["kernel_timing_pass_ms_per_step"] = round(ms_k / args.steps, 5)
    # the whole coarse step (graph replay: every level, explosions, side work) at the algorithmic
    # bytes of its cell updates, against the measured and the nominal bandwidth
    step_gbs = upd * 2 * 19 * BYTES_PER_VALUE[args.precision] / (ms / args.steps / 1e3) / 1e9
    roof["whole_step"] = {"achieved": round(step_gbs, 1), "unit": "GB/s", "frac": round(step_gbs / roof["peak"], 4),
                          "frac_of_nominal_7900": round(step_gbs / NOMINAL_HBM_GBS, 4)}
    roof["frac_of_nominal_7900"] = round(roof["achieved"] / NOMINAL_HBM_GBS, 4)
    cfg = _config(case, f)
    mass = f.reduce_mass_momentum()

    variants = {}
    if not args.no_variants and rank == 0:
        ref64 = None
        for prec in ("fp64", "fp32s", "fp16s"):
            k = max(args.steps // 4, 20)
            g, ms_v, lev_v = _run_timed(lbm, torch, case, prec, k, 3)
            entry = {"value": round(upd * k / (ms_v / 1e3) / 1e9, 3), "unit": UNIT,
                     "ms_per_step": round(ms_v / k, 4), "steps": k}
            r = _roofline(g, lev_v, prec, peaks, peak_kind)
            entry["roofline"] = {kk: r[kk] for kk in ("bound", "achieved", "peak", "unit", "frac", "traffic")}
            if prec == "fp64":
                entry["roofline_alu"] = _fp64_alu_roofline(r, _fp64_peak(lbm))
                ref64 = g
            else:
                entry["error_vs_fp64_after_%d_steps" % (k + 3)] = _precision_error(g, ref64)
                g.close()
            variants[prec] = entry
        if ref64 is not None:
            ref64.close()

    e2e = _e2e(lbm, torch, case, args.precision, min(args.steps, 200)) if rank == 0 and not args.no_e2e else None
    batch = _batch(lbm, torch) if rank == 0 and not args.no_batch else None
    net = _net(lbm, torch, peaks, peak_kind) if rank == 0 and not args.no_net else None
    lid = _lid(lbm, torch, peaks, peak_kind) if rank == 0 and not args.no_lid else None
    uni = _uniform_grid_leg(lbm, torch, peaks, peak_kind) if rank == 0 and not args.no_uniform else None
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = _cpu_baseline(case)
    line = {"metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": round(ms / args.steps, 5), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[args.precision], "data": "synthetic",
            "config": dict(cfg, precision=args.precision, parallelism="replicas" if world > 1 else "single"),
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
            "gpu_launches": int(launches * args.steps), "mass_total": mass[0]}
    if variants:
        line["precisions"] = variants
    if batch:
        line["batch"] = batch
    if net:
        line["warm_start_net"] = net
    if lid:
        line["paper_lid_benchmark"] = lid
    if uni:
        line["uniform_512"] = uni
    if rank == 0:
        print(json.dumps(line), flush=True)
    f.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
