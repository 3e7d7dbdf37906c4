"""Host-side helpers of bench.py (no GPU): the oracle's start field, the FP64 arithmetic roofline,
and the kernel-source hash the committed ncu traffic record is keyed on."""
import json
import os

import numpy as np

import bench
from paper_1508_07982_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_start_field_of_the_oracle_legs_is_the_case_plug():
    case = inputs.sphere_channel_case()
    field = bench._uniform(case)
    rho, u = field(0, np.zeros(3), np.zeros(3), np.zeros(3))
    assert np.allclose(rho, 1.0) and np.allclose(u[0], case["u_init"][0]) and np.allclose(u[1:], 0.0)


def test_fp64_arithmetic_roofline_converts_bandwidth_to_instructions():
    r = bench._fp64_alu_roofline({"achieved": 304.0}, 500.0)   # 1 G updates/s at 304 B per update
    assert abs(r["achieved"] - bench.FP64_INST_PER_UPDATE) < 0.05
    assert r["bound"] == "alu" and r["peak"] == 500.0
    assert abs(r["frac"] - bench.FP64_INST_PER_UPDATE / 500.0) < 1e-3


def test_kernel_hash_ignores_comments():
    base = {n: "int a;\n// note\nint b; // tail\n" for n in ("step_kernel.cuh", "kernels_impl.cuh", "kernels_f32.cu",
                                                            "kernels_f64.cu", "kernels_f16.cu", "kernels.h")}
    other = {n: "int a;\n\n// another note\nint b;\n" for n in base}
    assert bench._kernel_hash(base.__getitem__) == bench._kernel_hash(other.__getitem__)
    changed = dict(base, **{"kernels.h": "int a;\nint c;\n"})
    assert bench._kernel_hash(changed.__getitem__) != bench._kernel_hash(base.__getitem__)
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
        assert json.load(fh)["fp32s"]["dram_bytes_per_launch"] > 0
