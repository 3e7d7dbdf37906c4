"""CPU-only checks of the C-ABI library: it loads without a GPU, exports every entry point
declared in include/lbm_gb300.h, and its host-side forest planner agrees exactly with the
oracle's independent forest (leaf sets and cell counts are integer results: bit-exact)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1508_07982_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lbm():
    from paper_1508_07982_gb300 import build, lbm as mod
    build.build()
    return mod


def _declared():
    txt = open(os.path.join(ROOT, "include", "lbm_gb300.h")).read()
    return sorted(set(re.findall(r"^\s*(?:lbm_status|const char\*)\s+(lbm_\w+)\s*\(", txt, re.M)))


def test_library_exports_every_declared_symbol(lbm):
    lib = lbm.library()
    declared = _declared()
    assert len(declared) >= 20
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(lbm.EXPORTS) == declared


def test_lattice_order_matches_the_oracle(lbm, oracle_mod):
    e, w, opp = lbm.lbm_lattice()
    e2, w2, opp2 = oracle_mod.lattice()
    assert (e == e2).all() and (opp == opp2).all()
    assert np.abs(w - w2).max() == 0.0


def test_invalid_descriptions_are_rejected_on_the_host(lbm):
    bad = [
        dict(inputs.cavity_case(), B=12),
        dict(inputs.cavity_case(), lmax=9),
        dict(inputs.cavity_case(), bc=["periodic", "noslip", "noslip", "noslip", "noslip", "noslip"]),
        dict(inputs.cavity_case(), rho0=0.0),
        dict(inputs.cavity_case(), u_shift=(0.25, 0.2, 0.0)),       # |u_shift| >= 0.3
        dict(inputs.cavity_case(), u_shift=(float("nan"), 0.0, 0.0)),
    ]
    for case in bad:
        with pytest.raises(lbm.LBMError) as ei:
            lbm.Plan(case)
        assert ei.value.status == lbm.LBM_EINVAL


def _cases():
    yield "cavity", inputs.cavity_case(), None
    yield "channel", inputs.sphere_channel_case(H=32, B=8, radii=(20.0, 12.0, 6.5), inlet_outlet=True), None
    yield "poiseuille", inputs.plane_poiseuille_case(B=8, where="both"), None
    yield "lid-scaling", inputs.lid_scaling_case(roots=(3, 1, 3), B=8), None
    yield "free-slip", inputs.freeslip_box_case(lid=0.02, spheres=[(8.0, 1.0, 16.0, 4.0), (16.0, 16.0, 16.0, 2.5)]), None
    yield "periodic-ball", inputs.periodic_case(n=64, B=8, collision="trt", omega=1.7,
                                                regions=[("ball", 3, (5, 60, 33), 9.0)], lmax=3), None
    rng = np.random.default_rng(7)
    marks = {}

    def refine(L, x, y, z, user):
        k = (L, x, y, z)
        if k not in marks:
            marks[k] = rng.random() < (0.3 if L == 0 else 0.12)
        return int(marks[k])

    yield "random", dict(root=(3, 2, 2), B=8, lmax=3, collision="trt", rho0=1.0,
                         bc=["periodic", "periodic", "noslip", "noslip", "velocity", "velocity"],
                         bc_u=[(0, 0, 0)] * 4 + [(0.01, 0, 0)] * 2, spheres=[(9.0, 7.0, 5.0, 3.3)],
                         regions=[]), refine


def _rows(a):
    """Rows of a block list in lexicographic (z, y, x) order, to compare sets of blocks."""
    return a[np.lexsort((a[:, 0], a[:, 1], a[:, 2]))] if len(a) else a


def _forest_key(L, b, roots):
    """Root block in x-fastest order, then the Morton key within the root's octree."""
    root = ((int(b[2]) >> L) * roots[1] + (int(b[1]) >> L)) * roots[0] + (int(b[0]) >> L)
    k = 0
    for bit in range(L):
        for ax in range(3):
            k |= ((int(b[ax]) >> bit) & 1) << (3 * bit + ax)
    return (root << (3 * L)) | k


def test_block_lists_follow_the_forest_traversal(lbm):
    """Each level's leaf blocks (the block-major order of every per-level array) follow the
    traversal of the forest of octrees: roots in x-fastest order, the Morton curve within each
    root, so that the keys increase."""
    case = inputs.periodic_case(n=64, B=8, regions=[("box", 1, (8, 16, 0), (40, 48, 64)), ("box", 2, (16, 24, 8), (32, 40, 40))],
                                lmax=2)
    p = lbm.Plan(case)
    roots = case["root"]
    for L in range(p.nlev):
        keys = [_forest_key(L, b, roots) for b in p.leaves(L)]
        assert len(keys) > 8 and all(k1 < k2 for k1, k2 in zip(keys, keys[1:])), L
    # level 0 is the root grid, x fastest
    lv0 = p.leaves(0)
    assert [tuple(b) for b in lv0] == sorted((tuple(b) for b in lv0), key=lambda t: (t[2], t[1], t[0]))


@pytest.mark.parametrize("name", ["cavity", "channel", "poiseuille", "lid-scaling", "free-slip", "periodic-ball", "random"])
def test_host_planner_matches_the_oracle_forest(lbm, oracle_mod, name):
    case, refine = next((c, r) for n, c, r in _cases() if n == name)
    memo = {}

    def cached(L, x, y, z, user):        # both sides must see the same callback answers
        k = (L, x, y, z)
        if k not in memo:
            memo[k] = refine(L, x, y, z, user)
        return memo[k]

    cb = cached if refine else None
    p = lbm.Plan(case, refine=cb)
    o = oracle_mod.Oracle(case, refine=cb)
    assert p.nlev == o.nlev
    for L in range(p.nlev):
        a = p.leaves(L)
        b = o.leaves(L)
        assert a.shape == b.shape and (_rows(a) == _rows(b)).all(), "leaf set differs on level %d" % L
        c = p.counts(L)
        oc = o.counts(L)
        assert c["fluid"] == oc["fluid"]
        # the planner's ghost work list is the oracle's stream set minus its owned fluid cells
        assert c["ghost12"] == oc["stream"] - oc["fluid"]


def _golden_lid_table():
    rows = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "lid_driven_setup.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                k, *v = line.split()
                rows[k] = [float(x) for x in v]
    return rows


@pytest.mark.parametrize("roots,B", [((3, 3, 3), 32), ((3, 1, 3), 8), ((3, 4, 3), 16)])
def test_lid_scaling_forest_reproduces_the_benchmark_level_table(lbm, roots, B):
    """The benchmark's level table (Sec. 5.2) from the planner's leaf counts: coverage = blocks
    x 8^-L, workload = blocks x 2^L (cells per block are equal on every level, and level L takes
    2^L steps per coarse step), memory = blocks, each as a share of its sum, within one unit of
    the table's last digit (its memory row, 12/107 = 11.215 % printed as 11.22, sums to 100.00);
    7 / 12 / 24 / 64 leaf blocks per 3 x 1 x 3 roots."""
    p = lbm.Plan(inputs.lid_scaling_case(roots=roots, B=B))
    assert p.nlev == 4
    n = np.array([p.counts(L)["blocks"] for L in range(4)], dtype=float)
    k = roots[1]
    assert (n == np.array([7, 12, 24, 64]) * k).all()
    cov = n * 8.0 ** -np.arange(4)
    work = n * 2.0 ** np.arange(4)
    got = {"coverage": 100 * cov / cov.sum(), "workload": 100 * work / work.sum(), "memory": 100 * n / n.sum()}
    for key, ref in _golden_lid_table().items():
        assert np.abs(got[key] - np.array(ref)).max() <= 0.01 + 1e-9, (key, got[key], ref)
    # every leaf holds B^3 fluid cells (no obstacles)
    assert sum(p.counts(L)["fluid"] for L in range(4)) == int(n.sum()) * B ** 3


@pytest.mark.parametrize("B,levels", [(8, 1), (8, 2), (16, 1)])
def test_level_interfaces_meeting_free_slip_faces_are_planned(lbm, B, levels):
    """Sec. 4.1 lets level transitions meet free-slip boundaries by extending the boundary
    treatment to the ghost layers.  The planner resolves every needed free-slip mirror of an owned
    or ghost cell within ghost layer 3 (it fails with LBM_EINVAL otherwise), so a refined corner
    that reaches the y- and z- faces (and, with two levels, a second corner inside it) plans, with
    ghost work on every refined level.  The GPU parity tests check the values."""
    regions = [("box", 1, (0, 0, 0), (32, 16, 16)), ("box", 2, (0, 0, 0), (32, 8, 8))][:levels]
    case = dict(inputs.freeslip_box_case(n=32 if B == 8 else 64, B=B), regions=regions, lmax=levels)
    p = lbm.Plan(case)
    assert p.nlev == levels + 1
    for L in range(1, p.nlev):
        w = p.ghost_work(L)
        assert w["values1"] > 0 and w["values2"] > 0, (L, w)
