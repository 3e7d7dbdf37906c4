"""Seeded synthetic workloads for the refined-grid D3Q19 lattice Boltzmann method.

This module describes inputs only: domains, refinement regions, obstacles,
boundary conditions, relaxation parameters and initial (rho, u) fields.  It
holds none of the method's arithmetic.  Both the CUDA library (through its
binding) and the plain CPU oracle consume the same case dicts, each marshalling
them into its own C struct.

Case dict keys:
  root      (nx, ny, nz) root blocks (the octree roots, Sec. 3.2)
  B         cells per block edge on every level (Sec. 4: equal cell count per block)
  lmax      deepest level the refinement may create
  collision "srt" | "trt" (Sec. 2)
  rho0      reference density of the incompressible equilibrium (Eq. fequ)
  bc        six faces x-, x+, y-, y+, z-, z+: "periodic" | "noslip" | "velocity"
  bc_u      wall velocity per face (used by "velocity" faces)
  spheres   obstacles (cx, cy, cz, r) in level-0 cell units; a cell whose centre
            lies inside is a no-slip obstacle
  regions   refinement regions ("box", level, lo3, hi3) | ("ball", level, c3, r):
            a block below `level` that overlaps the region is split (Sec. 3.3)
  lambda_e0, magic, accel   coarse relaxation rate, TRT magic parameter, body
            acceleration on level 0 (Sec. 2.3 scales them per level)
  u_shift   optional: FP32S/FP16S storage holds f - f^eq(rho0, u_shift) (default 0)
All coordinates are in level-0 cell units; cell (i, j, k) of level L has its
centre at ((i + .5) / 2^L, ...).
"""
import math

import numpy as np

SEED = 20150827


# --------------------------------------------------------------------------- cases

def cavity_case(lid=0.05, lambda_e0=1.6, B=8):
    """Lid-driven cavity, 32^3 coarse cells, centre [8,24)^3 refined once.

    With B = 8 the roots are 4^3 blocks of 8^3 cells and the 2^3 central roots are
    split, giving 28,672 coarse + 32,768 fine cells.  Lid z = top moves with
    (lid, 0, 0); all other walls are no-slip (Sec. 5.2 benchmark boundaries).
    """
    n = 32 // B
    return dict(root=(n, n, n), B=B, lmax=1, collision="trt", rho0=1.0,
                bc=["noslip"] * 5 + ["velocity"],
                bc_u=[(0.0, 0.0, 0.0)] * 5 + [(lid, 0.0, 0.0)],
                spheres=[], regions=[("box", 1, (8, 8, 8), (24, 24, 24))],
                lambda_e0=lambda_e0, magic=3.0 / 16.0, accel=(0.0, 0.0, 0.0))


def lid_scaling_case(roots=(3, 3, 3), B=32, lid=0.05, lambda_e0=1.6, eps=1.0 / 32.0):
    """The lid-driven cavity of the performance benchmark (Sec. 5.2): lid z+ moving with
    (lid, 0, 0), no-slip elsewhere, and the regions where the lid meets the walls refined three
    times.

    Reading: the refined regions are the two lid edges perpendicular to the lid motion (x- and
    x+ at z+), where the moving lid runs into a wall; each is a box of thickness eps (level-0
    cell units, below one level-3 block) along the edge, so at every level exactly the blocks
    touching the edge are split.  On 3 x k x 3 roots this gives, per 3 x 1 x 3 roots, 7 / 12 /
    24 / 64 leaf blocks on levels 0-3, which reproduces the benchmark's table of coverage,
    workload and memory shares (77.78 / 16.67 / 4.17 / 1.39 %, 1.10 / 3.76 / 15.02 / 80.13 %,
    6.54 / 11.22 / 22.43 / 59.81 %).  Refining all four lid edges does not.  TRT with the magic
    parameter 3/16; lid speed and lambda_e0 are not given for the benchmark (those of the
    2-level cavity are used).
    """
    nx, ny, nz = (r * B for r in roots)
    return dict(root=tuple(roots), B=B, lmax=3, collision="trt", rho0=1.0,
                bc=["noslip"] * 5 + ["velocity"],
                bc_u=[(0.0, 0.0, 0.0)] * 5 + [(lid, 0.0, 0.0)],
                spheres=[],
                regions=[("box", 3, (0.0, 0.0, nz - eps), (eps, ny, nz)),
                         ("box", 3, (nx - eps, 0.0, nz - eps), (nx, ny, nz))],
                lambda_e0=lambda_e0, magic=3.0 / 16.0, accel=(0.0, 0.0, 0.0))


def _square_meets_circle(y0, y1, z0, z1, R):
    """The square [y0, y1] x [z0, z1] (coordinates from the circle's centre) meets the circle of
    radius R: its nearest point lies inside and its farthest outside (or on it)."""
    ny = 0.0 if y0 <= 0.0 <= y1 else min(abs(y0), abs(y1))
    nz = 0.0 if z0 <= 0.0 <= z1 else min(abs(z0), abs(z1))
    fy, fz = max(abs(y0), abs(y1)), max(abs(z0), abs(z1))
    return ny * ny + nz * nz <= R * R <= fy * fy + fz * fz


def pipe_poiseuille_case(D=60, B=8, lmax=0, where="wall", lambda_e0=0.6, accel=1e-6, paper_block=10):
    """Pipe Poiseuille flow (Sec. 5.1): a pipe of diameter D level-0 cells along x, periodic in x
    over one root block, driven by a body force; cells whose centre lies outside the pipe are
    no-slip obstacles (staircase).  TRT with the magic parameter 3/16.

    The cross-section is the smallest multiple of B that holds the pipe, with the pipe axis at
    its centre.  Refinement to lmax:
      "global"      every block;
      "wall"        the blocks the pipe wall passes through (this forest's own blocks);
      "wall-cover"  every block that overlaps (with positive area) a block the wall passes
                    through in the paper's forest, whose blocks have paper_block level-0 cells
                    per edge on a grid spanning the pipe (D = 60: 6 x 6 roots of 10^3 cells).
    With B = 8 the first refines a thinner band around the wall than the paper's 10^3 blocks do,
    the second a band that covers the paper's.  Returns (case, refine, flag, (centre, radius));
    refine and flag are the callbacks of lbm_create_forest."""
    n = -(-D // B)
    c = n * B / 2.0
    R = D / 2.0
    case = dict(root=(1, n, n), B=B, lmax=lmax, collision="trt", rho0=1.0,
                bc=["periodic"] * 2 + ["noslip"] * 4, bc_u=[(0.0, 0.0, 0.0)] * 6, spheres=[], regions=[],
                lambda_e0=lambda_e0, magic=3.0 / 16.0, accel=(accel, 0.0, 0.0))

    def refine(L, bx, by, bz, user):
        if L >= lmax:
            return 0
        if where == "global":
            return 1
        s = B / 2.0 ** L
        y0, y1, z0, z1 = by * s - c, (by + 1) * s - c, bz * s - c, (bz + 1) * s - c
        if where == "wall":
            return int(_square_meets_circle(y0, y1, z0, z1, R))
        P = paper_block / 2.0 ** L
        m = int(round(D / P))
        for j in range(m):          # the paper-grid blocks of level L that this block overlaps
            py0 = -R + j * P
            if min(y1, py0 + P) <= max(y0, py0):
                continue
            for k in range(m):
                pz0 = -R + k * P
                if min(z1, pz0 + P) > max(z0, pz0) and _square_meets_circle(py0, py0 + P, pz0, pz0 + P, R):
                    return 1
        return 0

    def flag(L, x, y, z, user):
        return int((y - c) ** 2 + (z - c) ** 2 >= R * R)

    return case, refine, flag, (c, R)


def freeslip_box_case(n=32, B=8, refine=True, lid=None, spheres=(), collision="trt", omega=1.6):
    """Box of n^3 level-0 cells, periodic in x, free-slip on the y and z faces (or the z+ face a
    velocity lid moving along x when lid is given); with refine, the central (n/4 .. 3n/4)^3 region
    (whole blocks, away from every face) is refined once.  Free-slip faces are named only in the
    paper (Sec. 4.1)."""
    r = n // B
    bc = ["periodic", "periodic", "freeslip", "freeslip", "freeslip", "velocity" if lid else "freeslip"]
    bc_u = [(0.0, 0.0, 0.0)] * 5 + [(lid or 0.0, 0.0, 0.0)]
    regions = [("box", 1, (n / 4 + 1, n / 4 + 1, n / 4 + 1), (3 * n / 4 - 1, 3 * n / 4 - 1, 3 * n / 4 - 1))] if refine else []
    return dict(root=(r, r, r), B=B, lmax=1 if refine else 0, collision=collision, rho0=1.0, bc=bc, bc_u=bc_u,
                spheres=list(spheres), regions=regions, lambda_e0=omega, magic=3.0 / 16.0, accel=(0.0, 0.0, 0.0))


def batch_cases(n=256, seed=SEED, B=16):
    """Small lid-driven cavities for stepping many forests together (the batched workload).

    Per case, drawn in turn from one seeded stream and redrawn until the leaf count lies in
    [8, 64]: root blocks per axis in {1..4}; 2 or 3 levels; lambda_e0 ~ U(1.5, 1.9); lid speed
    ~ U(0.02, 0.08) along x on the z+ face, no-slip elsewhere; TRT with Lambda = 3/16.  Level 1
    refines one random box of root blocks.  Level 2 refines one random box of level-1 blocks inside
    it, one level-1 block away from the level-1 box's faces (except where it reaches a wall), so
    that the forest is 2:1 balanced as drawn and its leaf count is known without building it:
    roots + 7 |box 1| + 7 |box 2|.  Each case carries that count as "leaves".
    """
    rng = np.random.default_rng(seed)
    cases = []
    while len(cases) < n:
        r = rng.integers(1, 5, size=3)
        lmax = int(rng.integers(1, 3))
        lo1 = np.array([rng.integers(0, r[a]) for a in range(3)])
        hi1 = np.array([rng.integers(lo1[a] + 1, r[a] + 1) for a in range(3)])
        n1 = int(np.prod(hi1 - lo1))
        regions = [("box", 1, tuple(int(v) * B for v in lo1), tuple(int(v) * B for v in hi1))]
        n2 = 0
        if lmax == 2:
            a_lo = 2 * lo1 + (lo1 > 0)
            a_hi = 2 * hi1 - (hi1 < r)
            if np.any(a_hi <= a_lo):
                continue
            lo2 = np.array([rng.integers(a_lo[a], a_hi[a]) for a in range(3)])
            hi2 = np.array([rng.integers(lo2[a] + 1, a_hi[a] + 1) for a in range(3)])
            n2 = int(np.prod(hi2 - lo2))
            regions.append(("box", 2, tuple(int(v) * B // 2 for v in lo2), tuple(int(v) * B // 2 for v in hi2)))
        leaves = int(np.prod(r)) + 7 * n1 + 7 * n2
        if not 8 <= leaves <= 64:
            continue
        lambda_e0 = float(rng.uniform(1.5, 1.9))
        lid = float(rng.uniform(0.02, 0.08))
        cases.append(dict(root=tuple(int(v) for v in r), B=B, lmax=lmax, collision="trt", rho0=1.0,
                          bc=["noslip"] * 5 + ["velocity"],
                          bc_u=[(0.0, 0.0, 0.0)] * 5 + [(lid, 0.0, 0.0)],
                          spheres=[], regions=regions, lambda_e0=lambda_e0, magic=3.0 / 16.0,
                          accel=(0.0, 0.0, 0.0), leaves=leaves))
    return cases


def warm_cases(n, seed=SEED, H=128, B=16, u_in=0.04, re_range=(20.0, 60.0)):
    """Channels H x H x H past 1-5 spheres, refined twice around them (the warm-start workload).

    Per case: sphere count uniform in 1..5, radii U(0.05, 0.15) H, centres uniform in the middle
    80 % of the box; Re uniform in re_range on the mean sphere diameter D (nu0 = u_in D / Re).
    No-slip walls at y = 0 and y = H, periodic x and z, driven by the body force a0 = 12 nu0 u_in
    / H^2 along x, whose plane Poiseuille flow has mean velocity u_in; TRT with Lambda = 3/16.
    Level 1 covers balls of radius r + H/16, level 2 balls of radius r + 3H/128 (level-0 units)
    around each sphere.
    """
    rng = np.random.default_rng(seed)
    cases = []
    for _ in range(n):
        k = int(rng.integers(1, 6))
        radii = rng.uniform(0.05, 0.15, k) * H
        centres = rng.uniform(0.1 * H, 0.9 * H, (k, 3))
        re = float(rng.uniform(*re_range))
        nu0 = u_in * 2.0 * float(radii.mean()) / re
        regions = [("ball", 1, tuple(float(v) for v in c), float(r) + H / 16.0) for c, r in zip(centres, radii)]
        regions += [("ball", 2, tuple(float(v) for v in c), float(r) + 3.0 * H / 128.0) for c, r in zip(centres, radii)]
        r0 = H // B
        cases.append(dict(root=(r0, r0, r0), B=B, lmax=2, collision="trt", rho0=1.0,
                          bc=["periodic", "periodic", "noslip", "noslip", "periodic", "periodic"],
                          bc_u=[(0.0, 0.0, 0.0)] * 6,
                          spheres=[tuple(float(v) for v in c) + (float(r),) for c, r in zip(centres, radii)],
                          regions=regions, lambda_e0=1.0 / (3.0 * nu0 + 0.5), magic=3.0 / 16.0,
                          accel=(12.0 * nu0 * u_in / H ** 2, 0.0, 0.0), u_init=(0.0, 0.0, 0.0), re=re,
                          u_in=u_in))
    return cases


def periodic_case(n=64, B=16, collision="srt", omega=1.9, regions=(), lmax=0):
    """Fully periodic cube of n^3 level-0 cells (uniform unless regions refine it)."""
    r = n // B
    return dict(root=(r, r, r), B=B, lmax=lmax, collision=collision, rho0=1.0,
                bc=["periodic"] * 6, bc_u=[(0.0, 0.0, 0.0)] * 6, spheres=[],
                regions=list(regions), lambda_e0=omega, magic=3.0 / 16.0,
                accel=(0.0, 0.0, 0.0))


SPHERE_CHANNEL_RADII = (34.0, 12.0, 6.0)


def sphere_channel_case(H=64, B=32, radii=SPHERE_CHANNEL_RADII, u_in=0.04, Re=100.0, inlet_outlet=False,
                        shift=True):
    """Channel 4H x H x H past a sphere of radius 0.1 H at (H, H/2, H/2), started from the plug
    flow (u_in, 0, 0).  With shift, FP32S/FP16S storage holds f - f^eq(rho0, plug) (u_shift).

    Four levels: blocks within radii[L-1] (level-0 cells, scaled with H/64) of the sphere centre
    are refined towards level L.  The relaxation rate follows from Re on the sphere diameter.
    By default every face is periodic (a periodic array of spheres in the stream; over 1000
    coarse steps the sphere's drag slows the mean flow by well under 1%).  With inlet_outlet the
    x faces are velocity walls with the plug instead: the plug outlet then clamps the wake on the
    under-resolved coarsest level and the run turns unstable after about 1,500-2,000 coarse steps
    at Re 100, so that variant serves short runs only.
    """
    s = H / 64.0
    c = (float(H), H / 2.0, H / 2.0)
    nu0 = u_in * (0.2 * H) / Re
    le0 = 1.0 / (3.0 * nu0 + 0.5)
    regions = [("ball", L + 1, c, r * s) for L, r in enumerate(radii)]
    bc = (["velocity", "velocity"] if inlet_outlet else ["periodic", "periodic"]) + ["periodic"] * 4
    return dict(root=(4 * H // B, H // B, H // B), B=B, lmax=len(radii), collision="trt",
                rho0=1.0, bc=bc, bc_u=[(u_in, 0.0, 0.0)] * 2 + [(0.0, 0.0, 0.0)] * 4,
                spheres=[(c[0], c[1], c[2], 0.1 * H)], regions=regions,
                lambda_e0=le0, magic=3.0 / 16.0, accel=(0.0, 0.0, 0.0), u_init=(u_in, 0.0, 0.0),
                u_shift=(u_in if shift else 0.0, 0.0, 0.0))


def plane_poiseuille_case(B=4, ny_roots=4, nxz_roots=1, where="bottom", lambda_e0=0.5, accel=1e-5):
    """Plane Poiseuille flow (Sec. 5.1): no-slip plates at y = 0 and y = H, periodic x and z,
    driven by a constant acceleration in x.  `where` refines one plate, both, or the middle."""
    H = ny_roots * B
    regs = []
    if where in ("bottom", "both"):
        regs.append(("box", 1, (0, 0, 0), (1e9, 0.5, 1e9)))
    if where in ("top", "both"):
        regs.append(("box", 1, (0, H - 0.5, 0), (1e9, H, 1e9)))
    if where == "middle":
        regs.append(("box", 1, (0, H / 2 - 0.5, 0), (1e9, H / 2 + 0.5, 1e9)))
    return dict(root=(nxz_roots, ny_roots, nxz_roots), B=B, lmax=1, collision="trt", rho0=1.0,
                bc=["periodic", "periodic", "noslip", "noslip", "periodic", "periodic"],
                bc_u=[(0.0, 0.0, 0.0)] * 6, spheres=[], regions=regs,
                lambda_e0=lambda_e0, magic=3.0 / 16.0, accel=(accel, 0.0, 0.0))


def plane_couette_case(B=4, nz_roots=4, nxy_roots=1, where=None, lambda_e0=0.5, u_wall=(0.05, 0.0, 0.0)):
    """Plane Couette flow: a velocity wall at z = H moving tangentially with u_wall, a no-slip wall
    at z = 0, periodic x and y, no force.  `where` refines the cells next to the moving wall
    ("top"), the fixed wall ("bottom"), both, or nothing (None)."""
    H = nz_roots * B
    regs = []
    if where in ("bottom", "both"):
        regs.append(("box", 1, (0, 0, 0), (1e9, 1e9, 0.5)))
    if where in ("top", "both"):
        regs.append(("box", 1, (0, 0, H - 0.5), (1e9, 1e9, H)))
    return dict(root=(nxy_roots, nxy_roots, nz_roots), B=B, lmax=1 if regs else 0, collision="trt", rho0=1.0,
                bc=["periodic"] * 4 + ["noslip", "velocity"],
                bc_u=[(0.0, 0.0, 0.0)] * 5 + [tuple(float(v) for v in u_wall)], spheres=[], regions=regs,
                lambda_e0=lambda_e0, magic=3.0 / 16.0, accel=(0.0, 0.0, 0.0))


# --------------------------------------------------------------------------- fields

def _splitmix64(x):
    """SplitMix64 finaliser (Steele, Lea & Flood 2014) on uint64 arrays."""
    x = (x + np.uint64(0x9E3779B97F4A7C15)) & np.uint64(0xFFFFFFFFFFFFFFFF)
    z = x
    z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & np.uint64(0xFFFFFFFFFFFFFFFF)
    z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & np.uint64(0xFFFFFFFFFFFFFFFF)
    return z ^ (z >> np.uint64(31))


def cell_normal(seed, X, Y, Z):
    """Standard normal deviate per cell, a pure function of (seed, x, y, z): counter-based,
    so any subset of cells can be generated in any order (Box-Muller on two SplitMix64 draws)."""
    with np.errstate(over="ignore"):
        key = (np.asarray(X, np.int64).astype(np.uint64)
               | (np.asarray(Y, np.int64).astype(np.uint64) << np.uint64(21))
               | (np.asarray(Z, np.int64).astype(np.uint64) << np.uint64(42)))
        h1 = _splitmix64(key ^ np.uint64(seed))
        h2 = _splitmix64(h1 ^ np.uint64(0xD1B54A32D192ED03))
    u1 = ((h1 >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)
    u2 = ((h2 >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


def taylor_green_modes(seed=SEED, nmodes=8, kmax=4):
    """Divergence-free Taylor-Green modes: integer wave vectors in {1..kmax}^3 and
    amplitudes drawn N(0,1) then projected orthogonal to k."""
    rng = np.random.default_rng(seed)
    modes = []
    for _ in range(nmodes):
        k = rng.integers(1, kmax + 1, size=3).astype(np.float64)
        a = rng.standard_normal(3)
        a -= k * (a @ k) / (k @ k)
        modes.append((k, a))
    return modes


def _tg_velocity(modes, N, Xc, Yc, Zc):
    X = 2.0 * math.pi * Xc / N
    Y = 2.0 * math.pi * Yc / N
    Z = 2.0 * math.pi * Zc / N
    u = [np.zeros(np.shape(X)) for _ in range(3)]
    for k, a in modes:
        sx, cx = np.sin(k[0] * X), np.cos(k[0] * X)
        sy, cy = np.sin(k[1] * Y), np.cos(k[1] * Y)
        sz, cz = np.sin(k[2] * Z), np.cos(k[2] * Z)
        u[0] += a[0] * cx * sy * sz
        u[1] += a[1] * sx * cy * sz
        u[2] += a[2] * sx * sy * cz
    return u


def taylor_green_field(N, seed=SEED, nmodes=8, kmax=4, umax=0.02, rho_sigma=1e-4):
    """Initial field of the periodic workload: a sum of Taylor-Green modes scaled so that
    max |u| over the N^3 level-0 cell centres is umax, and rho = 1 + N(0, rho_sigma^2).
    Returns field(level, X, Y, Z) -> (rho, (ux, uy, uz)) for integer level-L coordinates."""
    modes = taylor_green_modes(seed, nmodes, kmax)
    peak = 0.0
    ax = np.arange(N) + 0.5
    for z0 in range(0, N, 16):
        Zc, Yc, Xc = np.meshgrid(ax[z0:z0 + 16], ax, ax, indexing="ij")
        u = _tg_velocity(modes, N, Xc, Yc, Zc)
        peak = max(peak, float(np.sqrt(u[0] ** 2 + u[1] ** 2 + u[2] ** 2).max()))
    scale = umax / peak

    def field(level, X, Y, Z):
        s = 2.0 ** -level
        u = _tg_velocity(modes, N, (X + 0.5) * s, (Y + 0.5) * s, (Z + 0.5) * s)
        rho = 1.0 + rho_sigma * cell_normal(seed, X, Y, Z) if level == 0 else \
            1.0 + rho_sigma * cell_normal(seed + level, X, Y, Z)
        return rho, (u[0] * scale, u[1] * scale, u[2] * scale)

    return field


def uniform_field(rho=1.0, u=(0.0, 0.0, 0.0)):
    def field(level, X, Y, Z):
        return rho, u
    return field
