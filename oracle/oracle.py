"""ctypes wrapper of the plain CPU oracle in ``lbm_oracle.c``.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` use it; the product package never imports it.
It shares no code with the CUDA library.  Cases are plain dicts (see
``paper_1508_07982_gb300/inputs.py`` for the keys); this module marshals them
into the oracle's own C struct.
"""
import ctypes
import os
import subprocess

import numpy as np

Q = 19
_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liblbm_oracle.so")

_BC = {"periodic": 0, "noslip": 1, "velocity": 2, "freeslip": 3}
_COLL = {"srt": 0, "trt": 1}

CLS_OUT, CLS_OWNED, CLS_G1, CLS_G2, CLS_G3, CLS_G4, CLS_FINER, CLS_FAR = range(8)
FL_FLUID, FL_NOSLIP, FL_VEL = range(3)


def build(force=False):
    """Compiles the oracle with gcc (plain -O2, OpenMP, no FMA contraction)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if not force and os.path.exists(_OUT) and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC):
        return _OUT
    tmp = _OUT + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=gnu99", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _OUT)
    return _OUT


class _Desc(ctypes.Structure):
    _fields_ = [
        ("nroot", ctypes.c_int * 3),
        ("B", ctypes.c_int),
        ("lmax", ctypes.c_int),
        ("collision", ctypes.c_int),
        ("rho0", ctypes.c_double),
        ("bc", ctypes.c_int * 6),
        ("bcu", (ctypes.c_double * 3) * 6),
        ("nsph", ctypes.c_int),
        ("sph", (ctypes.c_double * 4) * 64),
        ("nreg", ctypes.c_int),
        ("reg", (ctypes.c_double * 8) * 64),
    ]


REFINE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p)
FLAG_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                           ctypes.c_void_p)

_lib_handle = None


def lib():
    global _lib_handle
    if _lib_handle is None:
        L = ctypes.CDLL(build())
        P = ctypes.c_void_p
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        L.orc_create.restype = P
        L.orc_create.argtypes = [ctypes.POINTER(_Desc), REFINE_FN, FLAG_FN, P]
        L.orc_destroy.argtypes = [P]
        L.orc_error.restype = ctypes.c_char_p
        L.orc_num_levels.argtypes = [P]
        L.orc_leaves.restype = ctypes.c_long
        L.orc_leaves.argtypes = [P, ctypes.c_int, ip]
        L.orc_window.argtypes = [P, ctypes.c_int, ip, ip, ip]
        L.orc_get_class.argtypes = [P, ctypes.c_int, P, P]
        L.orc_set_params.argtypes = [P, ctypes.c_double, ctypes.c_double, dp]
        L.orc_set_params_explicit.argtypes = [P, dp, dp, dp]
        L.orc_get_params.argtypes = [P, dp, dp, dp]
        L.orc_init_eq.argtypes = [P, ctypes.c_int, dp, dp]
        L.orc_step.argtypes = [P, ctypes.c_int]
        L.orc_get_f.argtypes = [P, ctypes.c_int, dp, ctypes.c_int]
        L.orc_set_f.argtypes = [P, ctypes.c_int, dp]
        L.orc_macro.argtypes = [P, ctypes.c_int, dp, dp]
        L.orc_mass_momentum.argtypes = [P, dp]
        for nm in ("orc_num_fluid", "orc_num_stream", "orc_num_ghost", "orc_num_coalesce"):
            getattr(L, nm).restype = ctypes.c_long
            getattr(L, nm).argtypes = [P, ctypes.c_int]
        L.orc_lattice.argtypes = [ip, dp, ip]
        L.orc_num_threads.restype = ctypes.c_int
        L.orc_feq.argtypes = [ctypes.c_double, dp, ctypes.c_double, dp]
        L.orc_collide.argtypes = [dp, ctypes.c_int, ctypes.c_double, ctypes.c_double, dp, ctypes.c_double]
        L.orc_scale_rate.restype = ctypes.c_double
        L.orc_scale_rate.argtypes = [ctypes.c_double, ctypes.c_int]
        L.orc_lambda_odd.restype = ctypes.c_double
        L.orc_lambda_odd.argtypes = [ctypes.c_double, ctypes.c_double]
        _lib_handle = L
    return _lib_handle


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def num_threads():
    return lib().orc_num_threads()


def lattice():
    e = np.zeros((Q, 3), np.int32)
    w = np.zeros(Q)
    opp = np.zeros(Q, np.int32)
    lib().orc_lattice(_ip(e), _dp(w), _ip(opp))
    return e, w, opp


def feq(rho, u, rho0=1.0):
    out = np.zeros(Q)
    uu = np.ascontiguousarray(u, dtype=np.float64)
    lib().orc_feq(rho, _dp(uu), rho0, _dp(out))
    return out


def collide(f, collision, le, lo, acc=(0.0, 0.0, 0.0), rho0=1.0):
    ff = np.array(f, dtype=np.float64)
    a = np.ascontiguousarray(acc, dtype=np.float64)
    lib().orc_collide(_dp(ff), _COLL[collision], le, lo, _dp(a), rho0)
    return ff


def scale_rate(w0, level):
    return lib().orc_scale_rate(w0, level)


def lambda_odd(le, magic):
    return lib().orc_lambda_odd(le, magic)


def _desc(case):
    d = _Desc()
    for a in range(3):
        d.nroot[a] = int(case["root"][a])
    d.B = int(case["B"])
    d.lmax = int(case.get("lmax", 0))
    d.collision = _COLL[case.get("collision", "trt")]
    d.rho0 = float(case.get("rho0", 1.0))
    bcs = case.get("bc", ["periodic"] * 6)
    bcu = case.get("bc_u", [(0.0, 0.0, 0.0)] * 6)
    for k in range(6):
        d.bc[k] = _BC[bcs[k]]
        for a in range(3):
            d.bcu[k][a] = float(bcu[k][a])
    sph = case.get("spheres", [])
    d.nsph = len(sph)
    for i, s in enumerate(sph):
        for a in range(4):
            d.sph[i][a] = float(s[a])
    reg = case.get("regions", [])
    d.nreg = len(reg)
    for i, r in enumerate(reg):
        if r[0] == "box":
            vals = [0.0, float(r[1])] + [float(v) for v in r[2]] + [float(v) for v in r[3]]
        else:
            vals = [1.0, float(r[1])] + [float(v) for v in r[2]] + [float(r[3]), 0.0, 0.0]
        for k in range(8):
            d.reg[i][k] = vals[k]
    return d


class Oracle:
    """One refined-grid simulation held by the C oracle."""

    def __init__(self, case, refine=None, flag=None):
        L = lib()
        self.case = case
        self._refine = REFINE_FN(refine) if refine else REFINE_FN()
        self._flag = FLAG_FN(flag) if flag else FLAG_FN()
        self._d = _desc(case)
        h = L.orc_create(ctypes.byref(self._d), self._refine, self._flag, None)
        if not h:
            raise ValueError("oracle rejected the case: " + L.orc_error().decode())
        self.h = h
        self.nlev = L.orc_num_levels(h)
        if "lambda_e0" in case:
            self.set_params(case["lambda_e0"], case.get("magic", 3.0 / 16.0), case.get("accel", (0.0, 0.0, 0.0)))

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_destroy(self.h)
            self.h = None

    # parameters -------------------------------------------------------------
    def set_params(self, lambda_e0, magic=3.0 / 16.0, accel=(0.0, 0.0, 0.0)):
        a = np.ascontiguousarray(accel, dtype=np.float64)
        lib().orc_set_params(self.h, lambda_e0, magic, _dp(a))

    def set_params_explicit(self, le, lo, acc):
        le = np.ascontiguousarray(le, dtype=np.float64)
        lo = np.ascontiguousarray(lo, dtype=np.float64)
        acc = np.ascontiguousarray(acc, dtype=np.float64).reshape(-1)
        lib().orc_set_params_explicit(self.h, _dp(le), _dp(lo), _dp(acc))

    def params(self):
        le = np.zeros(self.nlev)
        lo = np.zeros(self.nlev)
        acc = np.zeros((self.nlev, 3))
        lib().orc_get_params(self.h, _dp(le), _dp(lo), _dp(acc))
        return le, lo, acc

    # geometry ---------------------------------------------------------------
    def leaves(self, level):
        n = lib().orc_leaves(self.h, level, None)
        out = np.zeros((max(n, 1), 3), np.int32)
        lib().orc_leaves(self.h, level, _ip(out))
        return out[:n]

    def window(self, level):
        s = np.zeros(3, np.int32)
        n = np.zeros(3, np.int32)
        N = np.zeros(3, np.int32)
        lib().orc_window(self.h, level, _ip(s), _ip(n), _ip(N))
        return s, n, N

    def coords(self, level):
        """Global level coordinates (X, Y, Z) of every window cell, each shaped (nz, ny, nx).
        Periodic axes are wrapped into the domain; walled axes may hold outside cells."""
        s, n, N = self.window(level)
        per = [self.case.get("bc", ["periodic"] * 6)[2 * a] == "periodic" for a in range(3)]
        ax = []
        for a in range(3):
            g = s[a] + np.arange(n[a])
            if per[a]:
                g = np.mod(g, N[a])
            ax.append(g)
        Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
        return X, Y, Z

    def classes(self, level):
        s, n, N = self.window(level)
        cls = np.zeros(int(np.prod(n)), np.uint8)
        flg = np.zeros(int(np.prod(n)), np.uint8)
        if cls.size:
            lib().orc_get_class(self.h, level, cls.ctypes.data, flg.ctypes.data)
        shp = (n[2], n[1], n[0])
        return cls.reshape(shp), flg.reshape(shp)

    def num_fluid(self, level):
        return lib().orc_num_fluid(self.h, level)

    def counts(self, level):
        L = lib()
        return dict(fluid=L.orc_num_fluid(self.h, level), stream=L.orc_num_stream(self.h, level),
                    ghost=L.orc_num_ghost(self.h, level), coalesce=L.orc_num_coalesce(self.h, level))

    def cell_updates_per_coarse_step(self):
        return sum(self.num_fluid(L) * (1 << L) for L in range(self.nlev))

    # state ------------------------------------------------------------------
    def init_eq(self, level, rho=None, u=None):
        """rho: (nz,ny,nx) window array or None; u: (3,nz,ny,nx) or None."""
        r = None if rho is None else np.ascontiguousarray(rho, dtype=np.float64)
        v = None if u is None else np.ascontiguousarray(u, dtype=np.float64)
        lib().orc_init_eq(self.h, level, _dp(r) if r is not None else None, _dp(v) if v is not None else None)

    def init_fields(self, field):
        """Initial equilibrium from field(level, X, Y, Z) -> (rho, (ux, uy, uz)) on every level."""
        for L in range(self.nlev):
            s, n, N = self.window(L)
            if np.prod(n) == 0:
                continue
            X, Y, Z = self.coords(L)
            rho, u = field(L, X, Y, Z)
            rho = np.broadcast_to(np.asarray(rho, np.float64), X.shape)
            u = np.stack([np.broadcast_to(np.asarray(c, np.float64), X.shape) for c in u])
            self.init_eq(L, rho, u)

    def step(self, n=1):
        lib().orc_step(self.h, n)

    def get_f(self, level, post_collision=False):
        s, n, N = self.window(level)
        out = np.zeros((int(np.prod(n)), Q))
        if out.size:
            lib().orc_get_f(self.h, level, _dp(out), 1 if post_collision else 0)
        return out.reshape(n[2], n[1], n[0], Q)

    def set_f(self, level, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        lib().orc_set_f(self.h, level, _dp(f))

    def macro(self, level):
        s, n, N = self.window(level)
        m = int(np.prod(n))
        rho = np.zeros(m)
        u = np.zeros(3 * m)
        if m:
            lib().orc_macro(self.h, level, _dp(rho), _dp(u))
        shp = (n[2], n[1], n[0])
        return rho.reshape(shp), u.reshape((3,) + shp)

    def mass_momentum(self):
        out = np.zeros(4)
        lib().orc_mass_momentum(self.h, _dp(out))
        return out

    def lookup(self, level, X, Y, Z):
        """Window indices (iz, iy, ix) of global level coordinates; periodic axes wrap."""
        s, n, N = self.window(level)
        per = [self.case.get("bc", ["periodic"] * 6)[2 * a] == "periodic" for a in range(3)]
        idx = []
        for a, G in enumerate((X, Y, Z)):
            d = np.asarray(G) - s[a]
            if per[a]:
                d = np.mod(d, N[a])
            if np.any(d < 0) or np.any(d >= n[a]):
                raise IndexError("coordinate outside the oracle window on axis %d" % a)
            idx.append(d)
        return idx[2], idx[1], idx[0]
