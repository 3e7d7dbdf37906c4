"""Thin ctypes binding of the C-ABI in ``include/lbm_gb300.h``.

Argument marshalling only: every step of the method runs in the library's CUDA
kernels.  The shared library is the in-tree ``_lib/liblbm_gb300.so`` built by
``build.py``; importing this module fails loudly if it is missing.  PyTorch is
used for device buffers and streams (tensors are passed by ``data_ptr()``).
"""
import ctypes
import os

import numpy as np

from . import build as _build

_LIB_PATH = _build.LIB
Q = 19

LBM_OK, LBM_EINVAL, LBM_EUNBALANCED, LBM_ENOMEM, LBM_ECUDA, LBM_ETIMEOUT, LBM_ENONFINITE = range(7)
PRECISION = {"fp64": 0, "fp32s": 1, "fp16s": 2}
_BC = {"periodic": 0, "noslip": 1, "velocity": 2, "freeslip": 3}
_COLL = {"srt": 0, "trt": 1}

# Every entry point of include/lbm_gb300.h (checked by the tests).
EXPORTS = [
    "lbm_last_error", "lbm_lattice", "lbm_plan_create", "lbm_plan_num_levels", "lbm_plan_leaves",
    "lbm_plan_counts", "lbm_plan_ghost_work", "lbm_plan_destroy", "lbm_create_forest", "lbm_destroy", "lbm_num_levels",
    "lbm_get_block_table", "lbm_cell_updates_per_coarse_step", "lbm_set_level_params",
    "lbm_set_level_params_explicit", "lbm_init_equilibrium", "lbm_step_coarse", "lbm_get_macroscopic",
    "lbm_get_pdfs", "lbm_set_pdfs", "lbm_reduce_mass_momentum", "lbm_timing_begin", "lbm_timing_end",
    "lbm_launches_per_coarse_step", "lbm_set_kernel_config", "lbm_get_kernel_config",
    "lbm_mass_momentum_noalloc", "lbm_probe_fp64_fma", "lbm_autotune", "lbm_autotune_block_size",
    "lbm_batch_create", "lbm_batch_step",
    "lbm_batch_set_kernel_config", "lbm_batch_autotune", "lbm_batch_cell_updates_per_coarse_step",
    "lbm_batch_launches_per_coarse_step", "lbm_batch_destroy", "lbm_net_create", "lbm_net_destroy",
    "lbm_net_num_params", "lbm_net_get_params", "lbm_net_set_params", "lbm_net_forward", "lbm_net_predict",
    "lbm_net_gradient", "lbm_net_get_grads", "lbm_net_train_step", "lbm_velocity_residual",
    "lbm_warmstart_features", "lbm_warmstart_targets", "lbm_warmstart_fields", "lbm_net_set_backend",
    "lbm_net_set_wait_test",
]
NOALLOC_MAX_CELLS = 16384 * 4096


class LBMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("lbm status %d: %s" % (status, msg))
        self.status = status


class Desc(ctypes.Structure):
    _fields_ = [
        ("root_blocks", ctypes.c_int32 * 3),
        ("block_cells", ctypes.c_int32),
        ("max_level", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("collision", ctypes.c_int32),
        ("bc", ctypes.c_int32 * 6),
        ("bc_velocity", (ctypes.c_double * 3) * 6),
        ("rho0", ctypes.c_double),
        ("n_spheres", ctypes.c_int32),
        ("spheres", (ctypes.c_double * 4) * 64),
        ("n_regions", ctypes.c_int32),
        ("regions", (ctypes.c_double * 8) * 64),
        ("u_shift", ctypes.c_double * 3),
    ]


REFINE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p)
FLAG_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                           ctypes.c_void_p)

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
RELEASE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class Allocator(ctypes.Structure):
    """lbm_allocator: the device-memory hook of lbm_create_forest, lbm_batch_create and
    lbm_net_create."""
    _fields_ = [("alloc", ALLOC_FN), ("release", RELEASE_FN), ("user", ctypes.c_void_p)]


def _torch_alloc(nbytes, stream, user):
    try:
        import torch
        return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
    except Exception:        # out of memory (or torch torn down): the library returns LBM_ENOMEM
        return None


def _torch_release(ptr, nbytes, stream, user):
    try:
        import torch
        torch.cuda.caching_allocator_delete(int(ptr))
    except Exception:
        pass


_TORCH_ALLOCATOR = Allocator(ALLOC_FN(_torch_alloc), RELEASE_FN(_torch_release), None)


def _allocator(allocator):
    """"torch" (the default): torch's CUDA caching allocator; None: the library's cudaMalloc; or an
    Allocator the caller keeps alive for the object's lifetime."""
    if allocator == "torch":
        return ctypes.byref(_TORCH_ALLOCATOR)
    if allocator is None:
        return None
    return ctypes.byref(allocator)


_lib = None


def library():
    """Loads the in-tree library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise ImportError("CUDA library %s is missing: run __graft_entry__.build() first" % _LIB_PATH)
        L = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        i32p = ctypes.POINTER(ctypes.c_int32)
        i64p = ctypes.POINTER(ctypes.c_int64)
        dp = ctypes.POINTER(ctypes.c_double)
        L.lbm_last_error.restype = ctypes.c_char_p
        sig = {
            "lbm_lattice": [i32p, dp, i32p],
            "lbm_plan_create": [ctypes.POINTER(Desc), REFINE_FN, FLAG_FN, P, ctypes.POINTER(P)],
            "lbm_plan_num_levels": [P, i32p],
            "lbm_plan_leaves": [P, ctypes.c_int32, i32p, i32p],
            "lbm_plan_counts": [P, ctypes.c_int32, i64p],
            "lbm_plan_ghost_work": [P, ctypes.c_int32, i64p],
            "lbm_plan_destroy": [P],
            "lbm_create_forest": [ctypes.POINTER(Desc), REFINE_FN, FLAG_FN, P, P, ctypes.POINTER(Allocator),
                                  ctypes.POINTER(P)],
            "lbm_destroy": [P],
            "lbm_num_levels": [P, i32p],
            "lbm_get_block_table": [P, ctypes.c_int32, i32p, i32p],
            "lbm_cell_updates_per_coarse_step": [P, i64p],
            "lbm_set_level_params": [P, ctypes.c_double, ctypes.c_double, dp],
            "lbm_set_level_params_explicit": [P, dp, dp, dp],
            "lbm_init_equilibrium": [P, ctypes.c_int32, P, P, ctypes.c_int32],
            "lbm_step_coarse": [P, ctypes.c_int32],
            "lbm_get_macroscopic": [P, ctypes.c_int32, P, P, ctypes.c_int32],
            "lbm_get_pdfs": [P, ctypes.c_int32, P, ctypes.c_int32],
            "lbm_set_pdfs": [P, ctypes.c_int32, P, ctypes.c_int32],
            "lbm_reduce_mass_momentum": [P, dp],
            "lbm_timing_begin": [P, ctypes.c_int32],
            "lbm_timing_end": [P, dp, i64p, dp, i64p, dp, i64p],
            "lbm_launches_per_coarse_step": [P, i32p],
            "lbm_set_kernel_config": [P, ctypes.c_int32, ctypes.c_int32],
            "lbm_get_kernel_config": [P, i32p, i32p],
            "lbm_mass_momentum_noalloc": [P, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, dp, P, P],
            "lbm_autotune": [P, ctypes.c_int32, i32p, i32p, dp],
            "lbm_autotune_block_size": [ctypes.POINTER(Desc), REFINE_FN, FLAG_FN, P, ctypes.c_double, ctypes.c_double,
                                        dp, P, ctypes.POINTER(Allocator), ctypes.c_int32, i32p, dp],
            "lbm_batch_create": [ctypes.POINTER(P), ctypes.c_int32, ctypes.POINTER(Allocator), ctypes.POINTER(P)],
            "lbm_batch_step": [P, ctypes.c_int32],
            "lbm_batch_set_kernel_config": [P, ctypes.c_int32, ctypes.c_int32],
            "lbm_batch_autotune": [P, ctypes.c_int32, i32p, i32p, dp],
            "lbm_batch_cell_updates_per_coarse_step": [P, i64p],
            "lbm_batch_launches_per_coarse_step": [P, i32p],
            "lbm_batch_destroy": [P],
            "lbm_net_create": [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, P,
                               ctypes.POINTER(Allocator), ctypes.POINTER(P)],
            "lbm_net_destroy": [P],
            "lbm_net_num_params": [P, i64p],
            "lbm_net_get_params": [P, P],
            "lbm_net_set_params": [P, P],
            "lbm_net_forward": [P, P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P],
            "lbm_net_predict": [P, P, P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P],
            "lbm_net_gradient": [P, P, P, P, dp],
            "lbm_net_get_grads": [P, P],
            "lbm_net_train_step": [P, P, P, P, P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                   ctypes.c_float, dp],
            "lbm_velocity_residual": [P, dp],
            "lbm_probe_fp64_fma": [ctypes.c_int32, dp, P],
            "lbm_net_set_backend": [P, ctypes.c_int32],
            "lbm_net_set_wait_test": [P, ctypes.c_int32],
            "lbm_warmstart_features": [P, P, i32p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                       P, ctypes.c_int32, P, ctypes.c_int32, ctypes.c_double, ctypes.c_double, P, P, P],
            "lbm_warmstart_targets": [P, P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                      ctypes.c_double, P, P, P],
            "lbm_warmstart_fields": [P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                     ctypes.c_double, P, P, P],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.restype = ctypes.c_int
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status):
    if status != LBM_OK:
        raise LBMError(status, library().lbm_last_error().decode())


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ptr(x):
    """Pointer of a numpy array (host) or a torch tensor (host or device); None stays NULL."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def _host_f64(x):
    """Passes numpy FP64 arrays and torch tensors through; converts anything else to FP64."""
    if x is None or hasattr(x, "data_ptr") or (isinstance(x, np.ndarray) and x.dtype == np.float64
                                               and x.flags.c_contiguous):
        return x
    return np.ascontiguousarray(x, dtype=np.float64)


def lbm_lattice():
    e = np.zeros((Q, 3), np.int32)
    w = np.zeros(Q)
    opp = np.zeros(Q, np.int32)
    _check(library().lbm_lattice(e.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dp(w),
                                 opp.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))
    return e, w, opp


def make_desc(case, precision="fp64"):
    """Marshals a case dict (keys documented in inputs.py) into lbm_forest_desc."""
    d = Desc()
    for a in range(3):
        d.root_blocks[a] = int(case["root"][a])
    d.block_cells = int(case["B"])
    d.max_level = int(case.get("lmax", 0))
    d.precision = PRECISION[precision]
    d.collision = _COLL[case.get("collision", "trt")]
    bcs = case.get("bc", ["periodic"] * 6)
    bcu = case.get("bc_u", [(0.0, 0.0, 0.0)] * 6)
    for k in range(6):
        d.bc[k] = _BC[bcs[k]]
        for a in range(3):
            d.bc_velocity[k][a] = float(bcu[k][a])
    d.rho0 = float(case.get("rho0", 1.0))
    sph = case.get("spheres", [])
    d.n_spheres = len(sph)
    for i, s in enumerate(sph):
        for a in range(4):
            d.spheres[i][a] = float(s[a])
    reg = case.get("regions", [])
    d.n_regions = len(reg)
    for i, r in enumerate(reg):
        if r[0] == "box":
            vals = [0.0, float(r[1])] + [float(v) for v in r[2]] + [float(v) for v in r[3]]
        else:
            vals = [1.0, float(r[1])] + [float(v) for v in r[2]] + [float(r[3]), 0.0, 0.0]
        for k in range(8):
            d.regions[i][k] = vals[k]
    for a, v in enumerate(case.get("u_shift", (0.0, 0.0, 0.0))):
        d.u_shift[a] = float(v)
    return d


def lbm_probe_fp64_fma(reps=20, stream=None):
    """Measured FP64 FMA rate of the device in G FMA/s (see include/lbm_gb300.h)."""
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    r = ctypes.c_double()
    _check(library().lbm_probe_fp64_fma(reps, ctypes.byref(r), ctypes.c_void_p(stream)))
    return r.value


def lbm_mass_momentum_noalloc(pdfs, precision, n_cells, rho0, out, stream=None, u_shift=None):
    """Totals of a device PDF array without any allocation (see include/lbm_gb300.h).  pdfs and
    out are device tensors (or raw device addresses); out receives 5 doubles {rho, jx, jy, jz,
    skipped cells}.  u_shift: the storage shift of the shifted layouts (None = 0)."""
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    p = pdfs if isinstance(pdfs, int) else pdfs.data_ptr()
    o = out if isinstance(out, int) else out.data_ptr()
    us = None if u_shift is None else np.ascontiguousarray(u_shift, dtype=np.float64)
    _check(library().lbm_mass_momentum_noalloc(ctypes.c_void_p(p), PRECISION[precision], n_cells, rho0,
                                                _dp(us) if us is not None else None, ctypes.c_void_p(o),
                                                ctypes.c_void_p(stream)))


def autotune_block_size(case, precision="fp32s", n_steps=10, flag=None, stream=None, allocator="torch"):
    """lbm_autotune_block_size: the block size (8, 16 or 32) with the fewest ms per coarse step for
    this case's domain, regions and obstacles, and the ms of each candidate (-1: not buildable)."""
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    d = make_desc(case, precision)
    fl = FLAG_FN(flag) if flag else FLAG_FN()
    acc = np.ascontiguousarray(case.get("accel", (0.0, 0.0, 0.0)), dtype=np.float64)
    b = ctypes.c_int32()
    ms = np.zeros(3)
    _check(library().lbm_autotune_block_size(ctypes.byref(d), REFINE_FN(), fl, None, float(case["lambda_e0"]),
                                             float(case.get("magic", 3.0 / 16.0)), _dp(acc), ctypes.c_void_p(stream),
                                             _allocator(allocator), n_steps, ctypes.byref(b), _dp(ms)))
    return b.value, {8: ms[0], 16: ms[1], 32: ms[2]}


class Plan:
    """Host-only forest plan (lbm_plan_*): leaf set and per-level counts, no GPU needed."""

    def __init__(self, case, refine=None, flag=None):
        L = library()
        self._refine = REFINE_FN(refine) if refine else REFINE_FN()
        self._flag = FLAG_FN(flag) if flag else FLAG_FN()
        self._d = make_desc(case)
        h = ctypes.c_void_p()
        _check(L.lbm_plan_create(ctypes.byref(self._d), self._refine, self._flag, None, ctypes.byref(h)))
        self.h = h
        n = ctypes.c_int32()
        _check(L.lbm_plan_num_levels(self.h, ctypes.byref(n)))
        self.nlev = n.value

    def __del__(self):
        if getattr(self, "h", None):
            library().lbm_plan_destroy(self.h)
            self.h = None

    def leaves(self, level):
        n = ctypes.c_int32()
        _check(library().lbm_plan_leaves(self.h, level, ctypes.byref(n), None))
        out = np.zeros((max(n.value, 1), 3), np.int32)
        _check(library().lbm_plan_leaves(self.h, level, ctypes.byref(n), out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))
        return out[:n.value]

    def counts(self, level):
        c = np.zeros(4, np.int64)
        _check(library().lbm_plan_counts(self.h, level, c.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
        return dict(blocks=int(c[0]), fluid=int(c[1]), ghost12=int(c[2]), ghost_blocks=int(c[3]))

    def ghost_work(self, level):
        """Ghost stream work of the level's sub-steps: cells and (cell, direction) values."""
        c = np.zeros(4, np.int64)
        _check(library().lbm_plan_ghost_work(self.h, level, c.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
        return dict(cells1=int(c[0]), values1=int(c[1]), cells2=int(c[2]), values2=int(c[3]))


class Forest:
    """A refined-grid simulation on the current CUDA device (lbm_create_forest ... lbm_destroy).
    Its device memory comes from torch's caching allocator unless `allocator` says otherwise."""

    def __init__(self, case, precision="fp64", refine=None, flag=None, stream=None, allocator="torch"):
        L = library()
        self.case = case
        self.precision = precision
        self._refine = REFINE_FN(refine) if refine else REFINE_FN()
        self._flag = FLAG_FN(flag) if flag else FLAG_FN()
        self._d = make_desc(case, precision)
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        h = ctypes.c_void_p()
        self._alloc = allocator
        _check(L.lbm_create_forest(ctypes.byref(self._d), self._refine, self._flag, None,
                                   ctypes.c_void_p(stream), _allocator(allocator), ctypes.byref(h)))
        self.h = h
        n = ctypes.c_int32()
        _check(L.lbm_num_levels(self.h, ctypes.byref(n)))
        self.nlev = n.value
        self.B = int(case["B"])
        if "lambda_e0" in case:
            self.set_level_params(case["lambda_e0"], case.get("magic", 3.0 / 16.0), case.get("accel", (0.0, 0.0, 0.0)))

    def close(self):
        if getattr(self, "h", None):
            _check(library().lbm_destroy(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- tables
    def block_table(self, level):
        n = ctypes.c_int32()
        _check(library().lbm_get_block_table(self.h, level, ctypes.byref(n), None))
        out = np.zeros((max(n.value, 1), 3), np.int32)
        _check(library().lbm_get_block_table(self.h, level, ctypes.byref(n),
                                             out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))
        return out[:n.value]

    def n_cells(self, level):
        return len(self.block_table(level)) * self.B ** 3

    def cell_coords(self, level):
        """Global level coordinates (X, Y, Z) of the block-major cell order, each [n_cells]."""
        bt = self.block_table(level)
        B = self.B
        r = np.arange(B)
        lz, ly, lx = np.meshgrid(r, r, r, indexing="ij")
        X = (bt[:, 0:1] * B + lx.reshape(1, -1)).reshape(-1)
        Y = (bt[:, 1:2] * B + ly.reshape(1, -1)).reshape(-1)
        Z = (bt[:, 2:3] * B + lz.reshape(1, -1)).reshape(-1)
        return X, Y, Z

    def cell_updates_per_coarse_step(self):
        n = ctypes.c_int64()
        _check(library().lbm_cell_updates_per_coarse_step(self.h, ctypes.byref(n)))
        return n.value

    def launches_per_coarse_step(self):
        n = ctypes.c_int32()
        _check(library().lbm_launches_per_coarse_step(self.h, ctypes.byref(n)))
        return n.value

    # -- parameters and state
    def set_level_params(self, lambda_e0, magic=3.0 / 16.0, accel=(0.0, 0.0, 0.0)):
        a = np.ascontiguousarray(accel, dtype=np.float64)
        _check(library().lbm_set_level_params(self.h, lambda_e0, magic, _dp(a)))

    def set_level_params_explicit(self, le, lo, acc):
        le = np.ascontiguousarray(le, dtype=np.float64)
        lo = np.ascontiguousarray(lo, dtype=np.float64)
        acc = np.ascontiguousarray(acc, dtype=np.float64).reshape(-1)
        _check(library().lbm_set_level_params_explicit(self.h, _dp(le), _dp(lo), _dp(acc)))

    def init_equilibrium(self, level, rho=None, u=None, on_device=False):
        """rho [n_cells] and u [3][n_cells], FP64, block-major; numpy arrays, or torch tensors
        (host tensors may be pinned; device tensors need on_device=True)."""
        rho, u = _host_f64(rho), _host_f64(u)
        _check(library().lbm_init_equilibrium(self.h, level, _ptr(rho), _ptr(u), 1 if on_device else 0))

    def init_uniform(self, u=(0.0, 0.0, 0.0)):
        uu = np.ascontiguousarray(u, dtype=np.float64)
        _check(library().lbm_init_equilibrium(self.h, -1, None, uu.ctypes.data, 0))

    def init_fields(self, field):
        """f^eq from field(level, X, Y, Z) -> (rho, (ux, uy, uz)) on every level."""
        for L in range(self.nlev):
            X, Y, Z = self.cell_coords(L)
            if X.size == 0:
                self.init_equilibrium(L)
                continue
            rho, u = field(L, X, Y, Z)
            rho = np.broadcast_to(np.asarray(rho, np.float64), X.shape)
            u = np.stack([np.broadcast_to(np.asarray(c, np.float64), X.shape) for c in u])
            self.init_equilibrium(L, rho, u)

    def step_coarse(self, n=1):
        _check(library().lbm_step_coarse(self.h, n))

    def get_macroscopic(self, level, rho=None, u=None, on_device=False):
        """Returns (rho, u); allocates numpy outputs when none are given and on_device is False.  level = -1:
        every level, level 0 first, in one array."""
        if rho is None and u is None and not on_device:
            n = sum(self.n_cells(L) for L in range(self.nlev)) if level == -1 else self.n_cells(level)
            rho, u = np.zeros(n), np.zeros((3, n))
        _check(library().lbm_get_macroscopic(self.h, level, _ptr(rho), _ptr(u), 1 if on_device else 0))
        return rho, u

    def velocity_residual(self):
        """lbm_velocity_residual: relative velocity change since the previous call (inf first)."""
        r = ctypes.c_double()
        _check(library().lbm_velocity_residual(self.h, ctypes.byref(r)))
        return r.value

    def get_pdfs(self, level, out=None, on_device=False):
        if on_device:
            _check(library().lbm_get_pdfs(self.h, level, _ptr(out), 1))
            return out
        n = self.n_cells(level)
        out = np.zeros((Q, n))
        if n:
            _check(library().lbm_get_pdfs(self.h, level, out.ctypes.data, 0))
        return out

    def set_pdfs(self, level, pdfs, on_device=False):
        pdfs = _host_f64(pdfs)
        _check(library().lbm_set_pdfs(self.h, level, _ptr(pdfs), 1 if on_device else 0))

    def reduce_mass_momentum(self):
        out = np.zeros(4)
        _check(library().lbm_reduce_mass_momentum(self.h, _dp(out)))
        return out

    def set_kernel_config(self, cells_per_thread_log2, ctas_per_sm):
        _check(library().lbm_set_kernel_config(self.h, cells_per_thread_log2, ctas_per_sm))

    def kernel_config(self):
        a, b = ctypes.c_int32(), ctypes.c_int32()
        _check(library().lbm_get_kernel_config(self.h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def autotune(self, n_steps=10):
        """lbm_autotune: applies the fastest thread mapping; returns (cells_per_thread_log2,
        ctas_per_sm, ms per coarse step).  The state is left as it was."""
        a, b, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
        _check(library().lbm_autotune(self.h, n_steps, ctypes.byref(a), ctypes.byref(b), ctypes.byref(ms)))
        return a.value, b.value, ms.value

    def timing_begin(self, max_steps):
        _check(library().lbm_timing_begin(self.h, max_steps))

    def timing_end(self, explode=False, side=False):
        """Per level: (ms, launches) of the column-walk (stream-collide) kernels; with explode=True
        also the explosion kernels' (ms, launches); with side=True also the side kernels' (coupled
        cells and ghost work of the FP32/FP16 layouts)."""
        out = [np.zeros(self.nlev), np.zeros(self.nlev, np.int64), np.zeros(self.nlev), np.zeros(self.nlev, np.int64),
               np.zeros(self.nlev), np.zeros(self.nlev, np.int64)]
        i64 = ctypes.POINTER(ctypes.c_int64)
        _check(library().lbm_timing_end(self.h, _dp(out[0]), out[1].ctypes.data_as(i64), _dp(out[2]),
                                        out[3].ctypes.data_as(i64), _dp(out[4]), out[5].ctypes.data_as(i64)))
        res = tuple(out[:2])
        if explode:
            res += tuple(out[2:4])
        if side:
            res += tuple(out[4:6])
        return res


class Batch:
    """Independent forests stepped together, one launch per phase (lbm_batch_create ...
    lbm_batch_destroy).  The forests stay usable one by one and must outlive the batch."""

    def __init__(self, forests, allocator="torch"):
        self.forests = list(forests)
        arr = (ctypes.c_void_p * len(self.forests))(*[f.h.value for f in self.forests])
        h = ctypes.c_void_p()
        self._alloc = allocator
        _check(library().lbm_batch_create(arr, len(self.forests), _allocator(allocator), ctypes.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            _check(library().lbm_batch_destroy(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n_steps=1):
        _check(library().lbm_batch_step(self.h, n_steps))

    def set_kernel_config(self, cells_per_thread_log2, ctas_per_sm):
        _check(library().lbm_batch_set_kernel_config(self.h, cells_per_thread_log2, ctas_per_sm))

    def autotune(self, n_steps=10):
        a, b, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
        _check(library().lbm_batch_autotune(self.h, n_steps, ctypes.byref(a), ctypes.byref(b), ctypes.byref(ms)))
        return a.value, b.value, ms.value

    def cell_updates_per_coarse_step(self):
        n = ctypes.c_int64()
        _check(library().lbm_batch_cell_updates_per_coarse_step(self.h, ctypes.byref(n)))
        return n.value

    def launches_per_coarse_step(self):
        n = ctypes.c_int32()
        _check(library().lbm_batch_launches_per_coarse_step(self.h, ctypes.byref(n)))
        return n.value


class Net:
    """The warm-start convolutional net (lbm_net_create ... lbm_net_destroy).  Volumes are torch
    tensors on the device: inputs BF16 [nvol, D, H, W, 16]; skip, target FP32 [nvol, D, H, W, out];
    weight FP32 [nvol, D, H, W]."""

    def __init__(self, layers=5, in_channels=6, out_channels=4, seed=20150827, stream=None, allocator="torch"):
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        h = ctypes.c_void_p()
        self._alloc = allocator
        _check(library().lbm_net_create(layers, in_channels, out_channels, seed, ctypes.c_void_p(stream),
                                        _allocator(allocator), ctypes.byref(h)))
        self.h = h
        self.layers, self.in_channels, self.out_channels = layers, in_channels, out_channels

    def close(self):
        if getattr(self, "h", None):
            _check(library().lbm_net_destroy(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_wait_test(self, on):
        _check(library().lbm_net_set_wait_test(self.h, 1 if on else 0))

    def set_backend(self, backend):
        """"tcgen05" (default) or "mma.sync" for the convolutions."""
        _check(library().lbm_net_set_backend(self.h, {"mma.sync": 0, "tcgen05": 1}[backend]))

    def num_params(self):
        n = ctypes.c_int64()
        _check(library().lbm_net_num_params(self.h, ctypes.byref(n)))
        return n.value

    def params(self):
        p = np.zeros(self.num_params(), np.float32)
        _check(library().lbm_net_get_params(self.h, p.ctypes.data))
        return p

    def set_params(self, p):
        p = np.ascontiguousarray(p, np.float32)
        assert p.size == self.num_params()
        _check(library().lbm_net_set_params(self.h, p.ctypes.data))

    def grads(self):
        p = np.zeros(self.num_params(), np.float32)
        _check(library().lbm_net_get_grads(self.h, p.ctypes.data))
        return p

    def forward(self, x):
        import torch
        nvol, D, H, W, _ = x.shape
        z = torch.empty_like(x)
        _check(library().lbm_net_forward(self.h, _ptr(x), D, H, W, nvol, _ptr(z)))
        return z

    def predict(self, x, skip=None):
        import torch
        nvol, D, H, W, _ = x.shape
        pred = torch.empty((nvol, D, H, W, self.out_channels), dtype=torch.float32, device=x.device)
        _check(library().lbm_net_predict(self.h, _ptr(x), _ptr(skip), D, H, W, nvol, _ptr(pred)))
        return pred

    def gradient(self, target, skip=None, weight=None):
        """Loss and parameter gradients of the last forward/predict call's input."""
        loss = ctypes.c_double()
        _check(library().lbm_net_gradient(self.h, _ptr(skip), _ptr(target), _ptr(weight), ctypes.byref(loss)))
        return loss.value

    def train_step(self, x, target, skip=None, weight=None, lr=1e-3):
        nvol, D, H, W, _ = x.shape
        loss = ctypes.c_double()
        _check(library().lbm_net_train_step(self.h, _ptr(x), _ptr(skip), _ptr(target), _ptr(weight), D, H, W, nvol,
                                            lr, ctypes.byref(loss)))
        return loss.value


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def warmstart_features(coarse_rho, coarse_u, coarse_blocks, B, periodic_mask, level, halo, blocks, spheres,
                       rho_scale, u_scale):
    """lbm_warmstart_features on device tensors; returns (x BF16 [n, D, D, D, 16], skip FP32 [.., 4])."""
    import torch
    nb = blocks.shape[0]
    D = B + 2 * halo
    x = torch.empty((nb, D, D, D, 16), dtype=torch.bfloat16, device="cuda")
    skip = torch.empty((nb, D, D, D, 4), dtype=torch.float32, device="cuda")
    cb = np.ascontiguousarray(coarse_blocks, np.int32)
    ns = 0 if spheres is None else int(spheres.shape[0])
    _check(library().lbm_warmstart_features(_ptr(coarse_rho), _ptr(coarse_u), cb.ctypes.data_as(
        ctypes.POINTER(ctypes.c_int32)), B, periodic_mask, level, halo, _ptr(blocks), nb, _ptr(spheres), ns,
        rho_scale, u_scale, _ptr(x), _ptr(skip), _stream()))
    return x, skip


def warmstart_targets(rho, u, B, halo, nblocks, rho_scale, u_scale):
    import torch
    D = B + 2 * halo
    target = torch.empty((nblocks, D, D, D, 4), dtype=torch.float32, device="cuda")
    weight = torch.empty((nblocks, D, D, D), dtype=torch.float32, device="cuda")
    _check(library().lbm_warmstart_targets(_ptr(rho), _ptr(u), B, halo, nblocks, rho_scale, u_scale, _ptr(target),
                                           _ptr(weight), _stream()))
    return target, weight


def warmstart_fields(pred, B, halo, nblocks, rho_scale, u_scale):
    import torch
    n = nblocks * B ** 3
    rho = torch.empty(n, dtype=torch.float64, device="cuda")
    u = torch.empty((3, n), dtype=torch.float64, device="cuda")
    _check(library().lbm_warmstart_fields(_ptr(pred), B, halo, nblocks, rho_scale, u_scale, _ptr(rho), _ptr(u),
                                          _stream()))
    return rho, u
