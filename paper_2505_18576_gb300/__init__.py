"""GB300 AMGF-PCG: Python binding of the C ABI in include/amgf.h.

Argument marshalling only: every step of the solve runs in libamgf.so's CUDA
kernels.  Device vectors are passed as torch CUDA tensors (float64, contiguous)
or raw integer device pointers; PyTorch is used for device memory and streams.
There is no CPU fallback: importing works without a GPU, but every call that
needs the device raises AmgfError when libamgf.so cannot reach one.

Function names are those of the C ABI (amgf_setup, amgf_apply, amgf_pcg_solve,
...); ``Solver`` is a small object wrapper around a handle.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB as _LIB_PATH, build as _build

__all__ = ["AmgfError", "Options", "Stats", "Info", "Solver", "load_library", "amgf_options_default",
           "amgf_setup", "amgf_setup_host", "amgf_update_D", "amgf_apply", "amgf_vcycle", "amgf_matvec", "amgf_filter_solve",
           "amgf_filter_solve_noalloc", "amgf_filter_solve_host", "amgf_pcg_solve", "amgf_pcg_solve_host", "amgf_get_info", "amgf_export_matrix",
           "amgf_export_contact_set", "amgf_time_kernel", "amgf_destroy", "amgf_last_error", "EXPORTED",
           "amgf_setup_bounds", "amgf_update_bounds", "amgf_update_D_fine", "amgf_apply_stages", "amgf_mlp_grad",
           "amgf_profile_iteration"]

EXPORTED = ["amgf_options_default", "amgf_setup", "amgf_setup_host", "amgf_setup_bounds", "amgf_update_D",
            "amgf_update_bounds", "amgf_update_D_fine", "amgf_apply", "amgf_vcycle", "amgf_matvec",
            "amgf_filter_solve", "amgf_filter_solve_noalloc", "amgf_filter_solve_host", "amgf_pcg_solve",
            "amgf_pcg_solve_host",
            "amgf_get_info",
            "amgf_export_matrix", "amgf_export_contact_set", "amgf_time_kernel", "amgf_destroy",
            "amgf_last_error", "amgf_set_mlp", "amgf_mlp_train", "amgf_apply_stages", "amgf_mlp_grad",
            "amgf_profile_iteration"]

STATUS = {0: "OK", 1: "INVALID_ARG", 2: "NONFINITE", 3: "NOT_SPD", 4: "BREAKDOWN", 5: "NOT_CONVERGED",
          6: "CUDA", 7: "OOM"}


class AmgfError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Csr(ctypes.Structure):
    _fields_ = [("nrows", ctypes.c_int64), ("ncols", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class Options(ctypes.Structure):
    _fields_ = [("strength_theta", ctypes.c_double), ("rtol", ctypes.c_double),
                ("max_levels", ctypes.c_int), ("max_coarse", ctypes.c_int), ("num_functions", ctypes.c_int),
                ("nu", ctypes.c_int), ("filter", ctypes.c_int), ("contact_components", ctypes.c_int),
                ("maxit", ctypes.c_int), ("use_graph", ctypes.c_int), ("verbose", ctypes.c_int),
                ("precision", ctypes.c_int), ("filter_algo", ctypes.c_int),
                ("interp", ctypes.c_int), ("p_max", ctypes.c_int), ("update_in_place", ctypes.c_int),
                ("smoother", ctypes.c_int), ("cheby_lower", ctypes.c_double),
                ("stage_rows", ctypes.c_int), ("stage_depth", ctypes.c_int), ("sell_window", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("converged", ctypes.c_int), ("status", ctypes.c_int),
                ("nlevels", ctypes.c_int), ("rel_res_precond", ctypes.c_double), ("rz0", ctypes.c_double),
                ("t_solve_s", ctypes.c_double), ("kernel_launches", ctypes.c_int64),
                ("mlp_fallback", ctypes.c_int), ("rel_res_l2", ctypes.c_double), ("t_setup_s", ctypes.c_double)]


class LaunchRec(ctypes.Structure):
    _fields_ = [("op", ctypes.c_char * 64), ("level", ctypes.c_int), ("ms", ctypes.c_double),
                ("bytes", ctypes.c_double), ("flops", ctypes.c_double)]


class Info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("m", ctypes.c_int64), ("nc", ctypes.c_int64), ("nlevels", ctypes.c_int),
                ("level_rows", ctypes.c_int64 * 32), ("level_nnz", ctypes.c_int64 * 32),
                ("interp_nnz", ctypes.c_int64 * 32), ("filter_block", ctypes.c_int64),
                ("filter_nblocks", ctypes.c_int64), ("op_complexity", ctypes.c_double),
                ("t_setup_s", ctypes.c_double), ("t_assemble_s", ctypes.c_double),
                ("t_hierarchy_s", ctypes.c_double), ("t_filter_s", ctypes.c_double),
                ("staged_levels", ctypes.c_int64), ("sell_levels", ctypes.c_int64)]


_lib = None


def load_library(build_if_missing: bool = True):
    """Load libamgf.so (compiling it in place when missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build()
    if not os.path.exists(_LIB_PATH):
        raise AmgfError(6, f"{_LIB_PATH} is missing: build it with paper_2505_18576_gb300.build.build()")
    lib = ctypes.CDLL(_LIB_PATH)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
    sig = {
        "amgf_options_default": [vp],
        "amgf_setup": [vp, vp, vp, vp, vp],
        "amgf_setup_host": [vp, vp, vp, vp, vp],
        "amgf_setup_bounds": [vp, vp, vp, vp, vp, vp, i32, vp],
        "amgf_update_D": [vp, vp],
        "amgf_update_bounds": [vp, vp, vp, vp],
        "amgf_update_D_fine": [vp, vp],
        "amgf_apply": [vp, vp, vp, vp],
        "amgf_apply_stages": [vp, vp, vp, vp, vp, vp, vp, vp],
        "amgf_vcycle": [vp, vp, vp, vp],
        "amgf_matvec": [vp, vp, vp, vp],
        "amgf_filter_solve": [vp, vp, vp, vp],
        "amgf_filter_solve_noalloc": [vp, vp, vp, vp],
        "amgf_filter_solve_host": [vp, vp, vp],
        "amgf_pcg_solve": [vp, vp, vp, vp, vp],
        "amgf_pcg_solve_host": [vp, vp, vp, vp],
        "amgf_get_info": [vp, vp],
        "amgf_export_matrix": [vp, i32, i32, vp, vp, vp, vp, vp, vp],
        "amgf_export_contact_set": [vp, vp],
        "amgf_time_kernel": [vp, i32, i32, i32, vp, vp, vp],
        "amgf_destroy": [vp],
        "amgf_set_mlp": [vp, vp, i64],
        "amgf_mlp_train": [vp, vp, vp, vp, vp, i32, ctypes.c_float, ctypes.c_uint64, vp],
        "amgf_mlp_grad": [vp, vp, vp, vp, vp],
        "amgf_profile_iteration": [vp, vp, vp, i32, vp],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = i32
    lib.amgf_last_error.argtypes = []
    lib.amgf_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def amgf_last_error() -> str:
    return load_library().amgf_last_error().decode()


def _check(st: int):
    if st != 0:
        raise AmgfError(st, amgf_last_error())


def _ptr(t) -> ctypes.c_void_p:
    """Device or host pointer of a torch tensor / numpy array / int."""
    if t is None:
        return ctypes.c_void_p(0)
    if isinstance(t, int):
        return ctypes.c_void_p(t)
    if isinstance(t, np.ndarray):
        return ctypes.c_void_p(t.ctypes.data)
    return ctypes.c_void_p(t.data_ptr())


def _dev_vec(t, n: int, name: str):
    if isinstance(t, int):
        return ctypes.c_void_p(t)
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise AmgfError(1, f"{name}: expected a contiguous float64 CUDA tensor")
    if t.numel() != n:
        raise AmgfError(1, f"{name}: expected {n} entries, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def amgf_options_default(**overrides) -> Options:
    o = Options()
    _check(load_library().amgf_options_default(ctypes.byref(o)))
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


def _csr(mat, keep: list) -> Csr:
    rp = np.ascontiguousarray(mat.row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(mat.col_idx, dtype=np.int32)
    v = np.ascontiguousarray(mat.val, dtype=np.float64)
    keep += [rp, ci, v]
    ncols = getattr(mat, "ncols", None)
    if ncols is None:
        ncols = mat.shape[1]
    return Csr(len(rp) - 1, int(ncols), int(rp[-1]), rp.ctypes.data, ci.ctypes.data, v.ctypes.data)


def amgf_setup(K, J=None, D=None, opts: Options | None = None, host_only: bool = False) -> ctypes.c_void_p:
    """Host CSR K (n x n), J (m x n, optional), D (m) -> handle (c_void_p).

    host_only=True calls amgf_setup_host (hierarchy only, no device)."""
    lib = load_library()
    keep: list = []
    k = _csr(K, keep)
    j = _csr(J, keep) if J is not None else None
    d = np.ascontiguousarray(D, dtype=np.float64) if D is not None else None
    h = ctypes.c_void_p()
    fn = lib.amgf_setup_host if host_only else lib.amgf_setup
    _check(fn(ctypes.byref(k), ctypes.byref(j) if j is not None else None,
                          _ptr(d) if d is not None else None, ctypes.byref(opts) if opts else None,
                          ctypes.byref(h)))
    return h


def amgf_setup_bounds(K, J, D, d_lower, d_upper, opts: Options | None = None, host_only: bool = False):
    """Bound-constrained variant A = K + J^T D J + diag(d_lower + d_upper) -> handle."""
    lib = load_library()
    keep: list = []
    k = _csr(K, keep)
    j = _csr(J, keep) if J is not None else None
    d = np.ascontiguousarray(D, dtype=np.float64) if D is not None else None
    lo = np.ascontiguousarray(d_lower, dtype=np.float64) if d_lower is not None else None
    hi = np.ascontiguousarray(d_upper, dtype=np.float64) if d_upper is not None else None
    h = ctypes.c_void_p()
    _check(lib.amgf_setup_bounds(ctypes.byref(k), ctypes.byref(j) if j is not None else None,
                                 _ptr(d) if d is not None else None, _ptr(lo) if lo is not None else None,
                                 _ptr(hi) if hi is not None else None, ctypes.byref(opts) if opts else None,
                                 1 if host_only else 0, ctypes.byref(h)))
    return h


def amgf_update_bounds(h, D, d_lower, d_upper):
    d = np.ascontiguousarray(D, dtype=np.float64) if D is not None else None
    lo = np.ascontiguousarray(d_lower, dtype=np.float64) if d_lower is not None else None
    hi = np.ascontiguousarray(d_upper, dtype=np.float64) if d_upper is not None else None
    _check(load_library().amgf_update_bounds(h, _ptr(d) if d is not None else None,
                                             _ptr(lo) if lo is not None else None,
                                             _ptr(hi) if hi is not None else None))


def amgf_update_D_fine(h, D):
    """New D with the coarse levels of B kept from the last full setup (lagged hierarchy)."""
    d = np.ascontiguousarray(D, dtype=np.float64)
    _check(load_library().amgf_update_D_fine(h, _ptr(d)))


def amgf_update_D(h, D):
    d = np.ascontiguousarray(D, dtype=np.float64)
    _check(load_library().amgf_update_D(h, _ptr(d)))


def amgf_apply(h, r, z, n: int, stream=None):
    _check(load_library().amgf_apply(h, _dev_vec(r, n, "r"), _dev_vec(z, n, "z"), _stream(stream)))


def amgf_apply_stages(h, r, z, n: int, nc: int, y1=None, r1=None, w=None, r2=None, stream=None):
    """amgf_apply that also copies y1 = B r, r1 = r - A y1, w = A_w^{-1} P^T r1 and r2 = r1 - A P w."""
    _check(load_library().amgf_apply_stages(
        h, _dev_vec(r, n, "r"), _dev_vec(z, n, "z"), None if y1 is None else _dev_vec(y1, n, "y1"),
        None if r1 is None else _dev_vec(r1, n, "r1"), None if w is None else _dev_vec(w, nc, "w"),
        None if r2 is None else _dev_vec(r2, n, "r2"), _stream(stream)))


def amgf_vcycle(h, r, x, n: int, stream=None):
    _check(load_library().amgf_vcycle(h, _dev_vec(r, n, "r"), _dev_vec(x, n, "x"), _stream(stream)))


def amgf_matvec(h, x, y, n: int, stream=None):
    _check(load_library().amgf_matvec(h, _dev_vec(x, n, "x"), _dev_vec(y, n, "y"), _stream(stream)))


def amgf_filter_solve(h, v, w, nc: int, stream=None):
    _check(load_library().amgf_filter_solve(h, _dev_vec(v, nc, "v"), _dev_vec(w, nc, "w"), _stream(stream)))


def amgf_filter_solve_host(h, v: np.ndarray) -> np.ndarray:
    """w = A_w^{-1} v on the host (handles of amgf_setup_host), v in ascending-DOF order of I_c."""
    v = np.ascontiguousarray(v, dtype=np.float64)
    w = np.empty_like(v)
    _check(load_library().amgf_filter_solve_host(h, _ptr(v), _ptr(w)))
    return w


def amgf_filter_solve_noalloc(h, v, w, nc: int, stream=None):
    """amgf_filter_solve with its work vectors in the library's fixed array (allocates nothing)."""
    _check(load_library().amgf_filter_solve_noalloc(h, _dev_vec(v, nc, "v"), _dev_vec(w, nc, "w"),
                                                     _stream(stream)))


def amgf_pcg_solve(h, b, x, n: int, stream=None, check: bool = True) -> Stats:
    st = Stats()
    rc = load_library().amgf_pcg_solve(h, _dev_vec(b, n, "b"), _dev_vec(x, n, "x"), ctypes.byref(st),
                                       _stream(stream))
    if check and rc not in (0,):
        _check(rc)
    st.rc = rc
    return st


def amgf_pcg_solve_host(h, b: np.ndarray, x: np.ndarray, check: bool = True) -> Stats:
    assert b.dtype == np.float64 and x.dtype == np.float64 and b.flags.c_contiguous and x.flags.c_contiguous
    st = Stats()
    rc = load_library().amgf_pcg_solve_host(h, _ptr(b), _ptr(x), ctypes.byref(st))
    if check and rc != 0:
        _check(rc)
    st.rc = rc
    return st


def amgf_get_info(h) -> Info:
    info = Info()
    _check(load_library().amgf_get_info(h, ctypes.byref(info)))
    return info


def amgf_export_matrix(h, which: int, level: int):
    """(row_ptr, col_idx, val, shape) of A_l (which=0), P_l (1) or R_l (2)."""
    lib = load_library()
    nr, nc, nnz = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib.amgf_export_matrix(h, which, level, ctypes.byref(nr), ctypes.byref(nc), ctypes.byref(nnz),
                                  None, None, None))
    rp = np.empty(nr.value + 1, np.int64); ci = np.empty(nnz.value, np.int32); v = np.empty(nnz.value)
    _check(lib.amgf_export_matrix(h, which, level, ctypes.byref(nr), ctypes.byref(nc), ctypes.byref(nnz),
                                  _ptr(rp), _ptr(ci), _ptr(v)))
    return rp, ci, v, (nr.value, nc.value)


def amgf_export_contact_set(h, nc: int) -> np.ndarray:
    out = np.empty(max(nc, 1), np.int64)
    _check(load_library().amgf_export_contact_set(h, _ptr(out)))
    return out[:nc]


def amgf_time_kernel(h, which: int, warmup: int, reps: int, stream=None):
    ms, by = ctypes.c_double(), ctypes.c_double()
    _check(load_library().amgf_time_kernel(h, which, warmup, reps, _stream(stream), ctypes.byref(ms),
                                           ctypes.byref(by)))
    return ms.value, by.value


def amgf_set_mlp(h, weights):
    """Activate learned smoother weights (1313 floats) or restore theta = 1 (None)."""
    if weights is None:
        _check(load_library().amgf_set_mlp(h, None, 0))
        return
    w = np.ascontiguousarray(weights, dtype=np.float32)
    _check(load_library().amgf_set_mlp(h, _ptr(w), len(w)))


def amgf_mlp_train(h, params, adam_m, adam_v, adam_step, iters: int, lr: float, seed: int):
    """Adam steps on the smoother MLP for this handle's hierarchy; updates the float32 arrays in
    place and returns (new adam_step, losses)."""
    for a in (params, adam_m, adam_v):
        assert a.dtype == np.float32 and a.flags.c_contiguous and len(a) == 1313
    step = ctypes.c_int64(adam_step)
    loss = np.zeros(max(iters, 1), np.float32)
    _check(load_library().amgf_mlp_train(h, _ptr(params), _ptr(adam_m), _ptr(adam_v), ctypes.byref(step), iters,
                                         lr, seed, _ptr(loss)))
    return step.value, loss[:iters]


def amgf_mlp_grad(h, params, r_all):
    """(loss, gradient) of the training objective for weights `params` and the concatenated
    per-level vectors r_all (every level but the coarsest)."""
    w = np.ascontiguousarray(params, dtype=np.float32)
    r = np.ascontiguousarray(r_all, dtype=np.float64)
    assert len(w) == 1313
    g = np.zeros(1313, np.float32)
    loss = ctypes.c_double()
    _check(load_library().amgf_mlp_grad(h, _ptr(w), _ptr(r), _ptr(g), ctypes.byref(loss)))
    return loss.value, g


def amgf_profile_iteration(h, stream=None, cap: int = 4096):
    """Per-launch records of one PCG iteration: list of dicts (op, level, ms, bytes, flops)."""
    recs = (LaunchRec * cap)()
    n = ctypes.c_int()
    _check(load_library().amgf_profile_iteration(h, _stream(stream), recs, cap, ctypes.byref(n)))
    return [{"op": r.op.decode(), "level": r.level, "ms": r.ms, "bytes": r.bytes, "flops": r.flops}
            for r in recs[:min(n.value, cap)]]


def amgf_destroy(h):
    if h:
        load_library().amgf_destroy(h)


class Solver:
    """Owns one handle.  K, J: CSR objects with row_ptr/col_idx/val (contactgen.CSR works)."""

    def __init__(self, K, J=None, D=None, host_only=False, d_lower=None, d_upper=None, **opts):
        self.opts = amgf_options_default(**opts)
        if d_lower is not None or d_upper is not None:
            self.h = amgf_setup_bounds(K, J, D, d_lower, d_upper, self.opts, host_only=host_only)
        else:
            self.h = amgf_setup(K, J, D, self.opts, host_only=host_only)
        self.info = amgf_get_info(self.h)
        self.n = int(self.info.n)
        self.nc = int(self.info.nc)

    def close(self):
        if getattr(self, "h", None):
            amgf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def update_bounds(self, D, d_lower, d_upper):
        amgf_update_bounds(self.h, D, d_lower, d_upper)
        self.info = amgf_get_info(self.h)

    def update_D(self, D, keep_coarse: bool = False):
        (amgf_update_D_fine if keep_coarse else amgf_update_D)(self.h, D)
        self.info = amgf_get_info(self.h)

    def apply(self, r, z, stream=None):
        amgf_apply(self.h, r, z, self.n, stream)

    def apply_stages(self, r, z, y1=None, r1=None, w=None, r2=None, stream=None):
        amgf_apply_stages(self.h, r, z, self.n, self.nc, y1, r1, w, r2, stream)

    def mlp_grad(self, params, r_all):
        return amgf_mlp_grad(self.h, params, r_all)

    def profile_iteration(self, stream=None):
        return amgf_profile_iteration(self.h, stream)

    def vcycle(self, r, x, stream=None):
        amgf_vcycle(self.h, r, x, self.n, stream)

    def matvec(self, x, y, stream=None):
        amgf_matvec(self.h, x, y, self.n, stream)

    def filter_solve(self, v, w, stream=None):
        amgf_filter_solve(self.h, v, w, self.nc, stream)

    def pcg_solve(self, b, x, stream=None, check=True) -> Stats:
        return amgf_pcg_solve(self.h, b, x, self.n, stream, check)

    def pcg_solve_host(self, b, x, check=True) -> Stats:
        return amgf_pcg_solve_host(self.h, b, x, check)

    def export(self, which: int, level: int):
        import scipy.sparse as sp
        rp, ci, v, shape = amgf_export_matrix(self.h, which, level)
        return sp.csr_matrix((v, ci, rp), shape=shape)

    def contact_set(self):
        return amgf_export_contact_set(self.h, self.nc)

    def set_mlp(self, weights):
        amgf_set_mlp(self.h, weights)

    def time_kernel(self, which: int, warmup: int = 3, reps: int = 20, stream=None):
        return amgf_time_kernel(self.h, which, warmup, reps, stream)
