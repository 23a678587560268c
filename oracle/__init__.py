"""CPU FP64 oracle for AMGF-PCG -- TEST INFRASTRUCTURE ONLY.

Only tests/, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The GPU library never loads it, and it
never loads the GPU library; the two share only the seeded inputs of
``contactgen``.

The arithmetic lives in ``oracle.c`` (plain C loops in double precision, one
function per step of the method, each citing the paper's section or equation).
This module compiles it in place (``liboracle.so``) and wraps it with ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None

STATUS = {0: "OK", 1: "INVALID_ARG", 2: "NONFINITE", 3: "NOT_SPD", 4: "BREAKDOWN",
          5: "NOT_CONVERGED", 6: "CUDA", 7: "OOM"}


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (in place)."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class Opts(ctypes.Structure):
    _fields_ = [("strength_theta", ctypes.c_double), ("max_coarse", ctypes.c_int),
                ("max_levels", ctypes.c_int), ("num_functions", ctypes.c_int),
                ("nu", ctypes.c_int), ("filter", ctypes.c_int),
                ("contact_components", ctypes.c_int), ("build_amg", ctypes.c_int),
                ("interp", ctypes.c_int), ("p_max", ctypes.c_int), ("smoother", ctypes.c_int),
                ("cheby_lower", ctypes.c_double), ("hier_from_K", ctypes.c_int)]


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_SO)
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    lib.orc_opts_default.argtypes = [vp]
    lib.orc_create.argtypes = [i64, vp, vp, vp, i64, vp, vp, vp, vp, vp, vp]
    lib.orc_create.restype = i32
    lib.orc_create_bounds.argtypes = [i64, vp, vp, vp, i64, vp, vp, vp, vp, vp, vp, vp]
    lib.orc_create_bounds.restype = i32
    lib.orc_free.argtypes = [vp]
    lib.orc_error.argtypes = [vp]
    lib.orc_error.restype = ctypes.c_char_p
    for f in ("orc_S_apply", "orc_vcycle", "orc_filter_solve", "orc_apply"):
        getattr(lib, f).argtypes = [vp, vp, vp]
    lib.orc_pcg.argtypes = [vp, vp, vp, ctypes.c_double, i32, vp, vp, vp, vp]
    lib.orc_pcg.restype = i32
    lib.orc_num_levels.argtypes = [vp]
    lib.orc_num_levels.restype = i32
    for f in ("orc_n", "orc_nc", "orc_bandwidth"):
        getattr(lib, f).argtypes = [vp]
        getattr(lib, f).restype = i64
    lib.orc_get_Ic.argtypes = [vp, vp]
    lib.orc_mat_shape.argtypes = [vp, i32, i32, vp, vp, vp]
    lib.orc_mat_shape.restype = i32
    lib.orc_mat_get.argtypes = [vp, i32, i32, vp, vp, vp]
    lib.orc_mat_get.restype = i32
    for f in ("orc_get_cf", "orc_get_l1", "orc_get_func", "orc_get_theta"):
        getattr(lib, f).argtypes = [vp, i32, vp]
        getattr(lib, f).restype = i32
    lib.orc_set_mlp.argtypes = [vp, vp, i64]
    lib.orc_set_mlp.restype = i32
    lib.orc_mlp_loss.argtypes = [vp, vp, vp]
    lib.orc_mlp_loss.restype = i32
    lib.orc_set_threads.argtypes = [i32]
    lib.orc_set_threads.restype = i32
    _lib = lib
    return lib


def _p(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


class OracleError(RuntimeError):
    def __init__(self, status, msg=""):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def default_opts(**kw) -> Opts:
    o = Opts()
    _load().orc_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class Oracle:
    """AMGF (or plain AMG) preconditioner and PCG for A = K + J^T D J, on the CPU in FP64.

    K, J: (row_ptr int64, col_idx int32, val float64) host CSR triples (or objects
    with those attributes); D: barrier diagonal of length m (m may be 0); E: optional
    diagonal D_lo + D_hi of the bound-constraint variant (length n, >= 0), added to A.
    """

    def __init__(self, K, J=None, D=None, E=None, **opts):
        lib = _load()
        self._lib = lib
        self._h = ctypes.c_void_p()
        rp, ci, v = (np.ascontiguousarray(K.row_ptr, np.int64), np.ascontiguousarray(K.col_idx, np.int32),
                     np.ascontiguousarray(K.val, np.float64))
        n = len(rp) - 1
        if J is not None and J.nrows > 0:
            jrp, jci, jv = (np.ascontiguousarray(J.row_ptr, np.int64), np.ascontiguousarray(J.col_idx, np.int32),
                            np.ascontiguousarray(J.val, np.float64))
            m = len(jrp) - 1
            Dv = np.ascontiguousarray(D, np.float64)
        else:
            jrp = np.zeros(1, np.int64); jci = np.zeros(1, np.int32); jv = np.zeros(1); m = 0
            Dv = np.zeros(1)
        Ev = None if E is None else np.ascontiguousarray(E, np.float64)
        self._keep = (rp, ci, v, jrp, jci, jv, Dv, Ev)
        self.opts = default_opts(**opts)
        st = lib.orc_create_bounds(n, _p(rp), _p(ci), _p(v), m, _p(jrp), _p(jci), _p(jv), _p(Dv),
                                   None if Ev is None else _p(Ev), ctypes.byref(self.opts), ctypes.byref(self._h))
        if st != 0:
            msg = lib.orc_error(self._h).decode() if self._h else ""
            self.close()
            raise OracleError(st, msg)
        self.n = n
        self.m = m

    def close(self):
        if getattr(self, "_h", None):
            self._lib.orc_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- operators -------------------------------------------------------
    def S_apply(self, x):
        x = np.ascontiguousarray(x, np.float64); y = np.empty(self.n)
        self._lib.orc_S_apply(self._h, _p(x), _p(y)); return y

    def vcycle(self, r):
        r = np.ascontiguousarray(r, np.float64); x = np.empty(self.n)
        self._lib.orc_vcycle(self._h, _p(r), _p(x)); return x

    def apply(self, r):
        r = np.ascontiguousarray(r, np.float64); z = np.empty(self.n)
        self._lib.orc_apply(self._h, _p(r), _p(z)); return z

    def filter_solve(self, v):
        v = np.ascontiguousarray(v, np.float64); w = np.empty(self.nc)
        self._lib.orc_filter_solve(self._h, _p(v), _p(w)); return w

    def pcg(self, b, x0=None, tol=1e-8, maxit=5000):
        """Returns (x, iters, status, alphas, betas, relres)."""
        b = np.ascontiguousarray(b, np.float64)
        x = np.zeros(self.n) if x0 is None else np.array(x0, np.float64)
        al = np.zeros(maxit); be = np.zeros(maxit); rr = np.zeros(maxit + 1)
        it = ctypes.c_int(0)
        st = self._lib.orc_pcg(self._h, _p(b), _p(x), tol, maxit, ctypes.byref(it), _p(al), _p(be), _p(rr))
        k = it.value
        return x, k, st, al[:k], be[:k], rr[:k + 1]

    # --- introspection ---------------------------------------------------
    @property
    def nlev(self):
        return self._lib.orc_num_levels(self._h)

    @property
    def nc(self):
        return int(self._lib.orc_nc(self._h))

    @property
    def bandwidth(self):
        return int(self._lib.orc_bandwidth(self._h))

    def Ic(self):
        out = np.empty(self.nc, np.int64)
        self._lib.orc_get_Ic(self._h, _p(out)); return out

    def _mat(self, which, l):
        nr, nc_, nnz = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        if self._lib.orc_mat_shape(self._h, which, l, ctypes.byref(nr), ctypes.byref(nc_), ctypes.byref(nnz)):
            raise IndexError(l)
        rp = np.empty(nr.value + 1, np.int64); ci = np.empty(nnz.value, np.int32); v = np.empty(nnz.value)
        self._lib.orc_mat_get(self._h, which, l, _p(rp), _p(ci), _p(v))
        import scipy.sparse as sp
        return sp.csr_matrix((v, ci, rp), shape=(nr.value, nc_.value))

    def A(self, l):
        return self._mat(0, l)

    def P(self, l):
        return self._mat(1, l)

    def R(self, l):
        return self._mat(2, l)

    def S(self):
        return self._mat(3, 0)

    def cf(self, l):
        out = np.empty(self.A(l).shape[0], np.int8)
        if self._lib.orc_get_cf(self._h, l, _p(out)):
            raise IndexError(l)
        return out

    def l1(self, l):
        out = np.empty(self.A(l).shape[0])
        self._lib.orc_get_l1(self._h, l, _p(out)); return out

    def set_mlp(self, w):
        """Learned smoother weights (1313 values; None clears them: theta = 1)."""
        if w is None:
            self._lib.orc_set_mlp(self._h, None, 0)
            return
        w = np.ascontiguousarray(w, np.float64)
        self._mlp_w = w
        st = self._lib.orc_set_mlp(self._h, _p(w), len(w))
        if st:
            raise OracleError(st, "set_mlp")

    def mlp_loss(self, r_all):
        """Mean over the smoothed levels of ||(I - A_l W_l) r_l||^2 / ||r_l||^2 with the active
        weights; r_all holds the per-level vectors back to back (every level but the coarsest)."""
        r = np.ascontiguousarray(r_all, np.float64)
        out = ctypes.c_double()
        st = self._lib.orc_mlp_loss(self._h, _p(r), ctypes.byref(out))
        if st:
            raise OracleError(st, "mlp_loss")
        return out.value

    def theta(self, l):
        out = np.empty(self.A(l).shape[0])
        if self._lib.orc_get_theta(self._h, l, _p(out)):
            raise IndexError(l)
        return out

    def func(self, l):
        out = np.empty(self.A(l).shape[0], np.int32)
        self._lib.orc_get_func(self._h, l, _p(out)); return out


def set_threads(k: int) -> int:
    """Threads of the oracle's parallel loops (k <= 0 leaves them); returns the previous count."""
    return int(_load().orc_set_threads(int(k)))
