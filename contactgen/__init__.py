"""Seeded synthetic two-block contact problems (inputs only).

Produces K (Q1 linear elasticity on two stacked blocks), J (node-to-node normal
contact on the shared interface), the barrier diagonal D and a right-hand side
b: the data of the condensed interior-point Newton system A u = b with
A = K + J^T D J (Section 3, eq. (linsystem1)).  No solver arithmetic lives here;
both the CPU oracle and the GPU library consume these arrays.

The C source ``gen.c`` is compiled in place into ``libcontactgen.so`` on first
use (or by ``build()``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_SO = os.path.join(_HERE, "libcontactgen.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile gen.c into libcontactgen.so (in place)."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_SO)
    i64, vp = ctypes.c_int64, ctypes.c_void_p
    lib.cg_num_nodes.restype = i64
    lib.cg_num_dofs.restype = i64
    lib.cg_num_constraints.restype = i64
    lib.cg_K_rowptr.restype = i64
    lib.cg_J_fill.restype = i64
    for f in ("cg_num_nodes", "cg_num_dofs", "cg_num_constraints"):
        getattr(lib, f).argtypes = [vp]
    lib.cg_K_rowptr.argtypes = [vp, vp]
    lib.cg_K_fill.argtypes = [vp, vp, vp, vp]
    lib.cg_J_fill.argtypes = [vp, vp, vp, vp]
    lib.cg_node_xyz.argtypes = [vp, vp]
    lib.cg_element_stiffness.argtypes = [ctypes.c_double] * 5 + [vp]
    lib.cg_rng_raw.argtypes = [ctypes.c_uint64, i64, vp]
    lib.cg_splitmix_raw.argtypes = [ctypes.c_uint64, i64, vp]
    lib.cg_xoshiro_from_state.argtypes = [vp, i64, vp]
    lib.cg_draw_D_b.argtypes = [ctypes.c_uint64, i64, ctypes.c_double, ctypes.c_double, vp, i64, vp]
    _lib = lib
    return lib


class _Geom(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("clamp_bottom", ctypes.c_int), ("clamp_top", ctypes.c_int),
                ("E", ctypes.c_double), ("nu", ctypes.c_double)]


def _p(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


@dataclass
class CSR:
    """Host CSR matrix: int64 row pointers, int32 column indices, float64 values."""
    nrows: int
    ncols: int
    row_ptr: np.ndarray
    col_idx: np.ndarray
    val: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.col_idx, self.row_ptr), shape=(self.nrows, self.ncols))


# Workloads: elements per block (nx, ny, nz) and log10 range of D.
CONFIGS = {
    "tiny": dict(nx=8, ny=8, nz=4, d_lo=-2.0, d_hi=4.0),
    "c64": dict(nx=64, ny=64, nz=32, d_lo=-2.0, d_hi=8.0),
    "c96": dict(nx=96, ny=96, nz=48, d_lo=-2.0, d_hi=10.0),
    "c160": dict(nx=160, ny=160, nz=80, d_lo=-2.0, d_hi=12.0),
    "c202": dict(nx=202, ny=202, nz=101, d_lo=-2.0, d_hi=12.0),
}


@dataclass
class Problem:
    nx: int
    ny: int
    nz: int
    n: int
    m: int
    K: CSR
    J: CSR
    D: np.ndarray
    b: np.ndarray
    meta: dict = field(default_factory=dict)


def _geom(nx, ny, nz, clamp_bottom=True, clamp_top=True, E=1.0, nu=0.3):
    return _Geom(nx, ny, nz, int(clamp_bottom), int(clamp_top), E, nu)


def sizes(nx, ny, nz, clamp_bottom=True, clamp_top=True):
    lib = _load()
    g = _geom(nx, ny, nz, clamp_bottom, clamp_top)
    return int(lib.cg_num_dofs(ctypes.byref(g))), int(lib.cg_num_constraints(ctypes.byref(g)))


def stiffness(nx, ny, nz, clamp_bottom=True, clamp_top=True, E=1.0, nu=0.3) -> CSR:
    lib = _load()
    g = _geom(nx, ny, nz, clamp_bottom, clamp_top, E, nu)
    n = int(lib.cg_num_dofs(ctypes.byref(g)))
    rp = np.zeros(n + 1, dtype=np.int64)
    nnz = int(lib.cg_K_rowptr(ctypes.byref(g), _p(rp)))
    col = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz, dtype=np.float64)
    lib.cg_K_fill(ctypes.byref(g), _p(rp), _p(col), _p(val))
    return CSR(n, n, rp, col, val)


def contact_jacobian(nx, ny, nz, clamp_bottom=True, clamp_top=True) -> CSR:
    lib = _load()
    g = _geom(nx, ny, nz, clamp_bottom, clamp_top)
    n = int(lib.cg_num_dofs(ctypes.byref(g)))
    m = int(lib.cg_num_constraints(ctypes.byref(g)))
    rp = np.zeros(m + 1, dtype=np.int64)
    col = np.empty(2 * m, dtype=np.int32)
    val = np.empty(2 * m, dtype=np.float64)
    lib.cg_J_fill(ctypes.byref(g), _p(rp), _p(col), _p(val))
    return CSR(m, n, rp, col, val)


def contact_jacobian_curved(nx, ny, nz, curvature: float, clamp_bottom=True, clamp_top=True) -> CSR:
    """Node-to-node contact on an interface with tilted normals: row r constrains
    n_r . (u_upper - u_lower) for the node pair of row r of contact_jacobian, with the unit
    normal of the surface z = curvature ((x - 1/2)^2 + (y - 1/2)^2) at the pair's (x, y),
    n ~ (-2 c (x - 1/2), -2 c (y - 1/2), 1).  Six nonzeros per row (all displacement
    components of both nodes); curvature = 0 gives the z-only rows of contact_jacobian."""
    J0 = contact_jacobian(nx, ny, nz, clamp_bottom, clamp_top)
    xyz = node_xyz(nx, ny, nz, clamp_bottom, clamp_top)
    m = J0.nrows
    rp = np.arange(m + 1, dtype=np.int64) * 6
    col = np.empty(6 * m, dtype=np.int32)
    val = np.empty(6 * m, dtype=np.float64)
    for r in range(m):
        k0, k1 = J0.row_ptr[r], J0.row_ptr[r + 1]
        cols, vals = J0.col_idx[k0:k1], J0.val[k0:k1]
        up = int(cols[vals > 0][0]) // 3
        lo = int(cols[vals < 0][0]) // 3
        x, y = xyz[up, 0], xyz[up, 1]
        nrm = np.array([-2.0 * curvature * (x - 0.5), -2.0 * curvature * (y - 0.5), 1.0])
        nrm /= np.linalg.norm(nrm)
        a, b = (lo, up) if lo < up else (up, lo)
        sa = -1.0 if a == lo else 1.0
        for t, (node, sg) in enumerate(((a, sa), (b, -sa))):
            col[6 * r + 3 * t:6 * r + 3 * t + 3] = 3 * node + np.arange(3)
            val[6 * r + 3 * t:6 * r + 3 * t + 3] = sg * nrm
    return CSR(m, J0.ncols, rp, col, val)


def node_xyz(nx, ny, nz, clamp_bottom=True, clamp_top=True) -> np.ndarray:
    lib = _load()
    g = _geom(nx, ny, nz, clamp_bottom, clamp_top)
    nn = int(lib.cg_num_nodes(ctypes.byref(g)))
    xyz = np.empty(3 * nn, dtype=np.float64)
    lib.cg_node_xyz(ctypes.byref(g), _p(xyz))
    return xyz.reshape(nn, 3)


def element_stiffness(hx, hy, hz, E=1.0, nu=0.3) -> np.ndarray:
    lib = _load()
    Ke = np.empty(24 * 24, dtype=np.float64)
    lib.cg_element_stiffness(hx, hy, hz, E, nu, _p(Ke))
    return Ke.reshape(24, 24)


def rng_raw(seed: int, count: int) -> np.ndarray:
    lib = _load()
    out = np.empty(count, dtype=np.uint64)
    lib.cg_rng_raw(seed, count, _p(out))
    return out


def splitmix_raw(seed: int, count: int) -> np.ndarray:
    lib = _load()
    out = np.empty(count, dtype=np.uint64)
    lib.cg_splitmix_raw(seed, count, _p(out))
    return out


def xoshiro_from_state(state, count: int) -> np.ndarray:
    lib = _load()
    st = np.ascontiguousarray(state, dtype=np.uint64)
    out = np.empty(count, dtype=np.uint64)
    lib.cg_xoshiro_from_state(_p(st), count, _p(out))
    return out


def draw_D_b(seed: int, m: int, n: int, d_lo: float, d_hi: float):
    lib = _load()
    D = np.empty(m, dtype=np.float64)
    b = np.empty(n, dtype=np.float64)
    lib.cg_draw_D_b(seed, m, d_lo, d_hi, _p(D), n, _p(b))
    return D, b


def make_problem(config: str = "tiny", seed: int = 0, nx=None, ny=None, nz=None,
                 d_lo=None, d_hi=None, curvature: float = 0.0) -> Problem:
    """Generate one seeded two-block problem: K, J, D, b.  curvature != 0: contact rows with
    the tilted normals of contact_jacobian_curved instead of z-only rows."""
    c = dict(CONFIGS[config]) if config else {}
    nx = nx if nx is not None else c["nx"]
    ny = ny if ny is not None else c.get("ny", nx)
    nz = nz if nz is not None else c.get("nz", max(1, nx // 2))
    d_lo = d_lo if d_lo is not None else c.get("d_lo", -2.0)
    d_hi = d_hi if d_hi is not None else c.get("d_hi", 4.0)
    K = stiffness(nx, ny, nz)
    J = contact_jacobian_curved(nx, ny, nz, curvature) if curvature else contact_jacobian(nx, ny, nz)
    D, b = draw_D_b(seed, J.nrows, K.nrows, d_lo, d_hi)
    return Problem(nx, ny, nz, K.nrows, J.nrows, K, J, D, b,
                   meta=dict(config=config, seed=seed, d_lo=d_lo, d_hi=d_hi, curvature=curvature))
