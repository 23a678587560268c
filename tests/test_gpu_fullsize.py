"""GPU parity at the benchmark's full size (c64: n = 811,200, m = 4,225), in the launch
configuration bench.py times (default options, CUDA-graph PCG).

The oracle computes the whole apply and the whole solve at this size (seconds to a
minute on the host), so the comparison is element-by-element on full vectors:
  - AMGF apply: ||z_gpu - z_orc|| <= max(1e-12, 16 u kappa(A_w)) ||z_orc||, kappa(A_w) from
    sparse extreme eigenvalues (ARPACK, shift-invert for the smallest).
  - PCG on seed 0 at rtol 1e-8: iteration counts within +-1 and the A-norm bound
    ||x_gpu - x_orc||_A <= 2 rtol sqrt(kappa(MA)) ||x_orc||_A (kappa from the oracle's CG
    coefficients); at rtol 1e-12 the A-norm difference is at most max(1e-8, 10 f), f the FP64
    rounding floor measured on the oracle (see tests/test_gpu_parity.py).
  - Symmetry x^T M y = y^T M x of the GPU preconditioner, to max(1e-12, 16 u kappa(A_w)).
"""
import numpy as np
import pytest

import contactgen as cg
import oracle
from oracle.lanczos import kappa_estimate

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module")
def c64():
    import paper_2505_18576_gb300 as m
    p = cg.make_problem("c64", seed=0)
    o = oracle.Oracle(p.K, p.J, p.D)
    s = m.Solver(p.K, p.J, p.D)
    yield p, o, s
    s.close()
    o.close()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, np.float64)).cuda()


def kappa_Aw_sparse(o):
    import scipy.sparse.linalg as sla
    Ic = o.Ic()
    Aw = o.S()[Ic][:, Ic].tocsc()
    lmax = sla.eigsh(Aw, k=1, which="LA", return_eigenvectors=False)[0]
    lmin = sla.eigsh(Aw, k=1, sigma=0.0, which="LM", return_eigenvectors=False)[0]
    return lmax / lmin


def test_c64_apply_parity(c64):
    p, o, s = c64
    r = np.random.default_rng(11).standard_normal(p.n)
    z = torch.empty(p.n, dtype=torch.float64, device="cuda")
    s.apply(dev(r), z)
    torch.cuda.synchronize()
    zo = o.apply(r)
    tol = max(1e-12, 16 * EPS * kappa_Aw_sparse(o))
    err = np.linalg.norm(z.cpu().numpy() - zo) / np.linalg.norm(zo)
    print(f"c64 apply rel err {err:.3e} (tol {tol:.3e})")
    assert err <= tol


def test_c64_vcycle_parity(c64):
    p, o, s = c64
    r = np.random.default_rng(12).standard_normal(p.n)
    x = torch.empty(p.n, dtype=torch.float64, device="cuda")
    s.vcycle(dev(r), x)
    torch.cuda.synchronize()
    xo = o.vcycle(r)
    assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-12 * np.linalg.norm(xo)


def test_c64_preconditioner_symmetric(c64):
    p, o, s = c64
    rng = np.random.default_rng(13)
    a, b = rng.standard_normal(p.n), rng.standard_normal(p.n)
    za = torch.empty(p.n, dtype=torch.float64, device="cuda")
    zb = torch.empty(p.n, dtype=torch.float64, device="cuda")
    s.apply(dev(a), za)
    s.apply(dev(b), zb)
    torch.cuda.synchronize()
    x1 = float(b @ za.cpu().numpy())
    x2 = float(a @ zb.cpu().numpy())
    tol = max(1e-12, 16 * EPS * kappa_Aw_sparse(o))
    print(f"c64 symmetry {abs(x1 - x2) / max(abs(x1), abs(x2)):.3e} (tol {tol:.3e})")
    assert abs(x1 - x2) <= tol * max(abs(x1), abs(x2))


def test_c64_pcg_parity(c64):
    p, o, s = c64
    xo, ko, sto, al, be, _ = o.pcg(p.b, tol=1e-8)
    x = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    st = s.pcg_solve(dev(p.b), x)
    torch.cuda.synchronize()
    xg = x.cpu().numpy()
    S = o.S()
    d = xg - xo
    ea = np.sqrt(d @ (S @ d)) / np.sqrt(xo @ (S @ xo))
    kap, _, _ = kappa_estimate(al, be)
    xe = np.linalg.norm(d) / np.linalg.norm(xo)
    print(f"c64 pcg iters gpu {st.iters} oracle {ko}, A-norm diff {ea:.3e} (bound {2e-8*np.sqrt(kap):.3e}), "
          f"2-norm diff {xe:.3e}, t_solve {st.t_solve_s*1e3:.2f} ms")
    assert sto == 0 and st.status == 0
    assert abs(st.iters - ko) <= 1
    assert ea <= 2e-8 * np.sqrt(kap)


def test_c64_pcg_tight_solution_match(c64):
    import paper_2505_18576_gb300 as m
    p, o, s = c64
    xo, ko, sto, al, be, _ = o.pcg(p.b, tol=1e-12)
    s2 = m.Solver(p.K, p.J, p.D, rtol=1e-12)
    x = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    st = s2.pcg_solve(dev(p.b), x)
    torch.cuda.synchronize()
    d = x.cpu().numpy() - xo
    S = o.S()
    ea = np.sqrt(d @ (S @ d)) / np.sqrt(xo @ (S @ xo))
    xe = np.linalg.norm(d) / np.linalg.norm(xo)
    x2, *_ = o.pcg(p.b, x0=1e-10 * np.abs(p.b), tol=1e-12)
    d2 = x2 - xo
    floor = np.sqrt(d2 @ (S @ d2)) / np.sqrt(xo @ (S @ xo))
    print(f"c64 rtol 1e-12: iters gpu {st.iters} oracle {ko}, x diff A-norm {ea:.3e} 2-norm {xe:.3e}, "
          f"rounding floor {floor:.3e}")
    assert sto == 0 and st.status == 0 and abs(st.iters - ko) <= 1
    assert ea <= max(1e-8, 10 * floor)
    s2.close()
