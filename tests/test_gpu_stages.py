"""Step-by-step parity of one AMGF application on the GPU (Definition "AMGF", Section 5.1).

amgf_apply_stages returns the library's own intermediate vectors of z = M r:
    y1 = B r,  r1 = r - A y1,  w = A_w^{-1} P^T r1,  r2 = r1 - A P w,  z = y1 + P w + B r2.
Each step is checked against the oracle's operator applied to the GPU's input of that step,
so no tolerance depends on kappa(A_w) (which reaches 1e13 and more with D up to 1e12, where two
exact FP64 solves of A_w agree only to ~kappa(A_w) u):
  1. y1 against the oracle's V-cycle of r: 1e-12 relative (FP64); BF16 V-cycle: 5e-2.
  2. r1 against r - A y1 (oracle A, GPU y1), row by row within 2 gamma_k (|r| + |A||y1|)_i.
  3. w: normwise backward error ||A_w w - P^T r1|| <= 64 u ||A_w|| ||w||.
  4. P^T r2 = P^T r1 - A_w w vanishes to rounding: ||P^T r2|| <= 64 u ||A_w|| ||w||
     + 2 gamma_k || |A_w| |w| || + u ||P^T r1||; the rows of r2 outside I_c equal
     (r1 - A P w) row by row within 2 gamma_k (|r1| + |A| |P w|)_i.
  5. z against y1 + P w + (oracle V-cycle of the GPU's r2): 1e-12 of ||z|| (FP64).
Cases span D up to 1e12 (the full-form range), the tilted-normal contact rows whose filter
needed the Cholesky-factor reduction, and both exact filter algorithms.
"""
import numpy as np
import pytest

import contactgen as cg
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps

CASES = {
    "n16_d12": dict(nx=16, ny=12, nz=7, d_lo=-2, d_hi=12),
    "n24_d12": dict(nx=24, ny=24, nz=12, d_lo=-2, d_hi=12),
    "tilted8_d10": dict(nx=8, ny=8, nz=4, d_lo=-2, d_hi=10, curvature=1.0),
    "tilted16_d10": dict(nx=16, ny=16, nz=8, d_lo=-2, d_hi=10, curvature=1.0),
}


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def gam(k):
    return k * EPS / (1 - k * EPS)


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    p = cg.make_problem(None, seed=3, **CASES[request.param])
    o = oracle.Oracle(p.K, p.J, p.D)
    yield request.param, p, o
    o.close()


def norm2(M):
    """||M||_2 of a symmetric sparse matrix: dense for small ones, else Lanczos (ARPACK) with a
    1% margin on top of the converged largest-magnitude eigenvalue."""
    if M.shape[0] <= 4000:
        return np.linalg.norm(M.toarray(), 2)
    import scipy.sparse.linalg as spl
    ev = spl.eigsh(M, k=1, which="LM", return_eigenvectors=False, tol=1e-6)
    return 1.01 * float(np.abs(ev).max())


def run_stages(s, p, r):
    n, nc = p.n, s.nc
    z = torch.empty(n, dtype=torch.float64, device="cuda")
    y1, r1, r2 = (torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(3))
    w = torch.empty(nc, dtype=torch.float64, device="cuda")
    s.apply_stages(dev(r), z, y1=y1, r1=r1, w=w, r2=r2)
    return host(z), host(y1), host(r1), host(w), host(r2)


def check_stages(p, o, s, r, vtol):
    z, y1, r1, w, r2 = run_stages(s, p, r)
    S = o.S()
    absS = abs(S)
    k = np.diff(S.indptr)
    Ic = o.Ic()
    assert np.array_equal(s.contact_set(), Ic)
    # 1. first V-cycle
    yo = o.vcycle(r)
    e1 = np.linalg.norm(y1 - yo) / np.linalg.norm(yo)
    assert e1 <= vtol, e1
    # 2. r1 = r - A y1 in FP64, row by row
    ref = r - S @ y1
    assert np.all(np.abs(r1 - ref) <= 2 * gam(k + 1) * (np.abs(r) + absS @ np.abs(y1)) + 1e-300)
    # 3. filter solve: backward error on the GPU's own right-hand side
    Aw = S[Ic][:, Ic]
    nAw = norm2(Aw)
    v = r1[Ic]
    back = np.linalg.norm(Aw @ w - v) / (nAw * np.linalg.norm(w))
    assert back <= 64 * EPS, back
    # 4. P^T r2 = P^T r1 - A_w w vanishes to rounding (kappa-free); other rows as computed
    Pw = np.zeros(p.n)
    Pw[Ic] = w
    kw = np.diff(Aw.indptr)
    bound = (64 * EPS * nAw * np.linalg.norm(w) + 2 * gam(kw.max() + 1) * np.linalg.norm(abs(Aw) @ np.abs(w))
             + EPS * np.linalg.norm(v))
    ptr2 = np.linalg.norm(r2[Ic])
    assert ptr2 <= bound, (ptr2, bound)
    ref2 = r1 - S @ Pw
    assert np.all(np.abs(r2 - ref2) <= 2 * gam(k + 1) * (np.abs(r1) + absS @ np.abs(Pw)) + 1e-300)
    # 5. z = y2 + B r2 on the GPU's r2
    zref = y1 + Pw + o.vcycle(r2)
    e5 = np.linalg.norm(z - zref) / np.linalg.norm(z)
    assert e5 <= vtol, e5
    return dict(e1=e1, back=back, ptr2=ptr2 / max(np.linalg.norm(v), 1e-300), e5=e5)


@pytest.mark.parametrize("algo", [0, 1])
def test_apply_stages_fp64(case, algo):
    import paper_2505_18576_gb300 as m
    name, p, o = case
    s = m.Solver(p.K, p.J, p.D, filter_algo=algo)
    try:
        r = np.random.default_rng(4).standard_normal(p.n)
        res = check_stages(p, o, s, r, 1e-12)
        print(name, algo, {k: f"{v:.2e}" for k, v in res.items()})
        # the staged call computes exactly what amgf_apply computes
        z2 = torch.empty(p.n, dtype=torch.float64, device="cuda")
        s.apply(dev(r), z2)
        z1, *_ = run_stages(s, p, r)
        assert np.array_equal(host(z2), z1)
    finally:
        s.close()


def test_apply_stages_bf16(case):
    # precision 3 (BF16 storage of every V-cycle matrix): the V-cycles carry the BF16 error, the
    # FP64 steps 2-4 keep their rounding-level bounds
    import paper_2505_18576_gb300 as m
    name, p, o = case
    s = m.Solver(p.K, p.J, p.D, precision=3)
    try:
        r = np.random.default_rng(5).standard_normal(p.n)
        res = check_stages(p, o, s, r, 5e-2)
        print(name, "bf16", {k: f"{v:.2e}" for k, v in res.items()})
    finally:
        s.close()


def test_apply_stages_argument_checks(tiny):
    import paper_2505_18576_gb300 as m
    s = m.Solver(tiny.K, tiny.J, tiny.D, filter=0)
    z = torch.empty(tiny.n, dtype=torch.float64, device="cuda")
    r2 = torch.empty(tiny.n, dtype=torch.float64, device="cuda")
    with pytest.raises(m.AmgfError):  # r2 needs the filter
        s.apply_stages(dev(np.ones(tiny.n)), z, r2=r2)
    y1 = torch.empty(tiny.n, dtype=torch.float64, device="cuda")
    s.apply_stages(dev(np.ones(tiny.n)), z, y1=y1)  # M = B: y1 is the first V-cycle, z = B r
    torch.cuda.synchronize()
    assert torch.equal(y1, z)
    s.close()
