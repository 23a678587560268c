"""amgf_update_D_fine: a new barrier diagonal with the interpolation of the last full setup
reused (the coarse operators are updated to the Galerkin products of the new A; checked on
the host in tests/test_library_host.py).  What it must compute exactly is checked against the
oracle built for the new D: the fine-level operator A (row-wise dot-product bound), the filter
solve (kappa(A_w) bound), and the PCG solution (A-norm, within the FP64 rounding floor of the
oracle's own solve)."""
import numpy as np
import pytest

import contactgen as cg
import oracle
from oracle.lanczos import kappa_estimate

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
EPS = np.finfo(np.float64).eps


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, np.float64)).cuda()


@pytest.mark.parametrize("precision", [0, 3])
def test_lagged_update(precision):
    import paper_2505_18576_gb300 as m
    p = cg.make_problem(None, seed=6, nx=16, ny=12, nz=7, d_lo=-2, d_hi=6)
    D2, _ = cg.draw_D_b(77, p.m, p.n, -2.0, 10.0)
    s = m.Solver(p.K, p.J, p.D, precision=precision)
    P0_before = s.export(1, 0)
    s.update_D(D2, keep_coarse=True)
    assert (s.export(1, 0) != P0_before).nnz == 0  # interpolation reused
    o = oracle.Oracle(p.K, p.J, D2)
    S = o.S()
    assert (s.export(0, 0) != S).nnz == 0
    # fine-level operator
    x = np.random.default_rng(3).standard_normal(p.n)
    y = torch.empty(p.n, dtype=torch.float64, device="cuda")
    s.matvec(dev(x), y)
    yo = S @ x
    k = np.diff(S.indptr)
    gam = k * EPS / (1 - k * EPS)
    bound = 2 * gam * (abs(S) @ np.abs(x))
    assert np.all(np.abs(y.cpu().numpy() - yo) <= bound)
    # filter for the new D
    Ic = o.Ic()
    Aw = S[Ic][:, Ic].toarray()
    ev = np.linalg.eigvalsh(Aw)
    v = np.random.default_rng(4).standard_normal(len(Ic))
    w = torch.empty(len(Ic), dtype=torch.float64, device="cuda")
    s.filter_solve(dev(v), w)
    wo = o.filter_solve(v)
    assert np.linalg.norm(w.cpu().numpy() - wo) <= max(1e-12, 16 * EPS * ev[-1] / ev[0]) * np.linalg.norm(wo)
    # solve; bound as for the mixed solves: max(4 rtol sqrt(kappa), 10 f), f the FP64 rounding
    # floor of the oracle itself (A-norm spread of two solves started 1e-10 |b| apart)
    xo, ko, sto, al, be, _ = o.pcg(p.b, tol=1e-8)
    kap, _, _ = kappa_estimate(al, be)
    x2, *_ = o.pcg(p.b, x0=1e-10 * np.abs(p.b), tol=1e-8)
    d2 = x2 - xo
    floor = np.sqrt(d2 @ (S @ d2)) / np.sqrt(xo @ (S @ xo))
    xs = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    st = s.pcg_solve(dev(p.b), xs)
    d = xs.cpu().numpy() - xo
    ea = np.sqrt(d @ (S @ d)) / np.sqrt(xo @ (S @ xo))
    print(f"precision {precision}: lagged-hierarchy solve {st.iters} iterations (fresh oracle setup {ko}), "
          f"A-norm diff {ea:.2e}")
    assert st.converged == 1 and ea <= max(4e-8 * np.sqrt(kap), 10 * floor)
    s.close()


@pytest.mark.parametrize("precision,filter_algo,learned", [(0, 0, False), (3, 0, True), (0, 1, False), (2, 0, False)])
def test_in_place_update_equals_full_upload(precision, filter_algo, learned):
    # amgf_update_D_fine writing new values into the device image (default) and rebuilding the
    # image (update_in_place = 0) give the same preconditioner and the same solve, bit for bit,
    # over two successive updates (the second one from an in-place image)
    import paper_2505_18576_gb300 as m
    p = cg.make_problem(None, seed=8, nx=16, ny=12, nz=7, d_lo=-2, d_hi=6)
    Ds = [cg.draw_D_b(s_, p.m, p.n, -2.0, 10.0)[0] for s_ in (81, 82)]
    opts = dict(precision=precision, filter_algo=filter_algo, max_coarse=128)
    a = m.Solver(p.K, p.J, p.D, update_in_place=1, **opts)
    b = m.Solver(p.K, p.J, p.D, update_in_place=0, **opts)
    if learned:
        import os
        from paper_2505_18576_gb300.learned import load_weights
        w = load_weights(os.path.join(os.path.dirname(m.__file__), "weights", "smoother_c64.npz"))
        a.set_mlp(w)
        b.set_mlp(w)
    r = dev(np.random.default_rng(5).standard_normal(p.n))
    for D in Ds:
        a.update_D(D, keep_coarse=True)
        b.update_D(D, keep_coarse=True)
        assert a.info.nlevels == b.info.nlevels >= 3
        for lev in range(a.info.nlevels):
            assert (a.export(0, lev) != b.export(0, lev)).nnz == 0
        za = torch.empty(p.n, dtype=torch.float64, device="cuda")
        zb = torch.empty(p.n, dtype=torch.float64, device="cuda")
        a.apply(r, za)
        b.apply(r, zb)
        torch.cuda.synchronize()
        assert torch.equal(za, zb)
        xa = torch.zeros(p.n, dtype=torch.float64, device="cuda")
        xb = torch.zeros(p.n, dtype=torch.float64, device="cuda")
        sa = a.pcg_solve(dev(p.b), xa)
        sb = b.pcg_solve(dev(p.b), xb)
        assert sa.status == 0 and sa.iters == sb.iters and torch.equal(xa, xb)
    a.close()
    b.close()
