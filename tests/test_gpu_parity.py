"""GPU parity: the CUDA path (through the C ABI) against the CPU FP64 oracle.

Tolerances (FP64 on both sides; the hierarchy is bit-identical, see
tests/test_library_host.py, so every difference comes from the order of operations):
  - A x: per row, |y_gpu - y_orc| <= 2 gamma_k (|A| |x|)_i, gamma_k = k u / (1 - k u), k = nonzeros
    of the row (forward error bound of a dot product, applied to both sides).
  - V-cycle: ||x_gpu - x_orc|| <= 1e-12 ||x_orc||.
  - Filter solve w = A_w^{-1} v: both sides are exact solves (banded Cholesky vs block cyclic
    reduction, or block LDL^T sweeps with filter_algo = 1);
    two such FP64 solves agree only to ~ kappa(A_w) u, and kappa(A_w) grows with the spread of D
    (D couples the two contact faces).  Asserted: normwise backward error <= 64 u on the GPU
    result, and ||w_gpu - w_orc|| <= max(1e-12, 16 u kappa(A_w)) ||w_orc||.
  - AMGF apply: ||z_gpu - z_orc|| <= max(1e-12, 16 u kappa(A_w)) ||z_orc||; a case with
    D in [1, 10] (kappa(A_w) u < 1e-13) asserts the strict 1e-12.
  - PCG at rtol 1e-8: iteration counts within +-1, and ||x_gpu - x_orc||_A <= 2 rtol sqrt(kappa(MA))
    ||x_orc||_A (each iterate's A-norm error is at most rtol sqrt(kappa(MA)) ||x*||_A when
    lambda_max(MA) <= 1, x0 = 0), or 10 f where the rounding floor f (below) is larger (D up to
    1e12: f ~ 5e-5-8e-5 on these meshes); at rtol 1e-12 the A-norm difference is at most
    max(1e-8, 10 f), f = the FP64 rounding floor of the solve, measured as the A-norm spread of
    two oracle solves whose starting guesses differ by 1e-10 |b| (entries of A reach
    D_max ~ 1e8 while |x| ~ 1e2, so the true residual stalls near u |A||x| and two exact-
    arithmetic-equivalent solves differ by ~1e-8 in the A-norm).
"""
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


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.fixture(scope="module")
def amgf():
    import paper_2505_18576_gb300 as m
    m.load_library()
    return m


def _pair(p, **opts):
    import paper_2505_18576_gb300 as m
    return oracle.Oracle(p.K, p.J, p.D, **opts), m.Solver(p.K, p.J, p.D, **opts)


CASES = {
    "tiny": dict(nx=8, ny=8, nz=4, d_lo=-2, d_hi=4),
    "ragged": dict(nx=5, ny=3, nz=2, d_lo=-2, d_hi=8),
    "n16": dict(nx=16, ny=12, nz=7, d_lo=-2, d_hi=8),
    "n16_deep": dict(nx=16, ny=12, nz=7, d_lo=-2, d_hi=8),
    # the full-form barrier range, D up to 1e12: kappa(A_w) ~ 1e14, so the forward bounds of the
    # filter and the apply below are loose there; tests/test_gpu_stages.py checks every step of
    # the apply on these systems with kappa-free bounds
    "n16_d12": dict(nx=16, ny=12, nz=7, d_lo=-2, d_hi=12),
    "n24_d12": dict(nx=24, ny=24, nz=12, d_lo=-2, d_hi=12),
}
# the default hierarchy (coarsest <= 1200 rows, 4 weights per interpolation row) has two to
# four levels on these sizes; n16_deep keeps coarsening to 128 rows without truncation, so
# that every level kind (long coarse rows, a warp per row, tiny levels) runs
OPTS = {"n16_deep": dict(max_coarse=128, p_max=0)}


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    p = cg.make_problem(None, seed=1, **CASES[request.param])
    o, s = _pair(p, **OPTS.get(request.param, {}))
    yield request.param, p, o, s
    s.close()


def kappa_Aw(o):
    Ic = o.Ic()
    Aw = o.S()[Ic][:, Ic].toarray()
    ev = np.linalg.eigvalsh(Aw)
    return ev[-1] / ev[0], Aw


def kappa_tol(o):
    return max(1e-12, 16 * EPS * kappa_Aw(o)[0])


def test_matvec_rowwise_error_bound(case):
    name, p, o, s = case
    rng = np.random.default_rng(0)
    x = rng.standard_normal(p.n)
    y = torch.empty(p.n, dtype=torch.float64, device="cuda")
    s.matvec(dev(x), y)
    yg = host(y)
    yo = o.S_apply(x)
    S = o.S()
    absAx = abs(S) @ np.abs(x)
    k = np.diff(S.indptr)
    gam = k * EPS / (1 - k * EPS)
    assert np.all(np.abs(yg - yo) <= 2 * gam * absAx + 1e-300)


def test_vcycle_parity(case):
    name, p, o, s = case
    rng = np.random.default_rng(1)
    r = rng.standard_normal(p.n)
    x = torch.empty(p.n, dtype=torch.float64, device="cuda")
    s.vcycle(dev(r), x)
    xo = o.vcycle(r)
    assert np.linalg.norm(host(x) - xo) <= 1e-12 * np.linalg.norm(xo)


def test_filter_solve_parity(case):
    name, p, o, s = case
    kap, Aw = kappa_Aw(o)
    rng = np.random.default_rng(2)
    v = rng.standard_normal(o.nc)
    w = torch.empty(o.nc, dtype=torch.float64, device="cuda")
    s.filter_solve(dev(v), w)
    wg = host(w)
    wo = o.filter_solve(v)
    back = np.linalg.norm(Aw @ wg - v) / (np.linalg.norm(Aw, 2) * np.linalg.norm(wg))
    assert back <= 64 * EPS
    assert np.linalg.norm(wg - wo) <= max(1e-12, 16 * EPS * kap) * np.linalg.norm(wo)


def test_filter_sweep_algorithm_parity(case):
    # the alternative exact solver (sequential block LDL^T sweeps on one cluster) meets the same bounds
    import paper_2505_18576_gb300 as m
    name, p, o, _ = case
    kap, Aw = kappa_Aw(o)
    s1 = m.Solver(p.K, p.J, p.D, filter_algo=1, **OPTS.get(name, {}))
    try:
        rng = np.random.default_rng(2)
        v = rng.standard_normal(o.nc)
        w = torch.empty(o.nc, dtype=torch.float64, device="cuda")
        s1.filter_solve(dev(v), w)
        wg = host(w)
        wo = o.filter_solve(v)
        back = np.linalg.norm(Aw @ wg - v) / (np.linalg.norm(Aw, 2) * np.linalg.norm(wg))
        assert back <= 64 * EPS
        assert np.linalg.norm(wg - wo) <= max(1e-12, 16 * EPS * kap) * np.linalg.norm(wo)
    finally:
        s1.close()


def test_apply_parity(case):
    name, p, o, s = case
    rng = np.random.default_rng(3)
    r = rng.standard_normal(p.n)
    z = torch.empty(p.n, dtype=torch.float64, device="cuda")
    s.apply(dev(r), z)
    zo = o.apply(r)
    assert np.linalg.norm(host(z) - zo) <= kappa_tol(o) * np.linalg.norm(zo)


def test_apply_and_filter_strict_when_well_conditioned():
    # D in [1, 10]: kappa(A_w) ~ 1e3, so the strict 1e-12 bound applies
    p = cg.make_problem(None, seed=2, nx=8, ny=8, nz=4, d_lo=0.0, d_hi=1.0)
    o, s = _pair(p)
    kap, _ = kappa_Aw(o)
    assert kap < 1e4
    rng = np.random.default_rng(9)
    v = rng.standard_normal(o.nc)
    w = torch.empty(o.nc, dtype=torch.float64, device="cuda")
    s.filter_solve(dev(v), w)
    wo = o.filter_solve(v)
    assert np.linalg.norm(host(w) - wo) <= 1e-12 * np.linalg.norm(wo)
    r = rng.standard_normal(p.n)
    z = torch.empty(p.n, dtype=torch.float64, device="cuda")
    s.apply(dev(r), z)
    zo = o.apply(r)
    assert np.linalg.norm(host(z) - zo) <= 1e-12 * np.linalg.norm(zo)


def a_norm(S, v):
    return float(np.sqrt(v @ (S @ v)))


def test_pcg_parity(case):
    name, p, o, s = case
    xo, ko, sto, al, be, _ = o.pcg(p.b, tol=1e-8)
    x = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    st = s.pcg_solve(dev(p.b), x)
    assert sto == 0 and st.status == 0 and st.converged == 1
    assert abs(st.iters - ko) <= 1
    kap, _, _ = kappa_estimate(al, be)
    S = o.S()
    # with D up to 1e12 the FP64 rounding floor f of the A-norm comparison (two oracle solves
    # started 1e-10 |b| apart) lies above 2 rtol sqrt(kappa): u D_max |x| in the contact rows
    floor = rounding_floor(o, p.b, xo, 1e-8) if CASES[name]["d_hi"] > 8 else 0.0
    assert a_norm(S, host(x) - xo) <= max(2e-8 * np.sqrt(kap), 10 * floor) * a_norm(S, xo)


def rounding_floor(o, b, xo, tol):
    """A-norm spread of two oracle solves started 1e-10 |b| apart, relative to ||xo||_A."""
    x2, *_ = o.pcg(b, x0=1e-10 * np.abs(b), tol=tol)
    S = o.S()
    return a_norm(S, x2 - xo) / a_norm(S, xo)


def test_pcg_tight_solution_match(case):
    import paper_2505_18576_gb300 as m
    name, p, o, s = case
    xo, ko, sto, al, be, _ = o.pcg(p.b, tol=1e-12)
    st_ = m.Solver(p.K, p.J, p.D, rtol=1e-12, **OPTS.get(name, {}))
    x = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    st = st_.pcg_solve(dev(p.b), x)
    assert sto == 0 and st.status == 0
    assert abs(st.iters - ko) <= 1
    S = o.S()
    floor = rounding_floor(o, p.b, xo, 1e-12)
    assert a_norm(S, host(x) - xo) <= max(1e-8, 10 * floor) * a_norm(S, xo)
    st_.close()


def test_pcg_deterministic_and_graph_equals_stream(case):
    import paper_2505_18576_gb300 as m
    name, p, o, s = case
    x1 = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    x2 = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    s1 = s.pcg_solve(dev(p.b), x1)
    s2 = s.pcg_solve(dev(p.b), x2)
    assert s1.iters == s2.iters and torch.equal(x1, x2)
    s_ng = m.Solver(p.K, p.J, p.D, use_graph=0, **OPTS.get(name, {}))
    x3 = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    s3 = s_ng.pcg_solve(dev(p.b), x3)
    assert s3.iters == s1.iters and torch.equal(x1, x3)
    s_ng.close()


def test_host_buffers_solve_equals_device(case):
    name, p, o, s = case
    x = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    s.pcg_solve(dev(p.b), x)
    xh = np.zeros(p.n)
    st = s.pcg_solve_host(np.ascontiguousarray(p.b), xh)
    assert st.status == 0 and np.array_equal(xh, host(x))


# ---------------------------------------------------------------- special cases


def test_amg_only_mode(tiny):
    # M = B: no filter, the strict bound applies
    o, s = _pair(tiny, filter=0)
    r = np.random.default_rng(4).standard_normal(tiny.n)
    z = torch.empty(tiny.n, dtype=torch.float64, device="cuda")
    s.apply(dev(r), z)
    zo = o.apply(r)
    assert np.linalg.norm(host(z) - zo) <= 1e-12 * np.linalg.norm(zo)
    xo, ko, *_ = o.pcg(tiny.b)
    x = torch.zeros(tiny.n, dtype=torch.float64, device="cuda")
    st = s.pcg_solve(dev(tiny.b), x)
    assert abs(st.iters - ko) <= 1


def test_P_identity_exact_inverse(tiny):
    o, s = _pair(tiny, contact_components=2)
    r = np.random.default_rng(5).standard_normal(tiny.n)
    z = torch.empty(tiny.n, dtype=torch.float64, device="cuda")
    s.apply(dev(r), z)
    A = o.S().toarray()
    ref = np.linalg.solve(A, r)
    ev = np.linalg.eigvalsh(A)
    assert np.linalg.norm(host(z) - ref) <= max(1e-12, 16 * EPS * ev[-1] / ev[0]) * np.linalg.norm(ref)
    x = torch.zeros(tiny.n, dtype=torch.float64, device="cuda")
    st = s.pcg_solve(dev(r), x)
    assert st.iters == 1


def test_no_contact_two_B_minus_BAB(tiny):
    import paper_2505_18576_gb300 as m
    o = oracle.Oracle(tiny.K)
    s = m.Solver(tiny.K)
    assert s.nc == 0
    r = np.random.default_rng(6).standard_normal(tiny.n)
    z = torch.empty(tiny.n, dtype=torch.float64, device="cuda")
    s.apply(dev(r), z)
    zo = o.apply(r)
    assert np.linalg.norm(host(z) - zo) <= 1e-12 * np.linalg.norm(zo)


def test_zero_rhs_maxit_and_warm_start(tiny):
    import paper_2505_18576_gb300 as m
    o, s = _pair(tiny)
    x = torch.zeros(tiny.n, dtype=torch.float64, device="cuda")
    st = s.pcg_solve(torch.zeros(tiny.n, dtype=torch.float64, device="cuda"), x)
    assert st.status == 0 and st.iters == 0 and not torch.any(x)
    s3 = m.Solver(tiny.K, tiny.J, tiny.D, maxit=3)
    x = torch.zeros(tiny.n, dtype=torch.float64, device="cuda")
    st = s3.pcg_solve(dev(tiny.b), x, check=False)
    assert st.status == 5 and st.iters == 3 and st.rc == 5
    xo, *_ = o.pcg(tiny.b, tol=1e-12)
    x0 = xo + 1e-3 * np.random.default_rng(7).standard_normal(tiny.n)
    xw = dev(x0)
    st = s.pcg_solve(dev(tiny.b), xw)
    xr, kr, *_ = o.pcg(tiny.b, x0=x0)
    assert abs(st.iters - kr) <= 1
    assert np.linalg.norm(host(xw) - xr) <= 1e-8 * np.linalg.norm(xr)


def test_update_D_matches_fresh_oracle(tiny):
    import paper_2505_18576_gb300 as m
    s = m.Solver(tiny.K, tiny.J, tiny.D)
    D2, b2 = cg.draw_D_b(99, tiny.m, tiny.n, -2.0, 10.0)
    s.update_D(D2)
    o = oracle.Oracle(tiny.K, tiny.J, D2)
    r = np.random.default_rng(8).standard_normal(tiny.n)
    z = torch.empty(tiny.n, dtype=torch.float64, device="cuda")
    s.apply(dev(r), z)
    zo = o.apply(r)
    assert np.linalg.norm(host(z) - zo) <= kappa_tol(o) * np.linalg.norm(zo)


def test_invalid_device_arguments(tiny):
    import paper_2505_18576_gb300 as m
    s = m.Solver(tiny.K, tiny.J, tiny.D)
    with pytest.raises(m.AmgfError):
        s.apply(torch.zeros(tiny.n - 1, dtype=torch.float64, device="cuda"),
                torch.zeros(tiny.n, dtype=torch.float64, device="cuda"))
    with pytest.raises(m.AmgfError):
        s.apply(torch.zeros(tiny.n, dtype=torch.float32, device="cuda"),
                torch.zeros(tiny.n, dtype=torch.float64, device="cuda"))
    r = torch.zeros(tiny.n, dtype=torch.float64, device="cuda")
    with pytest.raises(m.AmgfError):
        s.apply(r, r)  # aliasing


def test_nonfinite_rhs_reports_status(tiny):
    import paper_2505_18576_gb300 as m
    s = m.Solver(tiny.K, tiny.J, tiny.D)
    b = tiny.b.copy(); b[3] = np.nan
    x = torch.zeros(tiny.n, dtype=torch.float64, device="cuda")
    st = s.pcg_solve(dev(b), x, check=False)
    assert st.status == 2


@pytest.mark.parametrize("dims", [(1, 1, 1), (2, 2, 1), (3, 2, 1), (4, 3, 2)])
def test_filter_solve_few_blocks(dims):
    # one, two and three diagonal blocks: cyclic reduction with 0, 1 and 2 reduction levels
    import paper_2505_18576_gb300 as m
    p = cg.make_problem(None, seed=4, nx=dims[0], ny=dims[1], nz=dims[2], d_lo=-2, d_hi=6)
    o = oracle.Oracle(p.K, p.J, p.D)
    kap, Aw = kappa_Aw(o)
    for algo in (0, 1):
        s = m.Solver(p.K, p.J, p.D, filter_algo=algo)
        v = np.random.default_rng(5).standard_normal(o.nc)
        w = torch.empty(o.nc, dtype=torch.float64, device="cuda")
        s.filter_solve(dev(v), w)
        wg = host(w)
        assert np.linalg.norm(Aw @ wg - v) <= 64 * EPS * np.linalg.norm(Aw, 2) * np.linalg.norm(wg)
        assert np.linalg.norm(wg - o.filter_solve(v)) <= max(1e-12, 16 * EPS * kap) * np.linalg.norm(wg)
        # one or two AMG levels (on one level the coarsest solve is the dense inverse of A)
        x = torch.zeros(p.n, dtype=torch.float64, device="cuda")
        st = s.pcg_solve(dev(p.b), x)
        xo, ko, *_ = o.pcg(p.b, tol=1e-8)
        assert st.converged == 1 and abs(st.iters - ko) <= 1
        assert np.linalg.norm(host(x) - xo) <= 1e-8 * np.linalg.norm(xo)
        s.close()


# ---------------------------------------------------------------- Chebyshev smoother
@pytest.mark.parametrize("nu,lo", [(2, 0.3), (3, 0.2), (1, 0.3)])
def test_chebyshev_smoother_parity(nu, lo):
    # degree-nu Chebyshev smoothing (options.smoother = 1): V-cycle within 1e-12 of the oracle's
    # recurrence (pinned there against the closed-form polynomial), AMGF apply within the
    # kappa(A_w) bound, PCG iterations within +-1, on a hierarchy deep enough for every level kind
    import paper_2505_18576_gb300 as m
    p = cg.make_problem(None, seed=2, nx=16, ny=12, nz=7, d_lo=-2, d_hi=8)
    opts = dict(smoother=1, nu=nu, cheby_lower=lo, max_coarse=128, p_max=0)
    o = oracle.Oracle(p.K, p.J, p.D, **opts)
    s = m.Solver(p.K, p.J, p.D, **opts)
    assert s.info.nlevels >= 4
    rng = np.random.default_rng(9)
    r = rng.standard_normal(p.n)
    x = torch.empty(p.n, dtype=torch.float64, device="cuda")
    s.vcycle(dev(r), x)
    xo = o.vcycle(r)
    assert np.linalg.norm(host(x) - xo) <= 1e-12 * np.linalg.norm(xo)
    z = torch.empty(p.n, dtype=torch.float64, device="cuda")
    s.apply(dev(r), z)
    zo = o.apply(r)
    assert np.linalg.norm(host(z) - zo) <= kappa_tol(o) * np.linalg.norm(zo)
    xo2, ko, sto, *_ = o.pcg(p.b, tol=1e-8)
    xs = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    st = s.pcg_solve(dev(p.b), xs)
    print(f"chebyshev degree {nu}, lower {lo}: {st.iters} iterations (oracle {ko})")
    assert sto == 0 and st.status == 0 and abs(st.iters - ko) <= 1
    s.close()
    o.close()


@pytest.mark.parametrize("precision", [1, 3])
def test_chebyshev_smoother_mixed(precision):
    # the FP32 / BF16 V-cycle with the Chebyshev smoother against the FP64 oracle's
    import paper_2505_18576_gb300 as m
    p = cg.make_problem(None, seed=2, nx=16, ny=12, nz=7, d_lo=-2, d_hi=8)
    opts = dict(smoother=1, nu=2, max_coarse=128, p_max=0)
    o = oracle.Oracle(p.K, p.J, p.D, **opts)
    s = m.Solver(p.K, p.J, p.D, precision=precision, **opts)
    r = np.random.default_rng(10).standard_normal(p.n)
    x = torch.empty(p.n, dtype=torch.float64, device="cuda")
    s.vcycle(dev(r), x)
    xo = o.vcycle(r)
    err = np.linalg.norm(host(x) - xo) / np.linalg.norm(xo)
    assert err <= (1e-4 if precision == 1 else 5e-2)
    xs = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    st = s.pcg_solve(dev(p.b), xs)
    _, ko, *_ = o.pcg(p.b, tol=1e-8)
    print(f"chebyshev precision {precision}: V-cycle rel diff {err:.2e}, {st.iters} iterations (oracle {ko})")
    assert st.status == 0 and st.iters <= ko + 3
    with pytest.raises(m.AmgfError):
        s.set_mlp(np.zeros(1313, np.float32))  # learned weights belong to the l1-Jacobi smoother
    s.close()
    o.close()
