"""Pins of the oracle's AMG hierarchy and V-cycle B (the B := AMG(A) of Section 5, Remark on l1 smoothers).

Each check compares the oracle with something other than itself: closed forms on
textbook matrices, hand-derived coarsenings, invariants of the interpolation, a
library sparse product, and the V-cycle's error-propagation identity evaluated
with dense matrices.
"""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from contactgen import CSR

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def csr_of(A):
    A = sp.csr_matrix(A)
    A.sort_indices()
    return CSR(A.shape[0], A.shape[1], A.indptr.astype(np.int64), A.indices.astype(np.int32),
               A.data.astype(np.float64))


def lap1d(n):
    return sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1], format="csr")


def lap2d(k):
    I = sp.identity(k)
    T = lap1d(k)
    return (sp.kron(I, T) + sp.kron(T, I)).tocsr()


def test_rs_1d_laplacian_closed_form():
    # 1D Dirichlet Laplacian, n = 2k+1: RS picks the odd points, direct interpolation is
    # linear interpolation (weights 1/2) and the Galerkin operator is (1/2) tridiag(-1, 2, -1)
    n = 33
    o = oracle.Oracle(csr_of(lap1d(n)), num_functions=1, max_coarse=4, filter=0, strength_theta=0.25)
    cf = o.cf(0)
    assert np.array_equal(np.nonzero(cf)[0], np.arange(1, n, 2))
    P = o.P(0).toarray()
    k = (n - 1) // 2
    Pref = np.zeros((n, k))
    for c in range(k):
        Pref[2 * c + 1, c] = 1.0
        Pref[2 * c, c] += 0.5
        Pref[2 * c + 2, c] += 0.5
    assert np.array_equal(P, Pref)
    assert np.array_equal(o.R(0).toarray(), Pref.T)
    assert np.allclose(o.A(1).toarray(), 0.5 * lap1d(k).toarray(), rtol=0, atol=1e-15)


def test_rs_2d_3x3_hand_derived():
    # 5-point Laplacian on a 3x3 grid (derivation in golden/rs_5pt_3x3.json)
    g = json.load(open(os.path.join(GOLDEN, "rs_5pt_3x3.json")))
    o = oracle.Oracle(csr_of(lap2d(3)), num_functions=1, max_coarse=2, filter=0, strength_theta=0.25)
    assert list(np.nonzero(o.cf(0))[0]) == g["C_points"]
    P = o.P(0).toarray()
    for row, w in g["P_rows"].items():
        assert np.allclose(P[int(row)], w, rtol=0, atol=1e-15)


def _golden_matrix(g):
    m = g["matrix"]
    A = np.diag(np.asarray(m["diag"], float))
    for i, j, a in m["offdiag"]:
        A[i, j] = A[j, i] = a
    return A


def test_classical_interpolation_hand_derived():
    # strong F-F couplings: classical weights differ from direct ones (golden/classical_6pt.json)
    g = json.load(open(os.path.join(GOLDEN, "classical_6pt.json")))
    A = _golden_matrix(g)
    assert np.all(np.linalg.eigvalsh(A) > 0)
    o = oracle.Oracle(csr_of(A), num_functions=1, max_coarse=2, filter=0, strength_theta=0.5)
    assert list(np.nonzero(o.cf(0))[0]) == g["C_points"]
    P = o.P(0).toarray()
    for row, w in g["P_rows"].items():
        assert np.allclose(P[int(row)], w, rtol=0, atol=1e-15)
    od = oracle.Oracle(csr_of(A), num_functions=1, max_coarse=2, filter=0, strength_theta=0.5, interp=1)
    Pd = od.P(0).toarray()
    for row, w in g["P_rows_direct"].items():
        assert np.allclose(Pd[int(row)], w, rtol=0, atol=1e-15)
    # truncation to one weight per row, rescaled to the row sum (hand-derived in the golden file)
    ot = oracle.Oracle(csr_of(A), num_functions=1, max_coarse=2, filter=0, strength_theta=0.5, p_max=1)
    Pt = ot.P(0).toarray()
    for row, w in g["P_rows_pmax1"].items():
        assert np.allclose(Pt[int(row)], w, rtol=0, atol=1e-15)
    assert np.array_equal(np.diff(ot.P(0).indptr), np.ones(6, dtype=np.int64))


def test_truncation_1d_laplacian_ties():
    # 1D Laplacian: every interior F point interpolates 1/2, 1/2 from its two C neighbours.
    # p_max = 1 keeps the tie's smaller coarse index and rescales it to the row sum 1; the
    # boundary F points have one weight (1/2) and stay as they are.
    n = 33
    k = (n - 1) // 2
    o = oracle.Oracle(csr_of(lap1d(n)), num_functions=1, max_coarse=4, filter=0, strength_theta=0.25, p_max=1)
    P = o.P(0).toarray()
    Pref = np.zeros((n, k))
    for c in range(k):
        Pref[2 * c + 1, c] = 1.0
    Pref[0, 0] = 0.5
    Pref[n - 1, k - 1] = 0.5
    for c in range(1, k):
        Pref[2 * c, c - 1] = 1.0
    assert np.array_equal(P, Pref)


def test_classical_guard_falls_back_to_direct():
    # a row whose lumped diagonal nearly cancels takes the direct weights
    # (golden/classical_guard_10pt.json)
    g = json.load(open(os.path.join(GOLDEN, "classical_guard_10pt.json")))
    A = _golden_matrix(g)
    assert np.all(np.linalg.eigvalsh(A) > 0)
    o = oracle.Oracle(csr_of(A), num_functions=1, max_coarse=3, filter=0, strength_theta=0.55)
    assert list(np.nonzero(o.cf(0))[0]) == g["C_points"]
    P = o.P(0).toarray()
    assert np.all(np.isfinite(P))
    for row, w in g["P_rows"].items():
        assert np.allclose(P[int(row)], w, rtol=0, atol=1e-14)


def test_rs_every_f_point_has_strong_c_neighbour():
    o = oracle.Oracle(csr_of(lap2d(17)), num_functions=1, max_coarse=10, filter=0, strength_theta=0.25)
    A = o.A(0)
    cf = o.cf(0)
    P = o.P(0)
    for i in np.nonzero(cf == 0)[0]:
        nb = A.indices[A.indptr[i]:A.indptr[i + 1]]
        assert np.any(cf[nb[nb != i]] == 1)
        assert P.indptr[i + 1] > P.indptr[i]


def _zero_rowsum_matrix(n, seed):
    # graph Laplacian of a random graph plus a few positive off-diagonal couplings,
    # diagonal chosen so that every row sums to zero, then a tiny shift for definiteness
    rng = np.random.default_rng(seed)
    A = sp.random(n, n, density=6.0 / n, random_state=rng, data_rvs=lambda k: -rng.uniform(0.5, 2.0, k))
    A = A + A.T
    pos = sp.random(n, n, density=1.0 / n, random_state=rng, data_rvs=lambda k: rng.uniform(0.01, 0.1, k))
    A = (A + pos + pos.T).tolil()
    A.setdiag(0)
    A = A.tocsr()
    d = -np.asarray(A.sum(axis=1)).ravel()
    return (A + sp.diags(d)).tocsr()


@pytest.mark.parametrize("p_max", [0, 2])
@pytest.mark.parametrize("interp", [0, 1])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_interpolation_preserves_constants(seed, interp, p_max):
    # For zero row sums, both classical interpolation (distributed strong F couplings, lumped
    # weak ones) and direct interpolation with the sign split reproduce constants exactly on
    # every F row that has a strong C neighbour (Ruge & Stueben's and Stueben's constructions);
    # truncation rescales the kept weights to the row sum, so it keeps that property.
    A = _zero_rowsum_matrix(400, seed)
    A = A + sp.identity(400) * 1e-12 * abs(A).max()
    o = oracle.Oracle(csr_of(A), num_functions=1, max_coarse=20, filter=0, strength_theta=0.25, interp=interp,
                      p_max=p_max)
    P = o.P(0)
    s = P @ np.ones(P.shape[1])
    has = np.diff(P.indptr) > 0
    assert has.sum() > 300
    assert np.allclose(s[has], 1.0, rtol=0, atol=1e-8)
    if p_max:
        assert np.diff(P.indptr).max() <= p_max
        full = oracle.Oracle(csr_of(A), num_functions=1, max_coarse=20, filter=0, strength_theta=0.25,
                             interp=interp).P(0)
        assert np.diff(full.indptr).max() > p_max  # the truncation had rows to act on


def test_galerkin_product_and_transpose(tiny):
    o = oracle.Oracle(tiny.K, tiny.J, tiny.D, max_coarse=128)
    assert o.nlev >= 3
    for l in range(o.nlev - 1):
        A, P, R, Ac = o.A(l), o.P(l), o.R(l), o.A(l + 1)
        assert (R != P.T).nnz == 0
        ref = (P.T @ A @ P).toarray()
        assert np.abs(Ac.toarray() - ref).max() <= 1e-13 * np.abs(ref).max()
        assert abs(Ac - Ac.T).max() <= 1e-13 * abs(Ac).max()
        # C points are injected: P restricted to C rows is the identity
        cf = o.cf(l)
        assert np.array_equal(P.toarray()[cf == 1], np.eye(P.shape[1]))
        # function (unknown) of each coarse point is inherited from its C point
        assert np.array_equal(o.func(l + 1), o.func(l)[cf == 1])
    assert np.array_equal(o.func(0), np.arange(tiny.n) % 3)


def test_strength_is_componentwise(tiny):
    # interpolation only couples DOFs of the same displacement component
    o = oracle.Oracle(tiny.K, tiny.J, tiny.D, max_coarse=128)
    for l in range(o.nlev - 1):
        P = o.P(l).tocoo()
        fc, ff = o.func(l + 1), o.func(l)
        assert np.array_equal(ff[P.row], fc[P.col])


def _cheb_q(A, k, lo):
    # closed form of the Chebyshev smoother's error propagation: q_k(W A) with
    # q_k(l) = T_k((c - l) / h) / T_k(c / h), c = (1 + lo) / 2, h = (1 - lo) / 2, W = diag(1/l1),
    # from the eigen-decomposition of the symmetric W^(1/2) A W^(1/2)
    from numpy.polynomial import chebyshev as C
    w = 1.0 / np.abs(A).sum(axis=1)
    sw = np.sqrt(w)
    lam, V = np.linalg.eigh(sw[:, None] * A * sw[None, :])
    c, h = 0.5 * (1 + lo), 0.5 * (1 - lo)
    Tk = np.zeros(k + 1)
    Tk[k] = 1.0
    q = C.chebval((c - lam) / h, Tk) / C.chebval(c / h, Tk)
    return sw[:, None] * (V * q) @ V.T / sw[None, :]


def _dense_B(o, l, cheb=None):
    A = o.A(l).toarray()
    if l == o.nlev - 1:
        return np.linalg.inv(A)
    n = A.shape[0]
    P = o.P(l).toarray()
    Bc = _dense_B(o, l + 1, cheb)
    I = np.eye(n)
    if cheb is None:
        S = I - np.diag(1.0 / np.abs(A).sum(axis=1)) @ A  # one l1-Jacobi sweep
    else:
        S = _cheb_q(A, *cheb)
    # error propagation of one V-cycle: S (I - P B_c P^T A) S = I - B A
    E = S @ (I - P @ Bc @ P.T @ A) @ S
    return (I - E) @ np.linalg.inv(A)


def test_vcycle_error_propagation_identity(tiny):
    o = oracle.Oracle(tiny.K, tiny.J, tiny.D, filter=0, max_coarse=128)
    n = tiny.n
    Bref = _dense_B(o, 0)
    rng = np.random.default_rng(3)
    X = rng.standard_normal((n, 6))
    for k in range(6):
        got = o.vcycle(X[:, k])
        ref = Bref @ X[:, k]
        assert np.linalg.norm(got - ref) <= 1e-9 * np.linalg.norm(ref)


@pytest.mark.parametrize("k,lo", [(2, 0.3), (3, 0.3), (2, 0.1)])
def test_vcycle_chebyshev_closed_form(tiny, k, lo):
    # the recurrence of the Chebyshev smoother against the closed-form polynomial q_k(W A);
    # B stays symmetric with eigenvalues of B A in (0, 1]
    o = oracle.Oracle(tiny.K, tiny.J, tiny.D, filter=0, max_coarse=128, smoother=1, nu=k, cheby_lower=lo)
    assert o.nlev >= 3
    n = tiny.n
    Bref = _dense_B(o, 0, (k, lo))
    rng = np.random.default_rng(4)
    for _ in range(4):
        x = rng.standard_normal(n)
        ref = Bref @ x
        assert np.linalg.norm(o.vcycle(x) - ref) <= 1e-9 * np.linalg.norm(ref)
    B = np.column_stack([o.vcycle(e) for e in np.eye(n)])
    assert np.abs(B - B.T).max() <= 1e-12 * np.abs(B).max()
    L = np.linalg.cholesky(o.S().toarray())
    ev = np.linalg.eigvalsh(L.T @ B @ L)
    assert ev.min() > 0 and ev.max() <= 1.0 + 1e-10
    # degree 1 with lo -> the interval's centre: one sweep x = W b / c
    o1 = oracle.Oracle(tiny.K, tiny.J, tiny.D, filter=0, max_coarse=128, smoother=1, nu=1, cheby_lower=lo)
    B1 = _dense_B(o1, 0, (1, lo))
    x = rng.standard_normal(n)
    assert np.linalg.norm(o1.vcycle(x) - B1 @ x) <= 1e-9 * np.linalg.norm(B1 @ x)


def test_vcycle_symmetric_convergent(tiny):
    o = oracle.Oracle(tiny.K, tiny.J, tiny.D, filter=0, max_coarse=128)
    n = tiny.n
    B = np.column_stack([o.vcycle(e) for e in np.eye(n)])
    assert np.abs(B - B.T).max() <= 1e-12 * np.abs(B).max()
    A = o.S().toarray()
    # generalized eigenvalues of (A, B^{-1}) = eig(BA): all in (0, 1] for an l1 smoother (omega = 1)
    L = np.linalg.cholesky(A)
    ev = np.linalg.eigvalsh(L.T @ B @ L)
    assert ev.min() > 0 and ev.max() <= 1.0 + 1e-10


def test_l1_row_sums(tiny):
    o = oracle.Oracle(tiny.K, tiny.J, tiny.D, max_coarse=128)
    for l in range(o.nlev):
        A = o.A(l)
        assert np.allclose(o.l1(l), np.asarray(abs(A).sum(axis=1)).ravel(), rtol=1e-14)


def test_assembled_schur_complement(tiny):
    o = oracle.Oracle(tiny.K, tiny.J, tiny.D, max_coarse=128)
    K, J = tiny.K.to_scipy(), tiny.J.to_scipy()
    ref = (K + J.T @ sp.diags(tiny.D) @ J).toarray()
    assert np.abs(o.S().toarray() - ref).max() <= 1e-15 * np.abs(ref).max()


def test_invalid_inputs(tiny):
    D = tiny.D.copy(); D[3] = np.nan
    with pytest.raises(oracle.OracleError) as e:
        oracle.Oracle(tiny.K, tiny.J, D)
    assert e.value.status == 2
    D = tiny.D.copy(); D[5] = -1.0
    with pytest.raises(oracle.OracleError) as e:
        oracle.Oracle(tiny.K, tiny.J, D)
    assert e.value.status == 3
    for bad in (dict(smoother=2), dict(smoother=1, cheby_lower=1.0), dict(cheby_lower=0.0)):
        with pytest.raises(oracle.OracleError) as e:
            oracle.Oracle(tiny.K, tiny.J, tiny.D, **bad)
        assert e.value.status == 1
