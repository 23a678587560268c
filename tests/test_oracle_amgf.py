"""Pins of the oracle's AMGF preconditioner (Definition "AMGF", Section 5.1).

  I - M A = (I - B A)(I - P A_w^{-1} P^T A)(I - B A),   A_w = P^T A P.

Checked against: the product form evaluated with dense matrices, the special
cases P = I (M = A^{-1}) and P = 0 (M = 2B - BAB), exactness of the filter step
on range(P), symmetry and positivity of M, and the lower-bound lemma
(A u, u) <= (M^{-1} u, u), i.e. lambda_max(M A) <= 1.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import contactgen as cg
import oracle


@pytest.fixture(scope="module")
def prob():
    return cg.make_problem("tiny", seed=0)


@pytest.fixture(scope="module")
def orc(prob):
    return oracle.Oracle(prob.K, prob.J, prob.D)


@pytest.fixture(scope="module")
def dense(prob, orc):
    n = prob.n
    A = orc.S().toarray()
    B = np.column_stack([orc.vcycle(e) for e in np.eye(n)])
    M = np.column_stack([orc.apply(e) for e in np.eye(n)])
    return A, B, M


def test_contact_set_is_nonzero_columns_of_J(prob, orc):
    Ic = orc.Ic()
    J = prob.J.to_scipy()
    assert np.array_equal(Ic, np.unique(J.indices))
    assert orc.nc == 2 * prob.m


def test_filter_solve_is_exact(prob, orc):
    Ic = orc.Ic()
    Aw = orc.S().toarray()[np.ix_(Ic, Ic)]
    rng = np.random.default_rng(0)
    v = rng.standard_normal(orc.nc)
    w = orc.filter_solve(v)
    ref = np.linalg.solve(Aw, v)
    assert np.linalg.norm(w - ref) <= 1e-10 * np.linalg.norm(ref)


def test_amgf_product_form(prob, orc, dense):
    A, B, M = dense
    n = prob.n
    Ic = orc.Ic()
    P = np.zeros((n, len(Ic))); P[Ic, np.arange(len(Ic))] = 1.0
    Aw = P.T @ A @ P
    I = np.eye(n)
    E = (I - B @ A) @ (I - P @ np.linalg.solve(Aw, P.T @ A)) @ (I - B @ A)
    Mref = (I - E) @ np.linalg.inv(A)
    assert np.abs(M - Mref).max() <= 1e-8 * np.abs(Mref).max()


def test_amgf_symmetric_spd_and_upper_bound(prob, dense):
    A, B, M = dense
    assert np.abs(M - M.T).max() <= 1e-10 * np.abs(M).max()
    L = np.linalg.cholesky(A)
    ev = np.linalg.eigvalsh(L.T @ (0.5 * (M + M.T)) @ L)   # spectrum of M A
    assert ev.min() > 0.0                  # M is SPD
    # (A u, u) <= (M^{-1} u, u): lambda_max(MA) <= 1.  The bound is attained (the
    # filter makes I - MA vanish on a subspace), so allow rounding of order eps * cond(A) ~ 1e-9
    assert ev.max() <= 1.0 + 1e-7
    assert ev.max() >= 1.0 - 1e-7


def test_symmetry_bilinear(prob, orc):
    rng = np.random.default_rng(5)
    x, y = rng.standard_normal(prob.n), rng.standard_normal(prob.n)
    a, b = x @ orc.apply(y), y @ orc.apply(x)
    assert abs(a - b) <= 1e-12 * max(abs(a), abs(b))


def test_filter_step_exact_on_range_P(prob, orc):
    # after y2 = y1 + P A_w^{-1} P^T r1 the residual vanishes on I_c
    rng = np.random.default_rng(1)
    r = rng.standard_normal(prob.n)
    Ic = orc.Ic()
    y1 = orc.vcycle(r)
    r1 = r - orc.S_apply(y1)
    y2 = y1.copy(); y2[Ic] += orc.filter_solve(r1[Ic])
    r2 = r - orc.S_apply(y2)
    assert np.abs(r2[Ic]).max() <= 1e-12 * np.abs(r1).max() * 1e3
    # an error lying in range(P) is annihilated by the middle factor
    e = np.zeros(prob.n); e[Ic] = rng.standard_normal(len(Ic))
    res = orc.S_apply(e)
    corr = np.zeros(prob.n); corr[Ic] = orc.filter_solve(res[Ic])
    assert np.linalg.norm(corr - e) <= 1e-9 * np.linalg.norm(e)


def test_P_identity_gives_exact_inverse(prob):
    # range(P) = whole space (generality remark: any full-rank P): I - MA = (I-BA) 0 (I-BA)
    o = oracle.Oracle(prob.K, prob.J, prob.D, contact_components=2)
    assert o.nc == prob.n
    A = o.S().toarray()
    rng = np.random.default_rng(2)
    r = rng.standard_normal(prob.n)
    z = o.apply(r)
    ref = np.linalg.solve(A, r)
    assert np.linalg.norm(z - ref) <= 1e-9 * np.linalg.norm(ref)
    x, k, st, *_ = o.pcg(r, tol=1e-8)
    assert st == 0 and k == 1


def test_P_empty_gives_two_B_minus_BAB(prob):
    # no contact constraints: I_c is empty, so M = 2B - BAB
    o = oracle.Oracle(prob.K, filter=1)
    assert o.nc == 0
    rng = np.random.default_rng(4)
    r = rng.standard_normal(prob.n)
    Br = o.vcycle(r)
    ref = 2 * Br - o.vcycle(o.S_apply(Br))
    assert np.linalg.norm(o.apply(r) - ref) <= 1e-12 * np.linalg.norm(ref)
    # and with the filter off, M = B
    o0 = oracle.Oracle(prob.K, filter=0)
    assert np.array_equal(o0.apply(r), o0.vcycle(r))


def test_xyz_contact_components(prob):
    o = oracle.Oracle(prob.K, prob.J, prob.D, contact_components=1)
    assert o.nc == 6 * prob.m
    nodes = np.unique(prob.J.col_idx // 3)
    assert np.array_equal(o.Ic(), np.sort((3 * nodes[:, None] + np.arange(3)).ravel()))
    rng = np.random.default_rng(6)
    x, y = rng.standard_normal(prob.n), rng.standard_normal(prob.n)
    a, b = x @ o.apply(y), y @ o.apply(x)
    assert abs(a - b) <= 1e-12 * max(abs(a), abs(b))
