"""The bound-constrained variant (Section 3, remark on bound constraints).

With bounds d_lo <= u - u_* <= d_hi the condensed matrix is K + J~^T D~ J~ with J~ = [J; I; -I]
and D~ = diag(D, D_lo, D_hi).  The oracle takes E = D_lo + D_hi as an added diagonal; these
pins check that against the matrix assembled from the stacked J~ and D~ themselves, the PCG
solution against a dense solve, and the AMGF properties that must survive the extra term.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import contactgen as cg
import oracle


def _bounds(n, seed):
    rng = np.random.default_rng(seed)
    return 10.0 ** rng.uniform(-3, 3, n), 10.0 ** rng.uniform(-3, 3, n)


def _stacked(p, dlo, dhi):
    J = p.J.to_scipy()
    n = p.n
    Jt = sp.vstack([J, sp.identity(n), -sp.identity(n)]).tocsr()
    Jt.sort_indices()
    Dt = np.concatenate([p.D, dlo, dhi])
    return cg.CSR(Jt.shape[0], n, Jt.indptr.astype(np.int64), Jt.indices.astype(np.int32), Jt.data), Dt


def test_bound_diagonal_equals_stacked_constraints(tiny):
    dlo, dhi = _bounds(tiny.n, 1)
    o = oracle.Oracle(tiny.K, tiny.J, tiny.D, E=dlo + dhi, build_amg=0)
    Jt, Dt = _stacked(tiny, dlo, dhi)
    ref = oracle.Oracle(tiny.K, Jt, Dt, build_amg=0)
    A, B = o.S(), ref.S()
    assert abs(A - B).max() <= 1e-14 * abs(B).max()
    # the only difference to the unbounded matrix is the diagonal
    A0 = oracle.Oracle(tiny.K, tiny.J, tiny.D, build_amg=0).S()
    assert abs((A - A0) - sp.diags(dlo + dhi)).max() <= 1e-14 * abs(B).max()


def test_bound_variant_pcg_matches_dense_solve():
    p = cg.make_problem(None, nx=6, ny=6, nz=3, d_lo=-2, d_hi=6)
    dlo, dhi = _bounds(p.n, 2)
    o = oracle.Oracle(p.K, p.J, p.D, E=dlo + dhi)
    x, k, st, *_ = o.pcg(p.b, tol=1e-13)
    assert st == 0
    ref = np.linalg.solve(o.S().toarray(), p.b)
    assert np.linalg.norm(x - ref) <= 1e-10 * np.linalg.norm(ref)


def test_bound_variant_keeps_contact_set_and_filter_exactness(tiny):
    dlo, dhi = _bounds(tiny.n, 3)
    o = oracle.Oracle(tiny.K, tiny.J, tiny.D, E=dlo + dhi)
    o0 = oracle.Oracle(tiny.K, tiny.J, tiny.D)
    assert np.array_equal(o.Ic(), o0.Ic())   # I_c = nonzero columns of J only
    # A_w^{-1} applied to A_w v returns v (exact filter solve on the bounded matrix)
    Ic = o.Ic()
    Aw = o.S()[Ic][:, Ic]
    v = np.random.default_rng(4).standard_normal(len(Ic))
    w = o.filter_solve(Aw @ v)
    assert np.linalg.norm(w - v) <= 1e-9 * np.linalg.norm(v)


def test_bound_variant_rejects_bad_diagonal(tiny):
    E = np.ones(tiny.n); E[3] = -1.0
    with pytest.raises(oracle.OracleError) as e:
        oracle.Oracle(tiny.K, tiny.J, tiny.D, E=E)
    assert e.value.status == 3
    E[3] = np.nan
    with pytest.raises(oracle.OracleError) as e:
        oracle.Oracle(tiny.K, tiny.J, tiny.D, E=E)
    assert e.value.status == 2
