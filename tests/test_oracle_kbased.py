"""The K-based hierarchy variant (hier_from_K) in the oracle, and what it does to PCG.

The variant keeps strength, coarsening and interpolation of the stiffness K alone
(K_{l+1} = R_l K_l P_l) and forms every level operator as A_l = K_l + J_l^T D J_l with
J_{l+1} = J_l P_l, so the coarse operators could be refreshed for a new D without a new setup.
It departs from B := AMG(A) (Remark after Lemma "condition number estimate", Section 5.1).
Pins:
  - A_l = K_l + J_l^T D J_l equals the Galerkin product R A_{l-1} P of the exported matrices;
  - the interpolation does not depend on D (two barrier diagonals, identical P_l bit for bit);
  - without contact rows the variant is the plain hierarchy (A = K), bit for bit.
Measured (seeded, D log-uniform in [1e-2, 1e12], PCG to 1e-8): the variant's AMGF-PCG needs about
twice the iterations of B := AMG(A) on 16x16x8 and three times on 32x32x16, and its plain AMG-PCG
does not converge, which is why the library builds B := AMG(A) for every D.
"""
import numpy as np
import pytest

import contactgen as cg
import oracle


def test_kbased_level_operators_are_galerkin():
    p = cg.make_problem(None, seed=0, nx=12, ny=12, nz=6, d_lo=-2, d_hi=10)
    o = oracle.Oracle(p.K, p.J, p.D, hier_from_K=1, max_coarse=128)
    assert o.nlev >= 3
    for l in range(1, o.nlev):
        A = o.A(l)
        G = (o.R(l - 1) @ o.A(l - 1) @ o.P(l - 1)).tocsr()
        d = (A - G).tocsr()
        scale = abs(o.R(l - 1)) @ abs(o.A(l - 1)) @ abs(o.P(l - 1))
        assert abs(d).max() <= 1e-12 * abs(scale).max()


def test_kbased_interpolation_independent_of_D():
    p = cg.make_problem(None, seed=0, nx=12, ny=12, nz=6, d_lo=-2, d_hi=10)
    D2, _ = cg.draw_D_b(77, p.m, p.n, -2.0, 4.0)
    o1 = oracle.Oracle(p.K, p.J, p.D, hier_from_K=1, max_coarse=128)
    o2 = oracle.Oracle(p.K, p.J, D2, hier_from_K=1, max_coarse=128)
    a1 = oracle.Oracle(p.K, p.J, p.D, max_coarse=128)
    assert o1.nlev == o2.nlev
    for l in range(o1.nlev - 1):
        P1, P2 = o1.P(l), o2.P(l)
        assert (P1 != P2).nnz == 0
    # B := AMG(A) does depend on D: the contact couplings are strong connections of A
    assert a1.P(0).shape != o1.P(0).shape or (a1.P(0) != o1.P(0)).nnz > 0


def test_kbased_without_contact_is_the_plain_hierarchy():
    p = cg.make_problem(None, seed=0, nx=8, ny=8, nz=4)
    o1 = oracle.Oracle(p.K, hier_from_K=1, max_coarse=128)
    o0 = oracle.Oracle(p.K, max_coarse=128)
    assert o1.nlev == o0.nlev
    for l in range(o0.nlev):
        assert (o1.A(l) != o0.A(l)).nnz == 0
    r = np.random.default_rng(0).standard_normal(p.n)
    assert np.array_equal(o1.apply(r), o0.apply(r))


def test_kbased_rejects_bound_terms():
    p = cg.make_problem("tiny", seed=0)
    with pytest.raises(oracle.OracleError):
        oracle.Oracle(p.K, p.J, p.D, E=np.ones(p.n), hier_from_K=1)


@pytest.mark.parametrize("dims,max_ratio", [((16, 16, 8), 1.5), ((32, 32, 16), 2.0)])
def test_kbased_hierarchy_converges_worse(dims, max_ratio):
    p = cg.make_problem(None, seed=0, nx=dims[0], ny=dims[1], nz=dims[2], d_lo=-2, d_hi=12)
    its = {}
    for from_k in (0, 1):
        for filt in (1, 0):
            o = oracle.Oracle(p.K, p.J, p.D, hier_from_K=from_k, filter=filt)
            _, k, st, *_ = o.pcg(p.b, tol=1e-8, maxit=400)
            its[(from_k, filt)] = (k, st)
            o.close()
    print(dims, "AMGF: A-based %d, K-based %d; AMG: A-based %d, K-based %d (status %d)" % (
        its[(0, 1)][0], its[(1, 1)][0], its[(0, 0)][0], its[(1, 0)][0], its[(1, 0)][1]))
    assert its[(0, 1)][1] == 0 and its[(1, 1)][1] == 0 and its[(0, 0)][1] == 0
    assert its[(1, 1)][0] >= max_ratio * its[(0, 1)][0]
    assert its[(1, 0)][1] == 5  # plain AMG-PCG on the K-based hierarchy misses 1e-8 in 400 iterations
