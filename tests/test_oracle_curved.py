"""AMG and AMGF on contact with tilted normals (Section 4: the filter removes the dependence
on the barrier diagonal D that contact adds to an AMG preconditioner).

With node-to-node contact along z the contact couplings are same-component couplings that
the unknown-approach AMG already captures, so plain AMG does not degrade (the z-only tests in
test_oracle_pcg.py).  With the normals of a curved interface every contact row couples all
three displacement components of both nodes; the AMG built on A = K + J^T D J (strength and
interpolation within one component) then misses the stiff contact modes, and AMG-PCG
degrades as D grows, while AMGF-PCG stays within the practical bound
kappa(M A) <= 2 (beta + 3) (beta = kappa of AMG on the contact-free K) at every D."""
import numpy as np
import pytest

import contactgen as cg
import oracle
from oracle.lanczos import kappa_estimate


def test_curved_rows_are_unit_normals():
    J0 = cg.contact_jacobian(4, 4, 2).to_scipy().toarray()
    assert np.array_equal(cg.contact_jacobian_curved(4, 4, 2, 0.0).to_scipy().toarray(), J0)
    Jc = cg.contact_jacobian_curved(6, 6, 3, 1.0).to_scipy()
    A = Jc.toarray()
    xyz = cg.node_xyz(6, 6, 3)
    for r in range(A.shape[0]):
        nz = np.nonzero(A[r])[0]
        nodes = sorted(set(nz // 3))
        assert len(nodes) == 2
        na, nb = A[r, 3 * nodes[0]:3 * nodes[0] + 3], A[r, 3 * nodes[1]:3 * nodes[1] + 3]
        assert np.allclose(na, -nb) and abs(np.linalg.norm(na) - 1.0) < 1e-14
        up = nodes[0] if xyz[nodes[0], 2] > xyz[nodes[1], 2] else nodes[1]
        n_up = A[r, 3 * up:3 * up + 3]
        x, y = xyz[up, 0], xyz[up, 1]
        ref = np.array([-2 * (x - 0.5), -2 * (y - 0.5), 1.0])
        assert np.allclose(n_up, ref / np.linalg.norm(ref), rtol=0, atol=1e-14)


def test_amgf_robust_where_amg_degrades():
    K = cg.stiffness(8, 8, 4)
    J = cg.contact_jacobian_curved(8, 8, 4, 1.0)
    okf = oracle.Oracle(K, filter=0)  # contact-free: beta = kappa of AMG-PCG on K
    _, b = cg.draw_D_b(0, J.nrows, K.nrows, -2.0, 2.0)
    _, _, st, al, be, _ = okf.pcg(b, tol=1e-12, maxit=1000)
    assert st == 0
    beta, _, _ = kappa_estimate(al, be)
    okf.close()
    its = {}
    for dh in (2.0, 10.0):
        D, b = cg.draw_D_b(0, J.nrows, K.nrows, -2.0, dh)
        o = oracle.Oracle(K, J, D)
        _, k, st, al, be, _ = o.pcg(b, tol=1e-12, maxit=1000)
        assert st == 0
        kap, _, _ = kappa_estimate(al, be)
        assert kap <= 2 * (beta + 3)
        _, its[dh], st, *_ = o.pcg(b, tol=1e-8)
        assert st == 0
        o.close()
        oa = oracle.Oracle(K, J, D, filter=0)  # plain AMG-PCG, M = B
        _, ka, sta, *_ = oa.pcg(b, tol=1e-8, maxit=400)
        if dh == 2.0:
            assert sta == 0 and ka >= 10 * its[dh]
        else:
            assert sta != 0  # not converged in 400 iterations
        oa.close()
    assert abs(its[10.0] - its[2.0]) <= 2
