"""The minimal interior-point driver (Section 3, Algorithm 1) on the CPU.

The linear solves go through an injected solver backed by the oracle (the IP loop itself only
knows the interface); the result is pinned against an independent solution of the same QP:
the contact pressures y = -lambda >= 0 minimise 1/2 y^T G y + q^T y with G = J K^-1 J^T and
q = J K^-1 f + g0 (the dual of the QP, a bound-constrained least-squares problem for scipy).
"""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spl
from scipy.optimize import lsq_linear

import oracle
from paper_2505_18576_gb300 import ip


class OracleSolver:
    def __init__(self, K, J, D, use_filter):
        self.K, self.J, self.filter = K, J, 1 if use_filter else 0
        self.o = oracle.Oracle(K, J, D, filter=self.filter)

    def update_D(self, D, keep_coarse=False):
        self.o.close()
        self.o = oracle.Oracle(self.K, self.J, D, filter=self.filter)

    def solve(self, b):
        x, k, st, *_ = self.o.pcg(b, tol=1e-10)
        assert st == 0
        return x, k, 0.0

    def close(self):
        self.o.close()


def dual_solution(K, J, f, g0):
    Ks = K.to_scipy().tocsc()
    Js = J.to_scipy()
    lu = spl.splu(Ks)
    KinvJt = lu.solve(Js.T.toarray())
    G = Js @ KinvJt
    q = Js @ lu.solve(f) + g0
    L = sla.cholesky(0.5 * (G + G.T), lower=True)
    # 1/2 y^T G y + q^T y = 1/2 |L^T y + L^-1 q|^2 + const
    res = lsq_linear(L.T, -sla.solve_triangular(L, q, lower=True), bounds=(0, np.inf), tol=1e-14,
                     lsmr_tol="auto", max_iter=10000)
    y = res.x
    u = lu.solve(f + Js.T @ y)
    return u, y


@pytest.mark.parametrize("policy", ["amgf", "amg", "switch"])
def test_ip_matches_dual_qp_solution(policy):
    K, J, f, g0 = ip.contact_qp(8, load=0.1, curvature=0.2)
    u, info = ip.solve(K, J, f, g0, tol=1e-7, policy=policy, switch_spread=1e6,
                       make_solver=lambda D, use_filter: OracleSolver(K, J, D, use_filter))
    assert info["converged"]
    u_ref, y_ref = dual_solution(K, J, f, g0)
    assert np.sum(y_ref > 0) >= 5                                   # contact is active somewhere
    assert np.linalg.norm(u - u_ref) <= 1e-5 * np.linalg.norm(u_ref)
    lam = info["lambda"]
    assert np.linalg.norm(-lam - y_ref) <= 1e-3 * np.linalg.norm(y_ref)
    gap = J.to_scipy() @ u + g0
    assert gap.min() >= -1e-8 * np.abs(g0).max()
    steps = info["steps"]
    # the barrier diagonal's spread grows by orders of magnitude over the IP iterations (Section 4)
    assert steps[-1]["spread"] >= 1e6 * min(r["spread"] for r in steps[:2])
    used = {r["preconditioner"] for r in steps}
    if policy == "switch":
        assert used == {"amg", "amgf"} and steps[0]["preconditioner"] == "amg"
    else:
        assert used == {policy}


def test_tilted_contact_amg_degrades_amgf_flat():
    # contact measured along the curved interface's normals: along the IP iterations the
    # PCG iterations of plain AMG grow with D's spread while AMGF's stay flat (Section 6)
    K, J, f, g0 = ip.contact_qp(8, tilted=True)
    its = {}
    for policy in ("amgf", "amg"):
        u, info = ip.solve(K, J, f, g0, tol=1e-6, policy=policy,
                           make_solver=lambda D, use_filter: OracleSolver(K, J, D, use_filter))
        assert info["converged"]
        its[policy] = [r["pcg_iters"] for r in info["steps"]]
        u_ref, y_ref = dual_solution(K, J, f, g0)
        assert np.linalg.norm(u - u_ref) <= 1e-4 * np.linalg.norm(u_ref)
    a, g = its["amgf"], its["amg"]
    assert max(a) - min(a) <= 3
    assert max(g[-3:]) >= 1.5 * g[0] and max(g[-3:]) >= 2.5 * max(a[-3:])
