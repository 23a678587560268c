"""The interior-point loop (Section 3, Algorithm 1) with the library's AMGF-PCG on the GPU.

ip.solve runs with its default linear solver, GpuSolver (amgf_setup / amgf_update_D +
amgf_pcg_solve), on the 8x8x4 two-block contact QP for the three preconditioner policies
(AMGF, plain AMG, and the switch from AMG to AMGF once D's spread reaches 1e6, the dynamic
strategy Section 6.3 suggests).  Checks:
  - the final displacement is within 1e-5 of the solution of the dual QP (solved by scipy);
  - every Newton system of the GPU run, solved again by the oracle with the same preconditioner,
    takes the same number of PCG iterations within +-1;
  - the same loop with the oracle as its linear solver takes as many Newton steps and makes the
    same preconditioner choice at every step.
"""
import numpy as np
import pytest

import oracle
from paper_2505_18576_gb300 import ip
from test_ip_driver import OracleSolver, dual_solution

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("policy", ["amgf", "amg", "switch"])
def test_ip_loop_with_gpu_solver(policy):
    K, J, f, g0 = ip.contact_qp(8, load=0.1, curvature=0.2)
    u, info = ip.solve(K, J, f, g0, tol=1e-7, policy=policy, switch_spread=1e6, rtol=1e-10, record_D=True)
    assert info["converged"]
    u_ref, y_ref = dual_solution(K, J, f, g0)
    assert np.linalg.norm(u - u_ref) <= 1e-5 * np.linalg.norm(u_ref)
    steps = info["steps"]
    gpu_its, orc_its = [], []
    for rec in steps:
        o = oracle.Oracle(K, J, rec["D"], filter=1 if rec["preconditioner"] == "amgf" else 0)
        _, ko, st, *_ = o.pcg(rec["b"], tol=1e-10)
        o.close()
        assert st == 0
        gpu_its.append(rec["pcg_iters"])
        orc_its.append(ko)
    print(policy, "PCG iterations per Newton step, GPU:", gpu_its, "oracle:", orc_its)
    assert all(abs(a - b) <= 1 for a, b in zip(gpu_its, orc_its))
    u2, info2 = ip.solve(K, J, f, g0, tol=1e-7, policy=policy, switch_spread=1e6,
                         make_solver=lambda D, use_filter: OracleSolver(K, J, D, use_filter))
    assert [r["preconditioner"] for r in steps] == [r["preconditioner"] for r in info2["steps"]]
    assert len(steps) == len(info2["steps"])
