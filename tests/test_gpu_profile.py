"""Reporting entry points on the GPU: the true residual in amgf_stats and the per-launch
records of amgf_profile_iteration (the byte model behind the per-kernel bandwidth tables)."""
import numpy as np
import pytest

import contactgen as cg
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_stats_true_residual_and_setup_time(tiny):
    import paper_2505_18576_gb300 as m
    s = m.Solver(tiny.K, tiny.J, tiny.D)
    o = oracle.Oracle(tiny.K, tiny.J, tiny.D, build_amg=0)
    x = torch.zeros(tiny.n, dtype=torch.float64, device="cuda")
    st = s.pcg_solve(torch.from_numpy(tiny.b).cuda(), x)
    torch.cuda.synchronize()
    xh = x.cpu().numpy()
    ref = np.linalg.norm(tiny.b - o.S_apply(xh)) / np.linalg.norm(tiny.b)
    assert st.status == 0 and st.t_setup_s > 0
    assert abs(st.rel_res_l2 - ref) <= 1e-6 * ref + 1e-15
    st0 = s.pcg_solve(torch.zeros(tiny.n, dtype=torch.float64, device="cuda"), x)
    assert st0.rel_res_l2 == 0.0
    s.close()


@pytest.mark.parametrize("precision", [0, 3])
def test_profile_iteration_records(precision):
    import paper_2505_18576_gb300 as m
    p = cg.make_problem(None, seed=1, nx=16, ny=12, nz=7, d_lo=-2, d_hi=8)
    s = m.Solver(p.K, p.J, p.D, precision=precision, max_coarse=128, p_max=0)
    x = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    st = s.pcg_solve(torch.from_numpy(p.b).cuda(), x)
    recs = s.profile_iteration()
    assert st.status == 0 and len(recs) > 10 and all(r["ms"] >= 0 for r in recs)
    assert recs[0]["op"] == "A p, p^T A p" and recs[0]["level"] == 0
    assert recs[-1]["op"] == "PCG: scalars and stop test"
    levels = {r["level"] for r in recs if r["level"] >= 0}
    assert levels == set(range(s.info.nlevels))
    # the fine-level post-smoother's record carries the same byte count as amgf_time_kernel's
    which = 1 if precision == 0 else 2
    _, kb = s.time_kernel(which, warmup=1, reps=2)
    post = [r for r in recs if r["level"] == 0 and "x + W (b - A x)" in r["op"]]
    assert len(post) == 2  # one per V-cycle
    # the bench's kernel reads no add vector and no dot partner; the V-cycle's second sweep adds y2
    assert min(r["bytes"] for r in post) == pytest.approx(kb, rel=1e-12)
    assert all(r["bytes"] > 0 and r["flops"] > 0 for r in recs if "A x" in r["op"] or "A p" in r["op"])
    s.close()
