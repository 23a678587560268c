"""Learned smoother on the GPU (FP32 MLP inference and training kernels) against the oracle.

  - weights giving theta = 1 reproduce the plain V-cycle (FP32 sigmoid: |theta - 1| ~ 1e-7,
    asserted to 1e-6 relative on the V-cycle output);
  - random weights: GPU V-cycle (FP32 MLP) vs oracle V-cycle (same weights, FP64 MLP) within
    1e-5 relative (theta differs by FP32 rounding of the 1313-weight forward pass, ~1e-6);
  - training lowers the smoothing loss; a learned solve converges; the fallback to theta = 1
    triggers when the learned weights miss the stop test.
"""
import numpy as np
import pytest

import contactgen as cg
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, np.float64)).cuda()


@pytest.fixture(scope="module")
def prob():
    return cg.make_problem(None, seed=7, nx=12, ny=12, nz=6, d_lo=-2, d_hi=8)


def unit_weights():
    from paper_2505_18576_gb300.learned import init_weights
    w = np.zeros(1313, np.float32)
    w[1312] = np.log(3.5)
    return w


def test_unit_weights_reproduce_plain(prob):
    import paper_2505_18576_gb300 as m
    s = m.Solver(prob.K, prob.J, prob.D)
    r = np.random.default_rng(0).standard_normal(prob.n)
    x0 = torch.empty(prob.n, dtype=torch.float64, device="cuda")
    x1 = torch.empty_like(x0)
    s.vcycle(dev(r), x0)
    s.set_mlp(unit_weights())
    s.vcycle(dev(r), x1)
    torch.cuda.synchronize()
    assert float(torch.linalg.norm(x1 - x0) / torch.linalg.norm(x0)) <= 1e-6
    s.set_mlp(None)
    x2 = torch.empty_like(x0)
    s.vcycle(dev(r), x2)
    torch.cuda.synchronize()
    assert torch.equal(x2, x0)


@pytest.mark.parametrize("precision", [0, 1])
def test_learned_vcycle_matches_oracle(prob, precision):
    import paper_2505_18576_gb300 as m
    w = (np.random.default_rng(5).standard_normal(1313) * 0.5).astype(np.float32)
    o = oracle.Oracle(prob.K, prob.J, prob.D)
    o.set_mlp(w.astype(np.float64))
    s = m.Solver(prob.K, prob.J, prob.D, precision=precision)
    s.set_mlp(w)
    r = np.random.default_rng(1).standard_normal(prob.n)
    x = torch.empty(prob.n, dtype=torch.float64, device="cuda")
    s.vcycle(dev(r), x)
    torch.cuda.synchronize()
    xo = o.vcycle(r)
    err = np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo)
    print(f"learned V-cycle precision {precision}: rel diff {err:.2e}")
    assert err <= 1e-5 if precision == 0 else err <= 1e-4


def test_training_lowers_loss_and_solve_converges(prob):
    import paper_2505_18576_gb300 as m
    from paper_2505_18576_gb300.learned import init_weights
    s = m.Solver(prob.K, prob.J, prob.D)
    w = init_weights(0)
    mm = np.zeros(1313, np.float32)
    vv = np.zeros(1313, np.float32)
    step, loss = m.amgf_mlp_train(s.h, w, mm, vv, 0, 40, 1e-2, 123)
    print("loss", loss[0], loss[-1])
    assert step == 40 and np.all(np.isfinite(loss)) and np.all(np.isfinite(w))
    assert loss[-1] < loss[0]
    s.set_mlp(w)
    x = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    st = s.pcg_solve(dev(prob.b), x)
    assert st.status == 0 and st.mlp_fallback == 0


def test_fallback_to_plain_weights(prob):
    import paper_2505_18576_gb300 as m
    s = m.Solver(prob.K, prob.J, prob.D)
    x = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    k_plain = s.pcg_solve(dev(prob.b), x).iters
    # theta = 0.3 everywhere: a weak smoother that needs more than k_plain iterations
    w = np.zeros(1313, np.float32)
    w[1312] = -30.0
    s2 = m.Solver(prob.K, prob.J, prob.D, maxit=k_plain)
    s2.set_mlp(w)
    x.zero_()
    st = s2.pcg_solve(dev(prob.b), x)
    assert st.status == 0 and st.mlp_fallback == 1 and st.iters == k_plain
