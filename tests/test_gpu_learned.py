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


def test_training_gradient_matches_oracle_finite_differences(tiny):
    # The device gradient of the training objective (mlp_backward_kernel, summed over levels by
    # mlp_grad_reduce_kernel) for given weights and given r_l, against central differences of
    # the oracle's FP64 objective (pinned there by the closed form on Fourier modes) for all
    # 1313 weights.  The step h = 1e-4 keeps the differences within ~2e-4 max|g| of the
    # derivative (ReLU kinks crossed by the step); the device computes the MLP in FP32.
    import paper_2505_18576_gb300 as m
    s = m.Solver(tiny.K, tiny.J, tiny.D, max_coarse=128)
    o = oracle.Oracle(tiny.K, tiny.J, tiny.D, max_coarse=128)
    ns = [int(s.info.level_rows[l]) for l in range(s.info.nlevels - 1)]
    assert ns == [o.A(l).shape[0] for l in range(o.nlev - 1)] and len(ns) >= 2
    rng = np.random.default_rng(11)
    w = (rng.standard_normal(1313) * 0.5).astype(np.float32)
    r = rng.uniform(-1, 1, sum(ns))
    loss, g = s.mlp_grad(w, r)
    w64 = w.astype(np.float64)
    o.set_mlp(w64)
    lo = o.mlp_loss(r)
    assert abs(loss - lo) <= 1e-5 * lo
    h = 1e-4
    fd = np.zeros(1313)
    for k in range(1313):
        wp = w64.copy(); wp[k] += h
        o.set_mlp(wp)
        lp = o.mlp_loss(r)
        wp[k] -= 2 * h
        o.set_mlp(wp)
        fd[k] = (lp - o.mlp_loss(r)) / (2 * h)
    gmax = np.abs(fd).max()
    err = np.abs(g.astype(np.float64) - fd)
    print(f"gradient: max|g| {gmax:.3e}, max abs diff {err.max():.3e}, loss {loss:.6f} (oracle {lo:.6f})")
    assert gmax > 0 and np.all(err <= 2e-3 * gmax + 2e-2 * np.abs(fd))
    # a learning-rate-scaled step along -g lowers the oracle's objective
    o.set_mlp(w64 - 1e-2 * g.astype(np.float64) / gmax)
    assert o.mlp_loss(r) < lo
    s.close()
    o.close()
