"""Pins of the oracle's learned-smoother path (per-row l1-Jacobi damping theta from an MLP).

Not in the paper: a per-row weight theta_i in [0.3, 1.2] multiplies the l1-Jacobi step
(W = diag(theta / l1)).  The pins: weights that give theta = 1 reproduce the plain V-cycle;
features and the 6-32-32-1 forward pass match a numpy evaluation from the exported hierarchy;
theta stays in [0.3, 1.2]; B stays SPD with spectrum of BA in (0, 2) (Assumption 1 with
omega < 2), and the AMGF preconditioner built on it stays SPD.
"""
import numpy as np
import pytest

import contactgen as cg
import oracle

MLP_NW = 1313


def unit_theta_weights():
    w = np.zeros(MLP_NW)
    w[1312] = np.log(3.5)  # 0.3 + 0.9 * sigmoid(log 3.5) = 1
    return w


def random_weights(seed, scale=0.5):
    return np.random.default_rng(seed).standard_normal(MLP_NW) * scale


def numpy_theta(w, f):
    W1 = w[:192].reshape(32, 6); b1 = w[192:224]
    W2 = w[224:1248].reshape(32, 32); b2 = w[1248:1280]
    w3 = w[1280:1312]; b3 = w[1312]
    h1 = np.maximum(f @ W1.T + b1, 0)
    h2 = np.maximum(h1 @ W2.T + b2, 0)
    o = h2 @ w3 + b3
    return 0.3 + 0.9 / (1 + np.exp(-o))


def numpy_features(o, p):
    J = p.J.to_scipy()
    d = np.asarray((J.multiply(J)).T @ p.D).ravel()
    c = (abs(J).sum(axis=0).A.ravel() != 0).astype(float)
    feats = []
    nlev = o.nlev
    for l in range(nlev - 1):
        A = o.A(l)
        aii = A.diagonal()
        l1 = o.l1(l)
        f = np.column_stack([np.log10(aii) / 10, np.log10(l1) / 10, aii / l1, c, np.log10(1 + d) / 10,
                             np.full(len(aii), l / (nlev - 1))])
        feats.append(f)
        cf = o.cf(l).astype(bool)
        d, c = d[cf], c[cf]
    return feats


def test_unit_weights_reproduce_plain_vcycle(tiny):
    o = oracle.Oracle(tiny.K, tiny.J, tiny.D)
    r = np.random.default_rng(0).standard_normal(tiny.n)
    x0 = o.vcycle(r)
    o.set_mlp(unit_theta_weights())
    assert np.allclose(o.theta(0), 1.0, rtol=0, atol=1e-15)
    assert np.linalg.norm(o.vcycle(r) - x0) <= 1e-14 * np.linalg.norm(x0)
    o.set_mlp(None)
    assert np.array_equal(o.vcycle(r), x0)


@pytest.mark.parametrize("seed", [1, 2])
def test_features_and_forward_match_numpy(tiny, seed):
    o = oracle.Oracle(tiny.K, tiny.J, tiny.D)
    w = random_weights(seed)
    o.set_mlp(w)
    for l, f in enumerate(numpy_features(o, tiny)):
        th = o.theta(l)
        assert np.allclose(th, numpy_theta(w, f), rtol=1e-13, atol=0)
        assert th.min() >= 0.3 and th.max() <= 1.2


def test_learned_vcycle_spd_and_convergent(tiny):
    o = oracle.Oracle(tiny.K, tiny.J, tiny.D, filter=0)
    o.set_mlp(random_weights(3, scale=1.0))
    n = tiny.n
    B = np.column_stack([o.vcycle(e) for e in np.eye(n)])
    assert np.abs(B - B.T).max() <= 1e-12 * np.abs(B).max()
    A = o.S().toarray()
    L = np.linalg.cholesky(A)
    ev = np.linalg.eigvalsh(L.T @ (0.5 * (B + B.T)) @ L)
    assert ev.min() > 0 and ev.max() < 2.0
    # and the AMGF preconditioner built on it is SPD
    of = oracle.Oracle(tiny.K, tiny.J, tiny.D)
    of.set_mlp(random_weights(3, scale=1.0))
    M = np.column_stack([of.apply(e) for e in np.eye(n)])
    evm = np.linalg.eigvalsh(L.T @ (0.5 * (M + M.T)) @ L)
    assert evm.min() > 0
    x, k, st, *_ = of.pcg(tiny.b)
    assert st == 0


def test_theta_inherited_contact_features(tiny):
    # rows of the contact DOFs see the flag and log10(1 + D) on the fine level
    o = oracle.Oracle(tiny.K, tiny.J, tiny.D)
    f0 = numpy_features(o, tiny)[0]
    Ic = o.Ic()
    assert np.all(f0[Ic, 3] == 1.0) and f0[:, 3].sum() == len(Ic)
    assert np.all(f0[Ic, 4] > 0)


# ---------------------------------------------------------------- training objective
class _Csr:
    def __init__(self, M):
        M = M.tocsr()
        M.sort_indices()
        self.row_ptr = M.indptr.astype(np.int64)
        self.col_idx = M.indices.astype(np.int32)
        self.val = M.data.astype(np.float64)
        self.nrows, self.ncols = M.shape


def _periodic_laplacian(N, s):
    import scipy.sparse as sp
    e = np.ones(N)
    A = sp.diags([-e[:-1], (2 + s) * e, -e[:-1]], [-1, 0, 1], format="lil")
    A[0, N - 1] = -1.0
    A[N - 1, 0] = -1.0
    return A.tocsr()


def _constant_theta_weights(beta):
    w = np.zeros(MLP_NW)
    w[1312] = beta
    return w


@pytest.mark.parametrize("k,beta", [(1, 0.0), (5, 1.5), (16, -2.0)])
def test_training_loss_closed_form_on_a_fourier_mode(k, beta):
    # A = circulant tridiag(-1, 2 + s, -1): every row has l1 = 4 + s, and r_i = cos(2 pi k i / N)
    # is an eigenvector with lambda_k = 2 + s - 2 cos(2 pi k / N).  With weights that make theta
    # constant (all but the output bias zero: theta = 0.3 + 0.9 sigmoid(beta)), one damped
    # l1-Jacobi step maps r to (1 - theta lambda_k / (4 + s)) r, so the objective of the one
    # smoothed level is (1 - theta lambda_k / (4 + s))^2; its derivative in beta follows.
    N, s = 64, 0.5
    A = _periodic_laplacian(N, s)
    o = oracle.Oracle(_Csr(A), num_functions=1, max_coarse=N // 2 + 10)
    assert o.nlev == 2 and np.allclose(o.l1(0), 4 + s)
    r = np.cos(2 * np.pi * k * np.arange(N) / N)
    lam = 2 + s - 2 * np.cos(2 * np.pi * k / N)
    q = lam / (4 + s)
    sig = 1 / (1 + np.exp(-beta))
    theta = 0.3 + 0.9 * sig
    o.set_mlp(_constant_theta_weights(beta))
    assert np.isclose(o.mlp_loss(r), (1 - theta * q) ** 2, rtol=1e-12, atol=1e-15)
    o.set_mlp(None)
    assert np.isclose(o.mlp_loss(r), (1 - q) ** 2, rtol=1e-12, atol=1e-15)
    # central difference of the oracle's loss in beta against the closed-form derivative
    h = 1e-5
    o.set_mlp(_constant_theta_weights(beta + h))
    lp = o.mlp_loss(r)
    o.set_mlp(_constant_theta_weights(beta - h))
    lm = o.mlp_loss(r)
    dref = 2 * (1 - theta * q) * (-q) * 0.9 * sig * (1 - sig)
    assert abs((lp - lm) / (2 * h) - dref) <= 1e-8 * max(1.0, abs(dref))


def test_training_loss_averages_levels(tiny):
    # the objective is a mean of per-level ratios ||e_l||^2 / ||r_l||^2: invariant under scaling
    # all vectors, or one level's vector alone, and equal for theta = 1 with or without a model
    # whose output is exactly 1
    o = oracle.Oracle(tiny.K, tiny.J, tiny.D, max_coarse=128)
    ns = [o.A(l).shape[0] for l in range(o.nlev - 1)]
    assert len(ns) >= 2
    r = np.random.default_rng(0).uniform(-1, 1, sum(ns))
    base = o.mlp_loss(r)
    assert np.isclose(o.mlp_loss(3.0 * r), base, rtol=1e-13)
    o.set_mlp(unit_theta_weights())
    assert np.isclose(o.mlp_loss(r), base, rtol=1e-13)
    r2 = r.copy()
    r2[:ns[0]] *= -7.0
    assert np.isclose(o.mlp_loss(r2), base, rtol=1e-13)
    assert 0.0 < base < 1.0
