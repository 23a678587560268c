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
