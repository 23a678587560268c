"""Pins of the seeded input generator (contactgen): Q1 elasticity, contact Jacobian, draws.

The generator is not the method; these checks make sure its K, J, D and b are the
linear-elasticity / node-to-node contact inputs of Section 2.2 and Section 3.
"""
import numpy as np
import pytest

import contactgen as cg


def lame(E=1.0, nu=0.3):
    return E * nu / ((1 + nu) * (1 - 2 * nu)), E / (2 * (1 + nu))


def test_sizes_match_workload_table():
    # n = 3 * free nodes, m = interface nodes; clamped faces eliminated
    assert cg.sizes(8, 8, 4) == (1944, 81)
    assert cg.sizes(64, 64, 32) == (811200, 4225)
    assert cg.sizes(96, 96, 48) == (2709792, 9409)
    assert cg.sizes(160, 160, 80) == (12442080, 25921)


def test_element_stiffness_closed_forms():
    h = 0.125
    Ke = cg.element_stiffness(h, h, h)
    lam, mu = lame()
    assert np.array_equal(Ke, Ke.T)
    # diagonal of the Q1 brick: int (lam+mu)(d_c phi)^2 + mu |grad phi|^2 = h (lam + 4 mu) / 9
    assert np.allclose(np.diag(Ke), h * (lam + 4 * mu) / 9, rtol=1e-14)
    # exactly six zero-energy modes (rigid motions), all other eigenvalues positive
    ev = np.linalg.eigvalsh(Ke)
    assert np.all(np.abs(ev[:6]) < 1e-12 * ev[-1])
    assert ev[6] > 1e-3 * ev[-1]


def _rigid_modes(xyz):
    nn = xyz.shape[0]
    modes = []
    for c in range(3):
        u = np.zeros((nn, 3)); u[:, c] = 1.0; modes.append(u.ravel())
    x, y, z = xyz[:, 0], xyz[:, 1], xyz[:, 2]
    for (a, b) in ((0, 1), (1, 2), (0, 2)):
        u = np.zeros((nn, 3)); u[:, a] = -xyz[:, b]; u[:, b] = xyz[:, a]; modes.append(u.ravel())
    return np.array(modes)


def test_unclamped_stiffness_null_space():
    K = cg.stiffness(4, 4, 2, clamp_bottom=False, clamp_top=False).to_scipy()
    xyz = cg.node_xyz(4, 4, 2, clamp_bottom=False, clamp_top=False)
    scale = abs(K).max()
    for u in _rigid_modes(xyz):
        assert np.abs(K @ u).max() < 1e-12 * scale
    # two separate blocks: 12 zero modes in total
    ev = np.linalg.eigvalsh(K.toarray())
    assert np.sum(ev < 1e-10 * ev[-1]) == 12


def test_patch_test_constant_strain():
    # a linear displacement field u = G x is an exact FE solution: interior rows of K u vanish
    nx, ny, nz = 4, 4, 4
    K = cg.stiffness(nx, ny, nz, clamp_bottom=False, clamp_top=False).to_scipy()
    xyz = cg.node_xyz(nx, ny, nz, clamp_bottom=False, clamp_top=False)
    rng = np.random.default_rng(1)
    G = rng.standard_normal((3, 3))
    u = (xyz @ G.T).ravel()
    f = (K @ u).reshape(-1, 3)
    eps = 1e-9
    zb = xyz[:, 2]
    interior = ((xyz[:, 0] > eps) & (xyz[:, 0] < 1 - eps) & (xyz[:, 1] > eps) & (xyz[:, 1] < 1 - eps)
                & (np.abs(zb - 0.0) > eps) & (np.abs(zb - 0.5) > eps) & (np.abs(zb - 1.0) > eps))
    assert interior.sum() > 0
    assert np.abs(f[interior]).max() < 1e-12 * np.abs(K).max()


def test_clamped_stiffness_spd_and_symmetric(tiny):
    K = tiny.K.to_scipy()
    assert abs(K - K.T).max() == 0.0
    np.linalg.cholesky(K.toarray())  # raises if not SPD
    # rows sorted, 27-point nodal stencil at most
    rp, ci = tiny.K.row_ptr, tiny.K.col_idx
    for i in range(0, tiny.n, 97):
        row = ci[rp[i]:rp[i + 1]]
        assert np.all(np.diff(row) > 0) and len(row) <= 81


def test_contact_jacobian(tiny):
    J = tiny.J.to_scipy().toarray()
    assert J.shape == (81, 1944)
    assert np.all((J != 0).sum(axis=1) == 2)
    assert np.all(J.sum(axis=1) == 0.0)            # +1 upper, -1 lower
    cols = np.nonzero(J)[1]
    assert np.all(cols % 3 == 2)                    # normal (z) components only
    xyz = cg.node_xyz(8, 8, 4)
    for r in range(81):
        lo, up = np.nonzero(J[r])[0]
        assert J[r, lo] == -1 and J[r, up] == 1
        assert np.allclose(xyz[lo // 3], xyz[up // 3])   # coincident interface nodes
        assert abs(xyz[lo // 3][2] - 0.5) < 1e-15


def test_rng_published_values():
    # SplitMix64 from state 0 (Steele, Lea, Flood 2014 reference code)
    assert [int(x) for x in cg.splitmix_raw(0, 3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                                         0x06C45D188009454F]
    # xoshiro256** (Blackman & Vigna) from state {1, 2, 3, 4}
    assert [int(x) for x in cg.xoshiro_from_state([1, 2, 3, 4], 3)] == [11520, 0, 1509978240]


def test_draws_distribution():
    D, b = cg.draw_D_b(7, 20000, 20000, -2.0, 8.0)
    lg = np.log10(D)
    assert lg.min() >= -2.0 and lg.max() < 8.0
    assert abs(lg.mean() - 3.0) < 0.1 and abs(lg.std() - 10 / np.sqrt(12)) < 0.05
    assert abs(b.mean()) < 0.03 and abs(b.std() - 1.0) < 0.03
    D2, b2 = cg.draw_D_b(7, 20000, 20000, -2.0, 8.0)
    assert np.array_equal(D, D2) and np.array_equal(b, b2)
    D3, _ = cg.draw_D_b(8, 20000, 20000, -2.0, 8.0)
    assert not np.array_equal(D, D3)
