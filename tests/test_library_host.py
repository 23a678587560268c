"""CPU checks of the C-ABI library: exported symbols, host setup vs the oracle, input errors.

No compute call reaches a device here; amgf_setup_host runs the host setup only.
"""
import ctypes
import os
import re

import numpy as np
import pytest

import contactgen as cg
import oracle
import paper_2505_18576_gb300 as amgf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "amgf.h")).read()
    return sorted(set(re.findall(r"^(?:int|const char\*)\s+(amgf_\w+)\s*\(", src, flags=re.M)))


def test_library_exports_every_declared_symbol():
    lib = amgf.load_library()
    names = declared_symbols()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(amgf.EXPORTED) == names


def _compare_hierarchy(p, **opts):
    o = oracle.Oracle(p.K, p.J, p.D, **opts)
    s = amgf.Solver(p.K, p.J, p.D, host_only=True, **opts)
    assert s.info.nlevels == o.nlev
    for l in range(o.nlev):
        A1, A2 = o.A(l), s.export(0, l)
        assert A1.shape == A2.shape
        assert np.array_equal(A1.indptr, A2.indptr) and np.array_equal(A1.indices, A2.indices)
        assert np.array_equal(A1.data, A2.data)
        if l + 1 < o.nlev:
            P1, P2 = o.P(l), s.export(1, l)
            assert np.array_equal(P1.indptr, P2.indptr) and np.array_equal(P1.indices, P2.indices)
            assert np.array_equal(P1.data, P2.data)
            R2 = s.export(2, l)
            assert (R2 != P2.T).nnz == 0
    if opts.get("filter", 1):
        assert np.array_equal(o.Ic(), s.contact_set())
    s.close()


@pytest.mark.parametrize("dims", [(8, 8, 4), (5, 3, 2), (16, 16, 8)])
def test_host_setup_matches_oracle_bitwise(dims):
    p = cg.make_problem(None, nx=dims[0], ny=dims[1], nz=dims[2], d_lo=-2, d_hi=8, seed=3)
    _compare_hierarchy(p)


def test_host_setup_matches_oracle_options(tiny):
    _compare_hierarchy(tiny, strength_theta=0.25)
    _compare_hierarchy(tiny, interp=1)
    _compare_hierarchy(tiny, interp=1, strength_theta=0.8)
    _compare_hierarchy(tiny, contact_components=1)
    _compare_hierarchy(tiny, max_coarse=400)
    _compare_hierarchy(tiny, p_max=4)
    _compare_hierarchy(tiny, p_max=2, interp=1)


def test_host_setup_truncated_matches_oracle_bitwise():
    # rows of the coarser levels carry many more weights than 4, so the truncation acts
    p = cg.make_problem(None, nx=16, ny=16, nz=8, d_lo=-2, d_hi=8, seed=3)
    _compare_hierarchy(p, p_max=4)
    _compare_hierarchy(p, p_max=3)


def test_host_setup_no_contact(tiny):
    o = oracle.Oracle(tiny.K)
    s = amgf.Solver(tiny.K, host_only=True)
    assert s.info.nc == 0 and s.info.nlevels == o.nlev
    for l in range(o.nlev):
        assert (o.A(l) != s.export(0, l)).nnz == 0


def test_host_only_handle_refuses_device_calls(tiny):
    s = amgf.Solver(tiny.K, tiny.J, tiny.D, host_only=True)
    lib = amgf.load_library()
    for fn in (lib.amgf_apply, lib.amgf_filter_solve_noalloc):
        st = fn(s.h, ctypes.c_void_p(8), ctypes.c_void_p(16), None)
        assert st == 1 and "host-only" in amgf.amgf_last_error()


def test_filter_block_structure(tiny):
    s = amgf.Solver(tiny.K, tiny.J, tiny.D, host_only=True)
    nb, nblk = s.info.filter_block, s.info.filter_nblocks
    assert nb >= 1 and nb * nblk >= s.info.nc and (nblk - 1) * nb < s.info.nc


def test_invalid_inputs(tiny):
    D = tiny.D.copy(); D[0] = np.inf
    with pytest.raises(amgf.AmgfError) as e:
        amgf.Solver(tiny.K, tiny.J, D, host_only=True)
    assert e.value.status == 2
    D = tiny.D.copy(); D[1] = 0.0
    with pytest.raises(amgf.AmgfError) as e:
        amgf.Solver(tiny.K, tiny.J, D, host_only=True)
    assert e.value.status == 3
    bad = cg.CSR(tiny.K.nrows, tiny.K.ncols, tiny.K.row_ptr.copy(), tiny.K.col_idx.copy(), tiny.K.val.copy())
    bad.col_idx[1], bad.col_idx[2] = bad.col_idx[2], bad.col_idx[1]   # unsorted row
    with pytest.raises(amgf.AmgfError) as e:
        amgf.Solver(bad, tiny.J, tiny.D, host_only=True)
    assert e.value.status == 1
    nanK = cg.CSR(tiny.K.nrows, tiny.K.ncols, tiny.K.row_ptr, tiny.K.col_idx, tiny.K.val.copy())
    nanK.val[5] = np.nan
    with pytest.raises(amgf.AmgfError) as e:
        amgf.Solver(nanK, tiny.J, tiny.D, host_only=True)
    assert e.value.status == 2
    with pytest.raises(amgf.AmgfError) as e:
        amgf.Solver(tiny.K, tiny.J, tiny.D, host_only=True, nu=0)
    assert e.value.status == 1
    with pytest.raises(amgf.AmgfError) as e:
        amgf.Solver(tiny.K, tiny.J, tiny.D, host_only=True, precision=4)
    assert e.value.status == 1
    for bad_opt in (dict(filter_algo=2), dict(interp=2), dict(p_max=-1), dict(update_in_place=2), dict(smoother=2),
                    dict(smoother=1, cheby_lower=1.0), dict(cheby_lower=0.0)):
        with pytest.raises(amgf.AmgfError) as e:
            amgf.Solver(tiny.K, tiny.J, tiny.D, host_only=True, **bad_opt)
        assert e.value.status == 1


def test_update_D_host(tiny):
    s = amgf.Solver(tiny.K, tiny.J, tiny.D, host_only=True)
    D2 = tiny.D * 10.0
    s.update_D(D2)
    o = oracle.Oracle(tiny.K, tiny.J, D2)
    for l in range(o.nlev):
        assert (o.A(l) != s.export(0, l)).nnz == 0


def test_device_setup_without_gpu_fails_loudly(tiny):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(amgf.AmgfError) as e:
        amgf.Solver(tiny.K, tiny.J, tiny.D)
    assert e.value.status == 6


def test_host_setup_bounds_matches_oracle_bitwise(tiny):
    rng = np.random.default_rng(7)
    dlo, dhi = 10.0 ** rng.uniform(-3, 3, tiny.n), 10.0 ** rng.uniform(-3, 3, tiny.n)
    o = oracle.Oracle(tiny.K, tiny.J, tiny.D, E=dlo + dhi)
    s = amgf.Solver(tiny.K, tiny.J, tiny.D, host_only=True, d_lower=dlo, d_upper=dhi)
    assert s.info.nlevels == o.nlev
    for l in range(o.nlev):
        A1, A2 = o.A(l), s.export(0, l)
        assert np.array_equal(A1.indptr, A2.indptr) and np.array_equal(A1.indices, A2.indices)
        assert np.array_equal(A1.data, A2.data)
    assert np.array_equal(o.Ic(), s.contact_set())
    # removing the bound term restores the plain hierarchy
    s.update_bounds(tiny.D, None, None)
    o0 = oracle.Oracle(tiny.K, tiny.J, tiny.D)
    assert np.array_equal(o0.A(1).data, s.export(0, 1).data)
    bad = dlo.copy(); bad[0] = -1.0
    with pytest.raises(amgf.AmgfError) as e:
        amgf.Solver(tiny.K, tiny.J, tiny.D, host_only=True, d_lower=bad)
    assert e.value.status == 3
    s.close()


@pytest.mark.parametrize("dims", [(8, 8, 4), (16, 12, 7)])
def test_update_D_fine_is_galerkin_for_reused_interpolation(dims):
    # amgf_update_D_fine keeps P_l, rewrites the contact rows of A_0 with the bits of a fresh
    # assembly, and brings every A_l to R_l A_new P_l (host setup only); two successive updates
    p = cg.make_problem(None, nx=dims[0], ny=dims[1], nz=dims[2], d_lo=-2, d_hi=8, seed=4)
    s = amgf.Solver(p.K, p.J, p.D, host_only=True, max_coarse=128)
    assert s.info.nlevels >= 3
    P_old = [s.export(1, l) for l in range(s.info.nlevels - 1)]
    for seed in (91, 92):
        D2, _ = cg.draw_D_b(seed, p.m, p.n, -2.0, 9.0)
        s.update_D(D2, keep_coarse=True)
        o = oracle.Oracle(p.K, p.J, D2, build_amg=0)
        A = o.S()
        assert (s.export(0, 0) != A).nnz == 0
        for l in range(s.info.nlevels - 1):
            P = s.export(1, l)
            assert (P != P_old[l]).nnz == 0
            A = (P.T @ A @ P).tocsr()
            Al = s.export(0, l + 1)
            assert abs(Al - A).max() <= 1e-12 * abs(A).max()
        o.close()
    s.close()


def test_host_setup_curved_contact_matches_oracle_bitwise():
    # contact rows with tilted normals (six nonzeros per row, all components in I_c)
    p = cg.make_problem(None, nx=10, ny=8, nz=5, d_lo=-2, d_hi=8, seed=3, curvature=1.0)
    _compare_hierarchy(p)
    _compare_hierarchy(p, max_coarse=128, p_max=0)


@pytest.mark.parametrize("algo", [0, 1])
@pytest.mark.parametrize("case", ["z8", "z16", "curved16_1e6", "curved16_1e10"])
def test_host_filter_solve_matches_oracle(case, algo):
    # the cyclic reduction factor applied on the host (the device solve's task semantics)
    # against the oracle's banded Cholesky: backward error and the kappa(A_w) forward bound.
    # With tilted contact normals and D up to 1e10, kappa(A_w) ~ 1e13: the Schur complements
    # are formed through the blocks' Cholesky factors, which keeps them positive definite
    dims, curv, dh = {"z8": ((8, 8, 4), 0.0, 8.0), "z16": ((16, 12, 7), 0.0, 8.0),
                      "curved16_1e6": ((16, 16, 8), 1.0, 6.0), "curved16_1e10": ((16, 16, 8), 1.0, 10.0)}[case]
    p = cg.make_problem(None, nx=dims[0], ny=dims[1], nz=dims[2], d_lo=-2, d_hi=dh, seed=2, curvature=curv)
    s = amgf.Solver(p.K, p.J, p.D, host_only=True, filter_algo=algo)
    o = oracle.Oracle(p.K, p.J, p.D)
    Ic = o.Ic()
    Aw = o.S()[Ic][:, Ic].toarray()
    ev = np.linalg.eigvalsh(Aw)
    v = np.random.default_rng(3).standard_normal(len(Ic))
    w = amgf.amgf_filter_solve_host(s.h, v)
    wo = o.filter_solve(v)
    eps = np.finfo(np.float64).eps
    back = np.linalg.norm(Aw @ w - v) / (np.linalg.norm(Aw, 2) * np.linalg.norm(w))
    assert back <= 64 * eps
    assert np.linalg.norm(w - wo) <= max(1e-12, 16 * eps * ev[-1] / ev[0]) * np.linalg.norm(wo)
    s.close()
    o.close()


def test_staged_sweep_options_rejected():
    # stage_rows in [0, 4096], stage_depth in [2, 8] when staging is on, sell_window >= 0; checked
    # before any device use
    p = cg.make_problem(None, seed=0, nx=4, ny=4, nz=2, d_lo=-2, d_hi=2)
    for kw in (dict(stage_rows=-1), dict(stage_rows=5000), dict(stage_rows=32, stage_depth=1),
               dict(stage_rows=32, stage_depth=9), dict(sell_window=-1)):
        with pytest.raises(amgf.AmgfError) as e:
            amgf.Solver(p.K, p.J, p.D, precision=3, host_only=True, **kw)
        assert e.value.status == 1
    # the binding's struct ends where the C struct ends: the last fields read back their defaults
    o = amgf.amgf_options_default()
    assert (o.stage_rows, o.stage_depth, o.sell_window) == (32, 2, 256)
    assert o.cheby_lower == 0.3


@pytest.mark.parametrize("cname,pyname", [("amgf_options", "Options"), ("amgf_stats", "Stats"),
                                          ("amgf_info", "Info")])
def test_binding_structs_follow_the_header(cname, pyname):
    # the ctypes mirrors of the ABI structs list the header's fields in the header's order
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "amgf.h")).read()
    body = hdr[:hdr.index("} " + cname + ";")]
    body = body[body.rindex("typedef struct {") + len("typedef struct {"):]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        # "type a, b, c" declares several fields
        names = decl.split(None, 1)[1]
        fields += [re.sub(r"\[.*\]", "", x).strip() for x in names.split(",")]
    assert [f[0] for f in getattr(amgf, pyname)._fields_] == fields
