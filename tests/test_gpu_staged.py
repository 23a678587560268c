"""Staged coarse-level sweeps of the mixed-precision V-cycle (csr_staged_kernel).

The staged kernel streams each tile's row pointers, column indices, BF16 values and epilogue
vectors into shared memory with bulk asynchronous copies, while the consumer warps only
gather x.  Each lane sums the same entries in the same order as csr_kernel, so the two are
compared bit for bit: the V-cycle output, the AMGF apply, and a whole PCG solve (iterations and
solution).  The cases span tiles of one pass of row groups up to tiles of about a hundred rows,
2 to 8 tiles in flight (8 is cut back until the stages fit in shared memory), ragged last
tiles and levels with fewer tiles than CTAs.  The mixed path itself is checked against the FP64
oracle in test_gpu_mixed.py with staging on (the default).
"""
import numpy as np
import pytest

import contactgen as cg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, np.float64)).cuda()


@pytest.fixture(scope="module")
def problems():
    return {
        "n24": cg.make_problem(None, seed=7, nx=24, ny=24, nz=12, d_lo=-2, d_hi=10),
        "n40": cg.make_problem(None, seed=8, nx=40, ny=40, nz=20, d_lo=-2, d_hi=12),
    }


@pytest.mark.parametrize("name,rows,depth", [("n24", 1, 2), ("n24", 32, 4), ("n24", 96, 3), ("n40", 32, 2),
                                             ("n40", 64, 2), ("n40", 48, 8)])
def test_staged_vcycle_and_apply_bitwise(problems, name, rows, depth):
    precision = 3
    import paper_2505_18576_gb300 as m
    p = problems[name]
    plain = m.Solver(p.K, p.J, p.D, precision=precision, stage_rows=0)
    staged = m.Solver(p.K, p.J, p.D, precision=precision, stage_rows=rows, stage_depth=depth)
    assert plain.info.staged_levels == 0
    mask = int(staged.info.staged_levels)
    print(f"{name} precision {precision} rows {rows} depth {depth}: staged levels mask {mask:#x} "
          f"of {staged.info.nlevels}")
    assert mask != 0 and (mask & 1) == 0  # some coarse level is staged, the fine level never
    r = dev(np.random.default_rng(3).standard_normal(p.n))
    for f in ("vcycle", "apply"):
        a = torch.empty(p.n, dtype=torch.float64, device="cuda")
        b = torch.empty(p.n, dtype=torch.float64, device="cuda")
        getattr(plain, f)(r, a)
        getattr(staged, f)(r, b)
        torch.cuda.synchronize()
        assert torch.all(torch.isfinite(b))
        assert torch.equal(a, b), f"{f}: staged and plain sweeps differ"
    plain.close()
    staged.close()


def test_staged_pcg_bitwise(problems):
    precision = 3
    import paper_2505_18576_gb300 as m
    p = problems["n40"]
    xs = []
    its = []
    for rows in (0, 32):
        s = m.Solver(p.K, p.J, p.D, precision=precision, stage_rows=rows)
        x = torch.zeros(p.n, dtype=torch.float64, device="cuda")
        st = s.pcg_solve(dev(p.b), x)
        torch.cuda.synchronize()
        xs.append(x.cpu().numpy())
        its.append(st.iters)
        s.close()
    print(f"precision {precision}: iterations plain {its[0]}, staged {its[1]}")
    assert its[0] == its[1]
    assert np.array_equal(xs[0], xs[1])


def test_staged_after_in_place_update(problems):
    # amgf_update_D_fine rewrites the coarse values in the same arrays; the staged sweeps read them
    import paper_2505_18576_gb300 as m
    p = problems["n24"]
    D2 = p.D * np.exp(np.random.default_rng(5).uniform(-1.0, 1.0, p.D.shape))
    out = []
    for rows in (0, 32):
        s = m.Solver(p.K, p.J, p.D, precision=3, stage_rows=rows)
        s.update_D(D2, keep_coarse=True)
        x = torch.empty(p.n, dtype=torch.float64, device="cuda")
        s.apply(dev(np.random.default_rng(9).standard_normal(p.n)), x)
        torch.cuda.synchronize()
        out.append(x.cpu().numpy())
        s.close()
    assert np.array_equal(out[0], out[1])



def test_staged_only_where_measured_faster(problems):
    # BF16 values and short rows (level 1 here); FP32 values never
    import paper_2505_18576_gb300 as m
    p = problems["n40"]
    for precision, staged in ((1, False), (2, False), (3, True)):
        s = m.Solver(p.K, p.J, p.D, precision=precision)
        assert (int(s.info.staged_levels) != 0) == staged, (precision, int(s.info.staged_levels))
        if staged:
            assert int(s.info.staged_levels) & 2  # level 1
        s.close()
