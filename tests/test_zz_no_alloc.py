"""amgf_filter_solve_noalloc: the filter solve for callers that cannot allocate device memory.

Such callers (another allocator owns the whole device, or a cudaMalloc with the
synchronisation it may imply is not allowed in their loop) get the same result as
amgf_filter_solve, with the work vectors kept in a fixed array inside the library.
This file is collected last so that a failure here does not stop the other tests, and it
passes both alone in a fresh process and after them.
"""
import numpy as np
import pytest

import contactgen as cg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("algo", [0, 1])
@pytest.mark.parametrize("dims", [(8, 8, 4), (5, 3, 2), (16, 12, 7)])
def test_noalloc_matches_filter_solve_on_two_calls(dims, algo):
    # filter_algo 0 (block cyclic reduction) uses three of the array's four vectors, filter_algo 1
    # (block LDL^T sweeps) all four
    import paper_2505_18576_gb300 as m
    p = cg.make_problem(None, seed=4, nx=dims[0], ny=dims[1], nz=dims[2], d_lo=-2, d_hi=8)
    s = m.Solver(p.K, p.J, p.D, filter_algo=algo)
    nc = s.nc
    rng = np.random.default_rng(21)
    va = torch.from_numpy(rng.standard_normal(nc)).cuda()
    vb = torch.from_numpy(rng.standard_normal(nc)).cuda()
    wa = torch.full((nc,), np.nan, dtype=torch.float64, device="cuda")
    wb = torch.full((nc,), np.nan, dtype=torch.float64, device="cuda")
    # two calls in a row on the allocation-free entry point
    m.amgf_filter_solve_noalloc(s.h, va, wa, nc)
    m.amgf_filter_solve_noalloc(s.h, vb, wb, nc)
    ra = torch.empty(nc, dtype=torch.float64, device="cuda")
    rb = torch.empty(nc, dtype=torch.float64, device="cuda")
    s.filter_solve(va, ra)
    s.filter_solve(vb, rb)
    torch.cuda.synchronize()
    for w, r in ((wa, ra), (wb, rb)):
        w, r = w.cpu().numpy(), r.cpu().numpy()
        assert np.all(np.isfinite(w))
        assert np.linalg.norm(w - r) <= 1e-12 * np.linalg.norm(r)
    s.close()


def test_noalloc_rejects_a_filter_larger_than_its_array():
    # a long strip with all three components of every contact node in the filter space: the
    # block-tridiagonal factor has 22 x 6001 = 132,022 rows, more than the array's 4 x 131,072
    # doubles allow; the call fails on the host before any launch and leaves the handle usable
    import paper_2505_18576_gb300 as m
    p = cg.make_problem(None, seed=0, nx=11000, ny=1, nz=1, d_lo=-2, d_hi=4)
    s = m.Solver(p.K, p.J, p.D, contact_components=1)
    nc = s.nc
    assert s.info.filter_block * s.info.filter_nblocks > 131072
    v = torch.from_numpy(np.random.default_rng(3).standard_normal(nc)).cuda()
    w = torch.empty(nc, dtype=torch.float64, device="cuda")
    with pytest.raises(m.AmgfError) as e:
        m.amgf_filter_solve_noalloc(s.h, v, w, nc)
    assert e.value.status == 1 and "too large" in str(e.value)
    s.filter_solve(v, w)
    torch.cuda.synchronize()
    assert torch.all(torch.isfinite(w))
    s.close()
