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


@pytest.mark.parametrize("dims", [(8, 8, 4), (5, 3, 2), (16, 12, 7)])
def test_noalloc_matches_filter_solve_on_two_calls(dims):
    import paper_2505_18576_gb300 as m
    p = cg.make_problem(None, seed=4, nx=dims[0], ny=dims[1], nz=dims[2], d_lo=-2, d_hi=8)
    s = m.Solver(p.K, p.J, p.D)
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
