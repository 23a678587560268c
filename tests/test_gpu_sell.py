"""FP64 coarse levels swept from the sliced-ELL copy (sell_kernel), one lane per row.

Each lane sums its row in CSR order in one FMA chain, so the result of a row does not depend on
where the length sort puts it: every sort window gives the same bits.  Against the lane-group
CSR kernel (partial sums per lane, then a shuffle reduction) the rows differ by rounding only:
the V-cycle agrees to 1e-13 relative and PCG takes the same iterations (within one).  The AMGF
apply passes that rounding difference through the exact filter solve, which amplifies it by
up to kappa(A_w) (about 1e10 with D up to 1e8 on these meshes), so the apply is held to
16 u kappa(A_w) = 2e-5 only.  The
oracle parity of the V-cycle at this size (1e-12) runs with the default options in
test_gpu_fullsize.py.  Values written in place by amgf_update_D_fine reach the sliced-ELL copy
too (bitwise equal to uploading the whole updated image).
"""
import numpy as np
import pytest

import contactgen as cg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, np.float64)).cuda()


@pytest.fixture(scope="module")
def c64():
    return cg.make_problem("c64", seed=1)


def outputs(s, p):
    r = dev(np.random.default_rng(4).standard_normal(p.n))
    out = []
    for f in ("vcycle", "apply"):
        z = torch.empty(p.n, dtype=torch.float64, device="cuda")
        getattr(s, f)(r, z)
        out.append(z)
    x = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    st = s.pcg_solve(dev(p.b), x)
    torch.cuda.synchronize()
    return [o.cpu().numpy() for o in out] + [x.cpu().numpy()], st.iters


def test_sell_against_csr_and_windows(c64):
    import paper_2505_18576_gb300 as m
    p = c64
    ref = m.Solver(p.K, p.J, p.D, sell_window=0)
    assert ref.info.sell_levels == 0
    o_ref, it_ref = outputs(ref, p)
    ref.close()
    got = {}
    for win in (1, 32, 256, 1 << 20):
        s = m.Solver(p.K, p.J, p.D, sell_window=win)
        mask = int(s.info.sell_levels)
        assert mask & 2 and not mask & 1  # level 1 (373,706 rows, the last slice ragged), never the fine level
        got[win] = outputs(s, p)
        s.close()
    o0, it0 = got[1]
    for win, (o, it) in got.items():
        assert it == it0
        for a, b in zip(o, o0):
            assert np.array_equal(a, b), f"window {win}: results depend on the sort window"
    for name, a, b, tol in zip(("vcycle", "apply"), o0[:2], o_ref[:2], (1e-13, 16 * 2.0**-53 * 1e10)):
        err = np.linalg.norm(a - b) / np.linalg.norm(b)
        print(f"{name}: sliced ELL vs CSR rel diff {err:.2e}")
        assert err <= tol
    assert abs(it0 - it_ref) <= 1


def test_sell_in_place_update(c64):
    import paper_2505_18576_gb300 as m
    p = c64
    D2 = p.D * np.exp(np.random.default_rng(6).uniform(-1.0, 1.0, p.D.shape))
    res = []
    for inplace in (1, 0):
        s = m.Solver(p.K, p.J, p.D, update_in_place=inplace)
        assert int(s.info.sell_levels) & 2
        s.update_D(D2, keep_coarse=True)
        z = torch.empty(p.n, dtype=torch.float64, device="cuda")
        s.apply(dev(np.random.default_rng(8).standard_normal(p.n)), z)
        torch.cuda.synchronize()
        res.append(z.cpu().numpy())
        s.close()
    assert np.array_equal(res[0], res[1])
