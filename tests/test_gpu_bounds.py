"""GPU parity of the bound-constrained variant A = K + J^T D J + diag(D_lo + D_hi)
(Section 3, remark on bound constraints) against the oracle, same tolerances as
tests/test_gpu_parity.py (V-cycle 1e-12; apply max(1e-12, 16 u kappa(A_w)); PCG iterations
within +-1 and the A-norm bound 2 rtol sqrt(kappa(MA)))."""
import numpy as np
import pytest

import contactgen as cg
import oracle
from oracle.lanczos import kappa_estimate

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
EPS = np.finfo(np.float64).eps


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, np.float64)).cuda()


@pytest.fixture(scope="module", params=["tiny", "n16"])
def case(request):
    import paper_2505_18576_gb300 as m
    dims = dict(tiny=dict(nx=8, ny=8, nz=4, d_lo=-2, d_hi=4), n16=dict(nx=16, ny=12, nz=7, d_lo=-2, d_hi=8))
    p = cg.make_problem(None, seed=3, **dims[request.param])
    rng = np.random.default_rng(11)
    dlo, dhi = 10.0 ** rng.uniform(-3, 4, p.n), 10.0 ** rng.uniform(-3, 4, p.n)
    o = oracle.Oracle(p.K, p.J, p.D, E=dlo + dhi)
    s = m.Solver(p.K, p.J, p.D, d_lower=dlo, d_upper=dhi)
    yield request.param, p, o, s, dlo, dhi
    s.close()


def test_bounds_vcycle_and_apply(case):
    name, p, o, s, *_ = case
    r = np.random.default_rng(1).standard_normal(p.n)
    x = torch.empty(p.n, dtype=torch.float64, device="cuda")
    s.vcycle(dev(r), x)
    xo = o.vcycle(r)
    assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-12 * np.linalg.norm(xo)
    Ic = o.Ic()
    ev = np.linalg.eigvalsh(o.S()[Ic][:, Ic].toarray())
    tol = max(1e-12, 16 * EPS * ev[-1] / ev[0])
    z = torch.empty(p.n, dtype=torch.float64, device="cuda")
    s.apply(dev(r), z)
    zo = o.apply(r)
    assert np.linalg.norm(z.cpu().numpy() - zo) <= tol * np.linalg.norm(zo)


@pytest.mark.parametrize("precision", [0, 3])
def test_bounds_pcg(case, precision):
    import paper_2505_18576_gb300 as m
    name, p, o, s0, dlo, dhi = case
    xo, ko, sto, al, be, _ = o.pcg(p.b, tol=1e-8)
    kap, _, _ = kappa_estimate(al, be)
    s = s0 if precision == 0 else m.Solver(p.K, p.J, p.D, d_lower=dlo, d_upper=dhi, precision=precision)
    x = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    st = s.pcg_solve(dev(p.b), x)
    S = o.S()
    d = x.cpu().numpy() - xo
    ea = np.sqrt(d @ (S @ d)) / np.sqrt(xo @ (S @ xo))
    print(f"{name} precision {precision}: iters {st.iters} (oracle {ko}), A-norm diff {ea:.2e}")
    assert st.converged == 1
    if precision == 0:
        assert abs(st.iters - ko) <= 1
        assert ea <= 2e-8 * np.sqrt(kap)
    else:
        assert st.iters <= 2 * ko + 5
        assert ea <= 4e-8 * np.sqrt(kap)
    if s is not s0:
        s.close()
