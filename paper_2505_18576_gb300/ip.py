"""Minimal interior-point driver for the two-block contact QP (Section 3, Algorithm 1).

The problem: minimise E(u) = 1/2 u^T K u - f^T u subject to the linearised node-to-node
gap g(u) = J u + g0 >= 0.  With slacks s (g(u) - s = 0, s > 0), multipliers lambda and the
dual variable z = mu / s, the primal-dual residuals of Section 3 are

    r_u = K u - f + J^T lambda,   r_s = -lambda - z,   r_lambda = J u + g0 - s,   r_z = z s - mu

(the lumped slack mass M_s is the identity for unit node-to-node weights).  Eliminating
z^, s^ and lambda^ from the Newton system leaves the condensed system of eq. (linsystem1),

    (K + J^T D J) u^ = b,   D = z / s,   b = -r_u - J^T (D r_lambda + r_s + r_z / s),

which each iteration solves with AMGF-PCG through the C ABI (amgf_update_D + amgf_pcg_solve),
then recovers s^ = J u^ + r_lambda, z^ = -(r_z + z s^) / s, lambda^ = r_s - z^.  Steps keep
s, z positive by the fraction-to-boundary rule (tau = 0.995); the problem is a convex QP, so
no line search is needed.  The optimality errors of Section 3 are measured in the problem's
units (forces by |f|_inf, lengths by |g0|_inf; the paper weights them by lumped mass
matrices instead), and the dimensionless mu decreases once the barrier subproblem's error
falls below kappa_eps mu (kappa_eps = 10), by mu <- max(tol / 10, min(kappa_mu mu, mu^1.5)).

The sequence of D it produces is the interior-point sequence the learned smoother trains on
and against which AMG and AMGF are compared (Section 6: AMG degrades in the late IP
iterations, AMGF stays flat).  `policy` chooses the preconditioner per solve:
  "amgf"  AMGF for every solve;  "amg"  M = B (one V-cycle) for every solve;
  "switch" AMG while the barrier diagonal's spread max(D)/min(D) stays below `switch_spread`,
          then AMGF (the dynamic strategy the paper suggests for future work: AMG in the early
          IP iterations, AMGF once the constraints dominate).
"""
from __future__ import annotations

import json
import time

import numpy as np


def contact_qp(nx: int, ny: int | None = None, nz: int | None = None, load: float = 0.1, curvature: float = 0.2,
               tilted: bool = False):
    """Two stacked blocks pressed together: a downward body force on the upper block (the
    lower block's bottom and the upper block's top are clamped) and an initial gap that
    opens quadratically from the interface centre, g0 = curvature ((x - 1/2)^2 + (y - 1/2)^2),
    so that the contact zone is a disc that grows with the load.  tilted: the gap is measured
    along the normal of that curved surface (contact rows n . (u_upper - u_lower), all three
    components) instead of along z."""
    import contactgen as cg
    ny = nx if ny is None else ny
    nz = max(1, nx // 2) if nz is None else nz
    K = cg.stiffness(nx, ny, nz)
    J = cg.contact_jacobian_curved(nx, ny, nz, curvature) if tilted else cg.contact_jacobian(nx, ny, nz)
    xyz = cg.node_xyz(nx, ny, nz)
    nn = xyz.shape[0]
    f = np.zeros(K.nrows)
    h3 = 0.5 / (nx * ny * nz)           # volume per node of one block
    f[3 * np.arange(nn // 2, nn) + 2] = -load * h3  # nodes of the upper block: body force -load
    Jz = cg.contact_jacobian(nx, ny, nz).to_scipy()  # the node pairs (z-only rows)
    up = Jz.indices[Jz.data > 0] // 3   # upper node of each constraint row (one +1 per row)
    rows = np.repeat(np.arange(Jz.shape[0]), np.diff(Jz.indptr))
    up_row = np.empty(Jz.shape[0], dtype=np.int64)
    up_row[rows[Jz.data > 0]] = up
    x, y = xyz[up_row, 0], xyz[up_row, 1]
    g0 = curvature * ((x - 0.5) ** 2 + (y - 0.5) ** 2)
    return K, J, f, g0


def _max_step(v, dv, tau=0.995):
    neg = dv < 0
    if not np.any(neg):
        return 1.0
    return float(min(1.0, tau * np.min(-v[neg] / dv[neg])))


class GpuSolver:
    """The condensed Newton system on the GPU: amgf_setup / amgf_update_D + amgf_pcg_solve."""

    def __init__(self, K, J, D, use_filter: bool, precision: int = 0, rtol: float = 1e-8, weights=None):
        import torch

        from . import Solver
        self.torch = torch
        self.s = Solver(K, J, D, precision=precision, filter=1 if use_filter else 0, rtol=rtol)
        if weights is not None:
            self.s.set_mlp(weights)
        self.b = torch.zeros(K.nrows, dtype=torch.float64, device="cuda")
        self.x = torch.zeros(K.nrows, dtype=torch.float64, device="cuda")

    def update_D(self, D, keep_coarse: bool = False):
        self.s.update_D(D, keep_coarse=keep_coarse)

    def solve(self, b):
        self.b.copy_(self.torch.from_numpy(np.ascontiguousarray(b)))
        self.x.zero_()
        st = self.s.pcg_solve(self.b, self.x)
        return self.x.cpu().numpy(), int(st.iters), float(st.t_solve_s)

    def close(self):
        self.s.close()


def solve(K, J, f, g0, tol: float = 1e-6, mu0: float = 1e-1, max_iter: int = 200, precision: int = 0,
          policy: str = "amgf", switch_spread: float = 1e6, weights=None, rtol: float = 1e-8,
          verbose: bool = False, record_D: bool = False, make_solver=None, lag: float | None = None):
    """Run the IP loop; returns (u, info) with one record per Newton step in info["steps"].

    make_solver(D, use_filter) -> object with update_D(D, keep_coarse), solve(b) -> (x, iters,
    seconds) and close(); default: GpuSolver (the library's AMGF-PCG on the current CUDA device).
    lag: None rebuilds the AMG hierarchy for every Newton system (B := AMG(A)); a number keeps
    the coarse levels of the last full setup (amgf_update_D_fine: new fine-level operator and
    filter only) until a solve needs more than (1 + lag) times the PCG iterations of the first
    solve after that setup."""
    if make_solver is None:
        def make_solver(D, use_filter):
            return GpuSolver(K, J, D, use_filter, precision=precision, rtol=rtol, weights=weights)
    Jsp = J.to_scipy()
    Ksp = K.to_scipy()
    n, m = K.nrows, J.nrows
    # residuals are measured in the problem's own units: forces by fs = |f|_inf, lengths by
    # gs = |g0|_inf (1 for a flat interface), complementarity and mu by fs * gs
    fs = float(np.abs(f).max()) or 1.0
    gs = float(np.abs(g0).max()) or 1.0
    u = np.zeros(n)
    s = np.maximum(g0, 1e-2 * gs)
    mu = mu0 * fs * gs
    z = mu / s
    lam = -z.copy()
    kappa_eps, kappa_mu = 10.0, 0.2

    def err(r_u, r_s, r_l, r_z):
        return max(np.abs(r_u).max() / fs, np.abs(r_s).max() / fs, np.abs(r_l).max() / gs,
                   np.abs(r_z).max() / (fs * gs))
    solvers = {}
    base_iters = {}  # PCG iterations of the first solve after each solver's last full setup
    full_next = {}
    log = []
    e0 = np.inf
    t_start = time.perf_counter()
    try:
        for it in range(max_iter):
            r_u = Ksp @ u - f + Jsp.T @ lam
            r_s = -lam - z
            r_l = Jsp @ u + g0 - s
            e0 = err(r_u, r_s, r_l, z * s)
            if e0 < tol:
                break
            mu_n = mu / (fs * gs)  # dimensionless barrier parameter
            while err(r_u, r_s, r_l, z * s - mu) < kappa_eps * mu_n and mu_n > tol / 10:
                mu_n = max(tol / 10, min(kappa_mu * mu_n, mu_n ** 1.5))
                mu = mu_n * fs * gs
            r_z = z * s - mu
            D = z / s
            spread = float(D.max() / D.min())
            use_filter = policy == "amgf" or (policy == "switch" and spread >= switch_spread)
            b = -r_u - Jsp.T @ (D * r_l + r_s + r_z / s)
            key = 1 if use_filter else 0
            t0 = time.perf_counter()
            lagged = False
            if key not in solvers:
                solvers[key] = make_solver(D, bool(key))
                full_next[key] = True
            else:
                lagged = lag is not None and not full_next.get(key, True)
                solvers[key].update_D(D, keep_coarse=lagged)
            t_setup = time.perf_counter() - t0
            du, kits, tsol = solvers[key].solve(b)
            if not lagged:
                base_iters[key] = kits
            full_next[key] = lag is None or kits > (1.0 + lag) * base_iters[key]
            ds = Jsp @ du + r_l
            dz = -(r_z + z * ds) / s
            dl = r_s - dz
            ap = _max_step(s, ds)
            ad = _max_step(z, dz)
            u += ap * du
            s += ap * ds
            lam += ap * dl
            z += ad * dz
            rec = {"iter": it, "mu": mu / (fs * gs), "e_opt": float(e0), "D_min": float(D.min()), "D_max": float(D.max()),
                   "spread": spread, "preconditioner": "amgf" if use_filter else "amg", "pcg_iters": kits,
                   "solve_s": tsol, "setup_s": t_setup, "lagged_setup": lagged, "alpha_p": ap, "alpha_d": ad,
                   "active": int(np.sum(z > s))}  # complementarity: active where z dominates s
            if record_D:
                rec["D"] = D.copy()
                rec["b"] = b.copy()
            log.append(rec)
            if verbose:
                print(json.dumps({k: v for k, v in rec.items() if k not in ("D", "b")}), flush=True)
    finally:
        for sv in solvers.values():
            sv.close()
    return u, {"steps": log, "wall_s": time.perf_counter() - t_start, "converged": bool(e0 < tol),
               "final_e_opt": float(e0), "mu": mu / (fs * gs), "lambda": lam, "slack": s}


if __name__ == "__main__":
    import argparse
    ap = argparse.ArgumentParser(description="interior-point solve of the two-block contact QP with AMGF-PCG")
    ap.add_argument("--nx", type=int, default=32)
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--precision", type=int, default=0)
    ap.add_argument("--policy", default="amgf", choices=["amgf", "amg", "switch"])
    ap.add_argument("--tilted", action="store_true", help="contact along the curved interface's normals")
    ap.add_argument("--switch-spread", type=float, default=1e6)
    ap.add_argument("--lag", type=float, default=None,
                    help="keep the coarse levels while PCG iterations stay within (1 + lag) of the last full setup's")
    ap.add_argument("--save-D", default=None, help="write the IP sequence of D to this .npz")
    ap.add_argument("--json", default=None)
    a = ap.parse_args()
    K, J, f, g0 = contact_qp(a.nx, tilted=a.tilted)
    u, info = solve(K, J, f, g0, tol=a.tol, precision=a.precision, policy=a.policy, switch_spread=a.switch_spread,
                    verbose=True, record_D=a.save_D is not None, lag=a.lag)
    steps = info["steps"]
    summary = {"nx": a.nx, "n": K.nrows, "m": J.nrows, "policy": a.policy, "lag": a.lag, "ip_iters": len(steps),
               "full_setups": sum(1 for r in steps if not r["lagged_setup"]),
               "converged": info["converged"], "final_e_opt": info["final_e_opt"],
               "pcg_iters_total": sum(r["pcg_iters"] for r in steps),
               "solve_s_total": sum(r["solve_s"] for r in steps), "setup_s_total": sum(r["setup_s"] for r in steps),
               "wall_s": info["wall_s"], "active_final": steps[-1]["active"] if steps else 0}
    print(json.dumps(summary), flush=True)
    if a.save_D:
        np.savez(a.save_D, D=np.array([r["D"] for r in steps]))
    if a.json:
        with open(a.json, "w") as fh:
            json.dump({"summary": summary, "steps": [{k: v for k, v in r.items() if k not in ("D", "b")} for r in steps]}, fh,
                      indent=1)
