"""Trainer driver of the learned l1-Jacobi smoother weights (not in the paper).

Two training sets: the synthetic barrier sequence below (`run_experiment`), and the barrier
diagonals of an actual interior-point run of the two-block contact QP (`run_ip_experiment`,
ip.py), evaluated on the Newton systems of a run with another load.

A small MLP (6 -> 32 -> 32 -> 1, ReLU) maps each row's features to a damping
theta in [0.3, 1.2] of the l1-Jacobi step (W = theta / l1).  It is trained on the
sequence of Schur complements A_k = K + J^T D_k J that an interior-point run produces:
the barrier diagonal's spread grows from 1e2 to 1e10 over the systems (Section 4 and
Fig. "cond(D)": D's condition number grows exponentially over the IP iterations).
Training minimises the smoothing loss mean_l ||(I - A_l W_l) r_l||^2 / ||r_l||^2 with
Adam; forward, backward and update run in the library's CUDA kernels
(amgf_mlp_train).  The result is measured by the PCG iteration count on held-out
systems, with theta = 1 (plain AMGF) as the fallback.
"""
from __future__ import annotations

import json
import os
import time

import numpy as np

from . import Solver, amgf_mlp_train

MLP_NW = 1313


def init_weights(seed: int = 0, scale: float = 0.1) -> np.ndarray:
    """Small random weights with the output bias set so that theta starts at 1."""
    rng = np.random.default_rng(seed)
    w = (rng.standard_normal(MLP_NW) * scale).astype(np.float32)
    w[1280:1312] = 0.0             # output layer starts flat
    w[1312] = np.float32(np.log(3.5))  # 0.3 + 0.9 * sigmoid(log 3.5) = 1
    return w


def ip_like_barriers(m: int, n_systems: int = 30, spread_lo: float = 2.0, spread_hi: float = 10.0,
                     seed0: int = 100, held_out: bool = False):
    """D_k log-uniform in [1e-2, 1e-2 * 10^s_k]: s_k grows linearly from spread_lo to spread_hi
    (training sequence, seeds seed0 + k), or is drawn uniformly in that range (held-out systems)."""
    import contactgen as cg
    out = []
    rng = np.random.default_rng(seed0)
    for k in range(n_systems):
        s = rng.uniform(spread_lo, spread_hi) if held_out else \
            spread_lo + (spread_hi - spread_lo) * k / max(1, n_systems - 1)
        D, _ = cg.draw_D_b(seed0 + k, m, 1, -2.0, -2.0 + s)
        out.append((s, D))
    return out


def train(K, J, barriers, iters_per_system: int = 20, lr: float = 1e-3, seed: int = 0, weights=None,
          verbose: bool = False):
    """Adam on the smoothing loss over the barrier sequence.  Returns (weights, log)."""
    w = init_weights(seed) if weights is None else np.array(weights, dtype=np.float32)
    m = np.zeros(MLP_NW, np.float32)
    v = np.zeros(MLP_NW, np.float32)
    step = 0
    log = []
    s = Solver(K, J, barriers[0][1], precision=0)
    try:
        for k, (spread, D) in enumerate(barriers):
            if k > 0:
                s.update_D(D)
            t0 = time.perf_counter()
            step, loss = amgf_mlp_train(s.h, w, m, v, step, iters_per_system, lr, seed * 1000003 + k)
            log.append({"system": k, "spread": float(spread), "loss_first": float(loss[0]),
                        "loss_last": float(loss[-1]), "seconds": time.perf_counter() - t0})
            if verbose:
                print(json.dumps(log[-1]), flush=True)
    finally:
        s.close()
    return w, log


def evaluate(K, J, barriers, b, weights, precision: int = 1, rtol: float = 1e-8):
    """PCG iterations and device time with theta = 1 and with the learned weights on each system."""
    import torch
    out = []
    s = Solver(K, J, barriers[0][1], precision=precision, rtol=rtol)
    try:
        bd = torch.from_numpy(np.ascontiguousarray(b)).cuda()
        x = torch.zeros(len(b), dtype=torch.float64, device="cuda")
        for k, (spread, D) in enumerate(barriers):
            if k > 0:
                s.update_D(D)
            s.set_mlp(None)
            x.zero_()
            st0 = s.pcg_solve(bd, x)
            xp = x.clone()
            s.set_mlp(weights)
            x.zero_()
            st1 = s.pcg_solve(bd, x)
            out.append({"system": k, "spread": float(spread), "plain_iters": st0.iters, "learned_iters": st1.iters,
                        "plain_s": st0.t_solve_s, "learned_s": st1.t_solve_s, "fallback": st1.mlp_fallback,
                        "rel_diff": float(torch.linalg.norm(x - xp) / torch.linalg.norm(xp))})
            s.set_mlp(None)
    finally:
        s.close()
    return out


def evaluate_systems(K, J, systems, weights, precision: int = 1, rtol: float = 1e-8):
    """Like evaluate, for a list of (D, b) pairs (each Newton system with its own right-hand side)."""
    import torch
    out = []
    s = Solver(K, J, systems[0][0], precision=precision, rtol=rtol)
    try:
        x = torch.zeros(K.nrows, dtype=torch.float64, device="cuda")
        for k, (D, b) in enumerate(systems):
            if k > 0:
                s.update_D(D)
            bd = torch.from_numpy(np.ascontiguousarray(b)).cuda()
            s.set_mlp(None)
            x.zero_()
            st0 = s.pcg_solve(bd, x)
            s.set_mlp(weights)
            x.zero_()
            st1 = s.pcg_solve(bd, x)
            out.append({"system": k, "spread": float(D.max() / D.min()), "plain_iters": st0.iters,
                        "learned_iters": st1.iters, "plain_s": st0.t_solve_s, "learned_s": st1.t_solve_s,
                        "fallback": st1.mlp_fallback})
            s.set_mlp(None)
    finally:
        s.close()
    return out


def run_ip_experiment(nx: int = 64, iters_per_system: int = 20, lr: float = 1e-3, seed: int = 0, precision: int = 1,
                      train_load: float = 0.1, train_curvature: float = 0.2, eval_load: float = 0.15,
                      eval_curvature: float = 0.3, out: str | None = None, verbose: bool = True) -> dict:
    """Train on the barrier diagonals of an actual interior-point run (ip.py, the two-block
    contact QP with one load) and evaluate on the Newton systems of a run with another load
    and gap, each with its own right-hand side."""
    from . import ip
    K, J, f, g0 = ip.contact_qp(nx, load=train_load, curvature=train_curvature)
    _, info = ip.solve(K, J, f, g0, record_D=True, precision=precision)
    train_set = [(r["spread"], r["D"]) for r in info["steps"]]
    _, _, f2, g2 = ip.contact_qp(nx, load=eval_load, curvature=eval_curvature)
    _, info2 = ip.solve(K, J, f2, g2, record_D=True, precision=precision)
    eval_sys = [(r["D"], r["b"]) for r in info2["steps"]]
    t0 = time.perf_counter()
    w, log = train(K, J, train_set, iters_per_system, lr, seed, verbose=verbose)
    t_train = time.perf_counter() - t0
    ev = evaluate_systems(K, J, eval_sys, w, precision=precision)
    plain = sum(e["plain_iters"] for e in ev)
    learned = sum(e["learned_iters"] for e in ev)
    res = {"nx": nx, "train_systems": len(train_set), "eval_systems": len(eval_sys), "train_seconds": t_train,
           "ip_iters_train": len(info["steps"]), "ip_iters_eval": len(info2["steps"]),
           "plain_iters_total": plain, "learned_iters_total": learned,
           "plain_s_total": sum(e["plain_s"] for e in ev), "learned_s_total": sum(e["learned_s"] for e in ev),
           "decision": "learned" if learned < plain else "fallback: theta = 1", "eval": ev, "train_log": log}
    if out:
        unit = np.zeros(MLP_NW, np.float32)
        unit[1312] = np.float32(np.log(3.5))
        save_weights(out, w if learned < plain else unit, {"nx": nx, "source": "interior-point run",
                                                            "decision": res["decision"]})
    if verbose:
        print(json.dumps({k: v for k, v in res.items() if k not in ("train_log", "eval")}), flush=True)
    return res


def save_weights(path: str, w, meta: dict | None = None):
    """Checkpoint: npz with the weights, a format version and free-form metadata."""
    np.savez(path, weights=np.asarray(w, np.float32), version=np.array([1]),
             meta=np.array(json.dumps(meta or {})))


def load_weights(path: str) -> np.ndarray:
    d = np.load(path)
    if int(d["version"][0]) != 1:
        raise ValueError("unknown smoother-weight checkpoint version")
    w = d["weights"].astype(np.float32)
    if w.shape != (MLP_NW,):
        raise ValueError("smoother-weight checkpoint has the wrong size")
    return w


def run_experiment(config: str = "c64", n_train: int = 30, n_eval: int = 10, iters_per_system: int = 20,
                   lr: float = 1e-3, seed: int = 0, precision: int = 1, out: str | None = None,
                   verbose: bool = True) -> dict:
    """Train on the IP-like sequence (seeds 100..), evaluate on held-out systems (seeds 200..)."""
    import contactgen as cg
    K = cg.stiffness(**{k: cg.CONFIGS[config][k] for k in ("nx", "ny", "nz")})
    J = cg.contact_jacobian(**{k: cg.CONFIGS[config][k] for k in ("nx", "ny", "nz")})
    train_set = ip_like_barriers(J.nrows, n_train, seed0=100)
    eval_set = ip_like_barriers(J.nrows, n_eval, seed0=200, held_out=True)
    _, b = cg.draw_D_b(0, J.nrows, K.nrows, -2.0, 8.0)
    t0 = time.perf_counter()
    w, log = train(K, J, train_set, iters_per_system, lr, seed, verbose=verbose)
    t_train = time.perf_counter() - t0
    ev = evaluate(K, J, eval_set, b, w, precision=precision)
    plain = sum(e["plain_iters"] for e in ev)
    learned = sum(e["learned_iters"] for e in ev)
    use = learned < plain
    res = {"config": config, "train_seconds": t_train, "train_log": log, "eval": ev,
           "plain_iters_total": plain, "learned_iters_total": learned,
           "plain_s_total": sum(e["plain_s"] for e in ev), "learned_s_total": sum(e["learned_s"] for e in ev),
           "decision": "learned" if use else "fallback: theta = 1"}
    if out:
        unit = np.zeros(MLP_NW, np.float32)
        unit[1312] = np.float32(np.log(3.5))  # theta = 1
        save_weights(out, w if use else unit, {"config": config, "decision": res["decision"]})
    if verbose:
        print(json.dumps({k: v for k, v in res.items() if k not in ("train_log", "eval")}), flush=True)
    return res


def run_evaluation(weights_path: str, config: str = "c64", n_eval: int = 10, precision: int = 1,
                   verbose: bool = True) -> dict:
    """Held-out evaluation of stored weights (no training): the systems of run_experiment's
    evaluation set (seeds 200.., spreads drawn in [1e2, 1e10]), theta = 1 against the weights."""
    import hashlib

    import contactgen as cg
    w = load_weights(weights_path)
    K = cg.stiffness(**{k: cg.CONFIGS[config][k] for k in ("nx", "ny", "nz")})
    J = cg.contact_jacobian(**{k: cg.CONFIGS[config][k] for k in ("nx", "ny", "nz")})
    eval_set = ip_like_barriers(J.nrows, n_eval, seed0=200, held_out=True)
    _, b = cg.draw_D_b(0, J.nrows, K.nrows, -2.0, 8.0)
    ev = evaluate(K, J, eval_set, b, w, precision=precision)
    res = {"config": config, "weights": os.path.basename(weights_path),
           "weights_sha256": hashlib.sha256(w.tobytes()).hexdigest(), "precision": precision,
           "plain_iters_total": sum(e["plain_iters"] for e in ev),
           "learned_iters_total": sum(e["learned_iters"] for e in ev),
           "plain_s_total": sum(e["plain_s"] for e in ev), "learned_s_total": sum(e["learned_s"] for e in ev),
           "fallbacks": sum(e["fallback"] for e in ev), "eval": ev}
    if verbose:
        print(json.dumps({k: v for k, v in res.items() if k != "eval"}), flush=True)
    return res


if __name__ == "__main__":
    import argparse
    ap = argparse.ArgumentParser(description="train the learned smoother weights and compare with theta = 1")
    ap.add_argument("--config", default="c64")
    ap.add_argument("--train", type=int, default=30)
    ap.add_argument("--eval", type=int, default=10)
    ap.add_argument("--iters", type=int, default=20)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--precision", type=int, default=1)
    ap.add_argument("--out", default=None)
    ap.add_argument("--json", default=None, help="write the full result (train log, per-system evaluation)")
    ap.add_argument("--ip", action="store_true",
                    help="train and evaluate on the Newton systems of interior-point runs (ip.py) instead")
    ap.add_argument("--nx", type=int, default=64, help="elements per side for --ip")
    ap.add_argument("--evaluate", default=None, metavar="WEIGHTS",
                    help="evaluate stored weights (.npz) on the held-out systems without training")
    a = ap.parse_args()
    if a.evaluate:
        r = run_evaluation(a.evaluate, a.config, a.eval, a.precision)
    elif a.ip:
        r = run_ip_experiment(a.nx, a.iters, a.lr, a.seed, a.precision, out=a.out)
    else:
        r = run_experiment(a.config, a.train, a.eval, a.iters, a.lr, a.seed, a.precision, a.out)
    if a.json:
        with open(a.json, "w") as f:
            json.dump(r, f, indent=1)
