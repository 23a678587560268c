#!/usr/bin/env python
"""Benchmark: AMGF-PCG seconds to a relative preconditioned residual of 1e-8 on one GB300.

Workload (default, the full form): the c160 two-block contact system -- two stacked Q1
linear-elastic blocks of 160x160x80 elements each (E=1, nu=0.3), node-to-node normal contact
on the 161x161 interface (m=25,921), barrier diagonal D log-uniform in [1e-2, 1e12],
n=12,442,080 DOFs, three seeded right-hand sides (seeds 0, 1, 2) cycled over the steps.
Synthetic data from contactgen (seeded).

One step = one full AMGF-PCG solve (x0 = 0) through the C ABI with inputs resident in HBM;
`value` is the plain FP64 solve (FP64 V-cycle, l1-Jacobi smoother with theta = 1).  The
working set (fine operator 8.6 GB plus hierarchy) is far larger than L2, so no flush is needed
between steps.  Prints one JSON line (rank 0).  Besides the contract's keys it carries
  - `variants`: the other V-cycle precisions and the learned smoother on the same workload
    (default: the mixed-precision + learned-smoother form, FP32 arithmetic with BF16 storage of
    every V-cycle matrix), each with its seconds per solve, PCG iterations, A-norm distance to
    the FP64 solution, true residual and the roofline of its dominant kernels;
  - `a_norm_rounding_floor`: the A-norm distance between two FP64 solves started 1e-10 |b|
    apart, the scale below which solutions cannot be told apart in FP64;
  - `roofline` (the FP64 fine-level sweep against the measured HBM copy bandwidth, with its
    FP64-pipe fraction as a secondary figure) and `roofline_coarse` (the level-1 sweep);
  - `iteration`: the algorithmic bytes (and flops, launches) of one PCG iteration summed over its
    launches, next to the timed seconds per iteration and the bandwidth that implies;
  - `cpu_baseline`: the CPU FP64 oracle on the host cores -- one complete PCG solve of the
    same system on all cores (setup reported separately) and a single-threaded sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl amgf|reference] [--config c160]

--impl reference times the CPU FP64 oracle on the host cores: each step runs a bounded
sample of PCG iterations of the same system, scaled to the full solve's iteration count
(`ms_per_step` is the measured time of a sampled step); one complete solve is timed as
well.  Under torchrun with N > 1 the GPU arm runs N independent replicas (the solve does
not shard; no collective on the data path); the reference arm runs on rank 0 only.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "AMGF-PCG seconds to 1e-8 rel. residual"
WORKLOADS = {
    "tiny": "two-block Q1 elasticity, 8x8x4 elements per block, n=1944, m=81 node-to-node contact rows, "
            "D log-uniform [1e-2,1e4]",
    "c64": "two-block Q1 elasticity, 64x64x32 elements per block, n=811200, m=4225 node-to-node contact rows, "
           "D log-uniform [1e-2,1e8], 3 seeded RHS",
    "c96": "two-block Q1 elasticity, 96x96x48 elements per block, n=2709792, m=9409 node-to-node contact rows, "
           "D log-uniform [1e-2,1e10], 3 seeded RHS",
    "c160": "two-block Q1 elasticity, 160x160x80 elements per block, n=12442080, m=25921 node-to-node contact "
            "rows, D log-uniform [1e-2,1e12], 3 seeded RHS",
    "c202": "two-block Q1 elasticity, 202x202x101 elements per block, n=24972654, m=41209 node-to-node contact "
            "rows, D log-uniform [1e-2,1e12], 3 seeded RHS",
}
PRECISIONS = ["FP64 V-cycle", "FP32 V-cycle", "FP32 V-cycle with BF16 fine-level K",
              "FP32 V-cycle with BF16 storage of every V-cycle matrix"]
# variant name -> (precision, learned smoother)
VARIANTS = {"fp64": (0, False), "fp32_vcycle": (1, False), "fp32_vcycle_bf16_K": (2, False),
            "fp32_vcycle_bf16_all": (3, False), "fp32_vcycle_bf16_K_learned": (2, True),
            "fp32_vcycle_bf16_all_learned": (3, True)}
DEFAULT_VARIANTS = "fp32_vcycle_bf16_all_learned"
# learned smoother weights trained by `python -m paper_2505_18576_gb300.learned --config c64 --out ...`
WEIGHTS = os.path.join(ROOT, "paper_2505_18576_gb300", "weights", "smoother_c64.npz")


def method_label(precision: int, learned: bool) -> str:
    smoother = "learned l1-Jacobi damping (MLP)" if learned else "l1-Jacobi, theta = 1"
    return f"AMGF-PCG in FP64 (flexible when mixed), {PRECISIONS[precision]}, {smoother}"


def workload_name(args, precision: int = 0, learned: bool = False) -> str:
    name = f"{args.config}: {WORKLOADS.get(args.config, args.config)}"
    if args.curvature:
        name += f"; contact along the normals of a curved interface (curvature {args.curvature:g})"
    return name + "; " + method_label(precision, learned)


def shared_config(args, p, precision: int = 0, learned: bool = False) -> dict:
    """`config` of both arms: the workload and the stop test (no implementation keys)."""
    return {"workload": workload_name(args, precision, learned), "n": int(p.n), "m": int(p.m), "rtol": 1e-8,
            "stop": "sqrt(r^T z / r0^T z0)", "l2": "working set larger than L2 (no flush)"}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id: str | None):
        self.bus_id = bus_id
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        rows = []
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 10:
                    continue
                if self.bus_id and self.bus_id.lower() not in parts[1].lower():
                    continue
                rows.append(parts)
            os.unlink(self.path)
        except Exception:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[6 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def make_inputs(config: str, curvature: float = 0.0):
    import contactgen as cg
    p = cg.make_problem(config, seed=0, curvature=curvature)
    c = cg.CONFIGS[config]
    rhs = [cg.draw_D_b(s, p.m, p.n, c["d_lo"], c["d_hi"])[1] for s in (0, 1, 2)]
    return p, rhs


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def cpu_oracle_baseline(p, rhs):
    """The CPU FP64 oracle on this host: setup, one complete PCG solve of seed 0's system on all
    cores, and a single-threaded sample (the initial residual, apply and one iteration) scaled by
    the all-core ratio of the complete solve to the same sample."""
    import oracle
    cores = os.cpu_count()
    threads = oracle.set_threads(0)
    t0 = time.perf_counter()
    o = oracle.Oracle(p.K, p.J, p.D)
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    _, k_full, st, *_ = o.pcg(rhs[0], tol=1e-8)
    t_full = time.perf_counter() - t0
    t0 = time.perf_counter()
    o.pcg(rhs[0], tol=1e-30, maxit=1)
    t_one_all = time.perf_counter() - t0
    oracle.set_threads(1)
    t0 = time.perf_counter()
    o.pcg(rhs[0], tol=1e-30, maxit=1)
    t_one_single = time.perf_counter() - t0
    oracle.set_threads(threads)
    o.close()
    single = t_one_single * (t_full / t_one_all)
    return {"value": t_full, "unit": "s", "cores": threads, "kind": "oracle",
            "sample": f"one complete oracle AMGF-PCG solve of the {p.n}-DOF system (seed 0), {k_full} iterations, "
                      f"status {st}, on {threads} threads; oracle setup {t_setup:.1f} s reported separately",
            "setup_s": round(t_setup, 2), "pcg_iters": int(k_full), "cpu_model": cpu_model(),
            "host_cores": cores,
            "single_thread": {"value": single, "unit": "s", "cores": 1,
                              "sample": f"initial residual, preconditioner apply and one PCG iteration on one "
                                        f"thread ({t_one_single:.2f} s; {t_one_all:.2f} s on {threads} threads), "
                                        f"scaled by the complete solve's time over the same sample on {threads} "
                                        f"threads"}}


def max_over_ranks(values, dist, device):
    """Element-wise maximum of per-rank timings (the slowest replica sets the job's time)."""
    if dist is None:
        return list(values)
    import torch
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def run_reference(args, rank, world):
    """The oracle on the host cores: K steps of a bounded sample of PCG iterations each."""
    if rank != 0:
        return 0
    import oracle
    p, rhs = make_inputs(args.config, args.curvature)
    threads = oracle.set_threads(0)
    t0 = time.perf_counter()
    o = oracle.Oracle(p.K, p.J, p.D)
    t_setup = time.perf_counter() - t0
    # one complete solve (untimed by the steps): the iteration count that scales each sample
    t0 = time.perf_counter()
    _, k_full, st, *_ = o.pcg(rhs[0], tol=1e-8)
    t_full = time.perf_counter() - t0
    k = max(1, args.ref_iters)
    times, step_s = [], []
    for step in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        o.pcg(rhs[step % 3], tol=1e-30, maxit=k)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            step_s.append(dt)
            # the sample's initial residual and preconditioner apply cost about one iteration
            times.append(dt / (k + 1) * (k_full + 1))
    o.close()
    value = statistics.mean(times)
    sample = (f"{k} oracle PCG iterations of the {args.config} solve per step after the initial residual and "
              f"preconditioner apply (oracle setup excluded), scaled by (k_full + 1) / ({k} + 1) with the complete "
              f"solve's k_full = {k_full} iterations; ms_per_step is the measured time of a sampled step")
    line = {"metric": METRIC, "value": value, "unit": "s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": statistics.mean(step_s) * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": shared_config(args, p),
            "parallelism": f"host cores ({threads} OpenMP threads)",
            "value_kind": "extrapolated from the sampled steps",
            "complete_solve": {"s": t_full, "pcg_iters": int(k_full), "status": int(st),
                               "setup_s": round(t_setup, 2)},
            "cpu_baseline": {"value": value, "unit": "s", "cores": threads, "kind": "oracle", "sample": sample,
                             "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def load_traffic(kind: str, precision: int, bytes_now: float):
    """DRAM bytes per launch of a kernel, from the ncu capture stored in profiles/: the ratio of
    measured DRAM bytes to algorithmic bytes at the captured size, times this launch's algorithmic
    bytes.  None when the kernel's source changed since the capture."""
    try:
        with open(os.path.join(ROOT, "profiles", "roofline_traffic.json")) as f:
            tr = json.load(f)
        ent = tr.get(f"{kind}:precision{precision}")
        if not ent or ent.get("kernel_source_sha") != kernel_source_sha(kind, precision):
            return None, None
        ratio = ent["dram_bytes_per_launch"] / ent["algorithmic_bytes_per_launch"]
        return ratio * bytes_now, f"{ent['capture']} (DRAM / algorithmic = {ratio:.3f}, scaled to this launch)"
    except Exception:
        return None, None


def level1_kernel(s) -> str:
    """Name of the kernel that runs the level-1 sweeps of this handle."""
    if int(s.info.sell_levels) & 2:
        return "sell_kernel<POST> (sliced ELL, one lane per row)"
    if int(s.info.staged_levels) & 2:
        return "csr_staged_kernel<POST> (tiles staged by cp.async.bulk)"
    return "csr_kernel<POST>"


def roofline_of(s, which: int, kind: str, precision: int, hbm_peak: float, peak_kind: str, sm_count: int,
                sm_mhz: float, label: str):
    kms, kbytes = s.time_kernel(which, warmup=5, reps=50)
    gbs = kbytes / (kms * 1e-3) / 1e9
    traffic, tsrc = load_traffic(kind, precision, kbytes)
    out = {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm_peak, "unit": "GB/s",
           "frac": round(gbs / hbm_peak, 4), "traffic": None if traffic is None else round(traffic),
           "kernel": label, "bytes_per_launch": kbytes, "ms_per_launch": kms,
           "peak_kind": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs, burst)"}
    if tsrc:
        out["traffic_source"] = tsrc
    if precision == 0:
        if which == 3:
            nnz = float(s.info.level_nnz[1])
            rows = float(s.info.level_rows[1])
        else:
            nnz = float(s.info.level_nnz[0])
            rows = float(s.info.n)
        flops = 2.0 * nnz + 4.0 * rows        # one FMA per nonzero; b - s, * w, + x, + add per row
        peak = sm_count * 2 * 2 * sm_mhz * 1e6 / 1e12
        tf = flops / (kms * 1e-3) / 1e12
        out["fp64_pipe"] = {"achieved": round(tf, 4), "peak": round(peak, 4), "unit": "TFLOP/s",
                            "frac": round(tf / peak, 4),
                            "peak_kind": f"derived: {sm_count} SMs x 2 FP64 FMA/clk x 2 flop x {sm_mhz:.0f} MHz"}
    return out


def iteration_model(s, s_per_iter: float, hbm_peak: float):
    """The bytes model of one PCG iteration next to its measured time: algorithmic bytes and flops
    summed over every launch of one iteration (amgf_profile_iteration records them launch by
    launch), over the timed solve's seconds per iteration."""
    recs = s.profile_iteration()
    by = sum(r["bytes"] for r in recs)
    fl = sum(r["flops"] for r in recs)
    gbs = by / s_per_iter / 1e9
    return {"algorithmic_bytes": round(by), "flops": round(fl), "launches": len(recs),
            "s_per_iteration": s_per_iter, "achieved_gbs": round(gbs, 1), "frac_of_hbm": round(gbs / hbm_peak, 4),
            "note": "bytes: stored values and indices at their precision, one read of every input vector, "
                    "one write of every output, summed over the launches of one iteration; time: the timed "
                    "solves' seconds per PCG iteration (includes the initial residual and apply)"}


def run_gpu(args, rank, world, local):
    import numpy as np
    import torch

    import paper_2505_18576_gb300 as amgf
    from paper_2505_18576_gb300.learned import load_weights

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist_
        dist_.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        dist = dist_

    def barrier():
        if dist is not None:
            dist.barrier()

    props = torch.cuda.get_device_properties(local)
    sm_count = int(props.multi_processor_count)
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            sm_mhz = float(json.load(f).get("sm_max_mhz", 2070.0))
    except Exception:
        sm_mhz = 2070.0
    hbm_peak, peak_kind = peaks()

    p, rhs = make_inputs(args.config, args.curvature)
    learned = bool(args.weights)
    t0 = time.perf_counter()
    s = amgf.Solver(p.K, p.J, p.D, use_graph=0 if args.no_graph else 1, precision=args.precision)
    t_setup = time.perf_counter() - t0
    if learned:
        s.set_mlp(load_weights(WEIGHTS if args.weights == "default" else args.weights))
    info = s.info
    n = p.n
    bdev = [torch.from_numpy(b).cuda() for b in rhs]
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for k in range(args.warmup):
        x.zero_()
        s.pcg_solve(bdev[k % 3], x)
    torch.cuda.synchronize()

    bus = getattr(props, "pci_bus_id", None)
    sampler = ClockSampler(None if bus is None else str(bus))
    sampler.start()
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    iters, launches, fallbacks, relres = [], 0, 0, []
    ev0.record(stream)
    for k in range(args.steps):
        x.zero_()
        st = s.pcg_solve(bdev[k % 3], x, stream=stream)
        iters.append(st.iters)
        fallbacks += st.mlp_fallback
        launches += st.kernel_launches
        relres.append(st.rel_res_l2)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    ms = max_over_ranks([ms], dist, "cuda")[0]

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    bh = [torch.from_numpy(b).pin_memory().numpy() for b in rhs]
    xh = torch.zeros(n, dtype=torch.float64).pin_memory().numpy()
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for k in range(args.steps):
        xh[:] = 0.0
        s.pcg_solve_host(bh[k % 3], xh)
    e2e_s = (time.perf_counter() - t0) / args.steps
    e2e_s = max_over_ranks([e2e_s], dist, "cuda")[0]

    # dominant kernels: the fine-level l1-Jacobi post-smoother (one pass over the fine operator with
    # the fused smoother epilogue) and the level-1 post-smoother, each timed alone with CUDA events
    fine_label = ("bsr3_kernel<POST>: fine-level FP64 l1-Jacobi sweep over A (3x3 node blocks)" if args.precision == 0
                  else "bsr3_mixed_kernel<POST>: fine-level FP32 l1-Jacobi sweep (K blocks + FP64 contact term)")
    roofline = roofline_of(s, 1 if args.precision == 0 else 2, "fine", args.precision, hbm_peak, peak_kind,
                           sm_count, sm_mhz, fine_label)
    roofline_coarse = None
    if info.nlevels >= 3:
        roofline_coarse = roofline_of(s, 3, "level1", args.precision, hbm_peak, peak_kind, sm_count, sm_mhz,
                                      f"{level1_kernel(s)}: level-1 l1-Jacobi sweep ({PRECISIONS[args.precision]})")
    iteration = iteration_model(s, ms * 1e-3 / max(1e-9, statistics.mean(iters)), hbm_peak)

    # the same workload with the other V-cycle precisions / the learned smoother (same timing method,
    # fewer steps), each with its A-norm distance to the timed configuration's solution of seed 0.
    # The timed solver is released first: at 25 M DOFs two hierarchies' host copies do not fit in
    # the host memory next to the GPU.
    variants, floor = {}, None
    wanted = [] if args.variants == "none" else (list(VARIANTS) if args.variants == "all"
                                                   else args.variants.split(","))
    x_ref = torch.zeros(n, dtype=torch.float64, device="cuda")
    s.pcg_solve(bdev[0], x_ref)

    def a_norm_rel(sol, xv):
        d = xv - x_ref
        yd = torch.empty_like(d)
        yr = torch.empty_like(d)
        sol.matvec(d, yd)          # A = K + J^T D J in FP64 in every precision
        sol.matvec(x_ref, yr)
        return float(torch.sqrt(torch.dot(d, yd) / torch.dot(x_ref, yr)))

    if wanted:
        # FP64 rounding floor of the A-norm comparison: the same solve started 1e-10 |b| away
        # from zero.  Two solves equal in exact arithmetic differ by about this much, because the
        # true residual stalls near u |A| |x| in the contact rows (entries up to D_max).
        x2 = (1e-10 * bdev[0].abs()).contiguous()
        s.pcg_solve(bdev[0], x2)
        floor = a_norm_rel(s, x2)
        del x2
    nlev, opc, nc = int(info.nlevels), float(info.op_complexity), int(info.nc)
    s.close()
    del s

    for name in wanted:
        prec, lrn = VARIANTS[name]
        if (prec, lrn) == (args.precision, learned) or (lrn and not os.path.exists(WEIGHTS)):
            continue
        t0 = time.perf_counter()
        sv = amgf.Solver(p.K, p.J, p.D, precision=prec)
        tv_setup = time.perf_counter() - t0
        if lrn:
            sv.set_mlp(load_weights(WEIGHTS))
        xv = torch.zeros(n, dtype=torch.float64, device="cuda")
        for k in range(2):
            xv.zero_()
            sv.pcg_solve(bdev[k % 3], xv)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        its, fb, rr = [], 0, []
        nst = max(3, min(args.steps, 10))
        e0.record(stream)
        for k in range(nst):
            xv.zero_()
            stv = sv.pcg_solve(bdev[k % 3], xv, stream=stream)
            its.append(stv.iters)
            fb += stv.mlp_fallback
            rr.append(stv.rel_res_l2)
        e1.record(stream)
        torch.cuda.synchronize()
        xv.zero_()
        sv.pcg_solve(bdev[0], xv)
        ent = {"workload": workload_name(args, prec, lrn), "s_per_solve": e0.elapsed_time(e1) / nst * 1e-3,
               "steps": nst, "pcg_iters": its, "rel_res_l2": rr, "setup_s": round(tv_setup, 3),
               "a_norm_rel_diff_vs_timed_solution": a_norm_rel(sv, xv)}
        if lrn:
            ent["mlp_fallbacks"] = fb
        if prec > 0:
            ent["roofline"] = roofline_of(sv, 2, "fine", prec, hbm_peak, peak_kind, sm_count, sm_mhz,
                                          "bsr3_mixed_kernel<POST>: fine-level l1-Jacobi sweep "
                                          f"({PRECISIONS[prec]}, FP64 contact term)")
            if sv.info.nlevels >= 3:
                ent["roofline_coarse"] = roofline_of(sv, 3, "level1", prec, hbm_peak, peak_kind, sm_count, sm_mhz,
                                                     f"{level1_kernel(sv)}: level-1 l1-Jacobi sweep ({PRECISIONS[prec]})")
        ent["iteration"] = iteration_model(sv, ent["s_per_solve"] / max(1e-9, statistics.mean(its)), hbm_peak)
        variants[name] = ent
        sv.close()
        del sv, xv

    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            del bdev, x, x_ref
            cpu = cpu_oracle_baseline(p, rhs)
        value = ms * 1e-3
        line = {
            "metric": METRIC, "value": value, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f64" if args.precision == 0 else "f64+f32" + ("+bf16" if args.precision >= 2 else ""),
            "data": "synthetic",
            "config": shared_config(args, p, args.precision, learned),
            "solve": {"nc": nc, "levels": nlev, "op_complexity": round(opc, 4), "pcg_iters": iters,
                      "rel_res_l2": relres, "setup_s": round(t_setup, 3), "mlp_fallbacks": fallbacks,
                      "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                      "aggregate_solves_per_s": world / (ms * 1e-3)},
            "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": 2 * n * 8, "d2h_bytes_per_step": n * 8},
            "gpu_launches": int(launches),
            "roofline": roofline,
            "clocks": clocks,
        }
        if roofline_coarse:
            line["roofline_coarse"] = roofline_coarse
        line["iteration"] = iteration
        if variants:
            line["variants"] = variants
            line["a_norm_rounding_floor"] = floor
        if cpu is not None:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def kernel_source_sha(kind: str = "fine", precision: int = 0):
    """Hash of the source a roofline kernel is built from: the fine-level FP64 BSR3 kernel
    (kind "fine", precision 0) or the mixed one (precision 1-3) with the host code that lays its
    operator out, or the level-1 kernels (CSR, sliced ELL, staged) with the host code that
    chooses and lays out their operators (kind "level1"; the hierarchy itself is pinned bit for
    bit to the oracle by the CPU tests).  DRAM traffic stored in profiles/roofline_traffic.json
    is used only while this hash is unchanged."""
    import hashlib
    h = hashlib.sha1()
    csrc = os.path.join(ROOT, "paper_2505_18576_gb300", "csrc")
    k = open(os.path.join(csrc, "kernels.cuh")).read()
    a = open(os.path.join(csrc, "amgf.cu")).read()
    c = open(os.path.join(csrc, "setup.cpp")).read()
    if kind == "level1":
        i = k.index("template <typename T, int K, int MODE, bool DOT, typename VT = T, int U = 4>")
        h.update(k[i:k.index("// Fine-level operator in 3x3 node blocks", i)].encode())
        i = a.index("static int lanes_for(")
        h.update(a[i:a.index("static int grid_for(", i)].encode())
        i = a.index("static int upload_csr(")
        h.update(a[i:a.index("static void fill_info(", i)].encode())
        i = c.index("void build_sell(")
        h.update(c[i:c.index("bool build_bsr3(", i)].encode())
        return h.hexdigest()[:12]
    mid = k.index("// Fine level of the FP32 V-cycle")
    if precision == 0:
        h.update(k[k.index("struct BsrArgs {"):mid].encode())
    else:
        i = k.index("bsr3_mixed_kernel(Bsr3MixedArgs<VT> a) {")
        h.update(k[mid:k.index("\n}\n", i) + 3].encode())
        i = a.index("// fine-level K in 3x3 blocks")
        h.update(a[i:a.index("// contact term J^T D J over all rows", i)].encode())
    i = c.index("bool build_bsr3(")
    h.update(c[i:c.index("\nint validate_csr(", i)].encode())
    return h.hexdigest()[:12]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="amgf", choices=["amgf", "reference"])
    ap.add_argument("--config", default="c160", choices=sorted(WORKLOADS))
    ap.add_argument("--curvature", type=float, default=0.0,
                    help="contact rows along the normals of a curved interface (0: z-only node-to-node rows)")
    ap.add_argument("--ref-iters", type=int, default=2, help="oracle PCG iterations per reference step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", type=int, default=0, choices=[0, 1, 2, 3],
                    help="V-cycle precision of the timed solve: 0 FP64, 1 FP32, 2 FP32 with BF16 fine-level K, "
                         "3 FP32 arithmetic with BF16 storage of every V-cycle matrix")
    ap.add_argument("--variants", default=DEFAULT_VARIANTS,
                    help="comma list of variants to time besides the main line (" + ", ".join(VARIANTS) +
                         "), 'all' or 'none'")
    ap.add_argument("--weights", default=None,
                    help="learned smoother weights (.npz) for the timed solve; 'default' = the packaged c64 weights")
    ap.add_argument("--no-graph", action="store_true",
                    help="launch the PCG kernels directly instead of one CUDA graph (for per-kernel profiling)")
    args = ap.parse_args()
    if args.variants not in ("all", "none"):
        for v in args.variants.split(","):
            if v not in VARIANTS:
                ap.error(f"unknown variant {v}")
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    return run_gpu(args, rank, world, local)


if __name__ == "__main__":
    sys.exit(main())
