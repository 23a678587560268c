#!/usr/bin/env python
"""Benchmark: AMGF-PCG seconds to a relative preconditioned residual of 1e-8 on one GB300.

Workload (default): the c64 two-block contact system -- two stacked Q1 linear-elastic
blocks of 64x64x32 elements each (E=1, nu=0.3), node-to-node normal contact on the
65x65 interface (m=4225), barrier diagonal D log-uniform in [1e-2, 1e8], n=811,200
DOFs, three seeded right-hand sides (seeds 0, 1, 2) cycled over the steps.  Synthetic
data from contactgen (seeded); FP64 arithmetic throughout.

One step = one full AMGF-PCG solve (x0 = 0) through the C ABI with inputs resident in
HBM.  The working set (fine operator ~0.76 GB plus hierarchy) is larger than L2, so
no flush is needed between steps.  Prints one JSON line (rank 0).  Besides the
contract's keys it carries `variants` (the other V-cycle precisions and the learned
smoother on the same workload, each with its A-norm distance to the timed solution) and
`a_norm_rounding_floor` (the A-norm distance between two FP64-equivalent solves started
1e-10 |b| apart: the scale below which solutions cannot be told apart in FP64).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl amgf|reference] [--config c64]

--impl reference times the CPU FP64 oracle on the host cores on a bounded sample of
the same workload (a few PCG iterations per step, scaled to the full solve's
iteration count).  Under torchrun with N > 1 the GPU arm runs N independent replicas
(the solve does not shard; no collective on the data path); the reference arm runs
on rank 0 only.
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
    "c64": "two-block Q1 elasticity, 64x64x32 elements per block, n=811200, m=4225 node-to-node contact rows, "
           "D log-uniform [1e-2,1e8], 3 seeded RHS, FP64 AMGF-PCG",
    "tiny": "two-block Q1 elasticity, 8x8x4 elements per block, n=1944, m=81, D log-uniform [1e-2,1e4]",
    "c96": "two-block Q1 elasticity, 96x96x48 elements per block, n=2709792, m=9409, D log-uniform [1e-2,1e10], "
           "FP64 AMGF-PCG",
    "c160": "two-block Q1 elasticity, 160x160x80 elements per block, n=12442080, m=25921, D log-uniform "
            "[1e-2,1e12], FP64 AMGF-PCG",
    "c202": "two-block Q1 elasticity, 202x202x101 elements per block, n=24972654, m=41209, D log-uniform "
            "[1e-2,1e12], FP64 AMGF-PCG",
}
# learned smoother weights trained by `python -m paper_2505_18576_gb300.learned --config c64 --out ...`
WEIGHTS = os.path.join(ROOT, "paper_2505_18576_gb300", "weights", "smoother_c64.npz")


def workload_name(args) -> str:
    name = f"{args.config}: {WORKLOADS.get(args.config, args.config)}"
    if args.curvature:
        name += f"; contact along the normals of a curved interface (curvature {args.curvature:g})"
    return name


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


def cpu_oracle_sample(p, rhs, iters_full: float, sample_iters: int, reps: int = 1):
    """Time `sample_iters` oracle PCG iterations (after its setup); scale to a full solve."""
    import oracle
    t0 = time.perf_counter()
    o = oracle.Oracle(p.K, p.J, p.D)
    t_setup = time.perf_counter() - t0
    per_iter = []
    for k in range(reps):
        t0 = time.perf_counter()
        o.pcg(rhs[k % len(rhs)], tol=1e-30, maxit=sample_iters)
        per_iter.append((time.perf_counter() - t0) / sample_iters)
    sec_iter = statistics.median(per_iter)
    o.close()
    return sec_iter * iters_full, sec_iter, t_setup


def max_over_ranks(values, dist, device):
    """Element-wise maximum of per-rank timings (the slowest replica sets the job's time)."""
    if dist is None:
        return list(values)
    import torch
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import oracle
    p, rhs = make_inputs(args.config, args.curvature)
    cores = os.cpu_count()
    o = oracle.Oracle(p.K, p.J, p.D)
    # iteration count of the full solve (untimed, once): scales the per-iteration sample
    _, k_full, st, *_ = o.pcg(rhs[0], tol=1e-8)
    times = []
    for step in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        o.pcg(rhs[step % 3], tol=1e-30, maxit=args.ref_iters)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt / args.ref_iters * k_full)
    value = statistics.mean(times)
    sample = (f"{args.ref_iters} PCG iterations of the {args.config} solve per step (oracle setup excluded), "
              f"scaled by the full solve's {k_full} iterations")
    line = {"metric": METRIC, "value": value, "unit": "s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": value * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": workload_name(args), "rtol": 1e-8,
                       "stop": "sqrt(r^T z / r0^T z0)", "parallelism": "host cores (OpenMP row loops)"},
            "cpu_baseline": {"value": value, "unit": "s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(args, rank, world, local):
    import numpy as np
    import torch

    import paper_2505_18576_gb300 as amgf

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist_
        dist_.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        dist = dist_

    def barrier():
        if dist is not None:
            dist.barrier()

    p, rhs = make_inputs(args.config, args.curvature)
    t0 = time.perf_counter()
    s = amgf.Solver(p.K, p.J, p.D, use_graph=0 if args.no_graph else 1, precision=args.precision)
    t_setup = time.perf_counter() - t0
    weights = None
    if args.weights:
        from paper_2505_18576_gb300.learned import load_weights
        weights = load_weights(WEIGHTS if args.weights == "default" else args.weights)
        s.set_mlp(weights)
    info = s.info
    n = p.n
    bdev = [torch.from_numpy(b).cuda() for b in rhs]
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for k in range(args.warmup):
        x.zero_()
        s.pcg_solve(bdev[k % 3], x)
    torch.cuda.synchronize()

    props = torch.cuda.get_device_properties(local)
    bus = getattr(props, "pci_bus_id", None)
    sampler = ClockSampler(None if bus is None else str(bus))
    sampler.start()
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    iters, launches, solve_s, fallbacks = [], 0, [], 0
    ev0.record(stream)
    for k in range(args.steps):
        x.zero_()
        st = s.pcg_solve(bdev[k % 3], x, stream=stream)
        iters.append(st.iters)
        fallbacks += st.mlp_fallback
        launches += st.kernel_launches
        solve_s.append(st.t_solve_s)
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

    # the same workload with the other V-cycle precisions (same timing method, fewer steps),
    # each with its A-norm distance to this run's solution of seed 0
    variants = {}
    floor = None
    if not args.no_variants:
        x_ref = torch.zeros(n, dtype=torch.float64, device="cuda")
        s.pcg_solve(bdev[0], x_ref)
        table = [("fp64", 0, False), ("fp32_vcycle", 1, False), ("fp32_vcycle_bf16_K", 2, False),
                 ("fp32_vcycle_bf16_all", 3, False)]
        if os.path.exists(WEIGHTS):
            table += [("fp32_vcycle_bf16_K_learned", 2, True), ("fp32_vcycle_bf16_all_learned", 3, True)]
        wanted = None if args.variants == "all" else set(args.variants.split(","))
        for name, prec, learned in table:
            if (prec, learned) == (args.precision, weights is not None) or (wanted and name not in wanted):
                continue
            sv = amgf.Solver(p.K, p.J, p.D, precision=prec)
            if learned:
                from paper_2505_18576_gb300.learned import load_weights
                sv.set_mlp(load_weights(WEIGHTS))
            xv = torch.zeros(n, dtype=torch.float64, device="cuda")
            for k in range(2):
                xv.zero_()
                sv.pcg_solve(bdev[k % 3], xv)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            its, fb = [], 0
            nst = max(2, min(args.steps, 5))
            e0.record(stream)
            for k in range(nst):
                xv.zero_()
                stv = sv.pcg_solve(bdev[k % 3], xv, stream=stream)
                its.append(stv.iters)
                fb += stv.mlp_fallback
            e1.record(stream)
            torch.cuda.synchronize()
            xv.zero_()
            sv.pcg_solve(bdev[0], xv)
            d = xv - x_ref
            yd = torch.empty_like(d)
            yr = torch.empty_like(d)
            s.matvec(d, yd)
            s.matvec(x_ref, yr)
            rel_a = float(torch.sqrt(torch.dot(d, yd) / torch.dot(x_ref, yr)))
            variants[name] = {
                "s_per_solve": e0.elapsed_time(e1) / nst * 1e-3, "pcg_iters": its,
                "a_norm_rel_diff_vs_timed_solution": rel_a}
            if learned:
                variants[name]["mlp_fallbacks"] = fb
            sv.close()
        # FP64 rounding floor of the A-norm comparison: the same solve started 1e-10 |b| away
        # from zero.  Two solves equal in exact arithmetic differ by about this much, because the
        # true residual stalls near u |A| |x| in the contact rows (entries up to D_max).
        x2 = (1e-10 * bdev[0].abs()).contiguous()
        s.pcg_solve(bdev[0], x2)
        d = x2 - x_ref
        yd = torch.empty_like(d)
        yr = torch.empty_like(d)
        s.matvec(d, yd)
        s.matvec(x_ref, yr)
        floor = float(torch.sqrt(torch.dot(d, yd) / torch.dot(x_ref, yr)))

    # dominant kernel: the fine-level l1-Jacobi post-smoother (one pass over the fine operator with
    # the fused smoother epilogue), timed alone with CUDA events.  In FP64 the pass is bound by the
    # FP64 pipe (2 FMA/clk/SM on this part), in the FP32 V-cycle by HBM bandwidth.
    which = 2 if s.info.n and args.precision else 1
    kms, kbytes = s.time_kernel(which, warmup=5, reps=50)
    hbm_peak, peak_kind = peaks()
    gbs = kbytes / (kms * 1e-3) / 1e9
    nnz0 = int(s.info.level_nnz[0])
    kflops = 2.0 * nnz0 + 4.0 * n          # 2 per nonzero, 4 per row (b - s, * w, + x, + add)
    tflops = kflops / (kms * 1e-3) / 1e12
    traffic = None
    try:
        with open(os.path.join(ROOT, "profiles", "roofline_traffic.json")) as f:
            tr = json.load(f)
        ent = tr.get(f"{args.config}:precision{args.precision}", {})
        if ent.get("kernel_source_sha") == kernel_source_sha(args.precision):
            traffic = ent.get("dram_bytes_per_launch")
    except Exception:
        pass
    if args.precision == 0:
        fp64_peak = fp64_peak_tflops()
        roofline = {"bound": "alu", "achieved": round(tflops, 4), "peak": round(fp64_peak, 4), "unit": "TFLOP/s",
                    "frac": round(tflops / fp64_peak, 4), "traffic": traffic,
                    "kernel": "bsr3_kernel<4,POST,0>: fine-level FP64 l1-Jacobi sweep over A (3x3 node blocks)",
                    "flops_per_launch": kflops, "bytes_per_launch": kbytes, "ms_per_launch": kms,
                    "hbm_gbs": round(gbs, 1), "hbm_frac": round(gbs / hbm_peak, 4),
                    "peak_kind": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz (FP64 pipe)"}
    else:
        roofline = {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm_peak, "unit": "GB/s",
                    "frac": round(gbs / hbm_peak, 4), "traffic": traffic,
                    "kernel": "bsr3_mixed_kernel<POST>: fine-level FP32 l1-Jacobi sweep (K blocks + FP64 contact term)",
                    "bytes_per_launch": kbytes, "ms_per_launch": kms, "peak_kind": f"{peak_kind} (burst)"}

    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            est, sec_iter, t_orc_setup = cpu_oracle_sample(p, rhs, float(np.mean(iters)), args.cpu_iters)
            cpu = {"value": est, "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
                   "sample": f"{args.cpu_iters} oracle PCG iterations on the {args.config} system (setup "
                             f"excluded, {t_orc_setup:.1f}s), {sec_iter * 1e3:.1f} ms/iteration scaled by the "
                             f"GPU solve's mean {np.mean(iters):.1f} iterations"}
        value = ms * 1e-3
        line = {
            "metric": METRIC, "value": value, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if args.precision == 0 else "f64+f32" + ("+bf16" if args.precision >= 2 else ""),
            "data": "synthetic",
            "config": {"workload": workload_name(args),
                       "precision": ["fp64", "fp32 V-cycle", "fp32 V-cycle, bf16 fine K",
                                     "fp32 V-cycle, bf16 storage of all V-cycle matrices"][args.precision],
                       "smoother": "l1-Jacobi, learned theta (MLP)" if weights is not None else "l1-Jacobi, theta = 1",
                       "n": n, "m": p.m, "nc": int(info.nc), "levels": int(info.nlevels),
                       "op_complexity": round(float(info.op_complexity), 4), "rtol": 1e-8,
                       "stop": "sqrt(r^T z / r0^T z0)", "pcg_iters": iters,
                       "l2": "working set larger than L2 (no flush)", "setup_s": round(t_setup, 3),
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "mlp_fallbacks": fallbacks,
                       "aggregate_solves_per_s": world / (ms * 1e-3)},
            "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": 2 * n * 8, "d2h_bytes_per_step": n * 8},
            "gpu_launches": int(launches),
            "roofline": roofline,
            "clocks": clocks,
        }
        if variants:
            line["variants"] = variants
            line["a_norm_rounding_floor"] = floor
        if cpu is not None:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    s.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def fp64_peak_tflops():
    """FP64 FMA pipe: 2 FMA per clock per SM on this part (nominal 1.25 TFLOP/s), 152 SMs, 2.07 GHz."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = float(json.load(f).get("sm_max_mhz", 2070.0))
    except Exception:
        mhz = 2070.0
    return 152 * 2 * 2 * mhz * 1e6 / 1e12


def kernel_source_sha(precision: int = 0):
    """Hash of the source the roofline kernel of this precision is built from: the fine-level
    FP64 BSR3 kernel (precision 0) or the mixed one (1-3), with the host code that lays its
    operator out.  DRAM traffic stored in profiles/roofline_traffic.json is used only while
    this hash is unchanged."""
    import hashlib
    h = hashlib.sha1()
    csrc = os.path.join(ROOT, "paper_2505_18576_gb300", "csrc")
    k = open(os.path.join(csrc, "kernels.cuh")).read()
    mid = k.index("// Fine level of the FP32 V-cycle")
    if precision == 0:
        h.update(k[k.index("struct BsrArgs {"):mid].encode())
    else:
        i = k.index("bsr3_mixed_kernel(Bsr3MixedArgs<VT> a) {")
        h.update(k[mid:k.index("\n}\n", i) + 3].encode())
        a = open(os.path.join(csrc, "amgf.cu")).read()
        i = a.index("// fine-level K in 3x3 blocks")
        h.update(a[i:a.index("// contact term J^T D J over all rows", i)].encode())
    c = open(os.path.join(csrc, "setup.cpp")).read()
    i = c.index("bool build_bsr3(")
    h.update(c[i:c.index("\nint validate_csr(", i)].encode())
    return h.hexdigest()[:12]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="amgf", choices=["amgf", "reference"])
    ap.add_argument("--config", default="c64", choices=sorted(WORKLOADS))
    ap.add_argument("--curvature", type=float, default=0.0,
                    help="contact rows along the normals of a curved interface (0: z-only node-to-node rows)")
    ap.add_argument("--cpu-iters", type=int, default=8, help="oracle PCG iterations timed for cpu_baseline")
    ap.add_argument("--ref-iters", type=int, default=4, help="oracle PCG iterations per reference step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", type=int, default=0, choices=[0, 1, 2, 3],
                    help="V-cycle precision of the timed solve: 0 FP64, 1 FP32, 2 FP32 with BF16 fine-level K, "
                         "3 FP32 arithmetic with BF16 storage of every V-cycle matrix")
    ap.add_argument("--no-variants", action="store_true", help="skip the mixed-precision variant timings")
    ap.add_argument("--variants", default="all",
                    help="comma list of variants to time (fp64, fp32_vcycle, fp32_vcycle_bf16_K, "
                         "fp32_vcycle_bf16_all, fp32_vcycle_bf16_K_learned, fp32_vcycle_bf16_all_learned) or 'all'")
    ap.add_argument("--weights", default=None,
                    help="learned smoother weights (.npz) for the timed solve; 'default' = the packaged c64 weights")
    ap.add_argument("--no-graph", action="store_true",
                    help="launch the PCG kernels directly instead of one CUDA graph (for per-kernel profiling)")
    args = ap.parse_args()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    return run_gpu(args, rank, world, local)


if __name__ == "__main__":
    sys.exit(main())
