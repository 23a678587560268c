"""Achieved bandwidth of every kernel of one PCG iteration (amgf_profile_iteration).

    python -m paper_2505_18576_gb300.kernel_table --config c160 [--precision 3 --weights default]

Sets up the seeded two-block system of `--config`, solves it once, then records `--iters`
PCG iterations launch by launch (a CUDA event after every kernel) and prints a markdown table:
one line per operation and level with its launches per iteration, mean time per launch,
algorithmic bytes per launch (values + indices at the stored precision, one read of every
input vector, one write of every output), achieved GB/s against the measured copy bandwidth,
and for FP64 launches the FP64-pipe fraction (2 flops per nonzero against 2 FP64 FMA per
clock per SM at the maximum SM clock).  Event times include the gap between back-to-back
launches, which dominates the kernels of a few microseconds.
"""
from __future__ import annotations

import argparse
import collections
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d.get("sm_max_mhz", 2070.0)), "measured"
    except Exception:
        return 6800.0, 2070.0, "fallback"


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", default="c160")
    ap.add_argument("--precision", type=int, default=0)
    ap.add_argument("--weights", default=None, help="learned smoother weights (.npz), 'default' = packaged")
    ap.add_argument("--iters", type=int, default=3)
    ap.add_argument("--stage-rows", type=int, default=None, help="amgf_options.stage_rows (default: library's)")
    ap.add_argument("--stage-depth", type=int, default=None, help="amgf_options.stage_depth")
    ap.add_argument("--set", action="append", default=[], metavar="FIELD=INT",
                    help="any other integer field of amgf_options, e.g. --set fuse_tail=0")
    args = ap.parse_args(argv)

    import torch

    import contactgen as cg
    import paper_2505_18576_gb300 as amgf

    torch.cuda.set_device(0)
    hbm, mhz, kind = peaks()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    fp64_peak = sms * 2 * 2 * mhz * 1e6  # flop/s
    p = cg.make_problem(args.config, seed=0)
    opts = {}
    if args.stage_rows is not None:
        opts["stage_rows"] = args.stage_rows
    if args.stage_depth is not None:
        opts["stage_depth"] = args.stage_depth
    for kv in args.set:
        k, v = kv.split("=", 1)
        opts[k] = int(v)
    s = amgf.Solver(p.K, p.J, p.D, precision=args.precision, **opts)
    if args.weights:
        from paper_2505_18576_gb300.learned import load_weights
        default = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "smoother_c64.npz")
        s.set_mlp(load_weights(default if args.weights == "default" else args.weights))
    b = torch.from_numpy(p.b).cuda()
    x = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    st = s.pcg_solve(b, x)
    s.profile_iteration()  # warm-up
    agg = collections.OrderedDict()
    total_ms = 0.0
    for _ in range(args.iters):
        for r in s.profile_iteration():
            key = (r["op"], r["level"])
            a = agg.setdefault(key, [0, 0.0, 0.0, 0.0])
            a[0] += 1
            a[1] += r["ms"]
            a[2] += r["bytes"]
            a[3] += r["flops"]
            total_ms += r["ms"]
    fp64 = args.precision == 0
    print(f"Workload {args.config} (n = {p.n}), precision {args.precision}"
          f"{', learned smoother' if args.weights else ''}: {st.iters} PCG iterations per solve, "
          f"{total_ms / args.iters:.3f} ms per profiled iteration ({args.iters} iterations), "
          f"copy-bandwidth peak {hbm:.1f} GB/s ({kind}), FP64 peak {fp64_peak / 1e12:.3f} TFLOP/s "
          f"({sms} SMs, {mhz:.0f} MHz); staged levels mask {int(s.info.staged_levels):#x}, "
          f"sliced-ELL levels mask {int(s.info.sell_levels):#x}.\n")
    print("| operation | level | launches / iteration | us / launch | MB / launch | GB/s | of peak | FP64 pipe | share |")
    print("|---|---|---|---|---|---|---|---|---|")
    for (op, lvl), (cnt, ms, by, fl) in sorted(agg.items(), key=lambda kv: -kv[1][1]):
        per = cnt / args.iters
        t = ms / cnt
        gbs = (by / cnt) / (t * 1e-3) / 1e9 if t > 0 else 0.0
        # FP64 arithmetic: every kernel of the FP64 path; in the mixed path the fine-level FP64
        # products A p, r1 = r - A y1 and the rows touching I_c, and the filter
        is64 = fp64 or (lvl == 0 and op in ("A p, p^T A p", "b - A x, W (b - A x)",
                                             "r2 = r1 - A P w (rows touching I_c)")) or op.startswith("filter")
        pipe = f"{(fl / cnt) / (t * 1e-3) / fp64_peak:.2f}" if is64 and fl > 0 and t > 0 else ""
        print(f"| {op} | {lvl if lvl >= 0 else ''} | {per:g} | {t * 1e3:.1f} | {by / cnt / 1e6:.2f} | {gbs:.0f} | "
              f"{gbs / hbm:.2f} | {pipe} | {100 * ms / total_ms:.1f}% |")
    s.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
