"""Launch one kernel of the solve phase a few times on a generated workload (for profilers).

    python -m paper_2505_18576_gb300.profile_kernel --config c64 --precision 3 --which 2 --reps 3

Sets up the seeded two-block system of `--config`, then runs `amgf_time_kernel(which)`
(0: fine-level A x, 1: fine-level FP64 post-smoother, 2: fine-level post-smoother of the mixed
V-cycle, 3: level-1 post-smoother) with `--warmup` untimed and `--reps` timed launches, and
prints the kernel's mean duration and algorithmic bytes per launch.  Under a profiler, select
the kernel by name and the launch count, e.g. `ncu -k regex:bsr3_mixed -s 1 -c 2`.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", default="c64")
    ap.add_argument("--precision", type=int, default=0)
    ap.add_argument("--which", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=1)
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--weights", default=None, help="learned smoother weights (.npz), 'default' = packaged")
    ap.add_argument("--stage-rows", type=int, default=None, help="amgf_options.stage_rows (default: library's)")
    ap.add_argument("--stage-depth", type=int, default=None, help="amgf_options.stage_depth")
    ap.add_argument("--set", action="append", default=[], metavar="FIELD=INT",
                    help="any other integer field of amgf_options, e.g. --set fuse_tail=0")
    args = ap.parse_args(argv)

    import torch

    import contactgen as cg
    import paper_2505_18576_gb300 as amgf

    torch.cuda.set_device(0)
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
    ms, nbytes = s.time_kernel(args.which, warmup=args.warmup, reps=args.reps)
    info = s.info
    print(json.dumps({"config": args.config, "precision": args.precision, "which": args.which, "ms": ms,
                      "algorithmic_bytes_per_launch": nbytes, "gbs": nbytes / (ms * 1e-3) / 1e9,
                      "levels": int(info.nlevels), "staged_levels": int(info.staged_levels),
                      "level_rows": [int(info.level_rows[l]) for l in range(info.nlevels)],
                      "level_nnz": [int(info.level_nnz[l]) for l in range(info.nlevels)]}))
    s.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
