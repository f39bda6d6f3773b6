"""A short run of the cumulative-update step for profilers (ncu launch lists
and counter captures): one context, seeded fields moved by a few sweeps of
the bare Ising action, their exact log weights, `--warmup` untimed steps and
`--steps` steps, then the number of library launches of each phase so that a
capture can skip to the step it wants.

  python -m paper_1612_03804_gb300.profile_run --L 16 --batch 128 --prec 3xtf32 --n-wrap 32
  python -m paper_1612_03804_gb300.profile_run --L 50 --beta 10 --dtau 0.1 --n-wrap 10 --batch 1

The launch counts are printed on stderr as JSON: {"setup": S, "per_step": P}
(library kernels; a profiler that counts every kernel of the process sees
the same launches, torch launches none between them).
"""
import argparse
import json
import math
import sys

import numpy as np

CLASSES = [[(1, 0, 0), (0, 1, 0)], [(1, 1, 0), (1, -1, 0)], [(2, 0, 0), (0, 2, 0)], [(0, 0, 1)]]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--L", type=int, default=16)
    ap.add_argument("--beta", type=float, default=8.0)
    ap.add_argument("--dtau", type=float, default=0.05)
    ap.add_argument("--mu", type=float, default=-0.5)
    ap.add_argument("--n-wrap", type=int, default=32)
    ap.add_argument("--batch", type=int, default=128)
    ap.add_argument("--prec", default="3xtf32")
    ap.add_argument("--kinetic", default="dense", choices=["dense", "separable"])
    ap.add_argument("--tile", type=int, default=64, choices=[64, 128])
    ap.add_argument("--warmup", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    args = ap.parse_args()
    import torch
    from . import build, sldqmc
    from .inputs import batch_uniform
    build.build()
    torch.cuda.set_device(0)
    ctx = sldqmc.Context(args.L, args.L, mu=args.mu, xi=1.0, beta=args.beta, dtau=args.dtau, n_wrap=args.n_wrap,
                         prec=args.prec, max_batch=args.batch)
    ctx.set_kinetic_form(args.kinetic)
    if args.prec != "fp64":
        ctx.set_tile_n(args.tile)
    kt = -0.5 * math.log(math.tanh(args.dtau * 2.774))
    ctx.set_effective_model(CLASSES, np.array([-args.dtau / args.beta, 0.0, 0.0, -kt / args.beta]))
    B = args.batch
    d_s = torch.from_numpy(batch_uniform(5000, B, ctx.M, ctx.N)).cuda()
    ctx.eff_sweeps_batch_dev(d_s, 2, 11, 0, -1)
    d_lw = torch.zeros(B, dtype=torch.float64, device="cuda")
    ctx.log_weight_batch_dev(d_s, d_lw)
    d_acc = torch.zeros(B, dtype=torch.int32, device="cuda")
    for w in range(args.warmup):
        ctx.cumulative_batch_dev(d_s, d_lw, 1, 123, w, 1, d_acc)
    ctx.sync()
    setup = ctx.kernel_launches()
    ctx.cumulative_batch_dev(d_s, d_lw, 1, 123, args.warmup, args.steps, d_acc)
    ctx.sync()
    per_step = (ctx.kernel_launches() - setup) / max(args.steps, 1)
    print(json.dumps({"setup": setup, "per_step": per_step}), file=sys.stderr)
    ctx.close()


if __name__ == "__main__":
    main()
