"""Precision sweep and large-lattice timing of the exact weight (GPU).

  python -m paper_1612_03804_gb300.precision_sweep            # 32x32, beta=10, M=200
  python -m paper_1612_03804_gb300.precision_sweep --large    # 100x100, beta=10, M=100

Sweep: seeded random +-1 fields on a 32x32 lattice (t=1, mu=-0.5, xi=1,
beta=10, dtau=0.05, M=200); for n_wrap in {5, 10, 20} the slice products run
in FP64, split-TF32 and BF16 (FP32 accumulation), with FP64 stabilisation in
every mode.  Reported per mode: relative and absolute log|det| error and
max|dG| against the FP64-product path (parity-checked against the FP64 CPU
oracle at smaller sizes; the oracle itself needs minutes per weight here),
and the relative error of the uniform-field closed form.

Large: one exact weight of a uniform field on 100x100 (N = 10^4, dtau=0.1,
M=100, n_wrap=10) in split-TF32 with the closed-form error, and the FP64
product time per slice measured on the same lattice (the full FP64 weight,
about 2*M*N^3 FP64 flops, is extrapolated from it and labelled so).
"""
import argparse
import json
import time

import numpy as np


def closed_form(L, beta, t, mu_eff):
    k = 2 * np.pi * np.arange(L) / L
    eps = (-2 * t * (np.cos(k)[None, :] + np.cos(k)[:, None])).ravel() - mu_eff
    return float(np.sum(np.logaddexp(0.0, -beta * eps)))


def sweep(args):
    import torch
    from . import sldqmc
    from .inputs import batch_uniform
    L, beta, dtau, mu = 32, 10.0, 0.05, -0.5
    M = int(round(beta / dtau))
    fields = torch.from_numpy(batch_uniform(1003, args.fields, M, L * L)).cuda()
    uniform = torch.ones((1, M, L * L), dtype=torch.int8, device="cuda")
    out = []
    for nw in (5, 10, 20):
        res = {}
        for prec in ("fp64", "3xtf32", "bf16x3", "bf16"):
            with sldqmc.Context(L, L, mu=mu, xi=1.0, beta=beta, dtau=dtau, n_wrap=nw, prec=prec,
                                max_batch=args.fields) as ctx:
                ld = torch.zeros(args.fields, dtype=torch.float64, device="cuda")
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                ctx.weight_batch_dev(fields, -1, ld)
                ctx.sync()
                dt = time.perf_counter() - t0
                G = torch.zeros((1, L * L, L * L), dtype=torch.float64, device="cuda")
                ctx.green_batch_dev(fields[:1], -1, 0, G)
                lu = torch.zeros(1, dtype=torch.float64, device="cuda")
                ctx.weight_batch_dev(uniform, -1, lu)
                ctx.sync()
                res[prec] = (ld.cpu().numpy(), G.cpu().numpy()[0], float(lu.item()), dt)
        ref_ld, ref_G = res["fp64"][0], res["fp64"][1]
        cf = closed_form(L, beta, 1.0, mu - 1.0)  # eta = -1, s = +1: mu -> mu - xi
        for prec in ("fp64", "3xtf32", "bf16x3", "bf16"):
            ld, G, lu, dt = res[prec]
            out.append({"n_wrap": nw, "prec": prec,
                        "logdet_rel_err_max": float(np.max(np.abs(ld - ref_ld) / np.abs(ref_ld))),
                        "logdet_abs_err_max": float(np.max(np.abs(ld - ref_ld))),
                        "max_abs_dG": float(np.max(np.abs(G - ref_G))),
                        "closed_form_rel_err": abs(lu - cf) / abs(cf),
                        "weights_per_s": args.fields / dt})
    return out


def large(args):
    import torch
    from . import sldqmc
    L, beta, dtau, mu, nw = 100, 10.0, 0.1, -0.5, 10
    M = int(round(beta / dtau))
    s = torch.ones((1, M, L * L), dtype=torch.int8, device="cuda")
    res = {}
    with sldqmc.Context(L, L, mu=mu, xi=1.0, beta=beta, dtau=dtau, n_wrap=nw, prec="3xtf32", max_batch=1) as ctx:
        ld = torch.zeros(1, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.weight_batch_dev(s, -1, ld)
        ctx.sync()
        res["split_tf32_s_per_weight"] = time.perf_counter() - t0
        cf = closed_form(L, beta, 1.0, mu - 1.0)
        res["split_tf32_closed_form_rel_err"] = abs(float(ld.item()) - cf) / abs(cf)
    # FP64 products: time one block of n_wrap slices (weight of a beta = n_wrap*dtau chain)
    with sldqmc.Context(L, L, mu=mu, xi=1.0, beta=nw * dtau, dtau=dtau, n_wrap=nw, prec="fp64", max_batch=1) as c64:
        s1 = torch.ones((1, nw, L * L), dtype=torch.int8, device="cuda")
        ld = torch.zeros(1, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c64.weight_batch_dev(s1, -1, ld)
        c64.sync()
        t_block = time.perf_counter() - t0
    res["fp64_s_per_block_of_10_slices"] = t_block
    res["fp64_s_per_weight_extrapolated"] = t_block * (M // nw)
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--fields", type=int, default=10)
    ap.add_argument("--large", action="store_true")
    args = ap.parse_args()
    import torch
    from . import build
    build.build()
    torch.cuda.set_device(0)
    print(json.dumps(large(args) if args.large else sweep(args), indent=1))


if __name__ == "__main__":
    main()
