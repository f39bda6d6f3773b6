"""Autotuner for the stabilisation interval n_wrap.

The paper cites the stabilised B-chain ("Basics of DQMC") but leaves the
re-orthogonalisation interval open.  On GB300 it sets the balance between
the cheap tensor-core slice products and the FP64 Cholesky-QR (about
3.3 N^3 FP64 flops per block), so it is chosen per lattice size, temperature
and precision mode by measurement:

  candidates: every n_wrap from a fixed ladder whose block condition bound
  n_wrap * dtau * (8|t| + 2|xi|) stays within the library's limit (16);
  accuracy: the log|det| of a batch of seeded fields must agree with an
  FP64-product evaluation at the smallest candidate within the mode's stated
  bound (FP64 1e-9, split-TF32 1e-6, BF16 1e-2, all relative);
  speed: the fastest accurate candidate wins (CUDA-event time of one batch).

autotune_schedule() tunes n_wrap together with the output tile of the
tensor-core slice products (128 x 64 with eight FP32 accumulators, or
128 x 128 with four: fewer shared-memory operand reads per flop, more
accumulation error per accumulator), keeping the fastest (n_wrap, tile)
pair whose log|det| meets the mode's bound.  The FP64 GEMM picks its own
tile (64 x 64 or 32 x 32) from the number of tiles a launch has.
"""
import math

LADDER = (2, 3, 4, 5, 6, 8, 10, 12, 16, 20, 25, 32, 40, 50, 64)
LIMIT = 16.0
TOL = {"fp64": 1e-9, "3xtf32": 1e-6, "bf16": 1e-2, "bf16x3": 1e-6}


def candidates(M, dtau, t=1.0, xi=1.0, limit=LIMIT):
    """n_wrap values of the ladder that the block condition bound allows (at most M)."""
    per = dtau * (8.0 * abs(t) + 2.0 * abs(xi))
    out = [n for n in LADDER if n <= M and (per == 0.0 or n * per <= limit)]
    return out or [1]


def autotune_nwrap(L, beta, dtau, mu, prec, t=1.0, xi=1.0, batch=16, reps=2, seed=4321, tol=None):
    """Returns (best n_wrap, [(n_wrap, ms per batch, max relative log-det deviation), ...])
    with the default 128 x 64 tensor-core tile."""
    nw, _, res = autotune_schedule(L, beta, dtau, mu, prec, t=t, xi=xi, batch=batch, reps=reps, seed=seed,
                                   tol=tol, tiles=(64,))
    return nw, [(r[0], r[2], r[3]) for r in res]


def autotune_schedule(L, beta, dtau, mu, prec, t=1.0, xi=1.0, batch=16, reps=2, seed=4321, tol=None,
                      tiles=(64, 128)):
    """Returns (best n_wrap, best tile width, [(n_wrap, tile, ms per batch, max relative
    log-det deviation), ...]); FP64 mode and lattices below 128 sites tune n_wrap only."""
    import torch
    from . import sldqmc
    from .inputs import batch_uniform

    M = int(round(beta / dtau))
    cands = candidates(M, dtau, t, xi)
    tol = TOL[prec] if tol is None else tol
    s = torch.from_numpy(batch_uniform(seed, batch, M, L * L)).cuda()
    ref = torch.zeros(batch, dtype=torch.float64, device="cuda")
    with sldqmc.Context(L, L, t=t, mu=mu, xi=xi, beta=beta, dtau=dtau, n_wrap=cands[0], prec="fp64",
                        max_batch=batch) as c0:
        c0.weight_batch_dev(s, -1, ref)
        c0.sync()
    if prec == "fp64" or L * L < 128:
        tiles = (64,)
    results = []
    for nw in cands:
        try:
            ctx = sldqmc.Context(L, L, t=t, mu=mu, xi=xi, beta=beta, dtau=dtau, n_wrap=nw, prec=prec,
                                 max_batch=batch)
        except sldqmc.SldqmcError:
            continue
        with ctx:
            for tile in tiles:
                ctx.set_tile_n(tile)
                ld = torch.zeros(batch, dtype=torch.float64, device="cuda")
                ctx.weight_batch_dev(s, -1, ld)
                ctx.sync()
                st = torch.cuda.current_stream()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(st)
                for _ in range(reps):
                    ctx.weight_batch_dev(s, -1, ld)
                e1.record(st)
                ctx.sync()
                ms = e0.elapsed_time(e1) / reps
                err = float(((ld - ref).abs() / ref.abs()).max())
                results.append((nw, tile, ms, err))
    ok = [r for r in results if math.isfinite(r[3]) and r[3] <= tol]
    best = min(ok, key=lambda r: r[2]) if ok else (cands[0], 64)
    return best[0], best[1], results
