"""Batched uneven chains: 64 independent SLDQMC chains, chain c on an L x L
lattice with L = (12, 16, 20, 24, 32)[c mod 5] and beta = (4, 8)[(c div 5)
mod 2], dtau = 0.05, mu = -0.5, xi = 1, split-TF32 products with FP64
stabilisation, n_wrap chosen per (L, beta) bucket by the autotuner, all ten
buckets stepped by one CUDA graph.  Every replay must equal the sequential
per-bucket cumulative updates bit for bit."""
import time

import numpy as np
import pytest

from paper_1612_03804_gb300.inputs import batch_uniform

pytestmark = pytest.mark.gpu

CLASSES = [[(1, 0, 0), (0, 1, 0)], [(1, 1, 0), (1, -1, 0)], [(2, 0, 0), (0, 2, 0)], [(0, 0, 1)]]
LS = (12, 16, 20, 24, 32)
BETAS = (4.0, 8.0)


def _buckets():
    counts = {}
    for c in range(64):
        key = (LS[c % 5], BETAS[(c // 5) % 2])
        counts[key] = counts.get(key, 0) + 1
    return counts


def _bare(beta, dtau=0.05, J=1.0, h=2.774):
    import math
    kt = -0.5 * math.log(math.tanh(dtau * h))
    return np.array([-dtau * J / beta, 0.0, 0.0, -kt / beta])


def test_sixty_four_uneven_chains_in_one_graph():
    import torch
    from paper_1612_03804_gb300 import build, sldqmc
    from paper_1612_03804_gb300.tune import autotune_nwrap
    build.build()
    torch.cuda.set_device(0)
    buckets = _buckets()
    assert sum(buckets.values()) == 64 and len(buckets) == 10
    members, refs = [], []
    for k, ((L, beta), B) in enumerate(sorted(buckets.items())):
        nw, _ = autotune_nwrap(L, beta, 0.05, -0.5, "3xtf32", batch=2, reps=1)
        for dst in (members, refs):
            ctx = sldqmc.Context(L, L, mu=-0.5, xi=1.0, beta=beta, dtau=0.05, n_wrap=nw, prec="3xtf32",
                                 max_batch=B)
            ctx.set_effective_model(CLASSES, _bare(beta))
            s = torch.from_numpy(batch_uniform(900 + k, B, ctx.M, ctx.N)).cuda()
            ctx.eff_sweeps_batch_dev(s, 20, 5, 0, -1)
            lw = torch.zeros(B, dtype=torch.float64, device="cuda")
            ctx.log_weight_batch_dev(s, lw)
            acc = torch.zeros(B, dtype=torch.int32, device="cuda")
            ctx.sync()
            dst.append((ctx, s, lw, acc, 7000 + k))
    g = sldqmc.Graph(members, n_eff=1, step0=3)
    g.launch(1)
    g.sync()
    t0 = time.perf_counter()
    g.launch(2)
    g.sync()
    dt = (time.perf_counter() - t0) / 2
    print(f"64 uneven chains: {dt * 1e3:.1f} ms per graph replay ({2 * 64 / dt:.1f} weight evals/s)")
    for ctx, s, lw, acc, sd in refs:
        ctx.cumulative_batch_dev(s, lw, 1, sd, 3, 3, acc)
        ctx.sync()
    for m, r in zip(members, refs):
        np.testing.assert_array_equal(m[1].cpu().numpy(), r[1].cpu().numpy())
        np.testing.assert_array_equal(m[3].cpu().numpy(), r[3].cpu().numpy())
        np.testing.assert_array_equal(m[2].cpu().numpy(), r[2].cpu().numpy())
    g.close()
