"""Uneven chain groups captured in one CUDA graph: every replay must equal
one step of sldqmc_cumulative_batch_dev for every member (same seeds, same
steps), bit for bit, across members of different lattice sizes, beta and
precision."""
import numpy as np
import pytest

from paper_1612_03804_gb300.inputs import batch_uniform

pytestmark = pytest.mark.gpu

CLASSES = [[(1, 0, 0), (0, 1, 0)], [(1, 1, 0), (1, -1, 0)], [(2, 0, 0), (0, 2, 0)], [(0, 0, 1)]]
J_EFF = np.array([-0.05, -0.01, 0.004, -0.45])


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    from paper_1612_03804_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _member(L, beta, dtau, nw, B, seed, prec="fp64"):
    import torch
    from paper_1612_03804_gb300 import sldqmc
    ctx = sldqmc.Context(L, L, mu=-0.5, xi=1.0, beta=beta, dtau=dtau, n_wrap=nw, prec=prec, max_batch=B)
    ctx.set_effective_model(CLASSES, J_EFF)
    s = torch.from_numpy(batch_uniform(seed, B, ctx.M, ctx.N)).cuda()
    lw = torch.zeros(B, dtype=torch.float64, device="cuda")
    ctx.log_weight_batch_dev(s, lw)
    acc = torch.zeros(B, dtype=torch.int32, device="cuda")
    ctx.sync()
    return ctx, s, lw, acc


@pytest.mark.parametrize("prec_big", ["fp64", "3xtf32"])
def test_graph_replays_equal_sequential_steps(prec_big):
    from paper_1612_03804_gb300 import sldqmc
    specs = [(4, 2.0, 0.1, 10, 3, 11, "fp64"), (6, 1.0, 0.1, 5, 2, 12, "fp64"), (12, 1.0, 0.05, 10, 2, 13, prec_big)]
    graph_m = [_member(*sp) for sp in specs]
    ref_m = [_member(*sp) for sp in specs]
    seeds = [101, 202, 303]
    g = sldqmc.Graph([(m[0], m[1], m[2], m[3], sd) for m, sd in zip(graph_m, seeds)], n_eff=1, step0=7)
    g.launch(3)
    g.sync()
    for (ctx, s, lw, acc), sd in zip(ref_m, seeds):
        ctx.cumulative_batch_dev(s, lw, 1, sd, 7, 3, acc)
        ctx.sync()
    for gm, rm in zip(graph_m, ref_m):
        np.testing.assert_array_equal(gm[1].cpu().numpy(), rm[1].cpu().numpy())
        np.testing.assert_array_equal(gm[3].cpu().numpy(), rm[3].cpu().numpy())
        np.testing.assert_array_equal(gm[2].cpu().numpy(), rm[2].cpu().numpy())
    g.close()
