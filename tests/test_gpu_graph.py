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


def test_uneven_graph_chains_against_oracle():
    """A small uneven set stepped by one CUDA graph, against the FP64 CPU oracle step by
    step: 12x12 at beta = 1 and 16x16 at beta = 2 (dtau = 0.05), split-TF32 products,
    bare-Ising H_eff, two chains each.  Decisions within the margin that the log-det
    bound allows (twice 1e-6 of the fermion part of log omega) are margin events, where
    the oracle takes the graph's outcome; every other decision, configuration and kept
    weight must agree."""
    import math

    import torch
    from oracle import oracle as O
    from paper_1612_03804_gb300 import sldqmc
    from paper_1612_03804_gb300.inputs import uniform_field
    bound = 1e-6
    specs = [(12, 1.0), (16, 2.0)]
    B, steps, step0 = 2, 4, 5
    members, models, states, seeds = [], [], [], []
    for k, (L, beta) in enumerate(specs):
        m = O.Model(L, L, mu=-0.5, xi=1.0, beta=beta, dtau=0.05, n_wrap=10, J=1.0, h=2.774)
        kt = -0.5 * math.log(math.tanh(m.dtau * m.h))
        J = np.array([-m.dtau * m.J / m.beta, 0.0, 0.0, -kt / m.beta])
        s0 = np.stack([O.eff_sweeps(m, uniform_field(4100 + 10 * k + b, m.M, m.N), CLASSES, J, 30, seed=7,
                                    step=b, direction=0)[0] for b in range(B)])
        ctx = sldqmc.Context(L, L, mu=-0.5, xi=1.0, beta=beta, dtau=0.05, n_wrap=10, prec="3xtf32", max_batch=B)
        ctx.set_effective_model(CLASSES, J)
        d_s = torch.from_numpy(s0).cuda()
        d_lw = torch.zeros(B, dtype=torch.float64, device="cuda")
        ctx.log_weight_batch_dev(d_s, d_lw)
        d_acc = torch.zeros(B, dtype=torch.int32, device="cuda")
        ctx.sync()
        seed = 5150 + k
        members.append((ctx, d_s, d_lw, d_acc, seed))
        models.append((m, J))
        states.append(([s0[b].copy() for b in range(B)], [O.log_weight_total(m, s0[b]) for b in range(B)]))
        seeds.append(seed)
    g = sldqmc.Graph(members, n_eff=1, step0=step0)
    compared = margin = 0
    for t in range(steps):
        before = [mb[3].cpu().numpy().copy() for mb in members]
        g.launch(1)
        g.sync()
        for k, (ctx, d_s, d_lw, d_acc, seed) in enumerate(members):
            m, J = models[k]
            so_l, lw_l = states[k]
            s_g, lw_g = d_s.cpu().numpy(), d_lw.cpu().numpy()
            acc_g = d_acc.cpu().numpy() - before[k]
            for b in range(B):
                fermion = abs(lw_l[b] - O.log_bare_weight(m, so_l[b]))
                mg = 4.0 * bound * fermion
                so, lwo, ao, lro, _, _ = O.cumulative_update(m, so_l[b], lw_l[b], CLASSES, J, 1,
                                                             seed=seed + (b << 32), step=step0 + t)
                lu = math.log(O.uniform(seed + (b << 32), 0, 0, step0 + t, 4))
                if abs(lro - lu) <= mg:
                    margin += 1
                    so_l[b], lw_l[b] = s_g[b].copy(), O.log_weight_total(m, s_g[b])
                    continue
                compared += 1
                assert acc_g[b] == ao, (k, b, t, lro, lu)
                np.testing.assert_array_equal(s_g[b], so)
                assert abs(lw_g[b] - lwo) <= 2.0 * bound * fermion
                so_l[b], lw_l[b] = so, lwo
    g.close()
    print(f"uneven graph vs oracle: {compared} decisions compared, {margin} margin events")
    assert compared >= len(specs) * B * steps - 2
