"""Observables of reduced-precision SLDQMC chains against the FP64 CPU oracle's
chains: both sample omega(C) exactly (Eq. 4), so the magnetisation moments
and the acceptance must agree within their statistical errors.

12x12 at the paper's critical point (beta = 1, dtau = 0.05, M = 20,
h = 2.774), bare-Ising effective action, 10 effective sweeps per cumulative
update.  GPU: 64 chains in split-TF32 and in FP64; oracle: 16 chains on the
host cores.  Error bars are standard errors of the per-chain means over
independent chains (which carry each chain's autocorrelation); agreement
within 3.5 sigma of the combined error."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1612_03804_gb300.inputs import uniform_field

pytestmark = pytest.mark.gpu

CLASSES = [[(1, 0, 0), (0, 1, 0)], [(1, 1, 0), (1, -1, 0)], [(2, 0, 0), (0, 2, 0)], [(0, 0, 1)]]
N_EFF = 10
BURN = 40


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    from paper_1612_03804_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _model():
    m = O.Model(12, 12, mu=-0.5, xi=1.0, beta=1.0, dtau=0.05, n_wrap=10, J=1.0, h=2.774)
    kt = -0.5 * math.log(math.tanh(m.dtau * m.h))
    return m, np.array([-m.dtau * m.J / m.beta, 0.0, 0.0, -kt / m.beta])


def _stats(series, V):
    """Per-chain means of |M|/V and (M/V)^2 after the burn-in: (mean, standard error) each."""
    x = series[BURN:].astype(np.float64) / V
    out = []
    for f in (np.abs(x), x * x):
        cm = f.mean(axis=0)
        out.append((cm.mean(), cm.std(ddof=1) / math.sqrt(len(cm))))
    return out


@pytest.fixture(scope="module")
def oracle_chains():
    m, J = _model()
    starts = [O.eff_sweeps(m, uniform_field(6000 + b, m.M, m.N), CLASSES, J, 100, seed=61, step=b,
                           direction=0)[0] for b in range(16)]
    series, acc = O.cumulative_chains(m, starts, CLASSES, J, N_EFF, [6100 + b for b in range(16)], 0, 160)
    return series, acc, 160


@pytest.mark.parametrize("prec", ["3xtf32", "fp64"])
def test_chain_observables_match_oracle(prec, oracle_chains):
    import torch
    from paper_1612_03804_gb300 import sldqmc
    from paper_1612_03804_gb300.inputs import batch_uniform
    m, J = _model()
    V = m.N * m.M
    B, steps = 64, 400
    with sldqmc.Context(12, 12, mu=-0.5, xi=1.0, beta=1.0, dtau=0.05, n_wrap=10, J=1.0, h=2.774, prec=prec,
                        max_batch=B) as ctx:
        ctx.set_effective_model(CLASSES, J)
        d_s = torch.from_numpy(batch_uniform(6200, B, m.M, m.N)).cuda()
        for k in range(100):
            ctx.eff_sweeps_batch_dev(d_s, 1, 62, k, -1)
        d_lw = torch.zeros(B, dtype=torch.float64, device="cuda")
        ctx.log_weight_batch_dev(d_s, d_lw)
        d_acc = torch.zeros(B, dtype=torch.int32, device="cuda")
        mags = torch.zeros((steps, B), dtype=torch.int64, device="cuda")
        for k in range(steps):
            ctx.cumulative_batch_dev(d_s, d_lw, N_EFF, 63, k, 1, d_acc)
            mags[k] = d_s.to(torch.int64).sum(dim=(1, 2))
        ctx.sync()
        g_series = mags.cpu().numpy()
        g_acc = d_acc.cpu().numpy()
    o_series, o_acc, o_steps = oracle_chains
    for name, (gm, ge), (om, oe) in zip(("|M|/V", "(M/V)^2"), _stats(g_series, V), _stats(o_series, V)):
        z = abs(gm - om) / math.sqrt(ge ** 2 + oe ** 2)
        print(f"{prec} {name}: GPU {gm:.5f} +- {ge:.5f}, oracle {om:.5f} +- {oe:.5f}, {z:.2f} sigma")
        assert z < 3.5, (name, gm, ge, om, oe)
    pg, po = g_acc.sum() / (B * steps), o_acc.sum() / (len(o_acc) * o_steps)
    eg = math.sqrt(pg * (1 - pg) / (B * steps)) * 3  # accept decisions are correlated in time
    eo = math.sqrt(po * (1 - po) / (len(o_acc) * o_steps)) * 3
    print(f"{prec} accept rate: GPU {pg:.4f}, oracle {po:.4f}")
    assert abs(pg - po) < 3.5 * math.sqrt(eg ** 2 + eo ** 2)
