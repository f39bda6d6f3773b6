"""The separable form of exp(-dtau K) in the slice products, against the FP64
CPU oracle through the C ABI.

exp(-dtau K) = e^{dtau mu} E1x (x) E1y holds exactly on the periodic lattice,
so the weight and G must equal the dense definition the oracle evaluates,
to the FP64 bar (1e-9 relative log|det|, 1e-9 absolute G) in the FP64 mode
and to the reduced-precision bar (1e-6, 1e-5) in the mixed modes, whose
split-FP32 convolutions carry 48-bit operands."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1612_03804_gb300.inputs import batch_uniform, domain_field, uniform_field

pytestmark = pytest.mark.gpu

BOUND = {"fp64": 1e-9, "3xtf32": 1e-6, "bf16x3": 1e-6}
G_BOUND = {"fp64": 1e-9, "3xtf32": 1e-5, "bf16x3": 1e-5}
CLASSES = [[(1, 0, 0), (0, 1, 0)], [(1, 1, 0), (1, -1, 0)], [(2, 0, 0), (0, 2, 0)], [(0, 0, 1)]]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    from paper_1612_03804_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _ctx(m, n_wrap, prec, max_batch):
    from paper_1612_03804_gb300 import sldqmc
    c = sldqmc.Context(m.Lx, m.Ly, t=m.t, mu=m.mu, xi=m.xi, beta=m.beta, dtau=m.dtau, n_wrap=n_wrap,
                       J=m.J, h=m.h, prec=prec, max_batch=max_batch)
    c.set_kinetic_form("separable")
    return c


CASES = [
    # Lx, Ly, mu, beta, dtau, n_wrap, field
    (4, 4, 0.0, 2.0, 0.1, 10, "uniform"),
    (5, 6, -0.5, 2.0, 0.1, 7, "domains"),    # Lx != Ly, odd Lx, ragged last block
    (2, 1, -0.5, 1.0, 0.25, 2, "uniform"),   # a direction of length 1 (no bond) and one of length 2
    (1, 1, 0.2, 1.0, 0.25, 3, "uniform"),
    (12, 12, -0.5, 2.0, 0.05, 20, "uniform"),
    (7, 3, 0.4, 1.5, 0.1, 5, "uniform"),
]


MIXED_CASES = [
    # the mixed modes need N >= 128 (their dense products use 128-row tensor-core tiles)
    (12, 12, -0.5, 2.0, 0.05, 20, "uniform"),
    (13, 11, 0.4, 1.5, 0.1, 5, "domains"),   # N = 143, Lx != Ly, both odd, ragged last block
    (16, 9, -0.5, 1.0, 0.1, 3, "uniform"),
]


@pytest.mark.parametrize("prec,Lx,Ly,mu,beta,dtau,nw,kind",
                         [("fp64",) + c for c in CASES] + [(p,) + c for p in ("3xtf32", "bf16x3") for c in MIXED_CASES])
def test_separable_weight_matches_oracle(prec, Lx, Ly, mu, beta, dtau, nw, kind):
    m = O.Model(Lx, Ly, mu=mu, xi=1.0, beta=beta, dtau=dtau, n_wrap=1)
    if kind == "uniform":
        fields = np.stack([uniform_field(300 + k, m.M, m.N) for k in range(3)])
    else:
        fields = np.stack([domain_field(300 + k, m.M, Lx, Ly, corr=2) for k in range(3)])
    with _ctx(m, nw, prec, 2) as ctx:
        for eta in (1, -1):
            ld, sg = ctx.weight_batch(fields, eta)
            for k in range(3):
                ref, rs = O.weight(m, fields[k], eta)
                assert sg[k] == rs
                assert abs(ld[k] - ref) <= BOUND[prec] * max(1.0, abs(ref)), (prec, k, eta, ld[k], ref)


@pytest.mark.parametrize("prec,Lx,Ly", [("fp64", 6, 5), ("3xtf32", 12, 11), ("bf16x3", 12, 11)])
def test_separable_green_matches_oracle(prec, Lx, Ly):
    m = O.Model(Lx, Ly, mu=-0.3, xi=1.0, beta=2.0, dtau=0.1, n_wrap=1)
    s = uniform_field(41, m.M, m.N)
    with _ctx(m, 10, prec, 1) as ctx:
        for tau in (0, 7):
            G, ld, sg = ctx.green(s, -1, tau)
            ref, rs, Gref = O.weight(m, s, -1, tau0=tau, want_G=True)
            assert sg == rs and abs(ld - ref) <= BOUND[prec] * abs(ref)
            assert np.abs(G - Gref).max() <= G_BOUND[prec]


@pytest.mark.parametrize("prec", ["fp64", "3xtf32"])
def test_separable_benchmark_size(prec):
    """16x16, beta = 8, dtau = 0.05 (M = 160), n_wrap = 32, B = 8 random fields."""
    m = O.Model(16, 16, mu=-0.5, xi=1.0, beta=8.0, dtau=0.05, n_wrap=10)
    B = 8
    fields = batch_uniform(2501, B, m.M, m.N)
    ref = O.weight_many(m, fields, -1)
    with _ctx(m, 32, prec, B) as ctx:
        ld, sg = ctx.weight_batch(fields, -1)
    r = np.array([x[0] for x in ref])
    np.testing.assert_array_equal(sg, [x[1] for x in ref])
    rel = np.abs(ld - r) / np.abs(r)
    print(f"separable {prec} 16x16 M=160: max rel log-det error {rel.max():.2e}")
    assert rel.max() <= BOUND[prec]


@pytest.mark.parametrize("prec", ["fp64", "3xtf32"])
def test_separable_uniform_field_closed_form(prec):
    L, beta, dtau, mu = 32, 10.0, 0.05, -0.5
    M = int(round(beta / dtau))
    k = 2 * np.pi * np.arange(L) / L
    m = O.Model(L, L, mu=mu, xi=1.0, beta=beta, dtau=dtau)
    with _ctx(m, 20, prec, 1) as ctx:
        s = np.ones((M, L * L), dtype=np.int8)
        ld, sg = ctx.weight(s, -1)
    eps = (-2 * (np.cos(k)[None, :] + np.cos(k)[:, None])).ravel() - (mu - 1.0)
    ref = float(np.sum(np.logaddexp(0.0, -beta * eps)))
    print(f"separable {prec} 32x32 closed form: rel err {abs(ld - ref) / ref:.2e}")
    assert sg == 1 and abs(ld - ref) <= BOUND[prec] * ref


def test_separable_cumulative_chain_bit_exact():
    """FP64 mode: a cumulative-update chain with the separable products follows the oracle."""
    m = O.Model(4, 4, mu=0.0, xi=1.0, beta=2.0, dtau=0.1, n_wrap=10, J=1.0, h=2.774)
    J = np.array([-0.05, -0.01, 0.004, -0.45])
    s = uniform_field(77, m.M, m.N)
    lw = O.log_weight_total(m, s)
    so, lwo = s.copy(), lw
    with _ctx(m, 10, "fp64", 1) as ctx:
        ctx.set_effective_model(CLASSES, J)
        for step in range(6):
            s, lw, a, lr = ctx.cumulative_update(s, lw, 1, seed=4242, step=step)
            so, lwo, ao, lro, _, mg = O.cumulative_update(m, so, lwo, CLASSES, J, 1, seed=4242, step=step)
            assert mg == 0 and a == ao
            np.testing.assert_array_equal(s, so)
            assert abs(lw - lwo) <= 1e-9 * abs(lwo)
            assert abs(lr - lro) <= 1e-8 * max(1.0, abs(lro))


def test_kinetic_form_rejects_bad_values():
    from paper_1612_03804_gb300 import sldqmc
    m = O.Model(4, 4, beta=1.0, dtau=0.1)
    with _ctx(m, 10, "fp64", 1) as ctx:
        with pytest.raises(sldqmc.SldqmcError):
            ctx.set_kinetic_form(7)
        ctx.set_kinetic_form("dense")
