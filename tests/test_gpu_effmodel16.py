"""The paper's 16-coupling effective model ("Results": 2 spatial, 10 temporal,
4 spatio-temporal couplings at L=8, beta=1, dtau=0.05, M=20) on the GPU
against the FP64 CPU oracle: features bit-exact, colour-ordered effective
sweeps bit-exact (both directions), the Eq. 3 fit, and a cumulative-update
chain whose decisions match outside the 1e-8 margin."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1612_03804_gb300 import effmodel as E
from paper_1612_03804_gb300.inputs import domain_field, uniform_field

pytestmark = pytest.mark.gpu

CLS = E.paper_classes()
J16 = np.concatenate([[-0.06, -0.01], -0.4 * 0.6 ** np.arange(10), [-0.01, -0.004, -0.003, -0.001]])


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    from paper_1612_03804_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _ctx(m, max_batch=2, n_wrap=10):
    from paper_1612_03804_gb300 import sldqmc
    c = sldqmc.Context(m.Lx, m.Ly, t=m.t, mu=m.mu, xi=m.xi, beta=m.beta, dtau=m.dtau, n_wrap=n_wrap,
                       J=m.J, h=m.h, max_batch=max_batch)
    c.set_effective_model(CLS, J16)
    return c


@pytest.mark.parametrize("L", [8, 16])
def test_features_16_classes(L):
    m = O.Model(L, L, beta=1.0, dtau=0.05)
    cfgs = np.stack([uniform_field(1, m.M, m.N), domain_field(2, m.M, L, L), np.ones((m.M, m.N), np.int8)])
    with _ctx(m) as ctx:
        F = ctx.features(cfgs)
    for k in range(3):
        np.testing.assert_array_equal(F[k], O.features(m, cfgs[k], CLS))


@pytest.mark.parametrize("L,nsw", [(8, 3), (12, 1)])
def test_eff_sweeps_16_classes_bit_exact(L, nsw):
    m = O.Model(L, L, beta=1.0, dtau=0.05)
    s0 = domain_field(31, m.M, L, L, corr=2)
    with _ctx(m) as ctx:
        for direction in (0, 1):
            sg, na = ctx.eff_sweeps(s0, nsw, seed=5, step=17, direction=direction)
            so, nao, mg = O.eff_sweeps(m, s0, CLS, J16, nsw, seed=5, step=17, direction=direction)
            assert mg == 0
            assert na == nao
            np.testing.assert_array_equal(sg, so)


def test_fit_16_classes_matches_oracle():
    m = O.Model(4, 4, mu=-0.5, xi=1.0, beta=1.0, dtau=0.05, n_wrap=10, J=1.0, h=2.774)
    cfgs = np.stack([domain_field(400 + k, m.M, 4, 4, corr=2) for k in range(60)])
    with _ctx(m, max_batch=8) as ctx:
        J, E0, r2 = ctx.fit_effective_action(cfgs)
    y = np.array([O.log_weight_total(m, c) for c in cfgs])
    F = np.array([O.features(m, c, CLS) for c in cfgs], dtype=np.float64)
    Jo, E0o, r2o = O.fit(F, y, m.beta)
    np.testing.assert_allclose(J, Jo, rtol=1e-6, atol=1e-9)
    assert abs(E0 - E0o) <= 1e-7 * abs(E0o)
    assert abs(r2 - r2o) < 1e-9


def test_cumulative_chain_16_classes():
    m = O.Model(8, 8, mu=-0.5, xi=1.0, beta=1.0, dtau=0.05, n_wrap=10, J=1.0, h=2.774)
    s = uniform_field(78, m.M, m.N)
    s, _, _ = O.eff_sweeps(m, s, CLS, J16, 20, seed=1, step=0, direction=0)
    lw = O.log_weight_total(m, s)
    so, lwo = s.copy(), lw
    n_acc = 0
    with _ctx(m) as ctx:
        for step in range(6):
            s, lw, a, lr = ctx.cumulative_update(s, lw, 2, seed=99, step=step)
            so, lwo, ao, lro, _, mg = O.cumulative_update(m, so, lwo, CLS, J16, 2, seed=99, step=step)
            assert mg == 0 and a == ao
            np.testing.assert_array_equal(s, so)
            assert abs(lw - lwo) <= 1e-9 * abs(lwo)
            n_acc += a
    print(f"16-class chain: {n_acc} of 6 accepted")
