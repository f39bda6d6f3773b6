"""GPU parity of the Monte Carlo paths against the FP64 CPU oracle, through
the C ABI: local DQMC sweeps, effective-model sweeps, features, the Eq. 3
fit and the Eq. 4 cumulative update.  Integer work (configurations, accept
counts) is bit-exact unless a decision fell within the 1e-8 margin."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1612_03804_gb300.inputs import batch_uniform, domain_field, uniform_field

pytestmark = pytest.mark.gpu

CLASSES = [[(1, 0, 0), (0, 1, 0)], [(1, 1, 0), (1, -1, 0)], [(2, 0, 0), (0, 2, 0)], [(0, 0, 1)]]
J_EFF = np.array([-0.05, -0.01, 0.004, -0.45])


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    from paper_1612_03804_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _ctx(m, n_wrap, max_batch=2):
    from paper_1612_03804_gb300 import sldqmc
    return sldqmc.Context(m.Lx, m.Ly, t=m.t, mu=m.mu, xi=m.xi, beta=m.beta, dtau=m.dtau, n_wrap=n_wrap,
                          J=m.J, h=m.h, max_batch=max_batch)


def test_log_bare_weight():
    m = O.Model(5, 4, beta=1.0, dtau=0.1, J=0.7, h=2.774)
    s = uniform_field(5, m.M, m.N)
    with _ctx(m, 10) as ctx:
        assert abs(ctx.log_bare_weight(s) - O.log_bare_weight(m, s)) < 1e-12


@pytest.mark.parametrize("Lx,Ly,beta,dtau,nw,mu,h", [(4, 4, 2.0, 0.1, 10, 0.0, 2.774),
                                                      (3, 3, 1.0, 0.1, 3, -0.5, 1.0),
                                                      (2, 1, 1.0, 0.25, 2, -0.5, 1.0)])
def test_local_sweep_trajectory(Lx, Ly, beta, dtau, nw, mu, h):
    """Same seed, same flips: the GPU chain follows the oracle chain exactly."""
    m = O.Model(Lx, Ly, mu=mu, xi=1.0, beta=beta, dtau=dtau, n_wrap=nw, J=1.0, h=h)
    s0 = uniform_field(2024, m.M, m.N)
    with _ctx(m, nw) as ctx:
        sg, stg = ctx.local_sweep(s0, seed=99, sweep0=0, n_sweeps=3)
    so, sto = O.local_sweep(m, s0, seed=99, sweep0=0, n_sweeps=3)
    assert sto["margin_events"] == 0 and stg["margin_events"] == 0
    assert stg["accepted"] == sto["accepted"]
    assert stg["proposed"] == sto["proposed"] == 3 * m.N * m.M
    np.testing.assert_array_equal(sg, so)
    assert stg["max_drift"] < 1e-8


def test_local_sweep_batched_chains():
    import torch
    m = O.Model(4, 4, mu=0.0, xi=1.0, beta=2.0, dtau=0.1, n_wrap=10, J=1.0, h=2.774)
    fields = batch_uniform(7, 3, m.M, m.N)
    seed = 12345
    with _ctx(m, 10, max_batch=3) as ctx:
        d_s = torch.from_numpy(fields).cuda()
        st = ctx.local_sweep_batch_dev(d_s, seed, 5, 2)
        out = d_s.cpu().numpy()
    for b in range(3):
        so, sto = O.local_sweep(m, fields[b], seed=seed + (b << 32), sweep0=5, n_sweeps=2)
        assert sto["margin_events"] == 0
        np.testing.assert_array_equal(out[b], so)
        assert st[b]["accepted"] == sto["accepted"]


@pytest.mark.parametrize("L,beta,dtau,nsw", [(4, 2.0, 0.1, 3), (5, 1.0, 0.1, 2), (16, 8.0, 0.05, 1)])
def test_eff_sweeps_bit_exact(L, beta, dtau, nsw):
    m = O.Model(L, L, beta=beta, dtau=dtau)
    s0 = domain_field(31, m.M, L, L, corr=2)
    with _ctx(m, 10) as ctx:
        ctx.set_effective_model(CLASSES, J_EFF)
        for direction in (0, 1):
            sg, na = ctx.eff_sweeps(s0, nsw, seed=5, step=17, direction=direction)
            so, nao, mg = O.eff_sweeps(m, s0, CLASSES, J_EFF, nsw, seed=5, step=17, direction=direction)
            assert mg == 0
            assert na == nao
            np.testing.assert_array_equal(sg, so)


def test_features_exact():
    m = O.Model(16, 16, beta=8.0, dtau=0.05)
    cfgs = np.stack([uniform_field(1, m.M, m.N), domain_field(2, m.M, 16, 16), np.ones((m.M, m.N), np.int8)])
    with _ctx(m, 10) as ctx:
        ctx.set_effective_model(CLASSES, J_EFF)
        F = ctx.features(cfgs)
    for k in range(3):
        np.testing.assert_array_equal(F[k], O.features(m, cfgs[k], CLASSES))


def test_fit_matches_oracle():
    m = O.Model(4, 4, mu=0.0, xi=1.0, beta=2.0, dtau=0.1, n_wrap=10)
    cfgs = np.stack([domain_field(300 + k, m.M, 4, 4, corr=2) for k in range(40)])
    with _ctx(m, 10, max_batch=8) as ctx:
        ctx.set_effective_model(CLASSES, J_EFF)
        J, E0, r2 = ctx.fit_effective_action(cfgs)          # ln omega evaluated on the GPU
    y = np.array([O.log_weight_total(m, c) for c in cfgs])
    F = np.array([O.features(m, c, CLASSES) for c in cfgs], dtype=np.float64)
    Jo, E0o, r2o = O.fit(F, y, m.beta)
    np.testing.assert_allclose(J, Jo, rtol=1e-7, atol=1e-10)
    assert abs(E0 - E0o) <= 1e-7 * abs(E0o)
    assert abs(r2 - r2o) < 1e-9


def test_cumulative_update_chain_matches_oracle():
    m = O.Model(4, 4, mu=0.0, xi=1.0, beta=2.0, dtau=0.1, n_wrap=10, J=1.0, h=2.774)
    s = uniform_field(77, m.M, m.N)
    lw = O.log_weight_total(m, s)
    so, lwo = s.copy(), lw
    acc_g = acc_o = 0
    with _ctx(m, 10) as ctx:
        ctx.set_effective_model(CLASSES, J_EFF)
        for step in range(6):
            s, lw, a, lr = ctx.cumulative_update(s, lw, 1, seed=4242, step=step)
            so, lwo, ao, lro, _, mg = O.cumulative_update(m, so, lwo, CLASSES, J_EFF, 1, seed=4242, step=step)
            assert mg == 0
            assert a == ao
            np.testing.assert_array_equal(s, so)
            assert abs(lw - lwo) <= 1e-9 * abs(lwo)
            assert abs(lr - lro) <= 1e-8 * max(1.0, abs(lro))
            acc_g += a
            acc_o += ao
    assert acc_g == acc_o


def test_cumulative_batch_dev_equals_single_chains():
    import torch
    m = O.Model(4, 4, mu=0.0, xi=1.0, beta=2.0, dtau=0.1, n_wrap=10, J=1.0, h=2.774)
    fields = batch_uniform(9, 3, m.M, m.N)
    seed = 777
    with _ctx(m, 10, max_batch=3) as ctx:
        ctx.set_effective_model(CLASSES, J_EFF)
        d_s = torch.from_numpy(fields).cuda()
        d_lw = torch.zeros(3, dtype=torch.float64, device="cuda")
        ctx.log_weight_batch_dev(d_s, d_lw)
        d_acc = torch.zeros(3, dtype=torch.int32, device="cuda")
        ctx.cumulative_batch_dev(d_s, d_lw, 1, seed, 0, 4, d_acc)
        ctx.sync()
        out = d_s.cpu().numpy()
        lw_out = d_lw.cpu().numpy()
        acc = d_acc.cpu().numpy()
    for b in range(3):
        s, lw = fields[b].copy(), O.log_weight_total(m, fields[b])
        na = 0
        for step in range(4):
            s, lw, a, _, _, mg = O.cumulative_update(m, s, lw, CLASSES, J_EFF, 1, seed=seed + (b << 32), step=step)
            assert mg == 0
            na += a
        np.testing.assert_array_equal(out[b], s)
        assert acc[b] == na
        assert abs(lw_out[b] - lw) <= 1e-9 * abs(lw)


def test_eff_sweeps_batch_dev_matches_oracle():
    import torch
    m = O.Model(6, 4, beta=2.0, dtau=0.1)
    fields = batch_uniform(21, 3, m.M, m.N)
    seed, step = 31, 5
    with _ctx(m, 10, max_batch=3) as ctx:
        ctx.set_effective_model(CLASSES, J_EFF)
        d_s = torch.from_numpy(fields).cuda()
        d_acc = torch.zeros(3, dtype=torch.int64, device="cuda")
        ctx.eff_sweeps_batch_dev(d_s, 2, seed, step, -1, d_acc)
        ctx.sync()
        out = d_s.cpu().numpy()
        acc = d_acc.cpu().numpy()
    for b in range(3):
        key = seed + (b << 32)
        direction = int(O.lib().or_random_word(key, 0, 0, step, 3)) & 1
        so, na, mg = O.eff_sweeps(m, fields[b], CLASSES, J_EFF, 2, seed=key, step=step, direction=direction)
        assert mg == 0
        np.testing.assert_array_equal(out[b], so)
        assert acc[b] == na
