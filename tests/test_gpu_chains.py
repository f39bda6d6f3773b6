"""Whole-chain GPU checks: the 4x4 local-DQMC run of 1000 sweeps against the
oracle, exact enumeration of a 2-site x 4-slice system with thousands of
batched GPU chains (local DQMC and cumulative updates with a poor H_eff),
checkpoint/resume of the cumulative chain, and the bounded-wait failure path."""
import numpy as np
import pytest
from scipy import stats

from oracle import oracle as O
from paper_1612_03804_gb300.inputs import uniform_field

pytestmark = pytest.mark.gpu

CLASSES = [[(1, 0, 0), (0, 1, 0)], [(1, 1, 0), (1, -1, 0)], [(2, 0, 0), (0, 2, 0)], [(0, 0, 1)]]
J_EFF = np.array([-0.05, -0.01, 0.004, -0.45])


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    from paper_1612_03804_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _ctx(m, n_wrap, max_batch=1):
    from paper_1612_03804_gb300 import sldqmc
    return sldqmc.Context(m.Lx, m.Ly, t=m.t, mu=m.mu, xi=m.xi, beta=m.beta, dtau=m.dtau, n_wrap=n_wrap,
                          J=m.J, h=m.h, max_batch=max_batch)


def test_small_dqmc_run_1000_sweeps():
    """4x4, mu=0, xi=1, beta=2, dtau=0.1, n_wrap=10: weight, G, then 1000 local sweeps -- the GPU
    chain equals the oracle chain."""
    m = O.Model(4, 4, t=1.0, mu=0.0, xi=1.0, beta=2.0, dtau=0.1, n_wrap=10, J=1.0, h=2.774)
    s = uniform_field(1001, m.M, m.N)
    with _ctx(m, 10) as ctx:
        for eta in (1, -1):
            ld, sg = ctx.weight(s, eta)
            ref, rs, Gref = O.weight(m, s, eta, want_G=True)
            assert sg == rs and abs(ld - ref) <= 1e-9 * abs(ref)
            G, _, _ = ctx.green(s, eta, 0)
            assert np.abs(G - Gref).max() < 1e-9
        sg, stg = ctx.local_sweep(s, seed=2024, sweep0=0, n_sweeps=1000)
    so, sto = O.local_sweep(m, s, seed=2024, sweep0=0, n_sweeps=1000)
    assert sto["margin_events"] == 0
    assert stg["accepted"] == sto["accepted"]
    np.testing.assert_array_equal(sg, so)
    assert stg["max_drift"] < 1e-8


ENUM = dict(Lx=2, Ly=1, t=1.0, mu=-0.5, xi=1.0, beta=1.0, dtau=0.25, n_wrap=2, J=1.0, h=1.0)


def _all_configs(M, N):
    n = M * N
    idx = np.arange(2 ** n)
    bits = (idx[:, None] >> np.arange(n)[None, :]) & 1
    return (2 * bits - 1).astype(np.int8).reshape(-1, M, N)


def _codes(S):
    b = (S.reshape(S.shape[0], -1) > 0).astype(np.int64)
    return (b << np.arange(b.shape[1])[None, :]).sum(axis=1)


def _chi2_p(counts, probs, min_expected=5.0):
    exp = probs * counts.sum()
    small = exp < min_expected
    c = np.append(counts[~small], counts[small].sum())
    e = np.append(exp[~small], exp[small].sum())
    return stats.chisquare(c, e).pvalue


@pytest.fixture(scope="module")
def enum_model():
    m = O.Model(**ENUM)
    cfgs = _all_configs(m.M, m.N)
    lw = np.array([O.log_weight_total(m, c) for c in cfgs])
    p = np.exp(lw - lw.max())
    return m, cfgs, lw, p / p.sum()


def test_enumeration_gpu_local_chains(enum_model):
    import torch
    m, cfgs, lw, p = enum_model
    B = 16384
    rng = np.random.Generator(np.random.PCG64(77))
    start = rng.choice(len(cfgs), size=B, p=p)
    with _ctx(m, 2, max_batch=B) as ctx:
        d_s = torch.from_numpy(np.ascontiguousarray(cfgs[start])).cuda()
        st = ctx.local_sweep_batch_dev(d_s, 31337, 0, 2)
        out = d_s.cpu().numpy()
    codes = _codes(out)
    assert np.mean(codes != start) > 0.3
    assert sum(x["margin_events"] for x in st) == 0
    assert _chi2_p(np.bincount(codes, minlength=len(cfgs)).astype(float), p) > 0.01


def test_enumeration_gpu_cumulative_chains_with_poor_model(enum_model):
    import torch
    m, cfgs, lw, p = enum_model
    B = 16384
    rng = np.random.Generator(np.random.PCG64(78))
    start = rng.choice(len(cfgs), size=B, p=p)
    with _ctx(m, 2, max_batch=B) as ctx:
        ctx.set_effective_model([[(1, 0, 0)], [(0, 0, 1)]], np.array([-0.2, -0.15]))
        d_s = torch.from_numpy(np.ascontiguousarray(cfgs[start])).cuda()
        d_lw = torch.from_numpy(lw[start].copy()).cuda()
        acc = torch.zeros(B, dtype=torch.int32, device="cuda")
        ctx.cumulative_batch_dev(d_s, d_lw, 1, 4242, 0, 1, acc)
        ctx.sync()
        out = d_s.cpu().numpy()
        lw_out = d_lw.cpu().numpy()
        na = int(acc.sum().item())
    codes = _codes(out)
    assert 0.05 * B < na < 0.98 * B
    np.testing.assert_allclose(lw_out, lw[codes], rtol=0, atol=1e-9)
    assert _chi2_p(np.bincount(codes, minlength=len(cfgs)).astype(float), p) > 0.01


def test_cumulative_checkpoint_resume_is_bit_identical():
    import torch
    m = O.Model(4, 4, mu=0.0, xi=1.0, beta=2.0, dtau=0.1, n_wrap=10, J=1.0, h=2.774)
    from paper_1612_03804_gb300.inputs import batch_uniform
    fields = batch_uniform(5, 4, m.M, m.N)
    with _ctx(m, 10, max_batch=4) as ctx:
        ctx.set_effective_model(CLASSES, J_EFF)
        a = torch.from_numpy(fields).cuda()
        la = torch.zeros(4, dtype=torch.float64, device="cuda")
        ctx.log_weight_batch_dev(a, la)
        acc = torch.zeros(4, dtype=torch.int32, device="cuda")
        ctx.cumulative_batch_dev(a, la, 1, 99, 0, 6, acc)
        # checkpoint after 3 steps: (s, log w, seed, step) to host and back
        b = torch.from_numpy(fields).cuda()
        lb = torch.zeros(4, dtype=torch.float64, device="cuda")
        ctx.log_weight_batch_dev(b, lb)
        ctx.cumulative_batch_dev(b, lb, 1, 99, 0, 3, acc)
        ckpt = (b.cpu().numpy().copy(), lb.cpu().numpy().copy())
        b2 = torch.from_numpy(ckpt[0]).cuda()
        lb2 = torch.from_numpy(ckpt[1]).cuda()
        ctx.cumulative_batch_dev(b2, lb2, 1, 99, 3, 3, acc)
        ctx.sync()
        np.testing.assert_array_equal(a.cpu().numpy(), b2.cpu().numpy())
        np.testing.assert_array_equal(la.cpu().numpy(), lb2.cpu().numpy())


def test_bounded_wait_times_out_and_context_survives():
    from paper_1612_03804_gb300 import sldqmc
    m = O.Model(4, 4, beta=1.0, dtau=0.1)
    with _ctx(m, 10) as ctx:
        ctx.wait_selftest(1 << 12)
        with pytest.raises(sldqmc.SldqmcError) as e:
            ctx.sync()
        assert e.value.status == -5
        s = uniform_field(3, m.M, m.N)
        ld, sg = ctx.weight(s, 1)
        ref, rs = O.weight(m, s, 1)
        assert sg == rs and abs(ld - ref) <= 1e-9 * abs(ref)
