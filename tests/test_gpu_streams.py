"""Contexts side by side, through the C ABI.

* Two contexts with different effective models (couplings and classes):
  each context's effective sweeps and features follow its own model,
  bit-exact against the FP64 oracle.
* A tensor-core context created on a non-blocking stream gives the same
  weights, bit for bit, as one on the default stream.
* The exact log weight evaluates its two flavours as one batch [s; -s] at
  eta = +1 on a second context and stream (B = 3), or as two batches on the
  two streams at once (B = 80: 2B above the SM count); the result equals
  2 ld(+1) + 2 ld(-1) + log phi from the single-flavour calls bit for bit,
  equals the sequential evaluation (profiling on), and agrees with the
  oracle within the split-TF32 bound.
* The identity behind that batch: ld(s, eta = -1) = ld(-s, eta = +1) and the
  same sign, bit for bit, in every precision mode (B_tau(-1) for s is
  B_tau(+1) for -s, Eq. 1).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1612_03804_gb300.inputs import batch_uniform, uniform_field

pytestmark = pytest.mark.gpu

CLASSES_A = [[(1, 0, 0), (0, 1, 0)], [(1, 1, 0), (1, -1, 0)], [(2, 0, 0), (0, 2, 0)], [(0, 0, 1)]]
J_A = np.array([-0.05, -0.01, 0.004, -0.45])
CLASSES_B = [[(0, 0, 1)], [(1, 0, 0), (0, 1, 0)]]
J_B = np.array([-0.7, 0.08])


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    from paper_1612_03804_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _ctx(m, n_wrap, prec="fp64", max_batch=2, stream=None):
    from paper_1612_03804_gb300 import sldqmc
    return sldqmc.Context(m.Lx, m.Ly, t=m.t, mu=m.mu, xi=m.xi, beta=m.beta, dtau=m.dtau, n_wrap=n_wrap,
                          J=m.J, h=m.h, prec=prec, max_batch=max_batch, stream=stream)


def test_two_effective_models_stay_apart():
    m = O.Model(6, 5, beta=1.0, dtau=0.1, mu=-0.5)
    s0 = uniform_field(41, m.M, m.N)
    with _ctx(m, 5) as a, _ctx(m, 5) as b:
        a.set_effective_model(CLASSES_A, J_A)
        b.set_effective_model(CLASSES_B, J_B)
        for ctx, classes, J in ((a, CLASSES_A, J_A), (b, CLASSES_B, J_B), (a, CLASSES_A, J_A)):
            sg, na = ctx.eff_sweeps(s0, 2, seed=9, step=4, direction=1)
            so, nao, mg = O.eff_sweeps(m, s0, classes, J, 2, seed=9, step=4, direction=1)
            assert mg == 0
            np.testing.assert_array_equal(sg, so)
            assert na == nao
            np.testing.assert_array_equal(ctx.features(s0[None])[0], O.features(m, s0, classes))


def test_tc_context_on_nonblocking_stream():
    import torch
    m = O.Model(12, 12, beta=1.0, dtau=0.1, mu=-0.5)  # N = 144: two ragged 128-row tiles
    B = 3
    fields = batch_uniform(77, B, m.M, m.N)
    d_s = torch.from_numpy(fields).cuda()
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    with _ctx(m, 5, "3xtf32", B) as c0, _ctx(m, 5, "3xtf32", B, stream=side.cuda_stream) as c1:
        out = []
        for ctx in (c0, c1):
            ld = torch.zeros(B, dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            ctx.weight_batch_dev(d_s, -1, ld)
            ctx.sync()
            out.append(ld.cpu().numpy())
    np.testing.assert_array_equal(out[0], out[1])
    ref = np.array([O.weight(m, f, -1)[0] for f in fields])
    assert np.max(np.abs(out[0] - ref) / np.abs(ref)) < 1e-6


@pytest.mark.parametrize("B", [3, 80])
def test_log_weight_flavours_on_two_streams(B):
    import torch
    m = O.Model(12, 12, beta=1.0, dtau=0.1, mu=-0.5)
    fields = batch_uniform(78, B, m.M, m.N)
    d_s = torch.from_numpy(fields).cuda()
    with _ctx(m, 5, "3xtf32", B) as ctx:
        lw = torch.zeros(B, dtype=torch.float64, device="cuda")
        ldp = torch.zeros(B, dtype=torch.float64, device="cuda")
        ldm = torch.zeros(B, dtype=torch.float64, device="cuda")
        ctx.log_weight_batch_dev(d_s, lw)
        ctx.weight_batch_dev(d_s, 1, ldp)
        ctx.weight_batch_dev(d_s, -1, ldm)
        ctx.sync()
        lw, ldp, ldm = lw.cpu().numpy(), ldp.cpu().numpy(), ldm.cpu().numpy()
        bare = np.array([ctx.log_bare_weight(f) for f in fields])
        np.testing.assert_array_equal(lw, (2.0 * ldp + 2.0 * ldm) + bare)
        # the sequential evaluation (profiling keeps one stream) is the same arithmetic
        ctx.profile(True)
        lw_seq = torch.zeros(B, dtype=torch.float64, device="cuda")
        ctx.log_weight_batch_dev(d_s, lw_seq)
        ctx.profile_read()
        ctx.profile(False)
        ctx.sync()
        np.testing.assert_array_equal(lw, lw_seq.cpu().numpy())
    ref = np.array([O.log_weight_total(m, f) for f in fields[:3]])
    assert np.max(np.abs(lw[:3] - ref) / np.abs(ref)) < 1e-6


@pytest.mark.parametrize("prec", ["fp64", "3xtf32", "bf16x3"])
def test_flavour_is_the_negated_field(prec):
    import torch
    m = O.Model(12, 12, beta=1.0, dtau=0.1, mu=-0.5)
    B = 3
    fields = batch_uniform(79, B, m.M, m.N)
    with _ctx(m, 5, prec, B) as ctx:
        ld = [torch.zeros(B, dtype=torch.float64, device="cuda") for _ in range(2)]
        sg = [torch.zeros(B, dtype=torch.int32, device="cuda") for _ in range(2)]
        ctx.weight_batch_dev(torch.from_numpy(fields).cuda(), -1, ld[0], sg[0])
        ctx.weight_batch_dev(torch.from_numpy(-fields).cuda(), 1, ld[1], sg[1])
        ctx.sync()
        np.testing.assert_array_equal(ld[0].cpu().numpy(), ld[1].cpu().numpy())
        np.testing.assert_array_equal(sg[0].cpu().numpy(), sg[1].cpu().numpy())
    ref = [O.weight(m, f, -1)[0] for f in fields]
    assert np.max(np.abs(ld[0].cpu().numpy() - ref) / np.abs(ref)) < (1e-9 if prec == "fp64" else 1e-6)
