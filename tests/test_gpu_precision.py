"""Mixed-precision slice products (3xTF32 and BF16 on tcgen05 tensor cores,
FP64 stabilisation and finalisation) against the parity-checked FP64 GPU
path, the closed form and the oracle.  The error is stated per mode:
3xTF32 must stay within 1e-6 relative in log|det| (the reduced-precision
target); BF16 is bounded at 1e-2 relative and reported."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1612_03804_gb300.inputs import batch_uniform, uniform_field

pytestmark = pytest.mark.gpu

BOUND = {"3xtf32": 1e-6, "bf16": 1e-2, "bf16x3": 1e-6}
G_BOUND = {"3xtf32": 1e-5, "bf16": 5e-2, "bf16x3": 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    from paper_1612_03804_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _ctx(L, beta, dtau, mu, nw, prec, max_batch=2):
    from paper_1612_03804_gb300 import sldqmc
    return sldqmc.Context(L, L, mu=mu, xi=1.0, beta=beta, dtau=dtau, n_wrap=nw, prec=prec, max_batch=max_batch)


@pytest.mark.parametrize("prec", ["3xtf32", "bf16", "bf16x3"])
def test_single_product_block_against_oracle(prec):
    """n_wrap = 1: every block is one tensor-core product; 12x12 has a ragged 128-tile."""
    m = O.Model(12, 12, mu=-0.5, xi=1.0, beta=1.0, dtau=0.1, n_wrap=1)
    s = uniform_field(3, m.M, m.N)
    with _ctx(12, 1.0, 0.1, -0.5, 1, prec) as ctx:
        for eta in (1, -1):
            ld, sg = ctx.weight(s, eta)
            ref, rs = O.weight(m, s, eta)
            assert sg == rs
            assert abs(ld - ref) <= BOUND[prec] * abs(ref), (prec, eta, ld, ref)


@pytest.mark.parametrize("prec", ["3xtf32", "bf16", "bf16x3"])
@pytest.mark.parametrize("L,beta,dtau,nw", [(16, 8.0, 0.05, 10), (12, 4.0, 0.05, 20)])
def test_against_fp64_path(prec, L, beta, dtau, nw):
    fields = batch_uniform(11, 3, int(round(beta / dtau)), L * L)
    with _ctx(L, beta, dtau, -0.5, nw, "fp64", 3) as c64, _ctx(L, beta, dtau, -0.5, nw, prec, 3) as cm:
        for eta in (1, -1):
            ref, rs = c64.weight_batch(fields, eta)
            ld, sg = cm.weight_batch(fields, eta)
            np.testing.assert_array_equal(sg, rs)
            rel = np.abs(ld - ref) / np.abs(ref)
            print(f"{prec} L={L} eta={eta}: max rel log-det error {rel.max():.2e}")
            assert rel.max() <= BOUND[prec]
        G64, _, _ = c64.green(fields[0], -1, 5)
        Gm, _, _ = cm.green(fields[0], -1, 5)
        err = np.abs(Gm - G64).max()
        print(f"{prec} L={L}: max|dG| {err:.2e}")
        assert err <= G_BOUND[prec]


@pytest.mark.parametrize("prec", ["3xtf32", "bf16", "bf16x3"])
def test_uniform_field_closed_form(prec):
    L, beta, dtau, mu = 16, 8.0, 0.05, -0.5
    M = int(round(beta / dtau))
    kx = 2 * np.pi * np.arange(L) / L
    with _ctx(L, beta, dtau, mu, 10, prec, 1) as ctx:
        for s0 in (1, -1):
            s = np.full((M, L * L), s0, dtype=np.int8)
            ld, sg = ctx.weight(s, -1)
            eps = (-2 * (np.cos(kx)[None, :] + np.cos(kx)[:, None])).ravel() - (mu - s0)
            ref = float(np.sum(np.logaddexp(0.0, -beta * eps)))
            assert sg == 1
            assert abs(ld - ref) <= BOUND[prec] * abs(ref)
