"""Delayed (rank-k) local updates against the FP64 CPU oracle: the same
flips and decisions as the immediate rank-1 updates ("Basics of DQMC"),
bit-exact configurations and accept counts; the Green's function is
carried as G0 - U V inside a block of k sites and corrected by one batched
GEMM per flavour after it."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1612_03804_gb300.inputs import batch_uniform

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    from paper_1612_03804_gb300 import build
    build.build()
    torch.cuda.set_device(0)


@pytest.mark.parametrize("L,beta,dtau,nw,k,sweeps", [
    (4, 2.0, 0.1, 10, 4, 3),      # four blocks per slice
    (4, 2.0, 0.1, 10, 32, 3),     # one block of 16 sites
    (8, 8.0, 0.05, 10, 32, 1),    # the training lattice: two blocks per slice
    (12, 1.0, 0.05, 10, 32, 1),   # N = 144: four blocks and a ragged one of 16
    (16, 2.0, 0.05, 10, 32, 1),   # N = 256
])
def test_delayed_trajectory_matches_oracle(L, beta, dtau, nw, k, sweeps):
    import torch
    from paper_1612_03804_gb300 import sldqmc
    m = O.Model(L, L, mu=-0.5, xi=1.0, beta=beta, dtau=dtau, n_wrap=nw, J=1.0, h=2.774)
    B, seed = 2, 31337
    fields = batch_uniform(2600 + L, B, m.M, m.N)
    with sldqmc.Context(L, L, mu=-0.5, xi=1.0, beta=beta, dtau=dtau, n_wrap=nw, J=1.0, h=2.774,
                        max_batch=B) as ctx:
        ctx.set_local_update_rank(k)
        d_s = torch.from_numpy(fields).cuda()
        st = ctx.local_sweep_batch_dev(d_s, seed, 0, sweeps)
        out = d_s.cpu().numpy()
    for b in range(B):
        so, sto = O.local_sweep(m, fields[b], seed=seed + (b << 32), sweep0=0, n_sweeps=sweeps)
        assert sto["margin_events"] == 0 and st[b]["margin_events"] == 0
        assert st[b]["proposed"] == sto["proposed"]
        assert st[b]["accepted"] == sto["accepted"]
        np.testing.assert_array_equal(out[b], so)
        assert st[b]["max_drift"] < 1e-8


def test_delayed_equals_immediate_on_the_gpu():
    """16 chains at 16x16: rank 1 and rank 32 give the same configurations."""
    import torch
    from paper_1612_03804_gb300 import sldqmc
    B = 16
    fields = batch_uniform(2700, B, 40, 256)
    outs = []
    for k in (1, 32):
        with sldqmc.Context(16, 16, mu=-0.5, xi=1.0, beta=2.0, dtau=0.05, n_wrap=10, max_batch=B) as ctx:
            ctx.set_local_update_rank(k)
            d_s = torch.from_numpy(fields).cuda()
            st = ctx.local_sweep_batch_dev(d_s, 99, 0, 2)
            outs.append((d_s.cpu().numpy(), [x["accepted"] for x in st]))
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    assert outs[0][1] == outs[1][1]


def test_local_update_rank_rejects_bad_values():
    from paper_1612_03804_gb300 import sldqmc
    with sldqmc.Context(4, 4, beta=1.0, dtau=0.1, n_wrap=10) as ctx:
        for k in (0, 33):
            with pytest.raises(sldqmc.SldqmcError):
                ctx.set_local_update_rank(k)
