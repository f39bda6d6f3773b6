"""The headline configuration, 100x100 (N = 10^4), beta = 10, dtau = 0.1 (M = 100),
n_wrap = 10, mu = -0.5, xi = 1, split-TF32 slice products (dense exp(-dtau K) as the
benchmark runs them, and the separable form) with the FP64-accurate digit-split
stabilisation, where the oracle's dense FP64 chain (about 10^14 flops per weight) is out of
reach.  Properties that hold at any size, through the C ABI:

  - the uniform field s = +1 is free fermions at mu + eta xi (B_tau of Eq. 1 with a
    constant field): log|det| within 1e-6 relative of sum_k log(1 + e^{-beta (eps_k -
    mu_eff)}), eps_k = -2t (cos kx + cos ky), and every element of G within 1e-5 of its
    translation-invariant closed form, both flavours;
  - a seeded random field obeys the particle-hole identity of the bipartite lattice,
    ld_eta(s; mu) - ld_-eta(s; -mu) = beta N mu + eta dtau xi sum s (pinned on the oracle
    at small sizes), within the two sides' 1e-6 bounds, both flavours.
"""
import numpy as np
import pytest

from paper_1612_03804_gb300.inputs import uniform_field

pytestmark = pytest.mark.gpu

L, BETA, DTAU, MU, XI, NW = 100, 10.0, 0.1, -0.5, 1.0, 10
M = int(round(BETA / DTAU))
N = L * L
LD_RTOL = 1e-6
G_ATOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    from paper_1612_03804_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _ctx(mu, kinetic):
    from paper_1612_03804_gb300 import sldqmc
    c = sldqmc.Context(L, L, mu=mu, xi=XI, beta=BETA, dtau=DTAU, n_wrap=NW, prec="3xtf32", max_batch=1)
    c.set_kinetic_form(kinetic)
    return c


def _closed(mu_eff):
    """log det(1 + e^{-beta K'}) and g(dy, dx) with G_ij = g(r_i - r_j) for K' = -tA - mu_eff."""
    k = 2 * np.pi * np.arange(L) / L
    eps = -2.0 * (np.cos(k)[None, :] + np.cos(k)[:, None]) - mu_eff
    ld = float(np.sum(np.logaddexp(0.0, -BETA * eps)))
    occ = 1.0 / (1.0 + np.exp(np.clip(-BETA * eps, -700, 700)))
    return ld, np.real(np.fft.ifft2(occ))


@pytest.mark.parametrize("kinetic", ["dense", "separable"])
def test_uniform_field_closed_form(kinetic):
    import torch
    u = torch.ones((1, M, N), dtype=torch.int8, device="cuda")
    idx = torch.arange(N, device="cuda")
    x, y = idx % L, idx // L
    with _ctx(MU, kinetic) as ctx:
        for eta in (1, -1):
            ld = torch.zeros(1, dtype=torch.float64, device="cuda")
            sg = torch.zeros(1, dtype=torch.int32, device="cuda")
            ctx.weight_batch_dev(u, eta, ld, sg)
            G = torch.zeros((1, N, N), dtype=torch.float64, device="cuda")
            ctx.green_batch_dev(u, eta, 0, G)
            ctx.sync()
            ref, g = _closed(MU + eta * XI)
            rel = abs(ld.item() - ref) / abs(ref)
            g = torch.from_numpy(g).cuda()
            dG = 0.0
            for r0 in range(0, N, 500):
                rows = idx[r0:r0 + 500]
                gref = g[(y[rows, None] - y[None, :]) % L, (x[rows, None] - x[None, :]) % L]
                dG = max(dG, float((G[0, r0:r0 + 500] - gref).abs().max()))
            print(f"100x100 uniform field, {kinetic}, eta={eta}: log-det rel err {rel:.2e}, max|dG| {dG:.2e}")
            assert sg.item() == 1
            assert rel <= LD_RTOL
            assert dG <= G_ATOL
            del G
            torch.cuda.empty_cache()


@pytest.mark.parametrize("kinetic", ["dense", "separable"])
def test_random_field_particle_hole(kinetic):
    import torch
    s = uniform_field(4242, M, N)
    d_s = torch.from_numpy(s[None]).cuda()
    out = {}
    for mu in (MU, -MU):
        with _ctx(mu, kinetic) as ctx:
            for eta in (1, -1):
                ld = torch.zeros(1, dtype=torch.float64, device="cuda")
                sg = torch.zeros(1, dtype=torch.int32, device="cuda")
                ctx.weight_batch_dev(d_s, eta, ld, sg)
                ctx.sync()
                out[(mu, eta)] = (ld.item(), sg.item())
    for eta in (1, -1):
        a, sa = out[(MU, eta)]
        b, sb = out[(-MU, -eta)]
        ref = BETA * N * MU + eta * DTAU * XI * float(s.astype(np.int64).sum())
        print(f"100x100 random field, {kinetic}, eta={eta}: ld(mu) - ld(-mu) - ref = {(a - b) - ref:.3e} "
              f"(bound {LD_RTOL * (abs(a) + abs(b)):.3e})")
        assert sa == sb
        assert abs((a - b) - ref) <= LD_RTOL * (abs(a) + abs(b))
