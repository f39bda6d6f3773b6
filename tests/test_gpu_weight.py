"""GPU parity of the exact fermion weight and Green's function (Eq. 1) against
the FP64 CPU oracle, through the C ABI.  Bar (FP64 mode): log|det| to 1e-9
relative, identical sign, G to 1e-9 absolute."""
import functools

import numpy as np
import pytest

from oracle import oracle as O
from paper_1612_03804_gb300.inputs import batch_uniform, domain_field, uniform_field

pytestmark = pytest.mark.gpu

LD_RTOL = 1e-9
G_ATOL = 1e-9


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    from paper_1612_03804_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _ctx(m, n_wrap, max_batch=2, prec="fp64"):
    from paper_1612_03804_gb300 import sldqmc
    return sldqmc.Context(m.Lx, m.Ly, t=m.t, mu=m.mu, xi=m.xi, beta=m.beta, dtau=m.dtau, n_wrap=n_wrap,
                          J=m.J, h=m.h, prec=prec, max_batch=max_batch)


CASES = [
    # Lx, Ly, mu, beta, dtau, n_wrap, field
    (4, 4, 0.0, 2.0, 0.1, 10, "uniform"),     # 4x4, beta=2, dtau=0.1 (the small DQMC case)
    (5, 5, -0.5, 2.0, 0.1, 7, "uniform"),     # ragged N=25, ragged last block 7,7,6
    (6, 7, 0.3, 3.0, 0.1, 5, "domains"),      # N=42, correlated domains
    (12, 12, -0.5, 2.0, 0.1, 10, "uniform"),  # N=144: three GEMM tiles with a ragged tail
    (2, 1, -0.5, 1.0, 0.25, 2, "uniform"),    # 2-site chain
    (1, 1, 0.2, 1.0, 0.25, 3, "uniform"),     # a single site
]


def _field(kind, seed, m):
    if kind == "uniform":
        return uniform_field(seed, m.M, m.N)
    return domain_field(seed, m.M, m.Lx, m.Ly, corr=2)


@pytest.mark.parametrize("Lx,Ly,mu,beta,dtau,nw,kind", CASES)
def test_weight_matches_oracle(Lx, Ly, mu, beta, dtau, nw, kind):
    m = O.Model(Lx, Ly, mu=mu, xi=1.0, beta=beta, dtau=dtau, n_wrap=1)
    with _ctx(m, nw, max_batch=2) as ctx:
        fields = np.stack([_field(kind, 100 + k, m) for k in range(3)])
        for eta in (1, -1):
            ld, sg = ctx.weight_batch(fields, eta)   # 3 configurations through a batch of 2
            for k in range(3):
                ref, rs = O.weight(m, fields[k], eta)
                assert sg[k] == rs
                assert abs(ld[k] - ref) <= LD_RTOL * max(1.0, abs(ref)), (k, eta, ld[k], ref)
        # bilayer weight 2 ld(+1) + 2 ld(-1)
        tot, _ = ctx.weight(fields[0], 0)
        ref = 2 * O.weight(m, fields[0], 1)[0] + 2 * O.weight(m, fields[0], -1)[0]
        assert abs(tot - ref) <= LD_RTOL * max(1.0, abs(ref))


def test_negative_sign_configurations():
    m = O.Model(2, 2, mu=-1.5, xi=6.0, beta=3.0, dtau=0.25, n_wrap=1)
    with _ctx(m, 2, max_batch=4) as ctx:
        fields = np.stack([uniform_field(seed, m.M, m.N) for seed in (4, 28, 0, 1)])
        ld, sg = ctx.weight_batch(fields, 1)
        ref = [O.weight(m, f, 1) for f in fields]
        assert [r[1] for r in ref].count(-1) >= 2
        for k in range(4):
            assert sg[k] == ref[k][1]
            assert abs(ld[k] - ref[k][0]) <= LD_RTOL * abs(ref[k][0])


@pytest.mark.parametrize("tau", [0, 1, 7, 19, 20])
def test_green_matches_oracle(tau):
    m = O.Model(4, 4, mu=0.0, xi=1.0, beta=2.0, dtau=0.1, n_wrap=1)
    s = uniform_field(1000, m.M, m.N)
    with _ctx(m, 10) as ctx:
        for eta in (1, -1):
            G, ld, sg = ctx.green(s, eta, tau)
            ref, rs, Gref = O.weight(m, s, eta, tau0=tau, want_G=True)
            assert sg == rs and abs(ld - ref) <= LD_RTOL * abs(ref)
            np.testing.assert_allclose(G, Gref, rtol=0, atol=G_ATOL)


def test_green_ragged_and_device_batch():
    import torch
    m = O.Model(5, 6, mu=-0.4, xi=1.0, beta=2.0, dtau=0.1, n_wrap=1)
    with _ctx(m, 6, max_batch=2) as ctx:
        fields = batch_uniform(77, 3, m.M, m.N)
        d_s = torch.from_numpy(fields).cuda()
        d_G = torch.zeros((3, m.N, m.N), dtype=torch.float64, device="cuda")
        d_ld = torch.zeros(3, dtype=torch.float64, device="cuda")
        d_sg = torch.zeros(3, dtype=torch.int32, device="cuda")
        ctx.green_batch_dev(d_s, -1, 11, d_G, d_ld, d_sg)
        ctx.sync()
        for k in range(3):
            ref, rs, Gref = O.weight(m, fields[k], -1, tau0=11, want_G=True)
            assert int(d_sg[k]) == rs
            assert abs(float(d_ld[k]) - ref) <= LD_RTOL * abs(ref)
            np.testing.assert_allclose(d_G[k].cpu().numpy(), Gref, rtol=0, atol=G_ATOL)


def test_lu_large_panels_and_interchanges():
    """29x29 (N = 841): the first LU panels have more than 800 rows (the global-memory panel
    kernel) and the last has 9 columns.  A random field against the oracle: the weight (LU
    without a right-hand side; in split-TF32 with digit-split trailing updates) and G (LU with
    one), so that the composed row interchanges of every panel reach the right columns."""
    m = O.Model(29, 29, mu=-0.3, xi=1.0, beta=0.5, dtau=0.1, n_wrap=5)
    s = uniform_field(5, m.M, m.N)
    ref_p, sp = O.weight(m, s, 1)
    ref_m, sm, Gref = O.weight(m, s, -1, tau0=2, want_G=True)
    with _ctx(m, 5, max_batch=1) as ctx:
        ld, sg = ctx.weight(s, 1)
        assert sg == sp and abs(ld - ref_p) <= LD_RTOL * abs(ref_p)
        G, ldg, sgg = ctx.green(s, -1, 2)
        assert sgg == sm and abs(ldg - ref_m) <= LD_RTOL * abs(ref_m)
        np.testing.assert_allclose(G, Gref, rtol=0, atol=G_ATOL)
    with _ctx(m, 5, max_batch=1, prec="3xtf32") as ctx:
        ld, sg = ctx.weight(s, 1)
        assert sg == sp and abs(ld - ref_p) <= 1e-6 * abs(ref_p)


def test_build_K_matches_oracle():
    m = O.Model(6, 5, t=1.3, mu=-0.4, beta=1.0, dtau=0.1)
    with _ctx(m, 10) as ctx:
        K, E, Ei = ctx.build_K()
    np.testing.assert_allclose(K, O.build_K(m), atol=0)
    np.testing.assert_allclose(E, O.build_E(m), atol=1e-14)
    np.testing.assert_allclose(Ei, O.build_E(m, -1.0), atol=1e-14)


def _closed(m, mu_eff):
    kx = 2 * np.pi * np.arange(m.Lx) / m.Lx
    ky = 2 * np.pi * np.arange(m.Ly) / m.Ly
    eps = (-2 * m.t * (np.cos(kx)[None, :] + np.cos(ky)[:, None])).ravel() - mu_eff
    return float(np.sum(np.logaddexp(0.0, -m.beta * eps)))


@pytest.mark.parametrize("L,beta,dtau,mu,nw", [(16, 8.0, 0.05, -0.5, 10), (32, 10.0, 0.05, -0.5, 20)])
def test_full_size_uniform_field_closed_form(L, beta, dtau, mu, nw):
    """Full sizes (16x16, beta=8, M=160; 32x32, beta=10, M=200): s = +-1 everywhere is free fermions at
    mu + eta xi s0, known in closed form."""
    m = O.Model(L, L, mu=mu, xi=1.0, beta=beta, dtau=dtau)
    with _ctx(m, nw, max_batch=1) as ctx:
        for s0 in (1, -1):
            s = np.full((m.M, m.N), s0, dtype=np.int8)
            for eta in (1, -1):
                ld, sg = ctx.weight(s, eta)
                ref = _closed(m, mu + eta * s0)
                assert sg == 1
                assert abs(ld - ref) <= LD_RTOL * abs(ref), (s0, eta, ld, ref)


def test_full_size_particle_hole_and_nwrap():
    """16x16, beta=8, dtau=0.05, random field: ld_eta(mu) - ld_-eta(-mu) = beta N mu + eta dtau xi sum s,
    and the result does not depend on n_wrap."""
    m = O.Model(16, 16, mu=-0.5, xi=1.0, beta=8.0, dtau=0.05)
    s = uniform_field(1001, m.M, m.N)
    res = {}
    for nw in (5, 10, 20):
        for mu in (-0.5, 0.5):
            with _ctx(m.replace(mu=mu), nw, max_batch=1) as ctx:
                for eta in (1, -1):
                    res[(nw, mu, eta)] = ctx.weight(s, eta)
    for nw in (5, 10, 20):
        for eta in (1, -1):
            a, sa = res[(nw, -0.5, eta)]
            b, sb = res[(nw, 0.5, -eta)]
            ref = m.beta * m.N * (-0.5) + eta * m.dtau * m.xi * float(s.sum())
            assert sa == sb
            assert abs((a - b) - ref) <= LD_RTOL * abs(a)
            assert abs(a - res[(10, -0.5, eta)][0]) <= LD_RTOL * abs(a)


def test_device_field_validation():
    import torch
    from paper_1612_03804_gb300 import sldqmc
    m = O.Model(4, 4, beta=1.0, dtau=0.1)
    with _ctx(m, 10) as ctx:
        s = torch.ones((1, m.M, m.N), dtype=torch.int8, device="cuda")
        s[0, 3, 5] = 0
        ld = torch.zeros(1, dtype=torch.float64, device="cuda")
        ctx.weight_batch_dev(s, 1, ld)
        with pytest.raises(sldqmc.SldqmcError) as e:
            ctx.sync()
        assert e.value.status == -1
        # the context stays usable
        s[0, 3, 5] = 1
        ctx.weight_batch_dev(s, 1, ld)
        ctx.sync()
        assert abs(float(ld[0]) - O.weight(m, s[0].cpu().numpy(), 1)[0]) < 1e-9 * abs(float(ld[0]))


def _tall_case():
    m = O.Model(36, 36, mu=-0.3, xi=1.0, beta=0.5, dtau=0.1, n_wrap=5)
    return m, domain_field(7, m.M, 36, 36, corr=3)


@functools.lru_cache(maxsize=1)
def _tall_ref():
    m, s = _tall_case()
    return O.weight(m, s, 1)


@pytest.mark.parametrize("prec", ["fp64", "3xtf32"])
def test_lu_tournament_pivoting_tall_panels(prec):
    """36x36 (N = 1296): the first 16 LU panels are taller than 800 rows and take the
    tournament-pivoting path (row blocks nominate pivots, one CTA chooses), the rest
    the shared-memory panel.  Weight (LU without a right-hand side; in split-TF32 with
    digit-split trailing updates) and, in FP64, G (LU with one) against the oracle."""
    m, s = _tall_case()
    bound = LD_RTOL if prec == "fp64" else 1e-6
    with _ctx(m, 5, max_batch=1, prec=prec) as ctx:
        ref_p, sp = _tall_ref()
        ld, sg = ctx.weight(s, 1)
        assert sg == sp and abs(ld - ref_p) <= bound * abs(ref_p), (ld, ref_p)
        if prec == "fp64":
            ref_m, sm, Gref = O.weight(m, s, -1, tau0=3, want_G=True)
            G, ldg, sgg = ctx.green(s, -1, 3)
            assert sgg == sm and abs(ldg - ref_m) <= LD_RTOL * abs(ref_m)
            np.testing.assert_allclose(G, Gref, rtol=0, atol=G_ATOL)


@pytest.mark.parametrize("prec", ["fp64", "3xtf32"])
def test_lattice_between_2048_and_4096_sites(prec):
    """48x48 (N = 2304): the pivot sort pads to 4096 columns, whose keys take exactly the
    default 48 KB of dynamic shared memory; the LU has tournament panels.  Uniform fields
    against the closed form, a random field against the particle-hole identity
    ld_eta(s; mu) - ld_-eta(s; -mu) = beta N mu + eta dtau xi sum s."""
    m = O.Model(48, 48, mu=-0.5, xi=1.0, beta=0.5, dtau=0.1)
    bound = LD_RTOL if prec == "fp64" else 1e-6
    with _ctx(m, 5, max_batch=1, prec=prec) as ctx:
        s = np.ones((m.M, m.N), dtype=np.int8)
        ld, sg = ctx.weight(s, -1)
        ref = _closed(m, m.mu - 1.0)
        assert sg == 1 and abs(ld - ref) <= bound * abs(ref), (ld, ref)
        r = uniform_field(48, m.M, m.N)
        ld_a, _ = ctx.weight(r, 1)
    with _ctx(m.replace(mu=0.5), 5, max_batch=1, prec=prec) as ctx:
        ld_b, _ = ctx.weight(r, -1)
    rhs = m.beta * m.N * m.mu + m.dtau * m.xi * float(r.astype(np.int64).sum())
    assert abs((ld_a - ld_b) - rhs) <= 2 * bound * max(abs(ld_a), abs(ld_b)), (ld_a - ld_b, rhs)
