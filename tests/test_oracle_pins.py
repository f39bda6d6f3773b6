"""Pins of the FP64 CPU oracle against facts fixed by the paper and by mathematics.

None of these re-type the oracle's own formula: each compares it with a closed
form, a library routine (scipy expm, numpy slogdet/lstsq, mpmath at 40
digits), an exact identity, published known-answer vectors, brute force or
exact enumeration.
"""
import math
import os

import mpmath
import numpy as np
import pytest
import scipy.linalg as sla
from scipy import stats

from oracle import oracle as O
from paper_1612_03804_gb300.inputs import domain_field, uniform_field

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------- RNG
def test_philox_known_answers():
    """Philox-4x32-10 against the published known-answer vectors (Salmon et al. SC'11)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = O.philox(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_uniform_is_top_53_bits():
    seed = 0x0123456789ABCDEF
    o = O.philox([5, 6, 7, 1], [seed & 0xFFFFFFFF, seed >> 32])
    w = (int(o[1]) << 32) | int(o[0])
    assert O.uniform(seed, 5, 6, 7, 1) == (w >> 11) / 2.0 ** 53


# ------------------------------------------------------------ hopping / E
@pytest.mark.parametrize("Lx,Ly", [(4, 4), (3, 5), (2, 1), (2, 2), (6, 1), (1, 1)])
def test_E_matches_expm(Lx, Ly):
    """E = exp(-dtau K) by Fourier sums vs scipy's Pade expm of K (slice matrix of Eq. 1)."""
    m = O.Model(Lx, Ly, t=1.3, mu=-0.4, beta=1.0, dtau=0.1)
    K = O.build_K(m)
    assert np.allclose(K, K.T)
    E = O.build_E(m)
    Ei = O.build_E(m, -1.0)
    np.testing.assert_allclose(E, sla.expm(-m.dtau * K), rtol=0, atol=1e-14)
    np.testing.assert_allclose(E @ Ei, np.eye(m.N), rtol=0, atol=1e-13)


def test_K_spectrum_is_tight_binding():
    """Eigenvalues of K are -2t(cos kx + cos ky) - mu on the periodic lattice (Eq. 6)."""
    m = O.Model(4, 6, t=0.7, mu=0.3, beta=1.0, dtau=0.1)
    ev = np.sort(np.linalg.eigvalsh(O.build_K(m)))
    kx = 2 * np.pi * np.arange(4) / 4
    ky = 2 * np.pi * np.arange(6) / 6
    ref = np.sort((-2 * 0.7 * (np.cos(kx)[None, :] + np.cos(ky)[:, None]) - 0.3).ravel())
    np.testing.assert_allclose(ev, ref, atol=1e-13)


# ------------------------------------------------------- closed-form weights
def _free_closed_form(m, mu_eff):
    kx = 2 * np.pi * np.arange(m.Lx) / m.Lx
    ky = 2 * np.pi * np.arange(m.Ly) / m.Ly
    ex = -2 * m.t * np.cos(kx) if m.Lx > 1 else np.zeros(1)
    ey = -2 * m.t * np.cos(ky) if m.Ly > 1 else np.zeros(1)
    eps = (ex[None, :] + ey[:, None]).ravel() - mu_eff
    return float(np.sum(np.logaddexp(0.0, -m.beta * eps)))


@pytest.mark.parametrize("L,beta,mu", [(4, 2.0, 0.0), (4, 10.0, -0.5), (6, 8.0, 0.3), (8, 4.0, -1.0)])
def test_free_fermion_product_formula(L, beta, mu):
    """xi = 0: det(1 + e^{-beta K}) = prod_k (1 + e^{-beta(eps_k - mu)}), G the Fermi function."""
    m = O.Model(L, L, t=1.0, mu=mu, xi=0.0, beta=beta, dtau=0.1, n_wrap=5)
    s = uniform_field(3, m.M, m.N)
    ld, sg, G = O.weight(m, s, -1, want_G=True)
    ref = _free_closed_form(m, mu)
    assert sg == 1
    assert abs(ld - ref) <= 1e-12 * abs(ref)
    # G_ij = (1/N) sum_k cos(k r_ij) / (1 + e^{-beta(eps_k - mu)})
    kx = 2 * np.pi * np.arange(L) / L
    eps = (-2 * (np.cos(kx)[None, :] + np.cos(kx)[:, None])).ravel() - mu
    nk = 1.0 / (1.0 + np.exp(-beta * eps))
    xs = np.arange(m.N) % L
    ys = np.arange(m.N) // L
    KX = np.repeat(kx[None, :], L, 0).ravel()
    KY = np.repeat(kx[:, None], L, 1).ravel()
    dx = xs[:, None] - xs[None, :]
    dy = ys[:, None] - ys[None, :]
    Gref = np.zeros((m.N, m.N))
    for q in range(m.N):
        Gref += np.cos(KX[q] * dx + KY[q] * dy) * nk[q]
    Gref /= m.N
    np.testing.assert_allclose(G, Gref, atol=1e-12)


@pytest.mark.parametrize("s0,eta", [(1, 1), (1, -1), (-1, 1), (-1, -1)])
def test_uniform_field_shifts_mu(s0, eta):
    """s = s0 everywhere: B = exp(-dtau (K - eta xi s0)), i.e. mu -> mu + eta xi s0."""
    m = O.Model(4, 4, t=1.0, mu=-0.5, xi=1.0, beta=8.0, dtau=0.05, n_wrap=10)
    s = np.full((m.M, m.N), s0, dtype=np.int8)
    ld, sg = O.weight(m, s, eta)
    ref = _free_closed_form(m, m.mu + eta * m.xi * s0)
    assert sg == 1
    assert abs(ld - ref) <= 1e-12 * abs(ref)


@pytest.mark.parametrize("L,beta,mu,seed", [(4, 4.0, 0.0, 1), (4, 8.0, -0.5, 2), (6, 6.0, 0.7, 3)])
def test_particle_hole_identity(L, beta, mu, seed):
    """Bipartite lattice: ld_eta(s; mu) - ld_-eta(s; -mu) = beta N mu + eta dtau xi sum s."""
    m = O.Model(L, L, mu=mu, xi=1.0, beta=beta, dtau=0.1, n_wrap=5)
    mneg = m.replace(mu=-mu)
    s = uniform_field(seed, m.M, m.N)
    for eta in (1, -1):
        a, sa = O.weight(m, s, eta)
        b, sb = O.weight(mneg, s, -eta)
        ref = m.beta * m.N * mu + eta * m.dtau * m.xi * float(s.sum())
        assert sa == sb
        assert abs((a - b) - ref) <= 1e-10 * max(abs(a), 1.0)


@pytest.mark.parametrize("Lx,Ly,mu,seed", [(4, 4, -0.5, 11), (3, 5, 0.3, 12)])
def test_flavours_are_the_negated_field(Lx, Ly, mu, seed):
    """Eq. 1: B_tau(eta) = e^{-dtau K} diag(e^{eta dtau xi s_tau}), so the eta = -1 weight of s
    is the eta = +1 weight of -s; and the total weight, log phi + 2 ld(+1) + 2 ld(-1), is
    invariant under s -> -s (H_s of Eq. 6 is Z2-symmetric).  An eta in the kinetic factor,
    one flavour counted twice, or a bare-weight term odd in s breaks one of the two."""
    m = O.Model(Lx, Ly, mu=mu, xi=1.0, beta=2.0, dtau=0.1, n_wrap=5, J=1.0, h=2.774)
    s = domain_field(seed, m.M, Lx, Ly, corr=2)
    a, sa = O.weight(m, s, -1)
    b, sb = O.weight(m, (-s).astype(np.int8), 1)
    assert sa == sb and abs(a - b) <= 1e-13 * abs(a)
    c, _ = O.weight(m, s, 1)
    assert abs(c - a) > 1e-6 * abs(a)  # the two flavours differ on this field
    lw, lw_neg = O.log_weight_total(m, s), O.log_weight_total(m, (-s).astype(np.int8))
    assert abs(lw - lw_neg) <= 1e-13 * abs(lw)


def _naive(m, s, eta):
    E = sla.expm(-m.dtau * O.build_K(m))
    B = np.eye(m.N)
    for tau in range(m.M):
        B = E @ np.diag(np.exp(eta * m.dtau * m.xi * s[tau])) @ B
    A = np.eye(m.N) + B
    sg, ld = np.linalg.slogdet(A)
    return ld, int(sg), np.linalg.inv(A)


@pytest.mark.parametrize("seed", [11, 12, 13])
def test_small_beta_naive_product(seed):
    """Small beta: unstabilised product + numpy slogdet/inv agree with the UDV oracle."""
    m = O.Model(4, 4, mu=-0.3, xi=1.0, beta=1.0, dtau=0.1, n_wrap=3)
    s = uniform_field(seed, m.M, m.N)
    for eta in (1, -1):
        ld, sg, G = O.weight(m, s, eta, want_G=True)
        ldn, sgn, Gn = _naive(m, s, eta)
        assert sg == sgn
        assert abs(ld - ldn) <= 1e-12 * abs(ldn)
        np.testing.assert_allclose(G, Gn, atol=1e-12)


def _mp_logdet(m, s, eta, dps=40):
    mpmath.mp.dps = dps
    E = mpmath.expm(-mpmath.mpf(m.dtau) * mpmath.matrix(O.build_K(m).tolist()))
    B = mpmath.eye(m.N)
    for tau in range(m.M):
        Dm = mpmath.diag([mpmath.exp(eta * mpmath.mpf(m.dtau) * m.xi * int(v)) for v in s[tau]])
        B = E * Dm * B
    d = mpmath.det(mpmath.eye(m.N) + B)
    return float(mpmath.log(abs(d))), (1 if d > 0 else -1)


def test_negative_sign_case():
    """A single flavour can have det(1+B) < 0; sign and log|det| agree with 40-digit mpmath."""
    m = O.Model(2, 2, mu=-1.5, xi=6.0, t=1.0, beta=3.0, dtau=0.25, n_wrap=4)
    found = 0
    for seed in (4, 28, 0, 1):
        s = uniform_field(seed, m.M, m.N)
        ref, sref = _mp_logdet(m, s, 1)
        for nw in (1, 2, 3, 4):
            ld, sg = O.weight(m, s, 1, n_wrap=nw)
            assert sg == sref
            assert abs(ld - ref) <= 1e-11 * max(1.0, abs(ref))
        found += sref < 0
    assert found >= 2


def test_mpmath_reference_moderate_beta():
    """beta = 4 (stabilisation needed in FP64): 40-digit mpmath product + det."""
    m = O.Model(2, 2, mu=-0.5, xi=1.0, beta=4.0, dtau=0.1, n_wrap=10)
    s = uniform_field(21, m.M, m.N)
    mpmath.mp.dps = 40
    K = O.build_K(m)
    Kmp = mpmath.matrix(K.tolist())
    E = mpmath.expm(-mpmath.mpf(m.dtau) * Kmp)
    for eta in (1, -1):
        B = mpmath.eye(m.N)
        for tau in range(m.M):
            Dm = mpmath.diag([mpmath.exp(eta * mpmath.mpf(m.dtau) * m.xi * int(v)) for v in s[tau]])
            B = E * Dm * B
        d = mpmath.det(mpmath.eye(m.N) + B)
        ld, sg = O.weight(m, s, eta)
        assert sg == (1 if d > 0 else -1)
        assert abs(ld - float(mpmath.log(abs(d)))) <= 1e-12 * abs(ld)


def test_cyclic_invariance():
    """det(1 + B_tau..B_1 B_M..B_tau+1) is independent of the starting slice."""
    m = O.Model(4, 4, mu=-0.5, beta=4.0, dtau=0.1, n_wrap=5)
    s = domain_field(5, m.M, 4, 4)
    ref, sref = O.weight(m, s, -1, tau0=0)
    for tau0 in (1, 7, 20, 39, 40):
        ld, sg = O.weight(m, s, -1, tau0=tau0)
        assert sg == sref
        assert abs(ld - ref) <= 1e-11 * abs(ref)


def test_nwrap_invariance():
    m = O.Model(4, 4, mu=-0.5, beta=10.0, dtau=0.1, n_wrap=1)
    s = uniform_field(6, m.M, m.N)
    ref, sref, Gref = O.weight(m, s, 1, want_G=True)
    for nw in (2, 5, 10, 20):
        ld, sg, G = O.weight(m, s, 1, n_wrap=nw, want_G=True)
        assert sg == sref
        assert abs(ld - ref) <= 1e-10 * abs(ref)
        np.testing.assert_allclose(G, Gref, atol=1e-10)


def test_green_is_inverse_of_cyclic_chain():
    """G(tau) from the oracle satisfies G (1 + B_tau..B_tau+1) = 1 (small beta, direct product)."""
    m = O.Model(3, 3, mu=0.2, beta=1.0, dtau=0.1, n_wrap=4)
    s = uniform_field(8, m.M, m.N)
    E = sla.expm(-m.dtau * O.build_K(m))
    tau0 = 4
    B = np.eye(m.N)
    for k in range(m.M):
        sl = (tau0 + k) % m.M
        B = E @ np.diag(np.exp(-m.dtau * m.xi * s[sl])) @ B
    _, _, G = O.weight(m, s, -1, tau0=tau0, want_G=True)
    np.testing.assert_allclose(G @ (np.eye(m.N) + B), np.eye(m.N), atol=1e-12)


# ---------------------------------------------------------- bare weight phi
def test_bare_weight_brute_force():
    """log phi against an explicit sum over bonds and time links on a 3x2 lattice."""
    m = O.Model(3, 2, beta=1.0, dtau=0.25, J=0.8, h=1.3)
    s = uniform_field(9, m.M, m.N)
    Kt = -0.5 * math.log(math.tanh(m.dtau * m.h))
    sp = 0
    for tau in range(m.M):
        for y in range(2):
            for x in range(3):
                i = x + 3 * y
                sp += s[tau, i] * s[tau, (x + 1) % 3 + 3 * y]  # x bonds
                sp += s[tau, i] * s[tau, x + 3 * ((y + 1) % 2)]  # y bonds (L=2: counted twice)
    tm = int(np.sum(s * np.roll(s, -1, axis=0)))
    ref = m.dtau * m.J * sp + Kt * tm
    assert abs(O.log_bare_weight(m, s) - ref) < 1e-12



def _tfim_trotter_factors(Lx, Ly, dtau, J, h):
    """Trotter factors of the transverse-field Ising model H_s = -J sum_<ij> sz sz - h sum_i sx
    (Eq. 6) on the 2^N spin basis, from scipy's matrix exponential of each term: the
    full off-diagonal factor expm(dtau h sum_i sx_i) and the diagonal of
    expm(dtau J sum_<ij> sz_i sz_j).  Basis index bit i set <=> s_i = -1."""
    N = Lx * Ly
    sx = np.array([[0.0, 1.0], [1.0, 0.0]])
    Hx = np.zeros((2 ** N, 2 ** N))
    for i in range(N):
        # site i is bit i of the basis index: the kron order puts site N-1 first
        op = np.array([[1.0]])
        for j in reversed(range(N)):
            op = np.kron(op, sx if j == i else np.eye(2))
        Hx += op
    Tx = sla.expm(dtau * h * Hx)
    # periodic adjacency: ring adjacency in each direction (a length-2 ring links its pair twice,
    # a length-1 ring not at all), A = A_x (x) I + I (x) A_y on site index x + Lx*y
    def ring(L):
        A = np.zeros((L, L))
        if L > 1:
            for a in range(L):
                A[a, (a + 1) % L] += 1
                A[a, (a - 1) % L] += 1
        return A
    A = np.kron(np.eye(Ly), ring(Lx)) + np.kron(ring(Ly), np.eye(Lx))
    spins = np.array([[1 - 2 * ((k >> i) & 1) for i in range(N)] for k in range(2 ** N)], dtype=np.float64)
    Hzz = 0.5 * np.einsum("ki,ij,kj->k", spins, A, spins)
    zz = np.diag(sla.expm(np.diag(dtau * J * Hzz)))
    return Tx, zz


def _basis_index(row):
    return int(sum(1 << i for i, v in enumerate(row) if v < 0))


@pytest.mark.parametrize("Lx,Ly,M", [(3, 2, 3), (4, 1, 3)])
def test_bare_weight_is_the_trotter_decomposition(Lx, Ly, M):
    """phi(C) is, up to one configuration-independent constant, the product over slices of
    <s_tau+1| expm(dtau h sum sx) |s_tau> expm(dtau J sum sz sz)[s_tau]: the Suzuki-Trotter
    path weight of H_s (Eq. 6).  A wrong temporal coupling (sign, factor 2, cosh/sinh
    swapped) or a missing spatial factor changes the ratio between configurations."""
    dtau, J, h = 0.2, 0.7, 1.9
    m = O.Model(Lx, Ly, beta=M * dtau, dtau=dtau, J=J, h=h)
    Tx, zz = _tfim_trotter_factors(Lx, Ly, dtau, J, h)
    rng = np.random.default_rng(5)
    diffs = []
    for _ in range(200):
        s = rng.choice(np.array([-1, 1], dtype=np.int8), size=(m.M, m.N))
        idx = [_basis_index(s[t]) for t in range(m.M)]
        path = sum(math.log(Tx[idx[(t + 1) % m.M], idx[t]]) + math.log(zz[idx[t]]) for t in range(m.M))
        diffs.append(O.log_bare_weight(m, s) - path)
    diffs = np.array(diffs)
    assert np.ptp(diffs) < 1e-11, np.ptp(diffs)
    # the constant is the normalisation of a time link: <s|expm(dtau h sx)|s'> = A e^{Kt s s'}
    # with A^2 = sinh cosh and e^{2 Kt} = cosh / sinh, so log phi - path = -M N log A
    A = math.sqrt(math.sinh(dtau * h) * math.cosh(dtau * h))
    assert abs(diffs[0] + m.M * m.N * math.log(A)) < 1e-11


def test_bare_weight_time_link_ratio_is_tanh():
    """Flipping one spin of a single-site chain breaks two time links: phi changes by the
    square of the off-diagonal / diagonal element of expm(dtau h sx), tanh(dtau h)^2."""
    dtau, h = 0.1, 2.774
    m = O.Model(1, 1, beta=0.6, dtau=dtau, J=1.0, h=h)
    T = sla.expm(dtau * h * np.array([[0.0, 1.0], [1.0, 0.0]]))
    s = np.ones((m.M, 1), dtype=np.int8)
    s2 = s.copy()
    s2[2, 0] = -1
    ratio = math.exp(O.log_bare_weight(m, s2) - O.log_bare_weight(m, s))
    assert abs(ratio - (T[0, 1] / T[0, 0]) ** 2) < 1e-14


def test_bare_weight_sums_to_trotter_partition_function():
    """Summing phi(C) over all 2^(N M) configurations gives Tr[(Tx Z)^M] times the same
    per-link constant (3x1 sites, 4 slices: 4096 configurations)."""
    Lx, Ly, M, dtau, J, h = 3, 1, 4, 0.25, 0.8, 1.3
    m = O.Model(Lx, Ly, beta=M * dtau, dtau=dtau, J=J, h=h)
    Tx, zz = _tfim_trotter_factors(Lx, Ly, dtau, J, h)
    Z_trotter = np.trace(np.linalg.matrix_power(Tx @ np.diag(zz), M))
    tot = 0.0
    for k in range(2 ** (m.N * m.M)):
        s = np.array([1 - 2 * ((k >> b) & 1) for b in range(m.N * m.M)], dtype=np.int8).reshape(m.M, m.N)
        tot += math.exp(O.log_bare_weight(m, s))
    A = math.sqrt(math.sinh(dtau * h) * math.cosh(dtau * h))
    assert abs(tot * A ** (m.N * m.M) / Z_trotter - 1.0) < 1e-12


# ------------------------------------------------------------ local sweeps
def _bruteforce_sweep(m, s, seed, sweep):
    """One local sweep where every ratio is a quotient of two full weights."""
    s = s.copy()
    acc = 0
    for tau in range(m.M):
        for i in range(m.N):
            lw0 = O.log_weight_total(m, s)
            s2 = s.copy()
            s2[tau, i] = -s2[tau, i]
            lw1 = O.log_weight_total(m, s2)
            u = O.uniform(seed, i, tau, sweep, 1)
            if math.log(u) < lw1 - lw0:
                s = s2
                acc += 1
    return s, acc


@pytest.mark.parametrize("n_wrap,seed", [(1, 3), (2, 4), (4, 5), (3, 6)])
def test_local_sweep_matches_bruteforce_ratios(n_wrap, seed):
    """Sherman-Morrison ratios, updates and wraps reproduce brute-force determinant ratios."""
    m = O.Model(2, 2, mu=-0.5, xi=1.0, beta=1.5, dtau=0.25, n_wrap=n_wrap, J=1.0, h=1.0)
    s = uniform_field(seed, m.M, m.N)
    sb = s.copy()
    tot = 0
    for sw in range(3):
        sb, a = _bruteforce_sweep(m, sb, seed, sw)
        tot += a
    so, st = O.local_sweep(m, s, seed, 0, 3)
    assert st["margin_events"] == 0
    assert st["accepted"] == tot
    np.testing.assert_array_equal(so, sb)
    assert st["max_drift"] < 1e-10


def test_local_sweep_nwrap_and_resume():
    m = O.Model(4, 4, mu=-0.5, xi=1.0, beta=2.0, dtau=0.1, n_wrap=10, J=1.0, h=2.774)
    s = uniform_field(1001, m.M, m.N)
    a, sa = O.local_sweep(m, s, 7, 0, 4)
    b, sb = O.local_sweep(m.replace(n_wrap=1), s, 7, 0, 4)
    np.testing.assert_array_equal(a, b)
    # resume after 2 sweeps is bit-identical (counter-based RNG)
    c, _ = O.local_sweep(m, s, 7, 0, 2)
    c, _ = O.local_sweep(m, c, 7, 2, 2)
    np.testing.assert_array_equal(a, c)
    assert sa["max_drift"] < 1e-9
    assert 0 < sa["accepted"] < sa["proposed"]


# ------------------------------------------------- exact enumeration (2x4)
ENUM = dict(Lx=2, Ly=1, t=1.0, mu=-0.5, xi=1.0, beta=1.0, dtau=0.25, n_wrap=2, J=1.0, h=1.0)


def _all_configs(M, N):
    n = M * N
    idx = np.arange(2 ** n)
    bits = (idx[:, None] >> np.arange(n)[None, :]) & 1
    return (2 * bits - 1).astype(np.int8).reshape(-1, M, N)


def _code(s):
    b = (s.reshape(-1) > 0).astype(np.int64)
    return int(np.sum(b << np.arange(b.size)))


@pytest.fixture(scope="module")
def enum_model():
    m = O.Model(**ENUM)
    cfgs = _all_configs(m.M, m.N)
    lw = np.array([O.log_weight_total(m, c) for c in cfgs])
    p = np.exp(lw - lw.max())
    return m, cfgs, lw, p / p.sum()


def _chi2_p(counts, probs, min_expected=5.0):
    """Pearson chi^2 p-value; cells expected below min_expected are pooled into one."""
    exp = probs * counts.sum()
    small = exp < min_expected
    c = np.append(counts[~small], counts[small].sum())
    e = np.append(exp[~small], exp[small].sum())
    return stats.chisquare(c, e).pvalue


def test_enumeration_weights_match_naive(enum_model):
    m, cfgs, lw, _ = enum_model
    for c in cfgs[::17]:
        ref = 0.0
        for eta in (1, -1):
            ldn, sgn, _ = _naive(m, c, eta)
            ref += 2 * ldn
        ref += O.log_bare_weight(m, c)
        lwc = O.log_weight_total(m, c)
        assert abs(lwc - ref) < 1e-12


@pytest.mark.slow
def test_enumeration_local_dqmc_chi2(enum_model):
    """Local DQMC from exact draws keeps the exact distribution (chi^2, 255 dof)."""
    m, cfgs, lw, p = enum_model
    rng = np.random.Generator(np.random.PCG64(424242))
    n_chain = 12000
    start = rng.choice(len(cfgs), size=n_chain, p=p)
    counts = np.zeros(len(cfgs))
    moved = 0
    for c in range(n_chain):
        s1, _ = O.local_sweep(m, cfgs[start[c]], seed=1000 + c, sweep0=0, n_sweeps=2)
        k = _code(s1)
        counts[k] += 1
        moved += k != start[c]
    assert moved > 0.3 * n_chain
    assert _chi2_p(counts, p) > 0.01


# -------------------------------------------------------- effective model
CLASSES_2D = [[(1, 0, 0), (0, 1, 0)], [(1, 1, 0), (1, -1, 0)], [(2, 0, 0), (0, 2, 0)], [(0, 0, 1)]]


def test_features_invariants():
    m = O.Model(4, 4, beta=1.0, dtau=0.1)
    ones = np.ones((m.M, m.N), dtype=np.int8)
    f = O.features(m, ones, CLASSES_2D)
    np.testing.assert_array_equal(f, [2 * m.N * m.M, 2 * m.N * m.M, 2 * m.N * m.M, m.N * m.M])
    s = uniform_field(4, m.M, m.N)
    np.testing.assert_array_equal(O.features(m, s, CLASSES_2D), O.features(m, -s, CLASSES_2D))
    # spatial checkerboard, uniform in time: NN bonds -1, diagonal +1, distance-2 +1, time +1
    x = np.arange(m.N) % 4
    y = np.arange(m.N) // 4
    cb = np.tile(np.where((x + y) % 2 == 0, 1, -1).astype(np.int8), (m.M, 1))
    np.testing.assert_array_equal(O.features(m, cb, CLASSES_2D),
                                  [-2 * m.N * m.M, 2 * m.N * m.M, 2 * m.N * m.M, m.N * m.M])


def test_coloring_is_proper_and_greedy():
    m = O.Model(5, 4, beta=0.7, dtau=0.1)
    nc, col = O.coloring(m, CLASSES_2D)
    N, M = m.N, m.M
    for v in range(N * M):
        tau, i = divmod(v, N)
        x, y = i % 5, i // 5
        for c in CLASSES_2D:
            for (dx, dy, dt) in c:
                for sg in (1, -1):
                    w = ((tau + sg * dt) % M) * N + (x + sg * dx) % 5 + 5 * ((y + sg * dy) % 4)
                    if w != v:
                        assert col[w] != col[v]
    # nearest neighbours only on an even periodic box: greedy gives the checkerboard
    m2 = O.Model(4, 4, beta=0.4, dtau=0.1)
    nc2, col2 = O.coloring(m2, [[(1, 0, 0), (0, 1, 0), (0, 0, 1)]])
    assert nc2 == 2


def test_fit_recovers_planted_model():
    """Eq. 3 on data generated from a known H_eff: exact J, E0 and R^2 = 1."""
    m = O.Model(4, 4, beta=1.0, dtau=0.1)
    rng = np.random.Generator(np.random.PCG64(77))
    Jt = np.array([-0.3, 0.05, 0.02, -0.6])
    E0 = 1.7
    F = np.array([O.features(m, domain_field(int(k), m.M, 4, 4, corr=2), CLASSES_2D)
                  for k in rng.integers(0, 2 ** 31, 60)], dtype=np.float64)
    y = -m.beta * (E0 + F @ Jt)
    J, e0, r2 = O.fit(F, y, m.beta)
    np.testing.assert_allclose(J, Jt, atol=1e-10)
    assert abs(e0 - E0) < 1e-9
    assert abs(r2 - 1.0) < 1e-12
    # with noise it equals numpy's least-squares solution
    y2 = y + rng.standard_normal(len(y)) * 0.5
    J2, e02, r22 = O.fit(F, y2, m.beta)
    A = np.hstack([np.ones((len(y2), 1)), F])
    coef = np.linalg.lstsq(A, y2, rcond=None)[0]
    np.testing.assert_allclose(-coef[1:] / m.beta, J2, rtol=1e-9, atol=1e-12)
    res = y2 - A @ coef
    assert abs(r22 - (1 - res @ res / np.sum((y2 - y2.mean()) ** 2))) < 1e-10


ENUM_CLASSES = [[(1, 0, 0)], [(0, 0, 1)]]


@pytest.mark.slow
def test_enumeration_effective_sweeps_chi2(enum_model):
    """Effective-model sweeps preserve exp(-beta H_eff) on the 2x4 system (both directions)."""
    m, cfgs, _, _ = enum_model
    J = np.array([-0.4, -0.3])
    F = np.array([O.features(m, c, ENUM_CLASSES) for c in cfgs], dtype=np.float64)
    le = -m.beta * (F @ J)
    pe = np.exp(le - le.max())
    pe /= pe.sum()
    rng = np.random.Generator(np.random.PCG64(99))
    n_chain = 12000
    start = rng.choice(len(cfgs), size=n_chain, p=pe)
    counts = np.zeros(len(cfgs))
    acc = 0
    for c in range(n_chain):
        s1, na, _ = O.eff_sweeps(m, cfgs[start[c]], ENUM_CLASSES, J, 1, seed=5000 + c, step=0,
                                 direction=c & 1)
        counts[_code(s1)] += 1
        acc += na
    assert acc > 0
    assert _chi2_p(counts, pe) > 0.01


@pytest.mark.slow
def test_enumeration_cumulative_update_chi2(enum_model):
    """Cumulative updates with a deliberately wrong H_eff keep the exact distribution (Eq. 4)."""
    m, cfgs, lw, p = enum_model
    # a poor effective model: the Eq. 4 acceptance must correct it
    J = np.array([-0.2, -0.15])
    rng = np.random.Generator(np.random.PCG64(31337))
    n_chain = 12000
    start = rng.choice(len(cfgs), size=n_chain, p=p)
    counts = np.zeros(len(cfgs))
    acc = 0
    for c in range(n_chain):
        s = cfgs[start[c]]
        l = lw[start[c]]
        s, l, a, lr, _, mg = O.cumulative_update(m, s, l, ENUM_CLASSES, J, 1, seed=9000 + c, step=0)
        acc += a
        counts[_code(s)] += 1
        assert abs(l - lw[_code(s)]) < 1e-12
    assert 0.05 * n_chain < acc < 0.98 * n_chain
    assert _chi2_p(counts, p) > 0.01


# --------------------------------------------------------- parallel helpers
def test_parallel_helpers_equal_sequential_calls():
    """weight_many and cumulative_chains only spread weight() and cumulative_update() over
    processes: same numbers as calling them one by one."""
    m = O.Model(3, 2, mu=-0.3, xi=1.0, beta=1.0, dtau=0.25, n_wrap=2, J=1.0, h=1.3)
    fields = [uniform_field(70 + k, m.M, m.N) for k in range(3)]
    assert O.weight_many(m, fields, 1, workers=2) == [O.weight(m, f, 1) for f in fields]
    classes = [[(1, 0, 0), (0, 1, 0)], [(0, 0, 1)]]
    J = np.array([-0.2, -0.5])
    series, acc = O.cumulative_chains(m, fields[:2], classes, J, 2, [11, 12], 5, 4, workers=2)
    for c in range(2):
        s, lw, n_acc = fields[c], O.log_weight_total(m, fields[c]), 0
        for k in range(4):
            s, lw, a, _, _, _ = O.cumulative_update(m, s, lw, classes, J, 2, 11 + c, 5 + k)
            n_acc += a
            assert series[k, c] == int(s.astype(np.int64).sum())
        assert acc[c] == n_acc
