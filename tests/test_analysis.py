"""tau_int estimator against the closed form of an AR(1) process:
x_t = rho x_{t-1} + noise has C(t) = rho^t, so tau_int = (1 + rho) / (2 (1 - rho))."""
import numpy as np

from paper_1612_03804_gb300.analysis import autocorr, tau_int


def _ar1(rho, T, chains, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    x = np.zeros((T, chains))
    x[0] = rng.standard_normal(chains) / np.sqrt(1 - rho * rho)
    for t in range(1, T):
        x[t] = rho * x[t - 1] + rng.standard_normal(chains)
    return x


def test_white_noise_tau_is_half():
    x = _ar1(0.0, 4000, 8, 1)
    tau, W = tau_int(x)
    assert abs(tau - 0.5) < 0.05


def test_ar1_tau_matches_closed_form():
    for rho in (0.5, 0.8):
        x = _ar1(rho, 20000, 8, 2)
        tau, W = tau_int(x)
        ref = (1 + rho) / (2 * (1 - rho))
        assert abs(tau - ref) < 0.1 * ref
        C = autocorr(x)
        assert abs(C[1] - rho) < 0.02
