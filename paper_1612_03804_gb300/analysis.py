"""Autocorrelation analysis of Monte Carlo series (host-side measurement).

The paper measures decorrelation through the autocorrelation function of the
total magnetisation, C(t) = (<M(0)M(t)> - <M>^2) / (<M^2> - <M>^2)
(caption of its Fig. 1), without fixing how tau is read off.  Here the
integrated time tau_int = 1/2 + sum_{t>=1} C(t) is estimated with the
automatic window of Madras and Sokal (J. Stat. Phys. 50, 109 (1988)): the
sum stops at the first W with W >= c * tau_int(W), c = 6.
"""
import numpy as np


def autocorr(series):
    """Normalised autocorrelation C(t) of one or several chains.

    series: array (T,) or (T, n_chains); the chains share one mean and
    variance and their lag products are pooled."""
    x = np.asarray(series, dtype=np.float64)
    if x.ndim == 1:
        x = x[:, None]
    T = x.shape[0]
    x = x - x.mean()
    var = np.mean(x * x)
    if var == 0.0:
        return np.ones(1)
    c = np.empty(T)
    for t in range(T):
        c[t] = np.mean(x[: T - t] * x[t:]) / var
    return c


def tau_int(series, c=6.0):
    """Integrated autocorrelation time with the Madras-Sokal window."""
    C = autocorr(series)
    tau = 0.5
    for W in range(1, len(C)):
        tau += C[W]
        if W >= c * tau:
            return max(tau, 0.5), W
    return max(tau, 0.5), len(C) - 1
