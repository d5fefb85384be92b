"""Integrated autocorrelation time of Monte Carlo time series (host-side analysis).

Convention (Sokal, "Monte Carlo methods in statistical mechanics", 1997):
tau_int = 1/2 + sum_{t>=1} rho(t), so uncorrelated samples have tau_int = 1/2
and N samples carry N / (2 tau_int) independent ones.  The sum is cut at the
automatic window W, the smallest W with W >= c * tau_int(W) (c = 6 by default).
Several independent chains are pooled by averaging their normalised
autocorrelation functions, each taken about its own chain mean.
"""
import numpy as np


def autocorrelation(series_list, t_max):
    """Pooled normalised autocorrelation rho(0..t_max) of equally long chains."""
    acc = np.zeros(t_max + 1)
    used = 0
    for x in series_list:
        x = np.asarray(x, dtype=np.float64)
        n = len(x)
        if n < 2:
            continue
        d = x - x.mean()
        c0 = np.dot(d, d) / n
        if not c0 > 0:
            continue
        T = min(t_max, n - 1)
        for t in range(T + 1):
            acc[t] += np.dot(d[: n - t], d[t:]) / (n - t) / c0
        used += 1
    return acc / max(used, 1)


def tau_int(series_list, c=6.0):
    """(tau_int, window, samples per chain) with Sokal's automatic window.

    Returns tau_int = 0.5 for constant or too-short series and flags a window
    that ran to the end of the series (window = -1): the estimate is then a
    lower bound."""
    series_list = [np.asarray(s, dtype=np.float64) for s in series_list if len(s) >= 2]
    if not series_list:
        return 0.5, 0, 0
    n = min(len(s) for s in series_list)
    series_list = [s[:n] for s in series_list]
    rho = autocorrelation(series_list, n - 1)
    tau = 0.5
    for w in range(1, n):
        tau += rho[w]
        if w >= c * tau:
            return max(tau, 0.5), w, n
    return max(tau, 0.5), -1, n
