"""Integrated autocorrelation time and binning error bars of Monte Carlo time
series (host-side analysis).

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


def binning_errors(series):
    """Standard errors of the mean of a correlated series by binning (the
    'standard binning analysis' of Sec. II.B for Monte Carlo error bars): the
    series is averaged in blocks of 1, 2, 4, ... consecutive samples and the
    naive standard error of the block means is returned for every block size
    with at least 16 blocks.  For correlated samples the error grows with the
    block size and levels off at the true one, sqrt(2 tau_int) times the naive
    value.  Returns (block sizes, errors)."""
    x = np.asarray(series, dtype=np.float64)
    sizes, errs = [], []
    b = 1
    while len(x) // b >= 16:
        nb = len(x) // b
        means = x[: nb * b].reshape(nb, b).mean(axis=1)
        sizes.append(b)
        errs.append(float(means.std(ddof=1) / np.sqrt(nb)))
        b *= 2
    return np.array(sizes, dtype=int), np.array(errs)


def binned_error(series, min_blocks=32):
    """Error bar of the mean: the binning error at the largest block size that
    still leaves at least min_blocks blocks (0 for fewer than 2 samples)."""
    x = np.asarray(series, dtype=np.float64)
    if len(x) < 2:
        return 0.0
    sizes, errs = binning_errors(x)
    if len(sizes) == 0:
        return float(x.std(ddof=1) / np.sqrt(len(x)))
    ok = [e for s, e in zip(sizes, errs) if len(x) // s >= min_blocks]
    return float(ok[-1] if ok else errs[0])


def twist_average(means, errors=None):
    """Twist-averaged estimate (Sec. III.C): the plain mean over the N_Theta twisted
    chains.  The chains are independent and each has its own expectation, so the
    statistical error of the average comes from the chains' own error bars,
    sqrt(sum_i err_i^2) / N_Theta, not from the spread between twists (which is
    the boundary-condition dependence TABC averages out).  Returns (mean, error);
    error is None without per-chain errors."""
    m = np.asarray(means, dtype=np.float64)
    if m.size == 0:
        raise ValueError("no twists")
    avg = float(m.mean(axis=0)) if m.ndim == 1 else m.mean(axis=0)
    if errors is None:
        return avg, None
    e = np.asarray(errors, dtype=np.float64)
    err = np.sqrt((e * e).sum(axis=0)) / m.shape[0]
    return avg, (float(err) if np.ndim(err) == 0 else err)
