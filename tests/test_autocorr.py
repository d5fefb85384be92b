"""The integrated-autocorrelation estimator used to correct the update rate,
checked against the closed form of a Gaussian AR(1) process
x_t = rho x_{t-1} + noise, whose autocorrelation is rho^t and whose
tau_int = 1/2 + sum_t rho^t = (1 + rho) / (2 (1 - rho))."""
import numpy as np
import pytest

from paper_2609_14668_b300.autocorr import tau_int, autocorrelation


def ar1(rho, n, seed):
    rng = np.random.default_rng(seed)
    e = rng.standard_normal(n)
    x = np.empty(n)
    x[0] = e[0] / np.sqrt(1 - rho * rho)
    for t in range(1, n):
        x[t] = rho * x[t - 1] + e[t]
    return x


@pytest.mark.parametrize("rho", [0.0, 0.5, 0.8])
def test_ar1_closed_form(rho):
    chains = [ar1(rho, 40000, s) for s in range(4)]
    tau, w, n = tau_int(chains)
    exact = (1 + rho) / (2 * (1 - rho))
    assert w > 0 and n == 40000
    assert abs(tau - exact) < 0.06 * exact + 0.02, (tau, exact)


def test_autocorrelation_of_ar1_is_geometric():
    x = ar1(0.7, 200000, 11)
    r = autocorrelation([x], 4)
    assert r[0] == pytest.approx(1.0)
    assert np.allclose(r[1:], 0.7 ** np.arange(1, 5), atol=0.02)


def test_degenerate_series():
    assert tau_int([np.ones(10)])[0] == 0.5
    assert tau_int([[1.0]]) == (0.5, 0, 0)
    # a monotone series stays positively correlated at short lags
    tau, w, n = tau_int([np.arange(40.0)])
    assert tau > 2.0 and n == 40


def test_binning_of_independent_samples_is_flat():
    """i.i.d. samples: every block size gives the naive error sigma / sqrt(n)."""
    from paper_2609_14668_b300.autocorr import binning_errors, binned_error
    x = np.random.default_rng(3).standard_normal(1 << 16)
    sizes, errs = binning_errors(x)
    assert sizes[0] == 1 and sizes[-1] == (1 << 16) // 16
    naive = x.std(ddof=1) / np.sqrt(len(x))
    assert errs[0] == pytest.approx(naive)
    assert np.all(np.abs(errs[:8] / naive - 1.0) < 0.15)
    assert abs(binned_error(x) / naive - 1.0) < 0.3


@pytest.mark.parametrize("rho", [0.5, 0.8])
def test_binning_of_ar1_reaches_the_correlated_error(rho):
    """AR(1): the error of the mean is sigma_x sqrt(2 tau_int / n) with
    sigma_x^2 = 1 / (1 - rho^2) and 2 tau_int = (1 + rho) / (1 - rho)."""
    from paper_2609_14668_b300.autocorr import binned_error
    n = 1 << 17
    x = ar1(rho, n, 5)
    exact = np.sqrt(1.0 / (1.0 - rho * rho) * (1.0 + rho) / (1.0 - rho) / n)
    assert abs(binned_error(x) / exact - 1.0) < 0.2
    naive = x.std(ddof=1) / np.sqrt(n)
    assert binned_error(x) > 1.5 * naive


def test_binning_degenerate():
    from paper_2609_14668_b300.autocorr import binned_error, binning_errors
    assert binned_error([1.0]) == 0.0
    s, e = binning_errors(np.arange(10.0))
    assert len(s) == 0
    assert binned_error(np.arange(10.0)) == pytest.approx(np.arange(10.0).std(ddof=1) / np.sqrt(10))


def test_twist_average_error_from_chain_errors():
    """Independent chains with different expectations: the error of the twist
    average is sqrt(sum err_i^2) / N, checked by repeating the experiment."""
    from paper_2609_14668_b300.autocorr import twist_average
    rng = np.random.default_rng(9)
    mu = np.linspace(-1.0, 1.0, 14)              # per-twist expectations
    sig = np.linspace(0.05, 0.2, 14)             # per-twist error bars
    draws = [twist_average(mu + sig * rng.standard_normal(14), sig) for _ in range(4000)]
    avgs = np.array([d[0] for d in draws])
    err = draws[0][1]
    assert err == pytest.approx(np.sqrt((sig ** 2).sum()) / 14)
    assert abs(avgs.mean() - mu.mean()) < 4 * err / np.sqrt(4000) + 1e-12
    assert abs(avgs.std() / err - 1.0) < 0.05
    assert twist_average([1.0, 3.0]) == (2.0, None)
    with pytest.raises(ValueError):
        twist_average([])
