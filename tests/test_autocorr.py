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
