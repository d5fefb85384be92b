"""Pins of the time-displaced oracle (oracle/tdgf.py): the free-fermion closed
forms of G(tau, 0) and G(0, tau), the exact HS sum of <H_I(tau) H_I(0)>
against the Trotterised ED, and dD/dU from the tau integral (Eq.
DouOccDerive) against a finite difference of the ED double occupancy."""
import itertools

import numpy as np
import pytest

from oracle import ed
from oracle import tdgf
from oracle.dqmc import Model
from synth import random_field


@pytest.mark.parametrize("theta", [(0.0, 0.0), (0.25, 0.5)])
def test_free_fermion_time_displaced(theta):
    m = Model(3, U=0.0, beta=2.0, dtau=0.1, theta=theta)
    f = random_field(m.M, m.N, 4)
    w, V = np.linalg.eigh(m.K)
    for l in (0, 3, 11, m.M):
        tau = l * m.dtau
        Gt0, G0t, _, _ = tdgf.greens(m, f, l)
        fermi = 1.0 / (1.0 + np.exp(-m.beta * w))       # (1 + e^{-beta K})^-1 spectrally
        ref_t0 = (V * (np.exp(-tau * w) * fermi)) @ V.conj().T
        ref_0t = -(V * ((1.0 - fermi) * np.exp(tau * w))) @ V.conj().T
        assert np.abs(Gt0 - ref_t0).max() < 1e-11
        assert np.abs(G0t - ref_0t).max() < 1e-11


def _hs_correlation(m):
    logw, hh, h1 = [], [], []
    for bits in itertools.product((1, -1), repeat=m.N * m.M):
        field = np.array(bits, dtype=np.int8).reshape(m.M, m.N)
        lw, _ = m.log_weight(field)
        logw.append(lw)
        row = [tdgf.hi_products(m, field, l) for l in range(m.M + 1)]
        hh.append([r[0] for r in row])
        h1.append(row[0][1])
    w = np.exp(np.array(logw) - max(logw))
    w /= w.sum()
    return w @ np.array(hh), w @ np.array(h1)


@pytest.mark.parametrize("theta", [(0.0, 0.0), (0.3, 0.0)])
def test_hs_sum_of_hi_correlation_equals_trotter_ed(theta):
    """Two-site cell (L = 1: A and B joined by the three bonds), 6 slices, all 2^12 fields."""
    m = Model(1, U=3.0, beta=1.2, dtau=0.2, theta=theta)
    hh, h1 = _hs_correlation(m)
    ref_hh, ref_h1 = ed.trotter_hi_correlation(m.lat, m.K, m.U, m.dtau, m.M)
    assert abs(h1 - ref_h1) < 1e-10
    assert np.abs(hh - ref_hh).max() < 1e-10


def test_dDdU_identity_and_tau_integral():
    """(1) For the Trotterised system, dD/dU = -dtau sum_l cov(D, H_I at mid-slice l)
    exactly (finite difference of the ED double occupancy, 1e-8).  (2) The estimator
    of Eq. DouOccDerive, -(2/N) int_0^{beta/2} C(tau) dtau by the trapezoidal rule
    over the slice times, converges to it as dtau^2: halving dtau cuts the gap >= 3x."""
    from oracle.lattice import Honeycomb
    lat = Honeycomb(1)
    K = lat.hopping_matrix()
    U, beta = 3.0, 1.2
    gaps = []
    for M in (12, 24):
        dtau = beta / M
        eps = 1e-5
        fd = (ed.trotter_averages(lat, K, U + eps, dtau, M)["double_occ"]
              - ed.trotter_averages(lat, K, U - eps, dtau, M)["double_occ"]) / (2 * eps)
        assert abs(ed.trotter_dDdU(lat, K, U, dtau, M) - fd) < 1e-8
        hh, h1 = ed.trotter_hi_correlation(lat, K, U, dtau, M)
        C = hh - h1 * h1
        assert np.allclose(C, C[::-1], atol=1e-12)                 # C(tau) = C(beta - tau)
        dDdU, _ = tdgf.integrals(C[: M // 2 + 1], dtau, lat.N)
        gaps.append(abs(dDdU - fd))
    assert gaps[1] < gaps[0] / 3.0, gaps


def test_trapezoid_convention():
    dD, chi = tdgf.integrals([1.0, 1.5, 2.0, 2.5], 0.5, 4)      # C = 1 + tau on [0, 1.5]
    assert abs(dD - (-2.0 / 4 * (1.5 + 1.5 ** 2 / 2))) < 1e-14
    assert abs(chi - 2.3125) < 1e-14                             # trapezoid of tau(1 + tau) on that grid
