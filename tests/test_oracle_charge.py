"""Pins of the oracle's charge-channel field (HS-n, Eq. DensityHS) against what
the paper and mathematics fix: the decoupling identity itself, the weight of
Eq. ConfgWeight written in the original (untransformed) basis with the p(x) of
Eq. BIOpnT, brute-force determinant ratios and inverses, the Hubbard atom, and
the Trotterised Fock-space ED, which both channels must reproduce exactly."""
import itertools

import numpy as np
import pytest

from oracle.dqmc import Model, Chain, local_ratio
from oracle import ed, enumerate as hs_enum
from synth import random_field

TW = (0.25, 0.5)


@pytest.mark.parametrize("U,dtau", [(3.73, 0.1), (4.0, 0.05), (1.0, 0.3), (8.0, 0.2)])
def test_charge_coupling_satisfies_decoupling_identity(U, dtau):
    """Eq. DensityHS on the four states of one site, with gamma_c = i arccos(e^{-dtau U/2})."""
    m = Model(1, U=U, beta=dtau, dtau=dtau, hs_channel=1)
    gc = 1j * m.alpha
    for nu, nd in itertools.product((0, 1), repeat=2):
        lhs = np.exp(-dtau * U * (nu * nd - 0.5 * (nu + nd)))
        rhs = np.exp(dtau * U / 2.0) / 2.0 * sum(np.exp(gc * x * (nu + nd - 1)) for x in (1, -1))
        assert abs(lhs - rhs) < 1e-14 * lhs


def _original_basis_log_weight(m, field):
    """log W(X) of Eq. ConfgWeight without the particle-hole transform: both spins
    share the hopping (and twist); B_up = e^{lam x} E and B_dn = e^{-lam x} E
    (spin channel, Eq. BIOpSz) or B_dn = B_up (charge channel, Eq. BIOpnT);
    P(X) = prod_l p(x_l) with p = 2^-N (spin) or e^{dtau U N/2} 2^-N e^{-gamma_c sum x} (charge).
    Complex: the phase must come out zero."""
    I = np.eye(m.N)
    Bup = np.eye(m.N, dtype=complex)
    Bdn = np.eye(m.N, dtype=complex)
    for l in range(m.M):
        x = field[l].astype(float)
        Bup = (np.exp(m.lam * x)[:, None] * m.E) @ Bup
        sdn = -m.lam if m.hs_channel == 0 else m.lam
        Bdn = (np.exp(sdn * x)[:, None] * m.E) @ Bdn
    logP = -m.M * m.N * np.log(2.0)
    if m.hs_channel == 1:
        logP += m.M * m.dtau * m.U * m.N / 2.0 - 1j * m.alpha * float(field.sum())
    return logP + np.log(np.linalg.det(I + Bup)) + np.log(np.linalg.det(I + Bdn))


@pytest.mark.parametrize("hs_channel", [0, 1])
@pytest.mark.parametrize("theta", [(0.0, 0.0), TW])
def test_weight_equals_original_basis_weight(hs_channel, theta):
    """The oracle's transformed weight (|det|^2, times e^{-gamma sum s} in the spin
    channel) is real, positive and differs from the original-basis weight by a
    field-independent constant."""
    m = Model(2, U=3.73, beta=0.6, dtau=0.1, theta=theta, hs_channel=hs_channel)
    diffs = []
    for seed in range(6):
        f = random_field(m.M, m.N, 300 + seed)
        w0 = _original_basis_log_weight(m, f)
        assert abs(np.sin(w0.imag)) < 1e-10            # real and positive
        lw, sign = m.log_weight(f)
        assert sign == 1.0 or (not m.is_complex and sign in (1.0, -1.0))
        diffs.append(w0.real - lw)
    assert np.ptp(diffs) < 1e-10


@pytest.mark.parametrize("theta", [(0.0, 0.0), TW])
def test_charge_ratio_equals_weight_ratio(theta):
    """R = |r|^2 equals W(X')/W(X) from brute-force determinants, and r the ratio of
    the complex up-spin determinants (Eqs. DRatio, rRatioLocal)."""
    m = Model(2, U=3.73, beta=1.0, dtau=0.1, theta=theta, hs_channel=1)
    field = random_field(m.M, m.N, 11)
    lw0, _ = m.log_weight(field)
    for l, i in ((1, 0), (4, 5), (10, 7)):
        G = m.green_direct(field, l)
        R, r, D = local_ratio(m, G, i, float(field[l - 1, i]))
        assert abs(abs(1.0 + D) - 1.0) < 1e-15 and abs(D.imag) > 1e-3
        assert abs(np.imag(r)) > 1e-6
        f2 = field.copy()
        f2[l - 1, i] *= -1
        lw1, _ = m.log_weight(f2)
        assert abs(R - np.exp(lw1 - lw0)) < 1e-10 * max(1.0, R)
        d0 = np.linalg.det(np.eye(m.N) + m.chain_product(field, 1, m.M))
        d1 = np.linalg.det(np.eye(m.N) + m.chain_product(f2, 1, m.M))
        assert abs(r - d1 / d0) < 1e-10 * max(1.0, abs(r))


def test_charge_green_is_complex_without_twist():
    m = Model(3, U=3.73, beta=1.0, dtau=0.1, hs_channel=1)
    f = random_field(m.M, m.N, 3)
    G = m.green_stable(f, 4, 5)
    assert np.abs(G.imag).max() > 1e-3
    assert np.abs(G - m.green_direct(f, 4)).max() < 1e-11


@pytest.mark.parametrize("theta", [(0.0, 0.0), TW])
@pytest.mark.parametrize("n_delay", [1, 4])
def test_charge_slice_update_matches_fresh_green(theta, n_delay):
    m = Model(3, U=3.73, beta=1.0, dtau=0.1, theta=theta, hs_channel=1)
    ch = Chain(m, n_delay=n_delay, n_stab=5, seed=9, field=random_field(m.M, m.N, 5))
    ch.G = m.wrap(ch.G, ch.field[0])
    ch.update_slice(1, 0)
    assert ch.accepted > 0
    assert np.abs(ch.G - m.green_direct(ch.field, 1)).max() < 1e-11


def test_charge_delayed_equals_local_sweep():
    m = Model(2, U=3.73, beta=1.0, dtau=0.1, hs_channel=1)
    a = Chain(m, n_delay=1, n_stab=5, seed=4, field=random_field(m.M, m.N, 21))
    b = Chain(m, n_delay=4, n_stab=5, seed=4, field=random_field(m.M, m.N, 21))
    a.sweep()
    b.sweep()
    assert np.array_equal(a.field, b.field) and a.accepted == b.accepted > 0
    assert np.abs(a.G - m.green_direct(a.field, 0)).max() < 1e-11
    assert np.abs(a.G - b.G).max() < 1e-11


def test_charge_hubbard_atom_closed_form():
    """t = 0: the decoupling is exact and slices commute: D = 1 / (2 (1 + e^{beta U / 2}))."""
    m = Model(1, t=0.0, U=3.0, beta=1.2, dtau=0.3, hs_channel=1)     # 2 sites, 4 slices, 2^8 fields
    avg = hs_enum.hs_average(m, keys=("double_occ",))
    assert abs(avg["double_occ"] - 1.0 / (2.0 * (1.0 + np.exp(m.beta * m.U / 2.0)))) < 1e-12


@pytest.mark.parametrize("theta", [(0.0, 0.0), (0.3, 0.7)])
def test_charge_hs_sum_equals_trotter_ed_two_sites(theta):
    """L = 1 (two sites, three bonds), M = 4: exhaustive HS-n sum equals the Trotterised ED."""
    m = Model(1, U=4.0, beta=0.8, dtau=0.2, theta=theta, hs_channel=1)
    ref = ed.trotter_averages(m.lat, m.K, m.U, m.dtau, m.M)
    got = hs_enum.hs_average(m, keys=("double_occ", "energy", "ekin", "Czz", "chi_e"))
    for k in ("double_occ", "energy", "ekin", "chi_e"):
        assert abs(got[k] - ref[k]) < 1e-10, k
    assert np.abs(got["Czz"] - ref["Czz"]).max() < 1e-10


@pytest.mark.slow
def test_charge_hs_sum_equals_trotter_ed_twisted():
    """L = 2 (8 sites), M = 2, twisted: the same exact identity on a cluster with distinct neighbours."""
    m = Model(2, U=4.0, beta=0.4, dtau=0.2, theta=TW, hs_channel=1)
    ref = ed.trotter_averages(m.lat, m.K, m.U, m.dtau, m.M)
    got = hs_enum.hs_average(m, keys=("double_occ", "energy", "ekin", "Czz", "chi_e"))
    for k in ("double_occ", "energy", "ekin", "chi_e"):
        assert abs(got[k] - ref[k]) < 1e-10, k
    assert np.abs(got["Czz"] - ref["Czz"]).max() < 1e-10
