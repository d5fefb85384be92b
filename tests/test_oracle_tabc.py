"""Twist-averaged boundary conditions (Sec. III.C): the quasi-random twist
sequence, pinned by the first terms of the van der Corput sequences, by the
elementary-interval property of the Halton sequence, and by what TABC is for
(a smaller finite-size error than periodic boundaries at U = 0); the library's
host-only generator must reproduce the oracle's values bit for bit."""
import itertools

import numpy as np
import pytest

from oracle import tabc
from oracle.lattice import Honeycomb


def test_first_terms_of_the_van_der_corput_sequences():
    assert [tabc.radical_inverse(m, 2) for m in range(8)] == [0, 1 / 2, 1 / 4, 3 / 4, 1 / 8, 5 / 8, 3 / 8, 7 / 8]
    from fractions import Fraction as F
    assert [tabc.radical_inverse(m, 3) for m in range(10)] == [
        F(0), F(1, 3), F(2, 3), F(1, 9), F(4, 9), F(7, 9), F(2, 9), F(5, 9), F(8, 9), F(1, 27)]


@pytest.mark.parametrize("a,b", [(1, 1), (2, 1), (3, 2), (4, 2), (2, 3)])
@pytest.mark.parametrize("block", [0, 1, 5])
def test_halton_elementary_intervals(a, b, block):
    """Any 2^a 3^b consecutive points starting at a multiple of 2^a 3^b put exactly
    one point in each box [i 2^-a, (i+1) 2^-a) x [j 3^-b, (j+1) 3^-b)."""
    n0 = 2 ** a * 3 ** b
    th = tabc.halton_twists(n0, start=block * n0)
    counts = np.zeros((2 ** a, 3 ** b), dtype=int)
    for t1, t2 in th:
        counts[int(t1 * 2 ** a), int(t2 * 3 ** b)] += 1
    assert (counts == 1).all()


def test_prefixes_stay_evenly_spread():
    """The cumulative property: every prefix of N points, N = 1..64, leaves no
    quarter of the square with more than N/4 + 2.5 points (i.i.d. uniform points
    exceed N/4 + 5 in half of the draws)."""
    th = tabc.halton_twists(64, start=1)
    for n in range(1, 65):
        q = np.zeros((2, 2), dtype=int)
        for t1, t2 in th[:n]:
            q[int(2 * t1), int(2 * t2)] += 1
        assert q.max() <= n / 4 + 2.5, n


def test_library_generator_matches_oracle():
    """afqmc_quasirandom_twists (host code of libafqmc.so, no device work)."""
    import paper_2609_14668_b300 as pkg
    for start, n in ((1, 14), (0, 50), (1000, 37), (2 ** 20 + 3, 8)):
        got = pkg.afqmc_quasirandom_twists(n, start)
        assert np.array_equal(got, tabc.halton_twists(n, start))
    assert pkg.afqmc_quasirandom_twists(0).shape == (0, 2)
    with pytest.raises(pkg.AfqmcError):
        pkg.afqmc_quasirandom_twists(-1)
    with pytest.raises(pkg.AfqmcError):
        pkg.afqmc_quasirandom_twists(10, 2 ** 31 - 5)


def _free_energy(L, theta, beta):
    """Kinetic energy per site of both spins at U = 0: (2 / N) sum_levels e f(e)."""
    lat = Honeycomb(L, theta=tuple(theta))
    w = np.linalg.eigvalsh(lat.hopping_matrix())
    return 2.0 * np.sum(w / (1.0 + np.exp(beta * w))) / lat.N


def _free_energy_bloch(L, theta, beta):
    """The same from the Bloch bands +-|f(k)| on the grid of Eq. kpoints (large L)."""
    lat = Honeycomb(L, theta=tuple(theta))
    e = np.abs(lat.f_of_k(lat.kvectors()))
    return 2.0 * np.sum(-e * np.tanh(beta * e / 2.0)) / lat.N


@pytest.mark.parametrize("L", [4, 5, 6, 7])
def test_twist_average_reduces_finite_size_error(L):
    """U = 0, beta t = 10: the mean over the first 14 twists of the sequence is at
    least 5x closer to the large-lattice value than the periodic lattice."""
    beta = 10.0
    assert abs(_free_energy_bloch(L, (0.3, 0.6), beta) - _free_energy(L, (0.3, 0.6), beta)) < 1e-12
    ref = _free_energy_bloch(300, (0.2, 0.7), beta)
    pbc = _free_energy(L, (0.0, 0.0), beta)
    tab = tabc.twist_average([_free_energy(L, t, beta) for t in tabc.halton_twists(14)])
    assert abs(tab - ref) * 5.0 < abs(pbc - ref)
