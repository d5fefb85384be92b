"""Pins of the CPU oracle against facts fixed by the paper and by mathematics:
closed forms (U = 0 Fermi function, Hubbard atom, Bloch spectrum), exact
diagonalisation, brute-force determinants and inverses, and library routines.
Each test targets a mistake the oracle could plausibly contain."""
import os

import numpy as np
import pytest
import scipy.linalg as sla

from oracle.lattice import Honeycomb
from oracle.linalg import expm_taylor, udt, stable_green
from oracle.dqmc import Model, Chain, local_ratio
from oracle.observables import measure
from oracle import ed, rng, enumerate as hs_enum
from synth import random_field

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- lattice
@pytest.mark.parametrize("L,theta", [(3, (0.0, 0.0)), (4, (0.0, 0.0)), (3, (0.25, 0.6)), (2, (0.5, 0.0))])
def test_spectrum_matches_bloch_function(L, theta):
    """Real-space K (built from bonds + Peierls phases) has eigenvalues +-|f(k)|
    on the twisted grid of Eq. kpoints (Eq. h0kMat)."""
    lat = Honeycomb(L, theta=theta)
    ev = np.sort(np.linalg.eigvalsh(lat.hopping_matrix()))
    fk = np.abs([lat.f_of_k(k) for k in lat.kvectors()])
    assert np.allclose(ev, np.sort(np.concatenate([fk, -fk])), atol=1e-12)


def test_neighbours_and_symmetry():
    for L in (2, 3, 6):
        lat = Honeycomb(L)
        K = lat.hopping_matrix()
        assert np.array_equal(K, K.T)
        # every site has exactly three distinct neighbours with hopping -t
        assert np.all((K != 0).sum(axis=1) == 3)
        assert np.allclose(K[K != 0], -1.0)
        # bipartite: no A-A or B-B hopping
        Nc = lat.Nc
        assert not K[:Nc, :Nc].any() and not K[Nc:, Nc:].any()


def test_dirac_points_present_when_L_multiple_of_3():
    """App. B: under PBC the Dirac points lie on the grid iff 3 | L."""
    for L, has in ((3, True), (6, True), (4, False), (5, False)):
        lat = Honeycomb(L)
        fk = np.abs([lat.f_of_k(k) for k in lat.kvectors()])
        assert (fk.min() < 1e-12) == has


# ---------------------------------------------------------------- linear algebra
def test_expm_taylor_vs_library():
    lat = Honeycomb(3)
    K = lat.hopping_matrix()
    for c in (-0.1, 0.05, 0.7, -2.5):
        w, V = np.linalg.eigh(K)                 # K is real symmetric: exact spectral exponential
        ref = (V * np.exp(c * w)) @ V.T
        assert np.linalg.norm(expm_taylor(c * K) - ref, 2) <= 1e-14 * np.linalg.norm(ref, 2)
        assert np.linalg.norm(expm_taylor(c * K) - sla.expm(c * K), 2) <= 1e-11 * np.linalg.norm(ref, 2)
    E = expm_taylor(-0.1 * K)
    assert np.allclose(E @ expm_taylor(0.1 * K), np.eye(lat.N), atol=1e-14)


def test_block_form_of_propagator():
    """U E U^+ is block diagonal with the 2x2 blocks e^{-dtau h(k)} (Eqs. NewBlMat, ExpLambda, FourierMat)."""
    L, dtau = 4, 0.1
    lat = Honeycomb(L)
    E = expm_taylor(-dtau * lat.hopping_matrix())
    ks = lat.kvectors()
    r = np.array([lat.bravais_vector(*lat.cell_coords(c)) for c in range(lat.Nc)])
    UA = np.exp(-1j * ks @ r.T) / L
    Ufull = sla.block_diag(UA, UA)
    Lam = Ufull @ E @ Ufull.conj().T
    for q, k in enumerate(ks):
        f = lat.f_of_k(k)
        h = np.array([[0, f], [np.conj(f), 0]])
        blk = Lam[np.ix_([q, lat.Nc + q], [q, lat.Nc + q])]
        assert np.allclose(blk, sla.expm(-dtau * h), atol=1e-13)
    # and nothing outside the blocks
    mask = np.ones_like(Lam, dtype=bool)
    for q in range(lat.Nc):
        mask[np.ix_([q, lat.Nc + q], [q, lat.Nc + q])] = False
    assert np.abs(Lam[mask]).max() < 1e-13


def test_udt_reconstructs():
    A = np.random.default_rng(1).standard_normal((12, 12)) * np.logspace(0, 12, 12)[None, :]
    U, D, T = udt(A)
    assert np.allclose(U.T @ U, np.eye(12), atol=1e-14)
    assert np.all(D > 0)
    assert np.allclose((U * D) @ T, A, rtol=1e-12, atol=1e-12 * np.abs(A).max())


# ---------------------------------------------------------------- closed forms
def fermi_green_U0(lat, beta):
    """G = (1 + e^{-beta K})^-1 from k space: G_k = 1/2 + tanh(beta|f|/2)/(2|f|) h(k) at the
    (shifted) momentum k = q + A, Fourier sum to r space over the cell grid q (Gauge-I)."""
    Nc = lat.Nc
    r = np.array([lat.bravais_vector(*lat.cell_coords(c)) for c in range(Nc)])
    G = np.zeros((lat.N, lat.N), dtype=complex)
    for k, q in zip(lat.kvectors(), lat.qvectors()):
        f = lat.f_of_k(k)
        af = abs(f)
        c = 0.5 * beta if af < 1e-14 else np.tanh(0.5 * beta * af) / (2.0 * af)
        Gk = np.array([[0.5, c * f], [c * np.conj(f), 0.5]])
        ph = np.exp(1j * r @ q)
        P = np.outer(ph, ph.conj()) / Nc                # e^{i k (r_I - r_J)} / Nc
        for a in (0, 1):
            for b in (0, 1):
                G[a * Nc:(a + 1) * Nc, b * Nc:(b + 1) * Nc] += Gk[a, b] * P
    return G


@pytest.mark.parametrize("L,beta,dtau,ns", [(2, 2.0, 0.1, 5), (3, 3.0, 0.1, 10), (6, 6.0, 0.1, 10), (3, 12.0, 0.1, 8)])
def test_U0_green_closed_form(L, beta, dtau, ns):
    m = Model(L, U=0.0, beta=beta, dtau=dtau)
    Gc = fermi_green_U0(m.lat, beta)
    assert np.abs(Gc.imag).max() < 1e-12
    field = random_field(m.M, m.N, 3)
    for l in (0, m.M // 2, m.M):
        G = m.green_stable(field, l, ns)
        assert np.abs(G - Gc.real).max() < 1e-12


def test_U0_observables_closed_form():
    L, beta = 3, 3.0
    m = Model(L, U=0.0, beta=beta, dtau=0.1)
    G = m.green_stable(random_field(m.M, m.N, 1), 0, 10)
    o = measure(m, G)
    fk = np.abs([m.lat.f_of_k(k) for k in m.lat.kvectors()])
    e_exact = -(2.0 / m.N) * np.sum(fk * np.tanh(0.5 * beta * fk))
    assert abs(o["double_occ"] - 0.25) < 1e-12
    assert abs(o["energy"] - e_exact) < 1e-12
    assert abs(o["density"] - 1.0) < 1e-12
    # n(k)_{ab} = [(1 + e^{beta h(k)})^-1]_{ba}  (Eq. nkMatrix)
    for q, k in enumerate(m.lat.kvectors()):
        f = m.lat.f_of_k(k)
        h = np.array([[0, f], [np.conj(f), 0]])
        nF = np.linalg.inv(np.eye(2) + sla.expm(beta * h))
        l1, l2 = q % L, q // L
        assert np.allclose(o["nk"][l2, l1], nF.T, atol=1e-12)


def test_hubbard_atom_closed_form():
    """t = 0: the HS identity is exact and slices commute: D = 1 / (2 (1 + e^{beta U / 2}))."""
    m = Model(1, t=0.0, U=3.0, beta=1.2, dtau=0.3)     # 2 sites, 4 slices, 2^8 fields
    avg = hs_enum.hs_average(m, keys=("double_occ",))
    assert abs(avg["double_occ"] - 1.0 / (2.0 * (1.0 + np.exp(m.beta * m.U / 2.0)))) < 1e-12


# ---------------------------------------------------------------- brute force
def test_stable_green_equals_plain_inverse():
    m = Model(3, U=3.73, beta=2.0, dtau=0.1)
    field = random_field(m.M, m.N, 7)
    for l in (0, 3, 10, 20):
        for ns in (1, 4, 10):
            assert np.abs(m.green_stable(field, l, ns) - m.green_direct(field, l)).max() < 1e-11


def test_wrap_moves_between_slices():
    m = Model(3, U=3.73, beta=2.0, dtau=0.1)
    field = random_field(m.M, m.N, 8)
    G = m.green_direct(field, 4)
    # the plain inverses carry ~1e-12 rounding at beta t = 2
    assert np.abs(m.wrap(G, field[4]) - m.green_direct(field, 5)).max() < 1e-11
    assert np.abs(m.unwrap(G, field[3]) - m.green_direct(field, 3)).max() < 1e-11


def test_ratio_equals_weight_ratio():
    """R = e^{2 gamma s} r^2 equals W(X')/W(X) from brute-force determinants (Eq. DRatio)."""
    m = Model(2, U=3.73, beta=1.0, dtau=0.1)
    field = random_field(m.M, m.N, 11)
    lw0, _ = m.log_weight(field)
    for l, i in ((1, 0), (4, 5), (10, 7)):
        G = m.green_direct(field, l)
        R, r, _ = local_ratio(m, G, i, float(field[l - 1, i]))
        f2 = field.copy()
        f2[l - 1, i] *= -1
        lw1, _ = m.log_weight(f2)
        assert abs(R - np.exp(lw1 - lw0)) < 1e-10 * max(1.0, R)
        # r itself: det(1 + B'..)/det(1 + B..) on the spin-up determinant
        d0 = np.linalg.det(np.eye(m.N) + m.chain_product(field, 1, m.M))
        d1 = np.linalg.det(np.eye(m.N) + m.chain_product(f2, 1, m.M))
        assert abs(r - d1 / d0) < 1e-10 * max(1.0, abs(r))


@pytest.mark.parametrize("n_delay", [1, 3, 64])
def test_slice_update_matches_fresh_green(n_delay):
    """After the delayed update of one slice, G equals (1 + R L)^-1 of the new field."""
    m = Model(3, U=3.73, beta=1.0, dtau=0.1)
    field = random_field(m.M, m.N, 5)
    ch = Chain(m, n_delay=n_delay, n_stab=5, seed=9, field=field)
    l = 1
    ch.G = m.wrap(ch.G, ch.field[0])
    ch.update_slice(l, 0)
    assert ch.accepted > 0
    assert np.abs(ch.G - m.green_direct(ch.field, l)).max() < 1e-11


def test_delayed_equals_local_sweep():
    m = Model(3, U=3.73, beta=1.0, dtau=0.1)
    f0 = random_field(m.M, m.N, 21)
    a = Chain(m, n_delay=1, n_stab=5, seed=4, field=f0)
    b = Chain(m, n_delay=4, n_stab=5, seed=4, field=f0)
    for _ in range(2):
        a.sweep()
        b.sweep()
    assert np.array_equal(a.field, b.field)
    assert np.abs(a.G - b.G).max() < 1e-11
    assert a.accepted == b.accepted > 0


def test_sweep_green_is_fresh_green():
    m = Model(3, U=3.73, beta=2.0, dtau=0.1)
    ch = Chain(m, n_delay=4, n_stab=10, seed=2)
    ch.sweep()
    assert ch.proposed == 2 * m.N * m.M
    assert np.abs(ch.G - m.green_direct(ch.field, 0)).max() < 1e-11


# ---------------------------------------------------------------- RNG
def test_splitmix64_published_outputs():
    vals = [int(x, 16) for x in open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) if x.startswith("0x")]
    assert [rng.mix64(n * rng.GAMMA) for n in (1, 2, 3)] == vals


def test_uniforms_in_unit_interval():
    key = rng.chain_key(123, 0)
    u = np.array([rng.uniform(key, n) for n in range(1, 20001)])
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.01


# ---------------------------------------------------------------- exact diagonalisation
SF_KEYS = ("S_af", "S_af_dk", "m2", "Czz_half")


def check_structure_factor(m, got, ref, twisted):
    """The oracle's structure-factor step (Eqs. SzSzCrF, SpinStrucF, CrfRatio and
    m^2 = S_zz(Gamma)/(2 N_c)) against the Fock-space structure factor computed
    from the spin density directly (oracle.ed, |sum_i e^{ik.r_i} s_i|^2 per
    sublattice; no C_zz involved): S_zz(Gamma), S_zz(Gamma + b1/L), m^2 and
    C_zz(floor(L/2), 0), all as exact averages over every HS field.  R_m^2 of a
    set of configurations is 1 - <S_zz(Gamma + dk)> / <S_zz(Gamma)> (the ratio of
    the expectation values, as Eq. CrfRatio defines it)."""
    S = ref["Szz"]                                    # [l2, l1]
    assert abs(got["S_af"] - S[0, 0]) < 1e-10
    assert abs(got["S_af_dk"] - S[0, 1]) < 1e-10      # dk = b1 / L: l1 = 1, l2 = 0
    assert abs(got["m2"] - ref["m2"]) < 1e-12
    assert abs(got["Czz_half"] - ref["Czz"][0, m.lat.L1 // 2]) < 1e-10
    R_ed = 1.0 - S[0, 1] / S[0, 0]
    assert abs((1.0 - got["S_af_dk"] / got["S_af"]) - R_ed) < 1e-9
    if twisted:
        # the twist breaks the a1 <-> a2 symmetry: dk along b2 or C_zz along a2
        # would fail the checks above by far more than their tolerance
        assert abs(S[0, 1] - S[1, 0]) > 1e-6
        assert abs(ref["Czz"][0, 1] - ref["Czz"][1, 0]) > 1e-6


@pytest.mark.slow
def test_hs_sum_equals_trotter_ed():
    """Exhaustive HS sum (oracle weights + Wick) equals the Trotterised Fock-space ED exactly (L=2, 8 sites, M=2)."""
    m = Model(2, U=4.0, beta=0.4, dtau=0.2)
    ref = ed.trotter_averages(m.lat, m.K, m.U, m.dtau, m.M)
    got = hs_enum.hs_average(m, keys=("double_occ", "energy", "ekin", "Czz", "chi_e") + SF_KEYS)
    for k in ("double_occ", "energy", "ekin", "chi_e"):
        assert abs(got[k] - ref[k]) < 1e-10
    assert np.abs(got["Czz"] - ref["Czz"]).max() < 1e-10
    check_structure_factor(m, got, ref, twisted=False)


def test_trotter_ed_converges_to_thermal_ed():
    """O(dtau^2) approach of the symmetric split to exact e^{-beta H} (L=1 two-site cell, three bonds)."""
    lat = Honeycomb(1)
    K = lat.hopping_matrix()
    ex = ed.thermal_averages(lat, K, 4.0, 2.0)
    errs = [abs(ed.trotter_averages(lat, K, 4.0, 2.0 / M, M)["double_occ"] - ex["double_occ"]) for M in (16, 32, 64)]
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5


# ---------------------------------------------------------------- twisted boundaries (complex G)
TW = (0.25, 0.5)


def test_block_form_of_twisted_propagator():
    """With a twist the same (untwisted) DFT block-diagonalises E; the blocks are
    e^{-dtau h(k)} at the shifted momenta k = ((l + theta)/L) b (Eqs. GaugeIPhase, kpoints)."""
    L, dtau = 4, 0.1
    lat = Honeycomb(L, theta=(0.3, 0.7))
    E = expm_taylor(-dtau * lat.hopping_matrix())
    q0 = Honeycomb(L).kvectors()
    r = np.array([lat.bravais_vector(*lat.cell_coords(c)) for c in range(lat.Nc)])
    UA = np.exp(-1j * q0 @ r.T) / L
    Ufull = sla.block_diag(UA, UA)
    Lam = Ufull @ E @ Ufull.conj().T
    for q, k in enumerate(lat.kvectors()):
        f = lat.f_of_k(k)
        h = np.array([[0, f], [np.conj(f), 0]])
        assert np.allclose(Lam[np.ix_([q, lat.Nc + q], [q, lat.Nc + q])], sla.expm(-dtau * h), atol=1e-13)
    mask = np.ones_like(Lam, dtype=bool)
    for q in range(lat.Nc):
        mask[np.ix_([q, lat.Nc + q], [q, lat.Nc + q])] = False
    assert np.abs(Lam[mask]).max() < 1e-13


def test_expm_taylor_complex_hermitian():
    K = Honeycomb(3, theta=TW).hopping_matrix()
    assert np.iscomplexobj(K) and np.allclose(K, K.conj().T)
    w, V = np.linalg.eigh(K)
    for c in (-0.1, 0.05, -2.5):
        ref = (V * np.exp(c * w)) @ V.conj().T
        assert np.linalg.norm(expm_taylor(c * K) - ref, 2) <= 1e-14 * np.linalg.norm(ref, 2)


def test_udt_reconstructs_complex():
    rng_ = np.random.default_rng(2)
    A = (rng_.standard_normal((12, 12)) + 1j * rng_.standard_normal((12, 12))) * np.logspace(0, 12, 12)[None, :]
    U, D, T = udt(A)
    assert np.allclose(U.conj().T @ U, np.eye(12), atol=1e-14)
    assert np.all(D > 0)
    assert np.allclose((U * D) @ T, A, rtol=1e-12, atol=1e-12 * np.abs(A).max())


@pytest.mark.parametrize("L,beta,ns,theta", [(2, 2.0, 5, (0.3, 0.1)), (3, 3.0, 10, TW), (6, 6.0, 10, (0.75, 0.25))])
def test_U0_green_closed_form_twisted(L, beta, ns, theta):
    m = Model(L, U=0.0, beta=beta, dtau=0.1, theta=theta)
    Gc = fermi_green_U0(m.lat, beta)
    assert np.abs(Gc.imag).max() > 1e-3          # genuinely complex
    field = random_field(m.M, m.N, 3)
    for l in (0, m.M // 2, m.M):
        assert np.abs(m.green_stable(field, l, ns) - Gc).max() < 1e-12


def test_U0_observables_closed_form_twisted():
    L, beta = 3, 3.0
    m = Model(L, U=0.0, beta=beta, dtau=0.1, theta=TW)
    o = measure(m, m.green_stable(random_field(m.M, m.N, 1), 0, 10))
    fk = np.abs([m.lat.f_of_k(k) for k in m.lat.kvectors()])
    assert abs(o["double_occ"] - 0.25) < 1e-12
    assert abs(o["energy"] + (2.0 / m.N) * np.sum(fk * np.tanh(0.5 * beta * fk))) < 1e-12
    for q, k in enumerate(m.lat.kvectors()):
        f = m.lat.f_of_k(k)
        nF = np.linalg.inv(np.eye(2) + sla.expm(beta * np.array([[0, f], [np.conj(f), 0]])))
        assert np.allclose(o["nk"][q // L, q % L], nF.T, atol=1e-12)


def test_stable_green_equals_plain_inverse_twisted():
    m = Model(3, U=3.73, beta=2.0, dtau=0.1, theta=TW)
    field = random_field(m.M, m.N, 7)
    for l in (0, 3, 10, 20):
        for ns in (1, 4, 10):
            assert np.abs(m.green_stable(field, l, ns) - m.green_direct(field, l)).max() < 1e-11


def test_ratio_equals_weight_ratio_twisted():
    """R = e^{2 gamma s} |r|^2 equals W(X')/W(X) = e^{...} |det'|^2/|det|^2, and r the
    ratio of the complex up-spin determinants."""
    m = Model(2, U=3.73, beta=1.0, dtau=0.1, theta=TW)
    field = random_field(m.M, m.N, 11)
    lw0, _ = m.log_weight(field)
    for l, i in ((1, 0), (4, 5), (10, 7)):
        G = m.green_direct(field, l)
        R, r, _ = local_ratio(m, G, i, float(field[l - 1, i]))
        assert abs(np.imag(r)) > 1e-6
        f2 = field.copy()
        f2[l - 1, i] *= -1
        lw1, _ = m.log_weight(f2)
        assert abs(R - np.exp(lw1 - lw0)) < 1e-10 * max(1.0, R)
        d0 = np.linalg.det(np.eye(m.N) + m.chain_product(field, 1, m.M))
        d1 = np.linalg.det(np.eye(m.N) + m.chain_product(f2, 1, m.M))
        assert abs(r - d1 / d0) < 1e-10 * max(1.0, abs(r))


@pytest.mark.parametrize("n_delay", [1, 4])
def test_slice_update_matches_fresh_green_twisted(n_delay):
    m = Model(3, U=3.73, beta=1.0, dtau=0.1, theta=TW)
    ch = Chain(m, n_delay=n_delay, n_stab=5, seed=9, field=random_field(m.M, m.N, 5))
    ch.G = m.wrap(ch.G, ch.field[0])
    ch.update_slice(1, 0)
    assert ch.accepted > 0
    assert np.abs(ch.G - m.green_direct(ch.field, 1)).max() < 1e-11


def test_sweep_green_is_fresh_green_twisted():
    m = Model(2, U=3.73, beta=1.0, dtau=0.1, theta=TW)
    a = Chain(m, n_delay=1, n_stab=5, seed=4, field=random_field(m.M, m.N, 21))
    b = Chain(m, n_delay=4, n_stab=5, seed=4, field=random_field(m.M, m.N, 21))
    a.sweep()
    b.sweep()
    assert np.array_equal(a.field, b.field) and a.accepted == b.accepted > 0
    assert np.abs(a.G - m.green_direct(a.field, 0)).max() < 1e-11
    assert np.abs(a.G - b.G).max() < 1e-11


@pytest.mark.slow
def test_hs_sum_equals_trotter_ed_twisted():
    """The same exact identity with complex hopping (twist): HS sum with weights
    e^{-gamma sum s}|det|^2 and complex Wick contractions equals the Trotterised ED."""
    m = Model(2, U=4.0, beta=0.4, dtau=0.2, theta=TW)
    ref = ed.trotter_averages(m.lat, m.K, m.U, m.dtau, m.M)
    got = hs_enum.hs_average(m, keys=("double_occ", "energy", "ekin", "Czz", "chi_e") + SF_KEYS)
    for k in ("double_occ", "energy", "ekin", "chi_e"):
        assert abs(got[k] - ref[k]) < 1e-10
    assert np.abs(got["Czz"] - ref["Czz"]).max() < 1e-10
    check_structure_factor(m, got, ref, twisted=True)


@pytest.mark.parametrize("L", [3, 6])
@pytest.mark.parametrize("theta", [(0.0, 0.0), TW])
def test_U0_structure_factor_closed_form(L, theta):
    """Free fermions at half filling: the spins are independent and the diagonal
    of the per-spin Fermi matrix (1 + e^{beta h(k)})^-1 is 1/2 at every k (h(k)
    has a zero diagonal), so <c_i^+ c_j> = delta_ij / 2 within a sublattice and
    <s_i s_j> = delta_ij / 8 there.  Hence S_zz(k) = 1/8 at every k,
    m^2 = 1 / (16 N_c), C_zz(r != 0) = 0 and R_m^2 = 0."""
    m = Model(L, U=0.0, beta=float(L), dtau=0.1, theta=theta)
    o = measure(m, m.green_stable(random_field(m.M, m.N, 4), 0, 10))
    assert abs(o["S_af"] - 0.125) < 1e-12 and abs(o["S_af_dk"] - 0.125) < 1e-12
    assert abs(o["m2"] - 1.0 / (16 * m.lat.Nc)) < 1e-14
    assert abs(o["R_m2"]) < 1e-11
    assert abs(o["Czz"][0, 0] - 0.125 / 1.0) < 1e-12
    off = o["Czz"].copy()
    off[0, 0] = 0.0
    assert np.abs(off).max() < 1e-12


@pytest.mark.parametrize("theta", [(0.0, 0.0), TW])
def test_U0_charge_compressibility_closed_form(theta):
    """Free fermions: chi_e = (beta / N_s) * 2 sum_lambda f (1 - f) over the
    single-particle levels (Eq. ChiCharge; two spins, independent modes)."""
    L, beta = 3, 3.0
    m = Model(L, U=0.0, beta=beta, dtau=0.1, theta=theta)
    o = measure(m, m.green_stable(random_field(m.M, m.N, 2), 0, 10))
    lam = np.linalg.eigvalsh(m.K)
    f = 1.0 / (1.0 + np.exp(beta * lam))
    assert abs(o["chi_e"] - beta / m.N * 2.0 * np.sum(f * (1.0 - f))) < 1e-12
