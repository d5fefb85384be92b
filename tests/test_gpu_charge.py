"""Charge-channel Ising field (HS-n, Eq. DensityHS) on the GPU against the oracle.

B_l = e^{i alpha diag(s_l)} E makes G complex even without a twist, so the
device holds it as its real 2N x 2N embedding and a flip is one complex rank-1
move, i.e. two simultaneous real moves of the embedding.  Tolerances as for the
spin channel: 1e-12 relative for one propagation, 1e-10 for stabilised G,
ratios and observables, exact fields and acceptance counts in lockstep."""
import numpy as np
import pytest

from synth import random_field, random_matrix

pytestmark = pytest.mark.gpu

TOL = 1e-10
TW = (0.25, 0.5)
PBC = (0.0, 0.0)


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_14668_b300 as p
    return p


def rel_err(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def make(pkg, L, beta, dtau, U, n_delay, n_stab, seed=1, measure=0, theta=PBC, precision=0):
    return pkg.Chain(pkg.make_params(L=L, beta=beta, dtau=dtau, U=U, n_delay=n_delay, n_stab=n_stab,
                                     seed=seed, measure=measure, theta=theta, precision=precision, hs_channel=1))


def model(L, beta, theta=PBC, U=3.73, dtau=0.1):
    from oracle.dqmc import Model
    return Model(L, U=U, beta=beta, dtau=dtau, theta=theta, hs_channel=1)


def cmatrix(N, seed):
    return random_matrix(N, seed) + 1j * random_matrix(N, seed + 1000)


@pytest.mark.parametrize("L,theta", [(2, PBC), (3, TW), (6, PBC)])
def test_wrap_parity_charge(pkg, L, theta):
    m = model(L, 0.4, theta)
    ch = make(pkg, L, 0.4, 0.1, 3.73, 4, 4, theta=theta)
    f = random_field(m.M, m.N, 100 + L)
    ch.set_field(f)
    A = cmatrix(m.N, 7 + L)
    l = 3
    assert rel_err(pkg.afqmc_wrap_matrix(ch.h, l, +1, A), m.wrap(A, f[l - 1])) < 1e-12
    assert rel_err(pkg.afqmc_wrap_matrix(ch.h, l, -1, A), m.unwrap(A, f[l - 1])) < 1e-12
    ch.close()


@pytest.mark.parametrize("L,beta,ns,theta", [(2, 2.0, 5, PBC), (3, 3.0, 10, TW), (6, 2.0, 10, PBC)])
def test_green_parity_charge(pkg, L, beta, ns, theta):
    m = model(L, beta, theta)
    f = random_field(m.M, m.N, 31 + L)
    ch = make(pkg, L, beta, 0.1, 3.73, 4, ns, theta=theta)
    ch.set_field(f)
    for l in (0, 1, m.M // 2 + 1, m.M):
        G = ch.green(l)
        assert G.dtype == np.complex128
        assert np.abs(G.imag).max() > 1e-3
        assert rel_err(G, m.green_stable(f, l, ns)) < TOL, l
    ch.close()


@pytest.mark.parametrize("theta", [PBC, TW])
def test_det_ratio_parity_charge(pkg, theta):
    from oracle.dqmc import local_ratio
    m = model(3, 1.0, theta)
    f = random_field(m.M, m.N, 5)
    ch = make(pkg, 3, 1.0, 0.1, 3.73, 4, 5, theta=theta)
    ch.set_field(f)
    for l, i in ((1, 0), (5, 7), (10, 17)):
        R, r = pkg.afqmc_det_ratio(ch.h, l, i)
        Ro, ro, _ = local_ratio(m, m.green_stable(f, l, 5), i, float(f[l - 1, i]))
        assert abs(np.imag(ro)) > 1e-8
        assert abs(R - Ro) <= TOL * abs(Ro) and abs(r - ro) <= TOL * abs(ro)
    ch.close()


@pytest.mark.parametrize("L,n_delay,theta", [(2, 1, PBC), (3, 4, TW), (6, 3, PBC), (6, 16, TW), (6, 64, PBC)])
def test_update_slice_lockstep_charge(pkg, L, n_delay, theta):
    """Complex flips as paired moves of the embedding take the oracle's decisions."""
    from oracle.dqmc import Chain
    m = model(L, 1.0, theta)
    f = random_field(m.M, m.N, 40 + L)
    oc = Chain(m, n_delay=n_delay, n_stab=5, seed=77, field=f)
    ch = make(pkg, L, 1.0, 0.1, 3.73, n_delay, 5, seed=77, theta=theta)
    ch.set_field(f)
    l = 4
    G0 = m.green_stable(f, l, 5)
    oc.G = G0.copy()
    oc.update_slice(l, 0)
    Gg, nacc = pkg.afqmc_update_slice(ch.h, l, 0, 0, G0)
    assert nacc == oc.accepted > 0
    assert np.array_equal(ch.field()[l - 1], oc.field[l - 1])
    assert rel_err(Gg, oc.G) < TOL
    ch.close()


@pytest.mark.parametrize("L,theta", [(2, PBC), (3, TW)])
def test_forced_flips_charge(pkg, L, theta):
    """Flipping a fixed set of sites of one slice (several pairs per window, across a
    window boundary at L = 3): the sum of log |r|^2 equals the brute-force
    log-weight change and G equals the fresh Green's function of the new field."""
    m = model(L, 1.0, theta)
    f = random_field(m.M, m.N, 90 + L)
    ch = make(pkg, L, 1.0, 0.1, 3.73, 4, 5, theta=theta)
    ch.set_field(f)
    l = 3
    mask = np.zeros(m.N, dtype=np.int8)
    mask[[0, 1, 3, m.N // 2, m.N - 2, m.N - 1]] = 1
    G, lr = pkg.afqmc_force_slice(ch.h, l, mask, m.green_direct(f, l))
    f2 = f.copy()
    f2[l - 1] = np.where(mask == 1, -f[l - 1], f[l - 1])
    assert np.array_equal(ch.field(), f2)
    lw0, _ = m.log_weight(f)
    lw1, _ = m.log_weight(f2)
    assert abs(lr - (lw1 - lw0)) < 1e-9
    assert rel_err(G, m.green_direct(f2, l)) < 1e-10
    ch.close()


@pytest.mark.parametrize("L,beta,n_delay,ns,theta", [(3, 3.0, 4, 10, PBC), (3, 2.0, 8, 5, TW), (6, 2.0, 32, 10, PBC)])
def test_sweep_lockstep_charge(pkg, L, beta, n_delay, ns, theta):
    from oracle.dqmc import Chain
    m = model(L, beta, theta)
    oc = Chain(m, n_delay=n_delay, n_stab=ns, seed=2024)
    ch = make(pkg, L, beta, 0.1, 3.73, n_delay, ns, seed=2024, theta=theta)
    assert np.array_equal(ch.field(), oc.field)
    st = ch.sweep(1)
    oc.sweep()
    assert st.proposed == 2 * m.N * m.M
    assert st.accepted == oc.accepted
    assert st.max_stab_drift < 1e-8
    assert np.array_equal(ch.field(), oc.field)
    assert rel_err(ch.green(0), oc.G) < TOL
    ch.close()


@pytest.mark.parametrize("theta", [PBC, TW])
def test_measure_parity_charge(pkg, theta):
    from oracle.observables import measure
    m = model(6, 2.0, theta)
    f = random_field(m.M, m.N, 9)
    ch = make(pkg, 6, 2.0, 0.1, 3.73, 8, 10, theta=theta)
    ch.set_field(f)
    got = ch.measure()
    ref = measure(m, m.green_stable(f, 0, 10))
    for k in ("energy", "double_occ", "ekin", "density", "m2", "S_af", "S_af_dk", "R_m2", "Czz_half", "chi_e"):
        assert abs(got[k] - ref[k]) <= TOL * max(1.0, abs(ref[k])), k
    assert rel_err(got["Czz"], ref["Czz"].reshape(-1)) < TOL
    assert rel_err(got["nk"], ref["nk"].reshape(m.lat.Nc, 2, 2)) < TOL
    ch.close()


@pytest.mark.parametrize("L,beta,ns,theta", [(2, 1.0, 5, PBC), (3, 1.2, 3, TW)])
def test_time_displaced_charge(pkg, L, beta, ns, theta):
    """C_{H_I}(tau) of one field through the charge-channel propagators (Eqs. DouOccDerive, fidelitysusp)."""
    from oracle import tdgf
    m = model(L, beta, theta)
    f = random_field(m.M, m.N, 17 + L)
    ch = make(pkg, L, beta, 0.1, 3.73, 4, ns, seed=3, theta=theta)
    ch.set_field(f)
    pkg.afqmc_measure_td(ch.h)
    C, dDdU, chiF, n = pkg.afqmc_get_td(ch.h)
    assert n == 1
    ref = [tdgf.hi_products(m, f, l) for l in range(m.M // 2 + 1)]
    Cref = np.array([r[0] - ref[0][1] ** 2 for r in ref])
    scale = max(np.abs([r[0] for r in ref]).max(), ref[0][1] ** 2)
    assert np.abs(C - Cref).max() <= 1e-9 * scale
    ch.close()


def test_charge_tensor_core_products_lockstep(pkg):
    """Precision bit 1 (FP64-accurate stabilisation products) keeps the oracle's decisions."""
    from oracle.dqmc import Chain
    m = model(6, 2.0, PBC)
    oc = Chain(m, n_delay=16, n_stab=10, seed=5)
    ch = make(pkg, 6, 2.0, 0.1, 3.73, 16, 10, seed=5, precision=2)
    ch.sweep(1)
    oc.sweep()
    assert np.array_equal(ch.field(), oc.field)
    assert rel_err(ch.green(0), oc.G) < TOL
    ch.close()


def test_charge_split_tf32_flush(pkg):
    """The split-TF32 flush also serves the paired complex moves: one slice update
    stays within the precision-1 tolerance of the FP64 oracle."""
    from oracle.dqmc import Chain
    m = model(6, 1.0, PBC)
    f = random_field(m.M, m.N, 61)
    oc = Chain(m, n_delay=16, n_stab=5, seed=3, field=f)
    ch = make(pkg, 6, 1.0, 0.1, 3.73, 16, 5, seed=3, precision=1)
    ch.set_field(f)
    G0 = m.green_stable(f, 2, 5)
    oc.G = G0.copy()
    oc.update_slice(2, 0)
    Gg, nacc = pkg.afqmc_update_slice(ch.h, 2, 0, 0, G0)
    assert nacc == oc.accepted > 0
    assert rel_err(Gg, oc.G) < 1e-5
    ch.close()


def test_charge_chain_matches_trotter_ed(pkg):
    """Two-site cluster (L = 1): the charge-channel chain reproduces the Trotterised
    ED within 4 sigma for D and e, as the spin channel does (both decouplings are exact)."""
    from oracle import ed
    from oracle.lattice import Honeycomb
    U, beta, dtau = 3.0, 1.2, 0.2
    lat = Honeycomb(1)
    ref = ed.trotter_averages(lat, lat.hopping_matrix(), U, dtau, 6)
    ch = make(pkg, 1, beta, dtau, U, 2, 3, seed=8, measure=1)
    ch.sweep(200)
    ch.observables()                           # discard the warm-up measurements
    bins = {"double_occ": [], "energy": []}
    for _ in range(30):
        ch.sweep(100)
        o = ch.observables()
        for k in bins:
            bins[k].append(o[k])
    for k, v in bins.items():
        v = np.array(v)
        mean, err = v.mean(), v.std(ddof=1) / np.sqrt(len(v))
        assert abs(mean - ref[k]) < 4.0 * err + 1e-12, (k, mean, err, ref[k])
    ch.close()
