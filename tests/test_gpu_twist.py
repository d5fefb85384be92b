"""Twisted boundaries (complex G, Sec. III.C) on the GPU against the oracle.

The device holds every complex matrix as its real 2N x 2N embedding; these
tests see only the complex N x N matrices of the C ABI.  Tolerances as for the
periodic path: 1e-12 relative for one propagation, 1e-10 for stabilised G,
ratios and observables, exact fields and acceptance counts in lockstep."""
import numpy as np
import pytest

from synth import random_field, random_matrix

pytestmark = pytest.mark.gpu

TOL = 1e-10
TW = (0.25, 0.5)


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_14668_b300 as p
    return p


def rel_err(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def make(pkg, L, beta, dtau, U, n_delay, n_stab, seed=1, measure=0, theta=TW, precision=0):
    return pkg.Chain(pkg.make_params(L=L, beta=beta, dtau=dtau, U=U, n_delay=n_delay, n_stab=n_stab,
                                     seed=seed, measure=measure, theta=theta, precision=precision))


def cmatrix(N, seed):
    return random_matrix(N, seed) + 1j * random_matrix(N, seed + 1000)


@pytest.mark.parametrize("L,theta", [(1, (0.5, 0.25)), (2, TW), (3, (0.1, 0.9)), (6, TW)])
def test_wrap_parity_twisted(pkg, L, theta):
    from oracle.dqmc import Model
    m = Model(L, U=3.73, beta=0.4, dtau=0.1, theta=theta)
    ch = make(pkg, L, 0.4, 0.1, 3.73, 4, 4, theta=theta)
    f = random_field(m.M, m.N, 100 + L)
    ch.set_field(f)
    A = cmatrix(m.N, 7 + L)
    l = 3
    assert rel_err(pkg.afqmc_wrap_matrix(ch.h, l, +1, A), m.wrap(A, f[l - 1])) < 1e-12
    assert rel_err(pkg.afqmc_wrap_matrix(ch.h, l, -1, A), m.unwrap(A, f[l - 1])) < 1e-12
    assert rel_err(pkg.afqmc_wrap_matrix(ch.h, l, 0, A), m.Eh @ A @ m.Ehinv) < 1e-12
    ch.close()


@pytest.mark.parametrize("L,beta,ns", [(2, 2.0, 5), (3, 3.0, 10), (6, 6.0, 10)])
def test_green_parity_twisted(pkg, L, beta, ns):
    from oracle.dqmc import Model
    m = Model(L, U=3.73, beta=beta, dtau=0.1, theta=TW)
    f = random_field(m.M, m.N, 31 + L)
    ch = make(pkg, L, beta, 0.1, 3.73, 4, ns)
    ch.set_field(f)
    for l in (0, 1, m.M // 2 + 1, m.M):
        G = ch.green(l)
        assert G.dtype == np.complex128
        assert rel_err(G, m.green_stable(f, l, ns)) < TOL, l
    ch.close()


def test_green_U0_twisted(pkg):
    """U = 0 with a twist: G = (1 + e^{-beta K'})^-1 of the complex hopping matrix."""
    from oracle.dqmc import Model
    m = Model(6, U=0.0, beta=6.0, dtau=0.1, theta=TW)
    ch = make(pkg, 6, 6.0, 0.1, 0.0, 4, 10)
    w, V = np.linalg.eigh(m.K)
    Gc = (V / (1.0 + np.exp(-m.beta * w))[None, :]) @ V.conj().T
    assert np.abs(Gc.imag).max() > 1e-3
    assert rel_err(ch.green(0), Gc) < 1e-12
    ch.close()


def test_det_ratio_parity_twisted(pkg):
    from oracle.dqmc import Model, local_ratio
    m = Model(3, U=3.73, beta=1.0, dtau=0.1, theta=TW)
    f = random_field(m.M, m.N, 5)
    ch = make(pkg, 3, 1.0, 0.1, 3.73, 4, 5)
    ch.set_field(f)
    for l, i in ((1, 0), (5, 7), (10, 17)):
        R, r = pkg.afqmc_det_ratio(ch.h, l, i)
        Ro, ro, _ = local_ratio(m, m.green_stable(f, l, 5), i, float(f[l - 1, i]))
        assert abs(np.imag(ro)) > 1e-8
        assert abs(R - Ro) <= TOL * abs(Ro) and abs(r - ro) <= TOL * abs(ro)
    ch.close()


@pytest.mark.parametrize("L,n_delay", [(2, 1), (3, 4), (6, 3), (6, 16), (6, 64)])
def test_update_slice_lockstep_twisted(pkg, L, n_delay):
    """Paired rank-1 moves of the embedding take the oracle's complex decisions."""
    from oracle.dqmc import Model, Chain
    m = Model(L, U=3.73, beta=1.0, dtau=0.1, theta=TW)
    f = random_field(m.M, m.N, 40 + L)
    oc = Chain(m, n_delay=n_delay, n_stab=5, seed=77, field=f)
    ch = make(pkg, L, 1.0, 0.1, 3.73, n_delay, 5, seed=77)
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


@pytest.mark.parametrize("L,beta,n_delay,ns", [(3, 3.0, 4, 10), (6, 2.0, 32, 10)])
def test_sweep_lockstep_twisted(pkg, L, beta, n_delay, ns):
    from oracle.dqmc import Model, Chain
    m = Model(L, U=3.73, beta=beta, dtau=0.1, theta=TW)
    oc = Chain(m, n_delay=n_delay, n_stab=ns, seed=2024)
    ch = make(pkg, L, beta, 0.1, 3.73, n_delay, ns, seed=2024)
    assert np.array_equal(ch.field(), oc.field)
    st = ch.sweep(1)
    oc.sweep()
    assert st.proposed == 2 * m.N * m.M
    assert st.accepted == oc.accepted
    assert st.max_stab_drift < 1e-8
    assert np.array_equal(ch.field(), oc.field)
    assert rel_err(ch.green(0), oc.G) < TOL
    ch.close()


def test_measure_parity_twisted(pkg):
    from oracle.dqmc import Model
    from oracle.observables import measure
    m = Model(6, U=3.73, beta=2.0, dtau=0.1, theta=TW)
    f = random_field(m.M, m.N, 9)
    ch = make(pkg, 6, 2.0, 0.1, 3.73, 8, 10)
    ch.set_field(f)
    got = ch.measure()
    ref = measure(m, m.green_stable(f, 0, 10))
    for k in ("energy", "double_occ", "ekin", "density", "m2", "S_af", "S_af_dk", "R_m2", "Czz_half", "chi_e"):
        assert abs(got[k] - ref[k]) <= TOL * max(1.0, abs(ref[k])), k
    assert rel_err(got["Czz"], ref["Czz"].reshape(-1)) < TOL
    assert rel_err(got["nk"], ref["nk"].reshape(m.lat.Nc, 2, 2)) < TOL
    ch.close()


def test_twisted_split_tf32_flush(pkg):
    """The split-TF32 flush also serves the embedding: one slice update stays
    within the precision-1 tolerance of the FP64 oracle."""
    from oracle.dqmc import Model, Chain
    m = Model(6, U=3.73, beta=1.0, dtau=0.1, theta=TW)
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
