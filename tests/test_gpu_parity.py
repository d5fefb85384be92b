"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerance (FP64 path): max |X_gpu - X_oracle| <= 1e-10 * max |X_oracle| for
G, ratios and observables after a stabilised recomputation; 1e-12 relative
for a single propagation step.  Accept/reject decisions and fields must agree
exactly (both sides decide in FP64 from the same counter-based uniforms)."""
import numpy as np
import pytest

from synth import random_field, random_matrix, WORKLOADS

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_14668_b300 as p
    return p


def rel_err(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def make(pkg, L, beta, dtau, U, n_delay, n_stab, seed=1, measure=0):
    return pkg.Chain(pkg.make_params(L=L, beta=beta, dtau=dtau, U=U, n_delay=n_delay, n_stab=n_stab,
                                     seed=seed, measure=measure))


@pytest.mark.parametrize("L", [1, 2, 3, 6, 24])
def test_wrap_parity(pkg, L):
    from oracle.dqmc import Model
    m = Model(L, U=3.73, beta=0.4, dtau=0.1)
    ch = make(pkg, L, 0.4, 0.1, 3.73, 4, 4)
    f = random_field(m.M, m.N, 100 + L)
    ch.set_field(f)
    A = random_matrix(m.N, 7 + L)
    l = 3
    got = pkg.afqmc_wrap_matrix(ch.h, l, +1, A)
    assert rel_err(got, m.wrap(A, f[l - 1])) < 1e-12
    got = pkg.afqmc_wrap_matrix(ch.h, l, -1, A)
    assert rel_err(got, m.unwrap(A, f[l - 1])) < 1e-12
    got = pkg.afqmc_wrap_matrix(ch.h, l, 0, A)
    assert rel_err(got, m.Eh @ A @ m.Ehinv) < 1e-12
    ch.close()


@pytest.mark.parametrize("L,beta,ns", [(2, 2.0, 5), (3, 3.0, 10), (6, 6.0, 10)])
def test_green_parity(pkg, L, beta, ns):
    from oracle.dqmc import Model
    m = Model(L, U=3.73, beta=beta, dtau=0.1)
    f = random_field(m.M, m.N, 31 + L)
    ch = make(pkg, L, beta, 0.1, 3.73, 4, ns)
    ch.set_field(f)
    for l in (0, 1, m.M // 2 + 1, m.M):
        assert rel_err(ch.green(l), m.green_stable(f, l, ns)) < TOL, l
    ch.close()


def test_green_U0_closed_form(pkg):
    """U = 0: G = (1 + e^{-beta K})^-1 for any field."""
    from oracle.dqmc import Model
    m = Model(6, U=0.0, beta=6.0, dtau=0.1)
    ch = make(pkg, 6, 6.0, 0.1, 0.0, 4, 10)
    w, V = np.linalg.eigh(m.K)
    Gc = (V / (1.0 + np.exp(-m.beta * w))[None, :]) @ V.T
    assert rel_err(ch.green(0), Gc) < 1e-12
    ch.close()


def test_det_ratio_parity(pkg):
    from oracle.dqmc import Model, local_ratio
    m = Model(3, U=3.73, beta=1.0, dtau=0.1)
    f = random_field(m.M, m.N, 5)
    ch = make(pkg, 3, 1.0, 0.1, 3.73, 4, 5)
    ch.set_field(f)
    for l, i in ((1, 0), (5, 7), (10, 17)):
        R, r = pkg.afqmc_det_ratio(ch.h, l, i)
        Ro, ro, _ = local_ratio(m, m.green_stable(f, l, 5), i, float(f[l - 1, i]))
        assert abs(R - Ro) <= TOL * abs(Ro) and abs(r - ro) <= TOL * abs(ro)
    ch.close()


@pytest.mark.parametrize("L,n_delay", [(3, 1), (3, 4), (6, 3), (6, 32), (6, 64)])
def test_update_slice_lockstep(pkg, L, n_delay):
    from oracle.dqmc import Model, Chain
    m = Model(L, U=3.73, beta=1.0, dtau=0.1)
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


@pytest.mark.parametrize("key", ["L3_beta3", "L6_beta6"])
def test_sweep_lockstep(pkg, key):
    """Same seed: the GPU chain and the oracle chain draw the same initial field,
    take the same decisions and end with the same G."""
    from oracle.dqmc import Model, Chain
    w = WORKLOADS[key]
    m = Model(w["L"], U=w["U"], beta=w["beta"], dtau=w["dtau"])
    oc = Chain(m, n_delay=w["n_delay"], n_stab=w["n_stab"], seed=2024)
    ch = make(pkg, w["L"], w["beta"], w["dtau"], w["U"], w["n_delay"], w["n_stab"], seed=2024)
    assert np.array_equal(ch.field(), oc.field)
    nsw = 2 if w["L"] <= 3 else 1
    acc = 0
    for _ in range(nsw):
        st = ch.sweep(1)
        oc.sweep()
        acc += st.accepted
        assert st.max_stab_drift < 1e-8
    assert acc == oc.accepted
    assert np.array_equal(ch.field(), oc.field)
    assert rel_err(ch.green(0), oc.G) < TOL
    ch.close()


def test_measure_parity(pkg):
    from oracle.dqmc import Model
    from oracle.observables import measure
    m = Model(6, U=3.73, beta=2.0, dtau=0.1)
    f = random_field(m.M, m.N, 9)
    ch = make(pkg, 6, 2.0, 0.1, 3.73, 8, 10)
    ch.set_field(f)
    got = ch.measure()
    ref = measure(m, m.green_stable(f, 0, 10))
    for k in ("energy", "double_occ", "ekin", "density", "m2", "S_af", "S_af_dk", "R_m2", "Czz_half", "chi_e"):
        assert abs(got[k] - ref[k]) <= TOL * max(1.0, abs(ref[k])), k
    assert rel_err(got["Czz"], ref["Czz"].reshape(-1)) < TOL
    nk_ref = ref["nk"].reshape(m.lat.Nc, 2, 2)
    assert rel_err(got["nk"], nk_ref) < TOL
    ch.close()


def test_sweep_measurements_accumulate(pkg):
    ch = make(pkg, 3, 3.0, 0.1, 3.73, 4, 10, measure=1)
    ch.sweep(2)
    o = ch.observables()
    assert o["n_samples"] == 2 * 2 * (30 // 10)
    assert abs(o["density"] - 1.0) < 1e-12
    assert 0.0 < o["double_occ"] < 0.25
    # correlation ratio of the averaged structure factors (Eq. CrfRatio on expectation values)
    assert abs(o["R_m2"] - (1.0 - o["S_af_dk"] / o["S_af"])) < 1e-14
    o2 = ch.observables()
    assert o2["n_samples"] == 0
    ch.close()


def test_full_size_slice_parity(pkg):
    """Full-size workload (L=24, N=1152): G at slice 0 from scratch, the first
    wrap and the first slice update (same uniforms) against the oracle."""
    from oracle.dqmc import Model, Chain
    w = WORKLOADS["L24_beta24"]
    m = Model(w["L"], U=w["U"], beta=w["beta"], dtau=w["dtau"])
    f = random_field(m.M, m.N, 424)
    ch = make(pkg, w["L"], w["beta"], w["dtau"], w["U"], w["n_delay"], w["n_stab"], seed=5)
    ch.set_field(f)
    G0 = m.green_stable(f, 0, w["n_stab"])
    assert rel_err(ch.green(0), G0) < TOL
    G1 = m.wrap(G0, f[0])
    assert rel_err(pkg.afqmc_wrap_matrix(ch.h, 1, +1, G0), G1) < 1e-12
    oc = Chain(m, n_delay=w["n_delay"], n_stab=w["n_stab"], seed=5, field=f)
    oc.G = G1.copy()
    oc.update_slice(1, 0)
    Gg, nacc = pkg.afqmc_update_slice(ch.h, 1, 0, 0, G1)
    assert nacc == oc.accepted > 0
    assert np.array_equal(ch.field()[0], oc.field[0])
    assert rel_err(Gg, oc.G) < TOL
    ch.close()


def test_handles_of_different_sizes_coexist(pkg):
    """Kernel shared-memory limits are process-wide: a handle created later with
    smaller needs (smaller lattice, FP64 flush) must not break an earlier one."""
    big = pkg.Chain(pkg.make_params(L=6, beta=1.0, dtau=0.1, U=3.73, n_delay=64, n_stab=5, seed=3, precision=1))
    small = pkg.Chain(pkg.make_params(L=2, beta=1.0, dtau=0.1, U=3.73, n_delay=2, n_stab=5, seed=3, precision=0))
    small.sweep(1)
    st = big.sweep(1)
    assert st.accepted > 0
    small.close()
    big.close()


def test_timing_mask_times_only_selected_families(pkg):
    ch = make(pkg, 3, 1.0, 0.1, 3.73, 4, 5)
    pkg.afqmc_set_timing(ch.h, ["update", "lu"])
    ch.sweep(1)
    t = pkg.afqmc_get_timing(ch.h)
    assert t["update"][0] == 2 * ch.M and t["update"][1] > 0
    assert t["lu"][0] > 0 and t["lu"][1] > 0
    for fam in ("propagate", "gemm", "qr"):
        assert t[fam][0] > 0 and t[fam][1] == 0.0
    with pytest.raises(pkg.AfqmcError) as e:
        pkg.afqmc_set_timing(ch.h, pkg.TIMING_ALL + 1)
    assert e.value.code == 1
    pkg.afqmc_set_timing(ch.h, 0)
    ch.close()
