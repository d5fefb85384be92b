"""Stabilisation products on the BF16 tensor cores with FP64 accuracy (Ozaki
scheme, precision bit 1), and the blocked solves of G whose couplings are such
products (precision bit 2).  Held to the FP64 parity bar: G recomputed from the
stacks matches the oracle to 1e-10 relative, a sweep takes the oracle's
decisions, with and without a twist and at the full L = 24 size.  The blocked
solves halve the system in units of 32 down to diagonal blocks of at most 64:
N = 18 and 36 are one block, N = 72 two blocks and one coupling, N = 144 and
the ragged N = 162 two levels, N = 1152 five."""
import numpy as np
import pytest

from synth import random_field, WORKLOADS

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


@pytest.mark.parametrize("L,beta,ns,theta,precision", [(3, 3.0, 10, (0.0, 0.0), 2), (6, 6.0, 10, (0.0, 0.0), 2),
                                                       (6, 6.0, 10, (0.0, 0.0), 3), (3, 3.0, 10, (0.25, 0.5), 2),
                                                       (3, 3.0, 10, (0.0, 0.0), 6), (6, 6.0, 10, (0.0, 0.0), 6),
                                                       (9, 2.0, 10, (0.0, 0.0), 7), (3, 3.0, 10, (0.25, 0.5), 6),
                                                       (6, 2.0, 10, (0.25, 0.5), 6)])
def test_green_parity(pkg, L, beta, ns, theta, precision):
    from oracle.dqmc import Model
    m = Model(L, U=3.73, beta=beta, dtau=0.1, theta=theta)
    f = random_field(m.M, m.N, 31 + L)
    ch = pkg.Chain(pkg.make_params(L=L, beta=beta, dtau=0.1, U=3.73, n_delay=4, n_stab=ns, seed=1, theta=theta,
                                   precision=precision))
    ch.set_field(f)
    for l in (0, 1, m.M // 2 + 1, m.M):
        assert rel_err(ch.green(l), m.green_stable(f, l, ns)) < TOL, l
    ch.close()


@pytest.mark.parametrize("precision", [2, 6])
def test_sweep_lockstep(pkg, precision):
    from oracle.dqmc import Model, Chain
    w = WORKLOADS["L6_beta6"]
    m = Model(w["L"], U=w["U"], beta=w["beta"], dtau=w["dtau"])
    oc = Chain(m, n_delay=w["n_delay"], n_stab=w["n_stab"], seed=2024)
    ch = pkg.Chain(pkg.make_params(L=w["L"], beta=w["beta"], dtau=w["dtau"], U=w["U"], n_delay=w["n_delay"],
                                   n_stab=w["n_stab"], seed=2024, precision=precision))
    st = ch.sweep(1)
    oc.sweep()
    assert st.accepted == oc.accepted
    assert st.max_stab_drift < 1e-8
    assert np.array_equal(ch.field(), oc.field)
    assert rel_err(ch.green(0), oc.G) < TOL
    ch.close()


_FULL = {}


def full_size_reference():
    """Field and oracle G(0) at L = 24 (cached: one dense N = 1152 recomputation)."""
    if not _FULL:
        from oracle.dqmc import Model
        w = WORKLOADS["L24_beta24"]
        m = Model(w["L"], U=w["U"], beta=w["beta"], dtau=w["dtau"])
        f = random_field(m.M, m.N, 424)
        _FULL.update(w=w, f=f, G0=m.green_stable(f, 0, w["n_stab"]))
    return _FULL


@pytest.mark.parametrize("precision", [3, 7])
def test_full_size_green(pkg, precision):
    ref = full_size_reference()
    w = ref["w"]
    ch = pkg.Chain(pkg.make_params(L=w["L"], beta=w["beta"], dtau=w["dtau"], U=w["U"], n_delay=w["n_delay"],
                                   n_stab=w["n_stab"], seed=5, precision=precision))
    ch.set_field(ref["f"])
    assert rel_err(ch.green(0), ref["G0"]) < TOL
    ch.close()
