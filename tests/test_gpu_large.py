"""Parity at the largest matrix dimensions of the column kernels (shape <4, 16>,
n up to 4096): the learned-proposal lattice L = 42 (real G, N = 3528) and the
L = 24 lattice with complex G (twist, and the charge channel; the device holds
the 2304 x 2304 real embedding).  For each: G at slice 0 recomputed from the
QR-stabilised stacks, the first wrap, and one full slice update (same
counter-based uniforms) against the FP64 CPU oracle; fields and accepted
counts exactly, G to 1e-10 relative (G at slice 0 of the charge channel: or
to 10 cond(1 + B_M...B_1) eps, where the field's conditioning puts the FP64
bound above 1e-10).  beta is kept short so that the dense
oracle finishes in seconds; the GPU kernels are the same at any beta."""
import numpy as np
import pytest

from synth import random_field

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


BETA, DTAU, U, NS, SEED = 1.0, 0.1, 3.73, 5, 17
_CACHE = {}


def oracle_case(L, theta, hs, n_delay):
    """Field, G(0), the first wrap and one oracle slice update (cached: the
    dense N = 3528 oracle takes tens of seconds), and for the charge channel
    the FP64 error bound of G(0) for this field, 10 cond(1 + B_M...B_1) eps
    (0 for the spin channel, whose G(0) is held to 1e-10 outright)."""
    key = (L, theta, hs, n_delay)
    if key not in _CACHE:
        from oracle.dqmc import Model, Chain
        m = Model(L, U=U, beta=BETA, dtau=DTAU, theta=theta, hs_channel=hs)
        f = random_field(m.M, m.N, 4200 + L + hs)
        G0 = m.green_stable(f, 0, NS)
        floor = 0.0
        if hs == 1:
            # charge channel: the FP64 error of any stable evaluation of
            # G = (1 + B_M...B_1)^-1 grows with cond(1 + B_M...B_1); the bound is
            # 10 cond eps (the oracle's own deviation from an iteratively refined
            # direct inverse, 9e-11 here, sits inside it)
            A = np.eye(m.N) + m.chain_product(f, 1, m.M)
            floor = 10.0 * np.linalg.cond(A) * np.finfo(float).eps
        G1 = m.wrap(G0, f[0])
        oc = Chain(m, n_delay=n_delay, n_stab=NS, seed=SEED, field=f)
        oc.G = G1.copy()
        oc.update_slice(1, 0)
        _CACHE[key] = (m.N, f, G0, G1, oc.G, oc.accepted, oc.field[0].copy(), floor)
    return _CACHE[key]


@pytest.mark.parametrize("L,theta,hs,n_delay,precision", [
    (42, (0.0, 0.0), 0, 64, 0),
    (42, (0.0, 0.0), 0, 64, 2),
    (42, (0.0, 0.0), 0, 64, 6),
    (24, (0.25, 0.5), 0, 32, 0),
    (24, (0.25, 0.5), 0, 32, 6),
    (24, (0.0, 0.0), 1, 32, 2),
])
def test_large_matrix_parity(pkg, L, theta, hs, n_delay, precision):
    N, f, G0, G1, G_upd, n_upd, f_upd, floor = oracle_case(L, theta, hs, n_delay)
    ch = pkg.Chain(pkg.make_params(L=L, beta=BETA, dtau=DTAU, U=U, n_delay=n_delay, n_stab=NS, seed=SEED,
                                   theta=theta, hs_channel=hs, precision=precision))
    assert ch.N == N
    ch.set_field(f)
    # 1e-10 relative, unless the field's conditioning puts the FP64 bound above
    # it: the random charge-channel field at L = 24 has cond(1 + B_M...B_1) ~ 1.4e6
    # and |G| up to ~1e5 (bound 10 cond eps ~ 1.5e-9)
    assert rel_err(ch.green(0), G0) < max(TOL, floor), floor
    assert rel_err(pkg.afqmc_wrap_matrix(ch.h, 1, +1, G0), G1) < 1e-12
    Gg, nacc = pkg.afqmc_update_slice(ch.h, 1, 0, 0, G1)
    assert nacc == n_upd > 0
    assert np.array_equal(ch.field()[0], f_upd)
    assert rel_err(Gg, G_upd) < TOL
    ch.close()


def test_dimension_above_the_column_kernels_is_rejected(pkg):
    with pytest.raises(pkg.AfqmcError) as e:
        pkg.Chain(pkg.make_params(L=48, beta=0.2, dtau=0.1, U=3.73, n_delay=8, n_stab=2, seed=1))
    assert e.value.code == 1 and "4096" in str(e.value)
