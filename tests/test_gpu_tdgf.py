"""Time-displaced measurement on the GPU against the oracle (oracle/tdgf.py)
and against the Trotterised ED.

* one field: the per-field estimators <H_I(tau_l) H_I(0)> and <H_I> for
  l = 0..M/2 match the oracle's dense-product Green's functions (1e-9
  relative), periodic and twisted, with recomputations from the stacks and
  propagation in between;
* a Markov chain's C(tau) and dD/dU match the Trotterised ED of the two-site
  cell within 4 sigma."""
import numpy as np
import pytest

from oracle import ed, tdgf
from synth import random_field

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_14668_b300 as p
    return p


@pytest.mark.parametrize("L,beta,ns,theta,precision", [(2, 1.2, 3, (0.0, 0.0), 0), (3, 1.0, 5, (0.25, 0.5), 0),
                                                       (6, 0.8, 4, (0.0, 0.0), 0), (3, 1.0, 5, (0.25, 0.5), 6),
                                                       (6, 0.8, 4, (0.0, 0.0), 6)])
def test_single_field_matches_oracle(pkg, L, beta, ns, theta, precision):
    """Precision 6: G(tau, 0) through the blocked solves as well (a second set of
    right-hand sides on the same LU)."""
    from oracle.dqmc import Model
    m = Model(L, U=3.73, beta=beta, dtau=0.1, theta=theta)
    f = random_field(m.M, m.N, 17 + L)
    ch = pkg.Chain(pkg.make_params(L=L, beta=beta, dtau=0.1, U=3.73, n_delay=4, n_stab=ns, seed=3, theta=theta,
                                   precision=precision))
    ch.set_field(f)
    pkg.afqmc_measure_td(ch.h)
    C, dDdU, chiF, n = pkg.afqmc_get_td(ch.h)
    assert n == 1
    ref = [tdgf.hi_products(m, f, l) for l in range(m.M // 2 + 1)]
    Cref = np.array([r[0] - ref[0][1] ** 2 for r in ref])
    scale = max(np.abs([r[0] for r in ref]).max(), ref[0][1] ** 2)
    assert np.abs(C - Cref).max() <= 1e-9 * scale
    d_ref, chi_ref = tdgf.integrals(Cref, m.dtau, m.N)
    assert abs(dDdU - d_ref) <= 1e-9 * scale and abs(chiF - chi_ref) <= 1e-9 * scale
    ch.close()


def test_chain_matches_trotter_ed(pkg):
    from oracle.lattice import Honeycomb
    U, beta, dtau = 3.0, 1.2, 0.2
    lat = Honeycomb(1)
    hh, h1 = ed.trotter_hi_correlation(lat, lat.hopping_matrix(), U, dtau, 6)
    C_ed = (hh - h1 * h1)[:4]
    d_ed, _ = tdgf.integrals(C_ed, dtau, lat.N)
    ch = pkg.Chain(pkg.make_params(L=1, beta=beta, dtau=dtau, U=U, n_delay=2, n_stab=3, seed=12))
    ch.sweep(200)
    pkg.afqmc_get_td(ch.h)
    bins_C, bins_d = [], []
    for _ in range(40):
        for _ in range(100):
            ch.sweep(1)
            pkg.afqmc_measure_td(ch.h)
        C, d, _, n = pkg.afqmc_get_td(ch.h)
        assert n == 100
        bins_C.append(C)
        bins_d.append(d)
    bins_C, bins_d = np.array(bins_C), np.array(bins_d)
    for l in range(4):
        mean, err = bins_C[:, l].mean(), bins_C[:, l].std(ddof=1) / np.sqrt(40)
        assert abs(mean - C_ed[l]) < 4.0 * err + 1e-12, (l, mean, err, C_ed[l])
    mean, err = bins_d.mean(), bins_d.std(ddof=1) / np.sqrt(40)
    assert abs(mean - d_ed) < 4.0 * err + 1e-12, (mean, err, d_ed)
    ch.close()
