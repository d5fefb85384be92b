"""Long physics run against the values the paper prints (Tables III and IV,
tests/golden/paper_tables_pbc.txt): L = 9, U/t = 3.75, PBC, spin channel,
beta t = L, dtau t = 0.05 (the paper's production step, Sec. II.B 'First').

The sweep uses B_l = e^V e^{-dtau K} and measures on the symmetric-split
Green's function, which has the weights and the density matrix of the paper's
symmetric Trotter form, so the discretised model is the same and only
statistics separate the two numbers.  32 independent chains swept together
(one CUDA graph per batched sweep); the error bar is the spread of the chain
means.  Several GPU-minutes: opt-in with `pytest -m paper` (not part of -m gpu)."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.paper

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_tables_pbc.txt")


def table_row(L, U):
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        v = [float(x) for x in line.split()]
        if int(v[0]) == L and abs(v[1] - U) < 1e-9:
            return dict(energy=(v[2], v[3]), double_occ=(v[4], v[5]))
    raise KeyError((L, U))


def test_L9_energy_and_double_occupancy_match_tables():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_14668_b300 as pkg
    L, U, dtau, n_chains, n_warm, n_meas = 9, 3.75, 0.05, 32, 20, 40
    ref = table_row(L, U)
    params = [pkg.make_params(L=L, beta=float(L), dtau=dtau, U=U, n_delay=32, n_stab=10, seed=900 + c,
                              chain=c, measure=1) for c in range(n_chains)]
    batch = pkg.Batch(params)
    batch.sweep(n_warm)
    for c in batch.chains:
        c.observables()                      # drop the warm-up measurements
    batch.sweep(n_meas)
    means = {k: np.array([c.observables()[k] for c in batch.chains]) for k in ref}
    batch.close()
    for k, (val, err) in ref.items():
        m = means[k].mean()
        se = means[k].std(ddof=1) / np.sqrt(n_chains)
        assert abs(m - val) < 4.0 * np.hypot(se, err), (k, m, se, val, err)
