"""Long physics run against the values the paper prints (App. C, Tables III
and IV, tests/golden/paper_tables_pbc.txt): L = 9, U/t = 3.50 and 3.75, PBC,
spin channel, beta t = L, dtau t = 0.05 (the paper's production step, Sec. II.B).

The sweep uses B_l = e^V e^{-dtau K} and measures on the symmetric-split
Green's function, which has the weights and the density matrix of the paper's
symmetric Trotter form, so the discretised model is the same and only
statistics separate the two numbers.  32 independent chains are swept together
(one CUDA graph per batched sweep); the error bar of a mean is the spread of
the 32 chain means.  Two checks per observable:
  * equilibration: the means of the first and second halves of the measurement
    sweeps agree within 3 combined standard errors (no drift left from the
    random start);
  * agreement with the table: |mean - value| < 2 sigma, sigma the combined
    standard error of our mean and the table's error bar.
Several GPU-minutes: opt-in with `pytest -m paper` (not part of -m gpu)."""
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


@pytest.mark.parametrize("U", [3.50, 3.75])
def test_L9_energy_and_double_occupancy_match_tables(U):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_14668_b300 as pkg
    L, dtau, n_chains, n_warm, n_meas = 9, 0.05, 32, 30, 60
    ref = table_row(L, U)
    params = [pkg.make_params(L=L, beta=float(L), dtau=dtau, U=U, n_delay=32, n_stab=10, seed=900 + c,
                              chain=c, measure=1) for c in range(n_chains)]
    batch = pkg.Batch(params)
    batch.sweep(n_warm)
    for c in batch.chains:
        c.observables()                      # drop the warm-up measurements
    series = {k: np.zeros((n_chains, n_meas)) for k in ref}
    for s in range(n_meas):
        batch.sweep(1)
        for i, c in enumerate(batch.chains):
            o = c.observables()
            for k in ref:
                series[k][i, s] = o[k]
    batch.close()
    half = n_meas // 2
    for k, (val, err) in ref.items():
        per_chain = series[k].mean(axis=1)
        m = per_chain.mean()
        se = per_chain.std(ddof=1) / np.sqrt(n_chains)
        a, b = series[k][:, :half].mean(axis=1), series[k][:, half:].mean(axis=1)
        se_ab = np.hypot(a.std(ddof=1), b.std(ddof=1)) / np.sqrt(n_chains)
        z_eq = (a.mean() - b.mean()) / se_ab
        z = (m - val) / np.hypot(se, err)
        print(f"PAPER_TABLE L={L} U={U} {k}: ours {m:.6f} +- {se:.6f}, table {val} +- {err}, "
              f"z = {z:+.2f}; halves {a.mean():.6f} / {b.mean():.6f}, z_eq = {z_eq:+.2f}")
        assert abs(z_eq) < 3.0, (k, "not equilibrated", a.mean(), b.mean(), se_ab)
        assert abs(z) < 2.0, (k, m, se, val, err)
