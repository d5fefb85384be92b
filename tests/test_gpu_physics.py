"""Full Markov chains on the GPU against exact results.

The HS sum reproduces the Trotterised density matrix exactly at any dtau, so
Monte Carlo averages of the GPU chain must agree with the Trotterised
exact diagonalisation of the 8-site (L=2) cluster within their statistical
error (tests/golden/ed_L2.json, written by tests/golden/make_ed_L2.py from the
oracle only).  Errors come from 40 bins of 100 sweeps; the bound is 4 sigma."""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "ed_L2.json")


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_14668_b300 as p
    return p


@pytest.mark.parametrize("case", [0, 1])
def test_chain_matches_trotter_ed(pkg, case):
    c = json.load(open(GOLDEN))["cases"][case]
    ch = pkg.Chain(pkg.make_params(L=c["L"], beta=c["beta"], dtau=c["dtau"], U=c["U"], n_delay=4, n_stab=4,
                                   seed=4242 + case, measure=1))
    ch.sweep(200)
    ch.observables()
    bins = {"double_occ": [], "energy": [], "Czz0": [], "Czz1": []}
    for _ in range(40):
        ch.sweep(100)
        o = ch.observables()
        assert o["n_samples"] == 100 * 2 * (ch.M // 4)
        bins["double_occ"].append(o["double_occ"])
        bins["energy"].append(o["energy"])
        bins["Czz0"].append(o["Czz"][0])
        bins["Czz1"].append(o["Czz"][1])
    ref = {"double_occ": c["double_occ"], "energy": c["energy"],
           "Czz0": c["Czz"][0][0], "Czz1": c["Czz"][0][1]}
    for k, v in bins.items():
        v = np.array(v)
        mean, err = v.mean(), v.std(ddof=1) / np.sqrt(len(v))
        assert abs(mean - ref[k]) < 4.0 * err + 1e-12, (k, mean, err, ref[k])
    ch.close()
