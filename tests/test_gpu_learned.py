"""Learned block proposals on the GPU against the oracle (oracle/learned.py)
and against exact results.

* the network's FP32 forward pass and gradient match the FP64 oracle (1e-5 and
  1e-4 relative: FP32 arithmetic over sums of <= 100 terms);
* the contexts and block values the kernels build match the oracle's geometry
  exactly;
* forced slice updates give the exact block weight ratio (brute-force
  determinants, 1e-9) and the fresh G of the new field (1e-10);
* block passes alone keep the chain's stationary distribution: averages match
  the Trotterised ED of the 8-site cluster within 4 sigma;
* a network trained on the GPU on configurations of the plain sampler proposes
  blocks that are accepted more often than an untrained one's."""
import json
import os

import numpy as np
import pytest

from oracle import learned as ln
from synth import random_field

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "ed_L2.json")


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_14668_b300 as p
    return p


def test_forward_and_gradient_match_oracle(pkg):
    net = pkg.Net(b=1, T=2, h=1, ht=1, hidden=16)
    p = ln.init_params(net.d_in, net.d_hid, net.d_out, seed=4)
    p["W2"] *= 20.0
    p["b1"] = np.linspace(-0.5, 0.5, net.d_hid)
    p32 = {k: v.astype(np.float32) for k, v in p.items()}
    net.set_params(p32)
    p64 = {k: v.astype(np.float64) for k, v in p32.items()}
    rng = np.random.default_rng(9)
    X = rng.choice([-1.0, 0.0, 1.0], size=(8, net.d_in))
    S = rng.choice([-1.0, 1.0], size=(8, net.d_out))
    _, Z_ref = ln.forward(p64, X)
    Z = pkg.afqmc_net_forward(net.net, X)
    assert np.abs(Z - Z_ref).max() <= 1e-5 * np.abs(Z_ref).max()
    g, loss = pkg.afqmc_net_gradient(net.net, X, S)
    g_ref = ln.grads(p64, X, S)
    flat = np.concatenate([np.ravel(g_ref[k]) for k in ("W1", "b1", "W2", "b2")])
    assert np.abs(g - flat).max() <= 1e-4 * np.abs(flat).max()
    assert abs(loss - ln.nll(p64, X, S)) <= 1e-5 * abs(loss)
    net.close()


def test_block_inputs_match_oracle_geometry(pkg):
    from oracle.lattice import Honeycomb
    L, M, b, T, h, ht = 4, 10, 2, 3, 1, 2
    lat = Honeycomb(L)
    fields = np.stack([random_field(M, lat.N, s) for s in range(3)])
    pos = [(0, 1, 0, 0), (2, 8, 3, 2), (1, 4, 2, 3)]          # context wraps in space and time
    net = pkg.Net(b=b, T=T, h=h, ht=ht, hidden=8)
    X, S = pkg.afqmc_net_inputs(net.net, fields, L, L, pos)
    for q, (c, l0, o1, o2) in enumerate(pos):
        assert np.array_equal(X[q], ln.context(lat, fields[c], l0, o1, o2, b, T, h, ht))
        assert np.array_equal(S[q], ln.block_values(lat, fields[c], l0, o1, o2, b, T))
    net.close()


def test_forced_slices_give_exact_block_ratio(pkg):
    from oracle.dqmc import Model
    m = Model(2, U=3.73, beta=0.6, dtau=0.1)
    f = random_field(m.M, m.N, 5)
    ch = pkg.Chain(pkg.make_params(L=2, beta=0.6, dtau=0.1, U=3.73, n_delay=2, n_stab=3, seed=1))
    ch.set_field(f)
    b, T, l0, o1, o2 = 1, 2, 3, 1, 1
    v = ln.block_values(m.lat, f, l0, o1, o2, b, T)
    new = v.copy()
    new[[0, 1, 3]] *= -1.0
    f_new = ln.with_block(m.lat, f, l0, o1, o2, b, T, new)
    G = ch.green(l0 - 1)
    tot = 0.0
    for t in range(T):
        l = l0 + t
        G = pkg.afqmc_wrap_matrix(ch.h, l, +1, G)
        mask = (f_new[l - 1] != f[l - 1]).astype(np.int8)
        G, lr = pkg.afqmc_force_slice(ch.h, l, mask, G)
        tot += lr
    assert abs(tot - ln.block_log_ratio(m, f, l0, o1, o2, b, T, new)) < 1e-9
    assert np.array_equal(ch.field(), f_new)
    ref = m.green_direct(f_new, l0 + T - 1)
    assert np.abs(G - ref).max() <= 1e-10 * np.abs(ref).max()
    ch.close()


@pytest.mark.parametrize("with_local", [False, True])
def test_block_moves_keep_the_distribution(pkg, with_local):
    c = json.load(open(GOLDEN))["cases"][0]
    ch = pkg.Chain(pkg.make_params(L=c["L"], beta=c["beta"], dtau=c["dtau"], U=c["U"], n_delay=4, n_stab=4,
                                   seed=77 + with_local, measure=1))
    net = pkg.Net(b=1, T=2, h=1, ht=1, hidden=16, seed=3)
    p = net.params()
    p["W2"] = p["W2"] * 30.0            # a strongly biased (untrained) proposal: the ratio must correct it
    net.set_params(p)

    def step():
        st = pkg.afqmc_block_sweep(ch.h, net.net)
        if with_local:
            ch.sweep(1)
        return st

    for _ in range(100):
        step()
    ch.observables()
    bins = {"double_occ": [], "energy": []}
    acc = prop = 0
    for _ in range(40):
        for _ in range(50):
            st = step()
            acc += st.accepted
            prop += st.proposed
        o = ch.observables()
        bins["double_occ"].append(o["double_occ"])
        bins["energy"].append(o["energy"])
    assert 0 < acc < prop
    for k, v in bins.items():
        v = np.array(v)
        mean, err = v.mean(), v.std(ddof=1) / np.sqrt(len(v))
        assert abs(mean - c[k]) < 4.0 * err + 1e-12, (k, mean, err, c[k])
    net.close()
    ch.close()


def test_trained_network_raises_block_acceptance(pkg):
    L, beta, dtau, U = 2, 1.0, 0.125, 4.0
    mk = lambda s: pkg.make_params(L=L, beta=beta, dtau=dtau, U=U, n_delay=4, n_stab=4, seed=s)
    sampler = pkg.Chain(mk(5))
    sampler.sweep(100)
    cfgs = []
    for _ in range(600):
        sampler.sweep(1)
        cfgs.append(sampler.field())
    cfgs = np.stack(cfgs)
    sampler.close()
    rates = {}
    for name, steps in (("untrained", 0), ("trained", 1500)):
        net = pkg.Net(b=1, T=2, h=1, ht=1, hidden=32, seed=8)
        loss0 = pkg.afqmc_net_train(net.net, cfgs, L, L, 1, 256, lr=0.0, seed=1)
        if steps:
            loss = pkg.afqmc_net_train(net.net, cfgs, L, L, steps, 256, lr=3e-3, seed=2)
            assert loss < loss0
        ch = pkg.Chain(mk(11))
        ch.sweep(50)
        acc = prop = 0
        for _ in range(60):
            st = pkg.afqmc_block_sweep(ch.h, net.net)
            acc += st.accepted
            prop += st.proposed
            ch.sweep(1)
        rates[name] = acc / prop
        ch.close()
        net.close()
    assert rates["trained"] > 1.2 * rates["untrained"], rates
