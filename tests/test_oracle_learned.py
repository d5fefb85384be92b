"""Pins of the learned-proposal oracle (oracle/learned.py): gradients against
central finite differences, normalisation of the proposal distribution, the
block geometry, the exact block weight ratio against the product of
single-flip ratios, and one Adam step against its closed form."""
import itertools

import numpy as np
import pytest

from oracle import learned as ln
from oracle.dqmc import Model, local_ratio
from synth import random_field


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    p = ln.init_params(12, 7, 5, seed=1)
    p["W2"] *= 10.0
    X = rng.choice([-1.0, 0.0, 1.0], size=(6, 12))
    S = rng.choice([-1.0, 1.0], size=(6, 5))
    g = ln.grads(p, X, S)
    eps = 1e-6
    for k in p:
        it = np.nditer(p[k], flags=["multi_index"])
        for _ in it:
            idx = it.multi_index
            old = p[k][idx]
            p[k][idx] = old + eps
            fp = ln.nll(p, X, S)
            p[k][idx] = old - eps
            fm = ln.nll(p, X, S)
            p[k][idx] = old
            assert abs((fp - fm) / (2 * eps) - g[k][idx]) < 1e-7, (k, idx)


def test_proposal_is_normalised():
    z = np.random.default_rng(3).standard_normal(8) * 3.0
    tot = sum(np.exp(ln.log_q(z, s)) for s in itertools.product((-1.0, 1.0), repeat=8))
    assert abs(tot - 1.0) < 1e-12
    # stable for large logits: log sigmoid(40) ~ -e^-40, log sigmoid(-40) ~ -40
    assert abs(ln.log_sigmoid(np.array([-40.0]))[0] + 40.0) < 1e-12


def test_block_geometry():
    m = Model(4, U=3.73, beta=0.8, dtau=0.1)
    f = random_field(m.M, m.N, 2)
    b, T, h, ht = 2, 3, 1, 1
    l0, o1, o2 = 6, 3, 1                       # context wraps around in space and time
    x = ln.context(m.lat, f, l0, o1, o2, b, T, h, ht)
    assert x.shape == ((T + 2 * ht) * (b + 2 * h) ** 2 * 2,)
    assert np.count_nonzero(x == 0.0) == b * b * 2 * T
    v = ln.block_values(m.lat, f, l0, o1, o2, b, T)
    assert np.array_equal(ln.with_block(m.lat, f, l0, o1, o2, b, T, v), f)
    v2 = -v
    f2 = ln.with_block(m.lat, f, l0, o1, o2, b, T, v2)
    assert np.count_nonzero(f2 != f) == v.size
    # the context does not see the block: flipping it leaves x unchanged
    assert np.array_equal(ln.context(m.lat, f2, l0, o1, o2, b, T, h, ht), x)


def test_block_ratio_is_product_of_single_flips():
    """W(X')/W(X) of a block move equals the product of the single-flip ratios
    R = e^{2 gamma s}|r|^2 taken one site after the other (slice by slice,
    ascending sites), each from the fresh G of the current field."""
    m = Model(2, U=3.73, beta=0.6, dtau=0.1)
    f = random_field(m.M, m.N, 5)
    b, T, l0, o1, o2 = 1, 2, 3, 1, 0
    v = ln.block_values(m.lat, f, l0, o1, o2, b, T)
    new = v.copy()
    new[[0, 2, 3]] *= -1.0
    ref = ln.block_log_ratio(m, f, l0, o1, o2, b, T, new)
    cur = f.copy()
    sites = ln.block_sites(m.lat, o1, o2, b)
    acc = 0.0
    for t in range(T):
        l = l0 + t
        for j, i in enumerate(sites):
            if new[t * len(sites) + j] != cur[l - 1, i]:
                R, _, _ = local_ratio(m, m.green_direct(cur, l), i, float(cur[l - 1, i]))
                acc += np.log(R)
                cur[l - 1, i] *= -1
    assert abs(acc - ref) < 1e-10
    assert np.array_equal(cur, ln.with_block(m.lat, f, l0, o1, o2, b, T, new))


def test_adam_first_step_closed_form():
    p = dict(w=np.array([1.0, -2.0, 0.5]))
    g = dict(w=np.array([0.3, -4.0, 1e-3]))
    m = dict(w=np.zeros(3))
    v = dict(w=np.zeros(3))
    ln.adam_step(p, g, m, v, 1, lr=0.01, eps=1e-8)
    # bias-corrected first step: lr * g / (|g| + eps)
    assert np.allclose(p["w"], np.array([1.0, -2.0, 0.5]) - 0.01 * g["w"] / (np.abs(g["w"]) + 1e-8), atol=1e-15)
