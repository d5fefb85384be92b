"""Learned block proposals for the HS field (test infrastructure, FP64 numpy).

This part is not in the paper: a small network proposes new values for a block
of the Ising field (b x b unit cells, both sublattices, T consecutive slices)
from the field around it, and every proposal is accepted or rejected by
Metropolis-Hastings with the exact weight ratio of the method, so the
stationary distribution stays exactly W(X) of Eq. ConfgWeight whatever the
network has learned.

Geometry.  A block at slice l0 (1-based, slices l0 .. l0+T-1) and cell offset
(o1, o2) holds the sites sub*Nc + cell(o1 + c1, o2 + c2), c1, c2 < b, sub in
{A, B}.  Its context is the field on the cells [o1-h, o1+b+h) x [o2-h, o2+b+h)
(periodic), both sublattices, slices [l0-ht, l0+T+ht) (periodic in imaginary
time), with the block's own entries set to 0.  Orders: context index
((t * W + w2) * W + w1) * 2 + sub with W = b + 2h; block index
((t * b + c2) * b + c1) * 2 + sub.

Network.  z = W2 tanh(W1 x + b1) + b2 with x the context (+1/-1/0) and z one
logit per block entry; the proposal draws every entry independently,
q(s'|x) = prod_i sigmoid(s'_i z_i).  Training minimises the mean negative
log-likelihood of block configurations taken from configurations of the plain
sampler, -mean_n sum_i log sigmoid(s_ni z_ni).

Acceptance.  The context does not change under the move, so
A = min(1, [W(X')/W(X)] q(s_old|x) / q(s_new|x)).
"""
import numpy as np


# ---------------------------------------------------------------- geometry
def block_sites(lat, o1, o2, b):
    """Site indices of the block's cells in block order (c2, c1, sub)."""
    out = []
    for c2 in range(b):
        for c1 in range(b):
            for sub in (0, 1):
                out.append(lat.site(sub, o1 + c1, o2 + c2))
    return np.array(out)


def context(lat, field, l0, o1, o2, b, T, h, ht):
    """Context vector of the block (float64, +1/-1, 0 on the block itself)."""
    M = field.shape[0]
    W = b + 2 * h
    x = np.zeros((T + 2 * ht) * W * W * 2)
    for t in range(T + 2 * ht):
        l = (l0 - 1 - ht + t) % M                 # 0-based slice
        inside_t = ht <= t < ht + T
        for w2 in range(W):
            for w1 in range(W):
                c1, c2 = w1 - h, w2 - h
                inside = inside_t and 0 <= c1 < b and 0 <= c2 < b
                for sub in (0, 1):
                    idx = ((t * W + w2) * W + w1) * 2 + sub
                    x[idx] = 0.0 if inside else float(field[l, lat.site(sub, o1 + c1, o2 + c2)])
    return x


def block_values(lat, field, l0, o1, o2, b, T):
    """The block's current field values in block order (float64)."""
    sites = block_sites(lat, o1, o2, b)
    return np.concatenate([field[l0 - 1 + t, sites].astype(float) for t in range(T)])


def with_block(lat, field, l0, o1, o2, b, T, values):
    """Copy of the field with the block replaced by `values` (block order)."""
    f = np.array(field, copy=True)
    sites = block_sites(lat, o1, o2, b)
    n = len(sites)
    for t in range(T):
        f[l0 - 1 + t, sites] = np.asarray(values[t * n:(t + 1) * n]).astype(np.int8)
    return f


# ---------------------------------------------------------------- network
def init_params(d_in, d_hid, d_out, seed):
    rng = np.random.default_rng(seed)
    return dict(W1=rng.standard_normal((d_hid, d_in)) / np.sqrt(d_in), b1=np.zeros(d_hid),
                W2=rng.standard_normal((d_out, d_hid)) / np.sqrt(d_hid) * 0.1, b2=np.zeros(d_out))


def forward(p, X):
    """X: (B, d_in) -> (hidden (B, d_hid), logits (B, d_out))."""
    H = np.tanh(X @ p["W1"].T + p["b1"])
    return H, H @ p["W2"].T + p["b2"]


def log_sigmoid(x):
    return -np.logaddexp(0.0, -x)


def nll(p, X, S):
    """Mean over the batch of -sum_i log sigmoid(s_i z_i)."""
    _, Z = forward(p, X)
    return float(-np.sum(log_sigmoid(S * Z)) / X.shape[0])


def grads(p, X, S):
    """Gradients of nll by the chain rule, written out layer by layer."""
    B = X.shape[0]
    H, Z = forward(p, X)
    dZ = -S / (1.0 + np.exp(S * Z)) / B          # d/dz of -log sigmoid(s z) = -s sigmoid(-s z)
    dW2 = dZ.T @ H
    db2 = dZ.sum(axis=0)
    dA = (dZ @ p["W2"]) * (1.0 - H * H)
    dW1 = dA.T @ X
    db1 = dA.sum(axis=0)
    return dict(W1=dW1, b1=db1, W2=dW2, b2=db2)


def log_q(z, s):
    """log q(s|x) = sum_i log sigmoid(s_i z_i)."""
    return float(np.sum(log_sigmoid(np.asarray(s) * np.asarray(z))))


def adam_step(p, g, m, v, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """Adam (Kingma & Ba 2015), bias-corrected, in place on p, m, v; step >= 1."""
    for k in p:
        m[k] = b1 * m[k] + (1.0 - b1) * g[k]
        v[k] = b2 * v[k] + (1.0 - b2) * g[k] * g[k]
        mh = m[k] / (1.0 - b1 ** step)
        vh = v[k] / (1.0 - b2 ** step)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)


# ---------------------------------------------------------------- exact ratio
def block_log_ratio(model, field, l0, o1, o2, b, T, values):
    """log W(X')/W(X) for replacing the block by `values`, by brute-force determinants."""
    lw0, _ = model.log_weight(field)
    lw1, _ = model.log_weight(with_block(model.lat, field, l0, o1, o2, b, T, values))
    return lw1 - lw0
