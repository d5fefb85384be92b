"""Exhaustive Hubbard-Stratonovich sum for tiny systems:
<O> = sum_X W(X) O(X) / sum_X W(X)  (Eq. GSObsQMC) with the oracle's weight
(Model.log_weight: e^{-gamma sum s} |det(1 + B_M...B_1)|^2 in the spin channel,
|det(1 + B_M...B_1)|^2 in the charge channel) and the oracle's Wick measurement
on G at slice 0."""
import itertools
import numpy as np

from .observables import measure


def hs_average(model, keys=("double_occ", "energy", "ekin", "Czz")):
    N, M = model.N, model.M
    logw, obs = [], []
    for bits in itertools.product((1, -1), repeat=N * M):
        field = np.array(bits, dtype=np.int8).reshape(M, N)
        lw, sign = model.log_weight(field)
        if not sign > 0:
            raise AssertionError("non-positive weight")
        logw.append(lw)
        o = measure(model, model.green_direct(field, M))
        obs.append({k: np.asarray(o[k], dtype=float) for k in keys})
    logw = np.array(logw)
    w = np.exp(logw - logw.max())
    w /= w.sum()
    return {k: sum(wi * oi[k] for wi, oi in zip(w, obs)) for k in keys}
