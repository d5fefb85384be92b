"""Python binding of libafqmc.so (include/afqmc.h): argument marshalling only.

Every computation runs in the CUDA kernels of the library; importing this
module fails loudly when the library is missing.  The functions carry the
names of the C entry points; ``Chain`` is a small convenience wrapper.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libafqmc.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("libafqmc.so is not built: run `python -m paper_2609_14668_b300.build` (nvcc, sm_103a)")

_lib = ctypes.CDLL(LIB_PATH)

STATUS = {0: "AFQMC_OK", 1: "AFQMC_E_INVALID", 2: "AFQMC_E_NOMEM", 3: "AFQMC_E_CUDA",
          4: "AFQMC_E_NUMERIC", 5: "AFQMC_E_TIMEOUT", 6: "AFQMC_E_STATE"}


class afqmc_params(ctypes.Structure):
    _fields_ = [("L1", ctypes.c_int32), ("L2", ctypes.c_int32), ("t", ctypes.c_double), ("U", ctypes.c_double),
                ("beta", ctypes.c_double), ("dtau", ctypes.c_double), ("theta1", ctypes.c_double),
                ("theta2", ctypes.c_double), ("hs_channel", ctypes.c_int32), ("n_delay", ctypes.c_int32),
                ("n_stab", ctypes.c_int32), ("precision", ctypes.c_int32), ("measure", ctypes.c_int32),
                ("chain", ctypes.c_int32), ("device", ctypes.c_int32), ("update_ctas", ctypes.c_int32),
                ("seed", ctypes.c_uint64)]


class afqmc_block_stats(ctypes.Structure):
    _fields_ = [("proposed", ctypes.c_uint64), ("accepted", ctypes.c_uint64), ("flipped", ctypes.c_uint64),
                ("max_stab_drift", ctypes.c_double)]


class afqmc_sweep_stats(ctypes.Structure):
    _fields_ = [("proposed", ctypes.c_uint64), ("accepted", ctypes.c_uint64), ("max_stab_drift", ctypes.c_double),
                ("launches", ctypes.c_uint64)]


KERNEL_FAMILIES = ["propagate", "update", "qr", "gemm", "qr_aux", "measure", "misc", "lu"]


class afqmc_timing(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_uint64 * len(KERNEL_FAMILIES)), ("ms", ctypes.c_double * len(KERNEL_FAMILIES))]


class afqmc_obs(ctypes.Structure):
    _fields_ = [("energy", ctypes.c_double), ("double_occ", ctypes.c_double), ("ekin", ctypes.c_double),
                ("density", ctypes.c_double), ("m2", ctypes.c_double), ("S_af", ctypes.c_double),
                ("S_af_dk", ctypes.c_double), ("R_m2", ctypes.c_double), ("Czz_half", ctypes.c_double),
                ("chi_e", ctypes.c_double), ("n_samples", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_H = ctypes.c_void_p
_P = ctypes.POINTER
_DP = _P(ctypes.c_double)
_FP = _P(ctypes.c_float)
_I8P = _P(ctypes.c_int8)

_SIGS = {
    "afqmc_create": ([_P(afqmc_params), ctypes.c_void_p, _P(_H)]),
    "afqmc_destroy": ([_H]),
    "afqmc_set_field": ([_H, _I8P, ctypes.c_uint64]),
    "afqmc_get_field": ([_H, _I8P]),
    "afqmc_sweep": ([_H, ctypes.c_int32, _P(afqmc_sweep_stats)]),
    "afqmc_measure": ([_H, _P(afqmc_obs), _DP, _DP]),
    "afqmc_get_obs": ([_H, _P(afqmc_obs), _DP, _DP]),
    "afqmc_get_G": ([_H, ctypes.c_int32, _DP]),
    "afqmc_wrap_matrix": ([_H, ctypes.c_int32, ctypes.c_int32, _DP]),
    "afqmc_update_slice": ([_H, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, _DP, _P(ctypes.c_int32)]),
    "afqmc_det_ratio": ([_H, ctypes.c_int32, ctypes.c_int32, _DP]),
    "afqmc_dims": ([_H, _P(ctypes.c_int32), _P(ctypes.c_int32), _P(ctypes.c_int32)]),
    "afqmc_set_timing": ([_H, ctypes.c_int32]),
    "afqmc_set_wait_limit": ([_H, ctypes.c_uint64]),
    "afqmc_update_slice_noalloc": ([_DP, _I8P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                    ctypes.c_uint64, ctypes.c_double, ctypes.c_double, ctypes.c_int32,
                                    ctypes.c_uint64, ctypes.c_int32, ctypes.c_void_p, _P(ctypes.c_int32)]),
    "afqmc_get_timing": ([_H, _P(afqmc_timing)]),
    "afqmc_batch_create": ([_P(afqmc_params), ctypes.c_int32, _P(_H)]),
    "afqmc_batch_destroy": ([_H]),
    "afqmc_batch_sweep": ([_H, ctypes.c_int32, _P(afqmc_sweep_stats)]),
    "afqmc_batch_autotune": ([_P(afqmc_params), ctypes.c_int32, _P(ctypes.c_int32), ctypes.c_int32,
                              _P(ctypes.c_int32), ctypes.c_int32, ctypes.c_int32, _P(ctypes.c_int32),
                              _P(ctypes.c_int32), _DP]),
    "afqmc_net_create": ([ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                          ctypes.c_uint64, ctypes.c_int32, _P(_H)]),
    "afqmc_net_destroy": ([_H]),
    "afqmc_net_dims": ([_H, _P(ctypes.c_int32)]),
    "afqmc_net_get_params": ([_H, _FP]),
    "afqmc_net_set_params": ([_H, _FP]),
    "afqmc_net_forward": ([_H, _FP, ctypes.c_int32, _FP]),
    "afqmc_net_inputs": ([_H, _I8P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                          _P(ctypes.c_int32), ctypes.c_int32, _FP, _FP]),
    "afqmc_net_gradient": ([_H, _FP, _FP, ctypes.c_int32, _FP, _DP]),
    "afqmc_net_train": ([_H, _I8P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                         ctypes.c_int32, ctypes.c_float, ctypes.c_uint64, _DP]),
    "afqmc_block_sweep": ([_H, _H, _P(afqmc_block_stats)]),
    "afqmc_force_slice": ([_H, ctypes.c_int32, _I8P, _DP, _DP]),
    "afqmc_measure_td": ([_H]),
    "afqmc_get_td": ([_H, _DP, _DP, _DP, _P(ctypes.c_int64)]),
    "afqmc_quasirandom_twists": ([ctypes.c_int32, ctypes.c_int32, _DP]),
}
for _name, _args in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = ctypes.c_int
_lib.afqmc_last_error.argtypes = [_H]
_lib.afqmc_last_error.restype = ctypes.c_char_p
_lib.afqmc_batch_last_error.argtypes = [_H]
_lib.afqmc_batch_last_error.restype = ctypes.c_char_p
_lib.afqmc_batch_chain.argtypes = [_H, ctypes.c_int32]
_lib.afqmc_batch_chain.restype = _H

_lib.afqmc_net_last_error.argtypes = [_H]
_lib.afqmc_net_last_error.restype = ctypes.c_char_p

EXPORTED = sorted(list(_SIGS) + ["afqmc_last_error", "afqmc_batch_last_error", "afqmc_batch_chain",
                                 "afqmc_net_last_error"])


class AfqmcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


def _check(code, handle):
    if code != 0:
        msg = _lib.afqmc_last_error(handle)
        raise AfqmcError(code, msg.decode() if msg else "")


def _dptr(a):
    return a.ctypes.data_as(_DP)


# ----------------------------------------------------------------- C names
# handles of complex-G chains (twisted boundaries or the charge-channel field):
# their G buffers are complex128
_COMPLEX = set()


def _params_complex(p):
    return p.theta1 != 0.0 or p.theta2 != 0.0 or p.hs_channel == 1


def _is_complex(h):
    return ctypes.cast(h, ctypes.c_void_p).value in _COMPLEX


def _gdtype(h):
    return np.complex128 if _is_complex(h) else np.float64


def afqmc_create(params, stream=None):
    h = _H()
    code = _lib.afqmc_create(ctypes.byref(params), ctypes.c_void_p(stream or 0), ctypes.byref(h))
    _check(code, None)
    if _params_complex(params):
        _COMPLEX.add(ctypes.cast(h, ctypes.c_void_p).value)
    return h


def afqmc_destroy(h):
    _COMPLEX.discard(ctypes.cast(h, ctypes.c_void_p).value)
    _check(_lib.afqmc_destroy(h), h)


def afqmc_dims(h):
    N, M, Nc = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(_lib.afqmc_dims(h, ctypes.byref(N), ctypes.byref(M), ctypes.byref(Nc)), h)
    return N.value, M.value, Nc.value


def afqmc_set_field(h, field, sweep_index=0):
    f = np.ascontiguousarray(field, dtype=np.int8)
    _check(_lib.afqmc_set_field(h, f.ctypes.data_as(_I8P), sweep_index), h)


def afqmc_get_field(h):
    N, M, _ = afqmc_dims(h)
    f = np.empty((M, N), dtype=np.int8)
    _check(_lib.afqmc_get_field(h, f.ctypes.data_as(_I8P)), h)
    return f


def afqmc_sweep(h, n_sweeps=1):
    st = afqmc_sweep_stats()
    _check(_lib.afqmc_sweep(h, n_sweeps, ctypes.byref(st)), h)
    return st


def _obs_call(fn, h):
    N, M, Nc = afqmc_dims(h)
    o = afqmc_obs()
    czz = np.empty(Nc)
    nk = np.empty(8 * Nc)
    _check(fn(h, ctypes.byref(o), _dptr(czz), _dptr(nk)), h)
    d = o.as_dict()
    d["Czz"] = czz
    d["nk"] = nk.view(np.complex128).reshape(Nc, 2, 2)
    return d


def afqmc_measure(h):
    return _obs_call(_lib.afqmc_measure, h)


def afqmc_get_obs(h):
    return _obs_call(_lib.afqmc_get_obs, h)


def afqmc_get_G(h, slice_):
    N, _, _ = afqmc_dims(h)
    G = np.empty((N, N), dtype=_gdtype(h))
    _check(_lib.afqmc_get_G(h, slice_, _dptr(G)), h)
    return G


def afqmc_wrap_matrix(h, slice_, direction, A):
    B = np.array(A, dtype=_gdtype(h), order="C", copy=True)
    _check(_lib.afqmc_wrap_matrix(h, slice_, direction, _dptr(B)), h)
    return B


def afqmc_update_slice(h, slice_, pas, sweep_index, G):
    B = np.array(G, dtype=_gdtype(h), order="C", copy=True)
    n = ctypes.c_int32()
    _check(_lib.afqmc_update_slice(h, slice_, pas, sweep_index, _dptr(B), ctypes.byref(n)), h)
    return B, n.value


def afqmc_det_ratio(h, slice_, site):
    """(R, r): r complex on the twisted path."""
    out = np.empty(3)
    _check(_lib.afqmc_det_ratio(h, slice_, site, _dptr(out)), h)
    return out[0], (complex(out[1], out[2]) if _is_complex(h) else out[1])


TIMING_ALL = (1 << len(KERNEL_FAMILIES)) - 1


def afqmc_set_wait_limit(h, wait_ns):
    """Test hook: limit (ns) of the device-side waits between CTAs; 0 = default."""
    _check(_lib.afqmc_set_wait_limit(h, int(wait_ns)), h)


def afqmc_set_timing(h, families):
    """families: True (all), False/0 (off), an int bit mask, or an iterable of family names."""
    if families is True:
        mask = TIMING_ALL
    elif families is False or families is None:
        mask = 0
    elif isinstance(families, int):
        mask = families
    else:
        mask = 0
        for f in families:
            mask |= 1 << KERNEL_FAMILIES.index(f)
    _check(_lib.afqmc_set_timing(h, mask), h)


def afqmc_get_timing(h):
    t = afqmc_timing()
    _check(_lib.afqmc_get_timing(h, ctypes.byref(t)), h)
    return {name: (int(t.launches[i]), float(t.ms[i])) for i, name in enumerate(KERNEL_FAMILIES)}


NOALLOC_MAX_N = 1152
NOALLOC_MAX_NDELAY = 64


def afqmc_update_slice_noalloc(G_dev_ptr, s_dev_ptr, N, M, slice_, pas, sweep_index, U, dtau, n_delay, seed,
                               chain=0, stream=None):
    """Allocation-free slice update on caller-owned device buffers (raw device
    pointers, e.g. torch tensor .data_ptr()); returns the accepted count."""
    n = ctypes.c_int32()
    code = _lib.afqmc_update_slice_noalloc(ctypes.cast(ctypes.c_void_p(G_dev_ptr), _DP),
                                           ctypes.cast(ctypes.c_void_p(s_dev_ptr), _I8P), N, M, slice_, pas,
                                           sweep_index, U, dtau, n_delay, seed, chain,
                                           ctypes.c_void_p(stream or 0), ctypes.byref(n))
    _check(code, None)
    return n.value


def _check_batch(code, b):
    if code != 0:
        msg = _lib.afqmc_batch_last_error(b)
        raise AfqmcError(code, msg.decode() if msg else "")


def afqmc_batch_create(params_list):
    arr = (afqmc_params * len(params_list))(*params_list)
    b = _H()
    _check_batch(_lib.afqmc_batch_create(arr, len(params_list), ctypes.byref(b)), None)
    for i, p in enumerate(params_list):
        if _params_complex(p):
            _COMPLEX.add(ctypes.cast(_lib.afqmc_batch_chain(b, i), ctypes.c_void_p).value)
    return b


def afqmc_batch_chain(b, i):
    h = _lib.afqmc_batch_chain(b, i)
    if not h:
        raise AfqmcError(1, f"no chain {i} in the batch")
    return _H(h)


def afqmc_batch_destroy(b, n=0):
    for i in range(n):
        _COMPLEX.discard(ctypes.cast(_lib.afqmc_batch_chain(b, i), ctypes.c_void_p).value)
    _lib.afqmc_batch_destroy(b)


def afqmc_batch_sweep(b, n_sweeps=1):
    st = afqmc_sweep_stats()
    _check_batch(_lib.afqmc_batch_sweep(b, n_sweeps, ctypes.byref(st)), b)
    return st


def afqmc_batch_autotune(params_list, n_delays, ctas, n_timed=1):
    arr = (afqmc_params * len(params_list))(*params_list)
    nd = (ctypes.c_int32 * len(n_delays))(*n_delays)
    cc = (ctypes.c_int32 * len(ctas))(*ctas)
    bn, bc, br = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
    _check_batch(_lib.afqmc_batch_autotune(arr, len(params_list), nd, len(n_delays), cc, len(ctas), n_timed,
                                           ctypes.byref(bn), ctypes.byref(bc), ctypes.byref(br)), None)
    return bn.value, bc.value, br.value


def afqmc_batch_last_error(b=None):
    m = _lib.afqmc_batch_last_error(b)
    return m.decode() if m else ""


def _check_net(code, net):
    if code != 0:
        msg = _lib.afqmc_net_last_error(net)
        raise AfqmcError(code, msg.decode() if msg else "")


def _fptr(a):
    return a.ctypes.data_as(_FP)


def afqmc_net_create(b, T, h, ht, hidden, seed=0, device=0):
    net = _H()
    _check_net(_lib.afqmc_net_create(b, T, h, ht, hidden, seed, device, ctypes.byref(net)), None)
    return net


def afqmc_net_destroy(net):
    _lib.afqmc_net_destroy(net)


def afqmc_net_dims(net):
    d = (ctypes.c_int32 * 4)()
    _check_net(_lib.afqmc_net_dims(net, d), net)
    return tuple(d)


def afqmc_net_get_params(net):
    p = np.empty(afqmc_net_dims(net)[3], dtype=np.float32)
    _check_net(_lib.afqmc_net_get_params(net, _fptr(p)), net)
    return p


def afqmc_net_set_params(net, p):
    p = np.ascontiguousarray(p, dtype=np.float32)
    _check_net(_lib.afqmc_net_set_params(net, _fptr(p)), net)


def afqmc_net_forward(net, X):
    X = np.ascontiguousarray(X, dtype=np.float32)
    d_in, _, d_out, _ = afqmc_net_dims(net)
    Z = np.empty((X.shape[0], d_out), dtype=np.float32)
    _check_net(_lib.afqmc_net_forward(net, _fptr(X), X.shape[0], _fptr(Z)), net)
    return Z


def afqmc_net_inputs(net, fields, L1, L2, pos):
    f = np.ascontiguousarray(fields, dtype=np.int8)
    p = np.ascontiguousarray(pos, dtype=np.int32).reshape(-1, 4)
    d_in, _, d_out, _ = afqmc_net_dims(net)
    X = np.empty((p.shape[0], d_in), dtype=np.float32)
    S = np.empty((p.shape[0], d_out), dtype=np.float32)
    _check_net(_lib.afqmc_net_inputs(net, f.ctypes.data_as(_I8P), f.shape[0], L1, L2, f.shape[1],
                                     p.ctypes.data_as(_P(ctypes.c_int32)), p.shape[0], _fptr(X), _fptr(S)), net)
    return X, S


def afqmc_net_gradient(net, X, S):
    X = np.ascontiguousarray(X, dtype=np.float32)
    S = np.ascontiguousarray(S, dtype=np.float32)
    g = np.empty(afqmc_net_dims(net)[3], dtype=np.float32)
    loss = ctypes.c_double()
    _check_net(_lib.afqmc_net_gradient(net, _fptr(X), _fptr(S), X.shape[0], _fptr(g), ctypes.byref(loss)), net)
    return g, loss.value


def afqmc_net_train(net, fields, L1, L2, n_steps, batch, lr=1e-3, seed=0):
    f = np.ascontiguousarray(fields, dtype=np.int8)
    loss = ctypes.c_double()
    _check_net(_lib.afqmc_net_train(net, f.ctypes.data_as(_I8P), f.shape[0], L1, L2, f.shape[1], n_steps, batch,
                                    lr, seed, ctypes.byref(loss)), net)
    return loss.value


def afqmc_net_last_error(net=None):
    m = _lib.afqmc_net_last_error(net)
    return m.decode() if m else ""


def afqmc_block_sweep(h, net):
    st = afqmc_block_stats()
    _check(_lib.afqmc_block_sweep(h, net, ctypes.byref(st)), h)
    return st


def afqmc_quasirandom_twists(n, start=1):
    """(n, 2) array of twist angles (theta1, theta2): the 2D Halton sequence in
    bases 2 and 3 from index start (host-only)."""
    out = np.zeros((max(n, 0), 2))
    _check(_lib.afqmc_quasirandom_twists(n, start, _dptr(out) if n > 0 else None), None)
    return out


def afqmc_measure_td(h):
    _check(_lib.afqmc_measure_td(h), h)


def afqmc_get_td(h):
    """(C(tau_l) for l = 0..M/2, dD/dU, chi_F, n_samples)."""
    _, M, _ = afqmc_dims(h)
    C = np.empty(M // 2 + 1)
    d, c, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
    _check(_lib.afqmc_get_td(h, _dptr(C), ctypes.byref(d), ctypes.byref(c), ctypes.byref(n)), h)
    return C, d.value, c.value, n.value


def afqmc_force_slice(h, slice_, mask, G):
    B = np.array(G, dtype=_gdtype(h), order="C", copy=True)
    m = np.ascontiguousarray(mask, dtype=np.int8)
    lr = ctypes.c_double()
    _check(_lib.afqmc_force_slice(h, slice_, m.ctypes.data_as(_I8P), _dptr(B), ctypes.byref(lr)), h)
    return B, lr.value


class Net:
    """Block-proposal network (owns an afqmc_net)."""

    def __init__(self, b, T, h, ht, hidden, seed=0, device=0):
        self.shape = (b, T, h, ht, hidden)
        self.net = afqmc_net_create(b, T, h, ht, hidden, seed, device)
        self.d_in, self.d_hid, self.d_out, self.n_params = afqmc_net_dims(self.net)

    def params(self):
        """Split parameter vector: W1, b1, W2, b2."""
        p = afqmc_net_get_params(self.net)
        a = self.d_hid * self.d_in
        W1 = p[:a].reshape(self.d_hid, self.d_in)
        b1 = p[a:a + self.d_hid]
        c = a + self.d_hid
        W2 = p[c:c + self.d_out * self.d_hid].reshape(self.d_out, self.d_hid)
        b2 = p[c + self.d_out * self.d_hid:]
        return dict(W1=W1, b1=b1, W2=W2, b2=b2)

    def set_params(self, d):
        afqmc_net_set_params(self.net, np.concatenate([np.ravel(d[k]) for k in ("W1", "b1", "W2", "b2")]))

    def close(self):
        if self.net:
            afqmc_net_destroy(self.net)
            self.net = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def afqmc_last_error(h=None):
    m = _lib.afqmc_last_error(h)
    return m.decode() if m else ""


def make_params(L, beta, dtau, U, n_delay, n_stab, t=1.0, seed=0, chain=0, measure=0, device=0, L2=None,
                precision=0, theta=(0.0, 0.0), update_ctas=0, hs_channel=0):
    return afqmc_params(L1=L, L2=L if L2 is None else L2, t=t, U=U, beta=beta, dtau=dtau,
                        theta1=float(theta[0]), theta2=float(theta[1]),
                        hs_channel=hs_channel, n_delay=n_delay, n_stab=n_stab, precision=precision,
                        measure=measure, chain=chain, device=device, update_ctas=update_ctas, seed=seed)


class Batch:
    """Independent chains swept together, one CUDA graph launch per batched sweep."""

    def __init__(self, params_list):
        self.params = list(params_list)
        self.b = afqmc_batch_create(self.params)
        self.chains = []
        for i, p in enumerate(self.params):
            c = Chain.__new__(Chain)
            c.params, c.h, c.borrowed = p, afqmc_batch_chain(self.b, i), True
            c.N, c.M, c.Nc = afqmc_dims(c.h)
            self.chains.append(c)

    def sweep(self, n=1):
        return afqmc_batch_sweep(self.b, n)

    def close(self):
        if self.b:
            for c in self.chains:
                c.h = None
            afqmc_batch_destroy(self.b, len(self.params))
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Chain:
    """One Markov chain on the GPU (owns an afqmc handle)."""
    borrowed = False

    def __init__(self, params, stream=None):
        self.params = params
        self.h = afqmc_create(params, stream)
        self.N, self.M, self.Nc = afqmc_dims(self.h)

    def close(self):
        if self.h and not self.borrowed:
            afqmc_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sweep(self, n=1):
        return afqmc_sweep(self.h, n)

    def set_field(self, f, sweep_index=0):
        afqmc_set_field(self.h, f, sweep_index)

    def field(self):
        return afqmc_get_field(self.h)

    def measure(self):
        return afqmc_measure(self.h)

    def observables(self):
        return afqmc_get_obs(self.h)

    def green(self, slice_=0):
        return afqmc_get_G(self.h, slice_)
