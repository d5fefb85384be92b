"""Finite-temperature AFQMC (DQMC) for the half-filled honeycomb Hubbard model:
periodic boundaries or twisted boundaries (Sec. III.C: Peierls phases on the
bonds, complex G), with the Ising field in the spin channel (HS-s^z, Eq. SzHS)
or in the charge channel (HS-n, Eq. DensityHS).

Follows Sec. II.B (Eqs. SzHS, DensityHS, coupling, BIOpSz, BIOpnT,
ConfgWeight, GrFMat and its five implementation notes) and
Sec. III.B (Eqs. DetailBalance, DRatio, GFupdate, rRatioLocal, GupdateLocal,
DelayG0, DelayRatio, DelayRgenk, FinalDelay).  Propagators are dense:
B_l = e^{lambda diag(s_l)} E with E = e^{-dtau H0} from a Taylor series (no
FFT), so this module is independent of the momentum-space propagation of
Sec. III.A that the CUDA path uses.  lambda is the coupling of Eq. coupling:
gamma_s = arccosh(e^{dtau U/2}) (spin channel, real) or
gamma_c = i arccos(e^{-dtau U/2}) (charge channel, imaginary).

Readings of the paper fixed here (the paper is silent or ambiguous):
  * the simulated spin is up; after the partial particle-hole transform the
    down-spin propagator is the complex conjugate of the up-spin one
    ('Fourth').  Spin channel: the transform leaves the scalar e^{-gamma sum s},
    so W(X) ~ e^{-gamma sum s} |det(1 + B_M...B_1)|^2 and a single flip at
    (l, i) has weight ratio R = e^{2 gamma s_i} |r|^2.  Charge channel: the
    scalar e^{+gamma_c sum s} of the transform cancels the e^{-gamma_c sum s}
    of p(x) (Eq. BIOpnT), so W(X) ~ |det(1 + B_M...B_1)|^2 and R = |r|^2.  In
    both, r = 1 + Delta (1 - G_ii) with Delta = e^{-2 lambda s_i} - 1 (real for
    the spin channel, a unit-circle point minus one for the charge channel);
  * a sweep is a forward pass l = 1..M (wrap into slice l, then propose every
    site i = 0..N-1 in ascending order) followed by a backward pass l = M..1
    (propose, then unwrap); accept iff u < R;
  * the delayed update flushes after n_delay accepted moves and at slice end;
    rejected moves do not use rank; the diagonal update of Eq. FinalDelay's
    text uses x_k (the printed x_m is read as x_k);
  * G is recomputed from the UDT stacks every n_stab slices (M % n_stab == 0):
    in the forward pass at l = c*n_stab after the slice update, in the backward
    pass at l-1 = c*n_stab after the unwrap.
"""
import numpy as np

from .lattice import Honeycomb
from .linalg import expm_taylor, udt_identity, udt_left_multiply, stable_green
from . import rng as _rng


class Model:
    """Static data: lattice, K, E = e^{-dtau K}, its inverse and half steps, gamma."""

    def __init__(self, L, t=1.0, U=3.73, beta=3.0, dtau=0.1, theta=(0.0, 0.0), hs_channel=0):
        self.lat = Honeycomb(L, t=t, theta=theta)
        self.N = self.lat.N
        self.M = int(round(beta / dtau))
        if abs(self.M * dtau - beta) > 1e-9:
            raise ValueError("beta must be a multiple of dtau")
        if hs_channel not in (0, 1):
            raise ValueError("hs_channel must be 0 (spin, Eq. SzHS) or 1 (charge, Eq. DensityHS)")
        self.t, self.U, self.beta, self.dtau = t, U, beta, dtau
        self.hs_channel = hs_channel
        self.K = self.lat.hopping_matrix()
        # Eq. coupling: gamma_s = arccosh(e^{dtau U / 2}), gamma_c = i arccos(e^{-dtau U / 2})
        self.gamma = np.arccosh(np.exp(dtau * U / 2.0))
        self.alpha = np.arccos(np.exp(-dtau * U / 2.0))
        self.lam = self.gamma if hs_channel == 0 else 1j * self.alpha
        self.is_complex = np.iscomplexobj(self.K) or hs_channel == 1
        self.E = expm_taylor(-dtau * self.K)
        self.Einv = expm_taylor(dtau * self.K)
        self.Eh = expm_taylor(-0.5 * dtau * self.K)
        self.Ehinv = expm_taylor(0.5 * dtau * self.K)

    # B_l = e^{H_I(x_l)} e^{-dtau H0}, H_I = lambda diag(s_l) for spin up (Eqs. BIOpSz, BIOpnT, ConfgWeight)
    def B(self, s_l):
        return np.exp(self.lam * s_l.astype(float))[:, None] * self.E

    def Binv(self, s_l):
        return self.Einv * np.exp(-self.lam * s_l.astype(float))[None, :]

    def flip_delta(self, s_i):
        """Delta = e^{-2 lambda s_i} - 1 of flipping s_i (Eq. DRatio)."""
        return np.exp(-2.0 * self.lam * s_i) - 1.0

    def weight_factor(self, s_i):
        """W(X')/W(X) = weight_factor * |r|^2 for a flip of s_i: e^{2 gamma s_i}
        from the scalar the particle-hole transform leaves in the spin channel,
        1 in the charge channel."""
        return np.exp(2.0 * self.gamma * s_i) if self.hs_channel == 0 else 1.0

    def wrap(self, G, s_l):
        """G -> B_l G B_l^-1 (Sec. III.A, first paragraph)."""
        return self.B(s_l) @ G @ self.Binv(s_l)

    def unwrap(self, G, s_l):
        """G -> B_l^-1 G B_l."""
        return self.Binv(s_l) @ G @ self.B(s_l)

    # ---- brute force (small beta only) -------------------------------------
    def chain_product(self, field, lo, hi):
        """B_hi ... B_lo (1-based, inclusive); identity when hi < lo."""
        P = np.eye(self.N)
        for l in range(lo, hi + 1):
            P = self.B(field[l - 1]) @ P
        return P

    def green_direct(self, field, l):
        """Eq. GrFMat by a plain inverse: (1 + B_l..B_1 B_M..B_{l+1})^-1."""
        R = self.chain_product(field, 1, l)
        Lm = self.chain_product(field, l + 1, self.M)
        return np.linalg.inv(np.eye(self.N) + R @ Lm)

    def log_weight(self, field):
        """log W(X) up to a field-independent constant: 2 log|det(1 + B_M..B_1)|,
        plus -gamma sum s in the spin channel.

        W is the up-spin determinant times its complex conjugate (Sec. II.B
        'Fourth'), so it is never negative; the returned sign is that of the
        real determinant (real path) or 1 (complex path)."""
        sign, ld = np.linalg.slogdet(np.eye(self.N) + self.chain_product(field, 1, self.M))
        if self.is_complex:
            sign = 1.0 if abs(sign) > 0 else 0.0
        scalar = -self.gamma * float(field.sum()) if self.hs_channel == 0 else 0.0
        return scalar + 2.0 * ld, sign

    # ---- stabilised chains -----------------------------------------------
    def udt_R(self, field, l, n_stab):
        """UDT of R = B_l ... B_1, re-orthogonalised after every n_stab factors."""
        out = udt_identity(self.N)
        lo = 1
        while lo <= l:
            hi = min(lo + n_stab - 1, l)
            out = udt_left_multiply(self.chain_product(field, lo, hi), out)
            lo = hi + 1
        return out

    def udt_Lt(self, field, l, n_stab):
        """UDT of L^T = (B_M ... B_{l+1})^T, built from the top slice down."""
        out = udt_identity(self.N)
        hi = self.M
        while hi > l:
            lo = max(hi - n_stab + 1, l + 1)
            out = udt_left_multiply(self.chain_product(field, lo, hi).T, out)
            hi = lo - 1
        return out

    def green_stable(self, field, l, n_stab):
        return stable_green(self.udt_R(field, l, n_stab), self.udt_Lt(field, l, n_stab))


def local_ratio(model, G, i, s_i):
    """Eq. rRatioLocal with the channel's Delta and the particle-hole weight factor.

    Returns (R, r, Delta): R = W(X')/W(X) = e^{2 gamma s_i} |r|^2 (spin channel)
    or |r|^2 (charge channel)."""
    Delta = model.flip_delta(s_i)
    r = 1.0 + Delta * (1.0 - G[i, i])
    return model.weight_factor(s_i) * (r * np.conj(r)).real, r, Delta


class Chain:
    """One Markov chain: field, G at the current slice, and the UDT stacks.

    Rstack[c]: UDT of B_{c n_s} ... B_1;  Lstack[c]: UDT of (B_M ... B_{c n_s + 1})^T.
    """

    def __init__(self, model, n_delay, n_stab, seed=0, chain=0, field=None, measure=None):
        self.m = model
        self.n_delay = int(n_delay)
        self.n_stab = int(n_stab)
        if model.M % self.n_stab:
            raise ValueError("M must be a multiple of n_stab")
        self.nc = model.M // self.n_stab
        self.key = _rng.chain_key(seed, chain)
        self.field = (_rng.initial_field(seed, chain, model.M, model.N) if field is None
                      else np.array(field, dtype=np.int8, copy=True))
        self.sweep_index = 0
        self.proposed = 0
        self.accepted = 0
        self.measure = measure          # optional callback measure(chain, G, l)
        self.init_stacks()

    def init_stacks(self):
        m, ns = self.m, self.n_stab
        self.Rstack = [None] * (self.nc + 1)
        self.Lstack = [None] * (self.nc + 1)
        self.Rstack[0] = udt_identity(m.N)
        self.Lstack[self.nc] = udt_identity(m.N)
        for c in range(self.nc - 1, -1, -1):
            C = m.chain_product(self.field, c * ns + 1, (c + 1) * ns)
            self.Lstack[c] = udt_left_multiply(C.T, self.Lstack[c + 1])
        self.G = stable_green(self.Rstack[0], self.Lstack[0])

    # ---- the delayed update of one slice (Sec. III.B) --------------------
    def update_slice(self, l, pas):
        m = self.m
        N = m.N
        s = self.field[l - 1]
        G0 = self.G.copy()
        X, Y, sites = [], [], []
        for i in range(N):
            sig = float(s[i])
            Delta = m.flip_delta(sig)
            # Eq. DelayRatio: r = 1 + Delta {1 - G0_ii + sum_m x_m(i) y_m(i)}
            corr = sum(X[q][i] * Y[q][i] for q in range(len(X)))
            r = 1.0 + Delta * (1.0 - G0[i, i] + corr)
            R = m.weight_factor(sig) * (r * np.conj(r)).real
            u = _rng.uniform(self.key, _rng.proposal_counter(self.sweep_index, pas, l, i, m.M, N))
            self.proposed += 1
            if u < R:                               # Eq. DetailBalance
                self.accepted += 1
                # Eq. DelayRgenk
                x = G0[:, i].copy()
                y = -G0[i, :].copy()
                y[i] += 1.0
                for q in range(len(X)):
                    x -= X[q] * Y[q][i]
                    y += X[q][i] * Y[q]
                x *= Delta / r
                X.append(x)
                Y.append(y)
                sites.append(i)
                s[i] = -s[i]
                if len(X) == self.n_delay:          # Eq. FinalDelay
                    G0 = G0 - np.array(X).T @ np.array(Y)
                    X, Y = [], []
        if X:
            G0 = G0 - np.array(X).T @ np.array(Y)
        self.G = G0

    def sweep(self):
        m, ns = self.m, self.n_stab
        # forward pass
        for l in range(1, m.M + 1):
            self.G = m.wrap(self.G, self.field[l - 1])
            self.update_slice(l, 0)
            if l % ns == 0:
                c = l // ns
                C = m.chain_product(self.field, (c - 1) * ns + 1, c * ns)
                self.Rstack[c] = udt_left_multiply(C, self.Rstack[c - 1])
                self.G = stable_green(self.Rstack[c], self.Lstack[c])
                if self.measure is not None:
                    self.measure(self, self.G, l)
        # backward pass
        for l in range(m.M, 0, -1):
            self.update_slice(l, 1)
            self.G = m.unwrap(self.G, self.field[l - 1])
            if (l - 1) % ns == 0:
                c = (l - 1) // ns
                C = m.chain_product(self.field, c * ns + 1, (c + 1) * ns)
                self.Lstack[c] = udt_left_multiply(C.T, self.Lstack[c + 1])
                self.G = stable_green(self.Rstack[c], self.Lstack[c])
                if self.measure is not None:
                    self.measure(self, self.G, l - 1)
        self.sweep_index += 1
