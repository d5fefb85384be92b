"""Time-displaced Green's functions and the interaction autocorrelation
C_{H_I}(tau) of Eqs. DouOccDerive and fidelitysusp (test infrastructure, FP64,
dense products: small beta only).

For one field, with B(l, 0) = B_l ... B_1 and G(0) = (1 + B(M, 0))^-1
(Eq. GrFMat at slice 0), the up-spin Green's functions at tau = l dtau > 0 are
  G(tau, 0)   = <c(tau) c^+(0)>  = B(l, 0) G(0),
  G(0, tau)   = -<c^+(tau) c(0)>^T = -(1 - G(0)) B(l, 0)^-1,
  G(tau, tau) = (1 + B(l, 0) B(M, l))^-1,
and at tau = 0 the limit 0+ (G(0, 0+) = G(0) - 1).  Observables use the
symmetric split, X_sym = e^{-dtau K/2} X e^{+dtau K/2} for all three.

Spin down follows from the partial particle-hole transform, c_i,dn ->
(-1)^i d_i^+, whose propagator is the complex conjugate of the up-spin one:
  G_dn(tau, 0)_ij = -(-1)^{i+j} conj(G_up(0, tau)_ji),
  G_dn(0, tau)_ij = -(-1)^{i+j} conj(G_up(tau, 0)_ji),
  G_dn(tau, tau)_ij = (-1)^{i+j} (delta_ij - conj(G_up(tau, tau)_ji)).
Wick, per spin s, tau > 0:
  <n_is(tau) n_js(0)> = n_is(tau) n_js(0) - G_s(0, tau)_ji G_s(tau, 0)_ij,
different spins factorise.  H_I = sum_i [n_i,up n_i,dn - (n_i,up + n_i,dn)/2].
"""
import numpy as np

from .observables import spin_down_green


def greens(model, field, l):
    """(G(tau,0), G(0,tau), G(tau,tau), G(0,0)) at tau = l dtau, 0 <= l <= M, unsymmetrised."""
    N = model.N
    I = np.eye(N)
    Bl0 = model.chain_product(field, 1, l)
    G00 = np.linalg.inv(I + model.chain_product(field, 1, model.M))
    Gt0 = Bl0 @ G00
    G0t = -(I - G00) @ np.linalg.inv(Bl0)
    Gtt = model.green_direct(field, l)
    return Gt0, G0t, Gtt, G00


def hi_products(model, field, l):
    """(<H_I(tau) H_I(0)>, <H_I>) for one field, tau = l dtau (Wick, complex arithmetic, real part)."""
    lat = model.lat
    N = model.N
    I = np.eye(N)
    sym = lambda X: model.Eh @ X @ model.Ehinv
    Gt0, G0t, Gtt, G00 = (sym(X) for X in greens(model, field, l))
    ps = lat.sublattice_sign()
    S = ps[:, None] * ps[None, :]
    up = dict(t0=Gt0, t0b=G0t, tt=Gtt, oo=G00)
    dn = dict(t0=-S * G0t.conj().T, t0b=-S * Gt0.conj().T,
              tt=spin_down_green(lat, Gtt), oo=spin_down_green(lat, G00))
    if l == 0:
        # equal time: the 0+ limit of G(0, tau) and G(tau, 0) = G(0)
        for d, G in ((up, G00), (dn, spin_down_green(lat, G00))):
            d["t0"], d["t0b"] = G, G - I

    def parts(d):
        a = 1.0 - np.diag(d["tt"])                 # <n_i(tau)>
        b = 1.0 - np.diag(d["oo"])                 # <n_j(0)>
        X = np.outer(a, b) - d["t0b"].T * d["t0"]  # <n_i(tau) n_j(0)>, [i, j]
        return a, b, X

    au, bu, Xu = parts(up)
    ad, bd, Xd = parts(dn)
    # <A_i(tau) B_j(0)>, A = n_up n_dn - (n_up + n_dn)/2, spins factorised
    AB = (Xu * Xd
          - 0.5 * (Xu * ad[:, None] + au[:, None] * Xd)
          - 0.5 * (Xu * bd[None, :] + bu[None, :] * Xd)
          + 0.25 * (Xu + Xd + np.outer(au, bd) + np.outer(ad, bu)))
    # equal-time <H_I> at slice 0: n_up n_dn factorises on one site
    b_up, b_dn = 1.0 - np.diag(up["oo"]), 1.0 - np.diag(dn["oo"])
    H = np.sum(b_up * b_dn - 0.5 * (b_up + b_dn))
    return float(np.real(AB.sum())), float(np.real(H))


def integrals(C, dtau, N):
    """(dD/dU, chi_F) from C(tau_l), l = 0 .. M/2, by the trapezoidal rule:
    dD/dU = -(2/N) int_0^{beta/2} C dtau (Eq. DouOccDerive), chi_F = int_0^{beta/2} tau C dtau
    (Eq. fidelitysusp)."""
    C = np.asarray(C, dtype=float)
    tau = dtau * np.arange(len(C))
    trap = lambda y: dtau * (y.sum() - 0.5 * (y[0] + y[-1]))
    return -2.0 / N * trap(C), trap(tau * C)
