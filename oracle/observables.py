"""Equal-time observables by Wick contraction (Sec. II.B 'Fifth', Sec. II.C, App. C).

Input: the spin-up Green's function G_ij = <c_i c_j^+> at a slice boundary of
the asymmetric Trotter product.  Readings:
  * observables are taken on G_sym = e^{-dtau H0/2} G e^{+dtau H0/2}, the
    Green's function of the symmetric third-order split used in production
    (the first implementation note of Sec. II.B); the weights of the two splits are identical;
  * spin down follows from the partial particle-hole transform with the
    staggered sign kept:  G_dn_ij = (-1)^{i+j} (delta_ij - conj(G_up_ji));
  * Wick:  <n_ia n_jb> = n_ia n_jb + delta_ab (delta_ij - G^a_ji) G^a_ij,
    n_ia = 1 - G^a_ii,  <c_i^+ c_j> = delta_ij - G_ji;
  * with a twist G is complex for one field: every Wick product is formed in
    complex arithmetic and its real part taken at the end (the weight is real
    and positive, and the imaginary parts average to zero);
  * R_m2 returned for one G is the per-field ratio 1 - S(Gamma+dk)/S(Gamma),
    used only for fixed-field parity; over many configurations Eq. CrfRatio
    is taken on the averages, 1 - <S(Gamma+dk)> / <S(Gamma)>.
Pins: tests/test_oracle_pins.py (exhaustive HS sum against Fock-space ED for
C_zz, S_zz(Gamma), S_zz(Gamma + b1/L), m^2, C_zz(L/2, 0); free-fermion closed
forms for S_zz, m^2, n(k), D, e, chi_e).
"""
import numpy as np


def spin_down_green(lat, Gup):
    ps = lat.sublattice_sign()
    return (ps[:, None] * ps[None, :]) * (np.eye(lat.N) - Gup.conj().T)


def measure(model, G):
    lat = model.lat
    N, Nc, L1, L2 = lat.N, lat.Nc, lat.L1, lat.L2
    Gu = model.Eh @ G @ model.Ehinv
    Gd = spin_down_green(lat, Gu)
    I = np.eye(N)
    nu = 1.0 - np.diag(Gu)
    nd = 1.0 - np.diag(Gd)
    # double occupancy D = N_s^-1 sum_i <n_i_up n_i_dn> (Sec. II.C, after Eq. ChiCharge)
    D = float(np.mean(nu * nd).real)
    # <H0> = sum_sigma sum_ij K_ij <c_i^+ c_j>  (App. C: E = <H0> + N_s U D)
    ekin = 0.0
    for Gs in (Gu, Gd):
        ekin += float(np.real(np.sum(model.K * (I - Gs.T))))
    energy = (ekin + N * model.U * D) / N
    # <s_i s_j> for all pairs, s = (n_up - n_dn)/2
    def nn(Ga, na, Gb, nb, same):
        out = np.outer(na, nb)
        if same:
            out = out + (I - Ga.T) * Ga
        return out
    ss = 0.25 * (nn(Gu, nu, Gu, nu, True) + nn(Gd, nd, Gd, nd, True)
                 - nn(Gu, nu, Gd, nd, False) - nn(Gd, nd, Gu, nu, False)).real
    # C_zz(r) = (1 / 2N_c) sum_i <s(r_i) s(r_i + r)>, r on the Bravais lattice (Eq. SzSzCrF)
    Czz = np.zeros((L2, L1))
    for sub in (0, 1):
        for n2 in range(L2):
            for n1 in range(L1):
                i = lat.site(sub, n1, n2)
                for d2 in range(L2):
                    for d1 in range(L1):
                        Czz[d2, d1] += ss[i, lat.site(sub, n1 + d1, n2 + d2)]
    Czz /= 2.0 * Nc
    # S_zz(k) = sum_r C_zz(r) e^{i k.r} (Eq. SpinStrucF); k.r = 2 pi (l1 d1/L1 + l2 d2/L2)
    def Szz(l1, l2):
        acc = 0.0 + 0.0j
        for d2 in range(L2):
            for d1 in range(L1):
                acc += Czz[d2, d1] * np.exp(2j * np.pi * (l1 * d1 / L1 + l2 * d2 / L2))
        return acc.real
    S0 = Szz(0, 0)
    Sdk = Szz(1, 0)                         # Gamma + b1/L (Eq. CrfRatio)
    # n_ab(k) = N_c^-1 sum_{I,J} e^{i q.(r_I - r_J)} <a_I^+ b_J>  (Eq. nkMatrix, spin up),
    # q the cell-DFT grid; with a twist (Gauge-I) this is the occupation at k = q + A
    cd = I - Gu.T                           # cd[i, j] = <c_i^+ c_j>
    nk = np.zeros((L2, L1, 2, 2), dtype=complex)
    for l2 in range(L2):
        for l1 in range(L1):
            k = lat.qvectors()[l1 + L1 * l2]
            ph = np.array([np.exp(1j * (k @ lat.bravais_vector(*lat.cell_coords(c)))) for c in range(Nc)])
            for a in (0, 1):
                for b in (0, 1):
                    blk = cd[a * Nc:(a + 1) * Nc, b * Nc:(b + 1) * Nc]
                    nk[l2, l1, a, b] = ph @ blk @ ph.conj() / Nc
    # charge compressibility (Eq. ChiCharge), one-configuration estimator:
    # chi_e = (beta / N_s) Re( sum_ij <n_i n_j> - N_s^2 ), n = n_up + n_dn, Wick for
    # every spin pair (the MC average of sum_i <n_i> is N_s at half filling)
    n_tot = nu + nd
    nn_sum = np.sum(np.outer(n_tot, n_tot))
    for Gs in (Gu, Gd):
        nn_sum = nn_sum + np.sum((I - Gs.T) * Gs)
    chi_e = float(model.beta / N * np.real(nn_sum - N * N))
    return dict(energy=energy, double_occ=D, ekin=ekin / N, Czz=Czz, S_af=S0, S_af_dk=Sdk, chi_e=chi_e,
                m2=S0 / (2.0 * Nc), R_m2=1.0 - Sdk / S0, Czz_half=Czz[0, L1 // 2], nk=nk,
                density=float(np.mean(nu + nd).real))
