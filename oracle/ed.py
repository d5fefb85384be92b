"""Fock-space exact diagonalisation of the Hubbard Hamiltonian of Eq. HubbModel
for small clusters, used to pin the oracle's weights and Wick contractions.

Two forms:
  * ``trotter_averages``: the Trotterised density matrix
    rho = (e^{-dtau H0/2} e^{-dtau H_U} e^{-dtau H0/2})^M  (first implementation note of Sec. II.B),
    which the Hubbard-Stratonovich sum reproduces exactly at any dtau;
  * ``thermal_averages``: exact e^{-beta H} by full diagonalisation (tiny clusters).

Each (N_up, N_dn) sector is the tensor product V_up x V_dn of one-species Fock
spaces; a state is a pair of bit masks, fermion signs by Jordan-Wigner order
(site index), all up operators ordered before all down operators.
"""
import itertools
import numpy as np
import scipy.linalg as sla


def species_basis(N, n):
    states = [sum(1 << i for i in c) for c in itertools.combinations(range(N), n)]
    return states, {s: a for a, s in enumerate(states)}


def species_hopping(K, states, index):
    """Matrix of sum_ij K_ij c_i^+ c_j in the fixed-particle-number basis."""
    N = K.shape[0]
    d = len(states)
    H = np.zeros((d, d), dtype=K.dtype)
    for a, s in enumerate(states):
        for j in range(N):
            if not (s >> j) & 1:
                continue
            s1 = s ^ (1 << j)
            sg1 = (-1) ** bin(s & ((1 << j) - 1)).count("1")
            for i in range(N):
                if K[i, j] == 0 or (s1 >> i) & 1:
                    continue
                s2 = s1 | (1 << i)
                sg2 = (-1) ** bin(s1 & ((1 << i) - 1)).count("1")
                H[index[s2], a] += K[i, j] * sg1 * sg2
    return H


def occupations(states, N):
    return np.array([[(s >> i) & 1 for i in range(N)] for s in states], dtype=float)


def _sector_data(K, N, nu, nd):
    su, iu = species_basis(N, nu)
    sd, idd = species_basis(N, nd)
    return (species_hopping(K, su, iu), species_hopping(K, sd, idd),
            occupations(su, N), occupations(sd, N))


def _observables_diag(occ_u, occ_d, U, bravais_pairs):
    """Diagonal observables on the product basis, arrays of shape (du, dd)."""
    nu = occ_u[:, None, :]
    nd = occ_d[None, :, :]
    docc = (nu * nd).sum(axis=2)                       # sum_i n_i_up n_i_dn
    hu = U * (nu * nd - 0.5 * (nu + nd)).sum(axis=2)  # H_U eigenvalues
    sz = 0.5 * (nu - nd)                                # (du, dd, N)
    czz = {key: sum((sz[..., i] * sz[..., j]) for i, j in pairs) for key, pairs in bravais_pairs.items()}
    return docc, hu, czz


def _structure_diag(occ_u, occ_d, lat):
    """Spin structure factor of every basis state, computed directly from the
    spin density (no detour through C_zz): for each k = (l1/L1) b1 + (l2/L2) b2,
    S(k) = (|sum_{i in A} e^{ik.r_i} s_i|^2 + |sum_{i in B} e^{ik.r_i} s_i|^2) / (2 N_c),
    r_i the Bravais vector of site i's cell, s_i = (n_up - n_dn)/2.  Summed over
    i and j of one sublattice this is the double sum that Eq. SpinStrucF applied
    to Eq. SzSzCrF amounts to on the periodic lattice.  Shape (du, dd, N_c),
    k index l1 + L1 * l2."""
    Nc, L1, L2 = lat.Nc, lat.L1, lat.L2
    sz = 0.5 * (occ_u[:, None, :] - occ_d[None, :, :])
    ph = np.empty((Nc, Nc), dtype=complex)           # ph[k, cell] = e^{i k.r_cell}
    for l2 in range(L2):
        for l1 in range(L1):
            for c in range(Nc):
                n1, n2 = lat.cell_coords(c)
                ph[l1 + L1 * l2, c] = np.exp(2j * np.pi * (l1 * n1 / L1 + l2 * n2 / L2))
    amp_a = sz[..., :Nc] @ ph.T
    amp_b = sz[..., Nc:] @ ph.T
    return (np.abs(amp_a) ** 2 + np.abs(amp_b) ** 2) / (2.0 * Nc)


def bravais_pair_table(lat):
    """For C_zz(r): r=(d1,d2) -> list of site pairs (i, i+r) on the same sublattice."""
    out = {}
    for d2 in range(lat.L2):
        for d1 in range(lat.L1):
            pairs = []
            for sub in (0, 1):
                for n2 in range(lat.L2):
                    for n1 in range(lat.L1):
                        pairs.append((lat.site(sub, n1, n2), lat.site(sub, n1 + d1, n2 + d2)))
            out[(d1, d2)] = pairs
    return out


def trotter_averages(lat, K, U, dtau, M):
    """<D>, <e>, C_zz under the Trotterised density matrix (exact for the HS sum)."""
    N = lat.N
    pairs = bravais_pair_table(lat)
    Z = 0.0
    acc_d = acc_kin = acc_n1 = acc_n2 = 0.0
    acc_c = {k: 0.0 for k in pairs}
    acc_s = np.zeros(lat.Nc)
    acc_m = 0.0
    for nu in range(N + 1):
        for nd in range(N + 1):
            Ku, Kd, ou, od = _sector_data(K, N, nu, nd)
            du, dd = Ku.shape[0], Kd.shape[0]
            Su = sla.expm(-0.5 * dtau * Ku)
            Sd = sla.expm(-0.5 * dtau * Kd)
            docc, hu, czz = _observables_diag(ou, od, U, pairs)
            eU = np.exp(-dtau * hu)
            X = np.eye(du * dd).reshape(du, dd, du * dd)
            for _ in range(M):
                X = np.tensordot(Su, X, axes=(1, 0))
                X = np.matmul(Sd, X)
                X = eU[:, :, None] * X
                X = np.tensordot(Su, X, axes=(1, 0))
                X = np.matmul(Sd, X)
            ia, ib = np.divmod(np.arange(du * dd), dd)
            diag = X[ia, ib, np.arange(du * dd)].reshape(du, dd)
            Z += diag.sum()
            acc_n1 += (nu + nd) * diag.sum()                # N is conserved: sector weight x N
            acc_n2 += (nu + nd) ** 2 * diag.sum()
            acc_d += (docc * diag).sum()
            for key in pairs:
                acc_c[key] += (czz[key] * diag).sum()
            acc_s += np.real((_structure_diag(ou, od, lat) * diag[..., None]).sum(axis=(0, 1)))
            # squared sublattice magnetisations (sum_{i in A} s_i)^2 + (sum_{i in B} s_i)^2
            sz = 0.5 * (ou[:, None, :] - od[None, :, :])
            ms = sz[..., :lat.Nc].sum(axis=2) ** 2 + sz[..., lat.Nc:].sum(axis=2) ** 2
            acc_m += np.real((ms * diag).sum())
            KX = np.tensordot(Ku, X, axes=(1, 0)) + np.matmul(Kd, X)
            acc_kin += KX[ia, ib, np.arange(du * dd)].sum()
    # with a twist the sector matrices are complex; the traces are real up to rounding
    Z, acc_d, acc_kin = np.real(Z), np.real(acc_d), np.real(acc_kin)
    acc_n1, acc_n2 = np.real(acc_n1), np.real(acc_n2)
    D = acc_d / Z / N
    ekin = acc_kin / Z
    Czz = np.zeros((lat.L2, lat.L1))
    for (d1, d2), v in acc_c.items():
        Czz[d2, d1] = np.real(v) / Z / (2.0 * lat.Nc)
    # Eq. ChiCharge: (beta / N_s) (<N^2> - <N>^2), beta = M dtau
    chi_e = M * dtau / N * (acc_n2 / Z - (acc_n1 / Z) ** 2)
    # S_zz(k) from the spin density itself, and m^2 = <M_A^2 + M_B^2> / (2 N_c)^2
    # (the Neel order parameter squared, Sec. II.C below Eq. SpinStrucF)
    Szz = (acc_s / Z).reshape(lat.L2, lat.L1)
    m2 = acc_m / Z / (2.0 * lat.Nc) ** 2
    return dict(double_occ=D, energy=(ekin + N * U * D) / N, ekin=ekin / N, Czz=Czz, chi_e=chi_e, Szz=Szz, m2=m2)


def thermal_averages(lat, K, U, beta):
    """Exact thermal <D> and <e> by full diagonalisation (only for tiny N)."""
    N = lat.N
    Z = acc_d = acc_kin = 0.0
    for nu in range(N + 1):
        for nd in range(N + 1):
            Ku, Kd, ou, od = _sector_data(K, N, nu, nd)
            du, dd = Ku.shape[0], Kd.shape[0]
            docc, hu, _ = _observables_diag(ou, od, U, {})
            H0 = np.kron(Ku, np.eye(dd)) + np.kron(np.eye(du), Kd)
            H = H0 + np.diag(hu.reshape(-1))
            w, V = np.linalg.eigh(H)
            p = np.exp(-beta * w)
            Z += p.sum()
            acc_d += np.einsum("n,in,i,in->", p, V.conj(), docc.reshape(-1), V).real
            acc_kin += np.einsum("n,in,ij,jn->", p, V.conj(), H0, V).real
    D = acc_d / Z / N
    ekin = acc_kin / Z
    return dict(double_occ=D, energy=(ekin + N * U * D) / N, ekin=ekin / N)


def trotter_hi_correlation(lat, K, U, dtau, M):
    """<H_I(tau_l) H_I(0)> and <H_I> under the Trotterised density matrix
    rho = S^M, S = e^{-dtau H0/2} e^{-dtau H_U} e^{-dtau H0/2}, for l = 0..M:
    Tr[S^{M-l} H_I S^l H_I] / Tr[S^M] with H_I = sum_i [n_up n_dn - (n_up + n_dn)/2]
    (diagonal in the occupation basis).  Dense per sector: tiny clusters only."""
    N = lat.N
    Z = 0.0
    hh = np.zeros(M + 1)
    h1 = 0.0
    for nu in range(N + 1):
        for nd in range(N + 1):
            Ku, Kd, ou, od = _sector_data(K, N, nu, nd)
            du, dd = Ku.shape[0], Kd.shape[0]
            Sh = np.kron(sla.expm(-0.5 * dtau * Ku), sla.expm(-0.5 * dtau * Kd))
            nuu = ou[:, None, :]
            ndd = od[None, :, :]
            hi = (nuu * ndd - 0.5 * (nuu + ndd)).sum(axis=2).reshape(-1)
            S = Sh @ (np.exp(-dtau * U * hi)[:, None] * Sh)
            P = [np.eye(du * dd)]
            for _ in range(M):
                P.append(P[-1] @ S)
            Z += np.trace(P[M])
            h1 += np.trace(P[M] * hi[None, :])      # Tr[S^M H_I]
            for l in range(M + 1):
                hh[l] += np.real(np.sum((P[M - l] * hi[None, :]) * (P[l] * hi[None, :]).T))
    Z = np.real(Z)
    return hh / Z, np.real(h1) / Z


def trotter_dDdU(lat, K, U, dtau, M):
    """dD/dU of the Trotterised density matrix, exactly: with S = Eh e^{-dtau U H_I} Eh
    (Eh = e^{-dtau H0/2}), d(S^M)/dU = -dtau sum_l S^{M-1-l} (Eh H_I e^{-dtau U H_I} Eh) S^l,
    so dD/dU = -dtau sum_l cov(D, H_I at the middle of slice l), D = N^-1 sum_i n_up n_dn."""
    N = lat.N
    Z = dsum = dmid = 0.0
    cross = 0.0
    for nu in range(N + 1):
        for nd in range(N + 1):
            Ku, Kd, ou, od = _sector_data(K, N, nu, nd)
            du, dd = Ku.shape[0], Kd.shape[0]
            Eh = np.kron(sla.expm(-0.5 * dtau * Ku), sla.expm(-0.5 * dtau * Kd))
            nuu = ou[:, None, :]
            ndd = od[None, :, :]
            hi = (nuu * ndd - 0.5 * (nuu + ndd)).sum(axis=2).reshape(-1)
            docc = (nuu * ndd).sum(axis=2).reshape(-1) / N
            eU = np.exp(-dtau * U * hi)
            S = Eh @ (eU[:, None] * Eh)
            Smid = Eh @ ((hi * eU)[:, None] * Eh)
            P = [np.eye(du * dd)]
            for _ in range(M):
                P.append(P[-1] @ S)
            Z += np.trace(P[M])
            dsum += np.trace(P[M] * docc[None, :])
            dmid += np.trace(P[M - 1] @ Smid)
            for l in range(M):
                cross += np.trace(P[M - 1 - l] @ Smid @ (P[l] * docc[None, :]))
    Z, dsum, dmid, cross = (np.real(x) for x in (Z, dsum, dmid, cross))
    return -dtau * (cross / Z - M * (dsum / Z) * (dmid / Z))
