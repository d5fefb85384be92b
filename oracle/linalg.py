"""Dense FP64 linear algebra used by the oracle.

* ``expm_taylor``: matrix exponential by scaling-and-squaring of a truncated
  Taylor series (Moler & Van Loan, "Nineteen dubious ways to compute the
  exponential of a matrix", methods 1 and 3).  Used for e^{-dtau H0}; it never
  touches the momentum-space form of Sec. III.A, so the FFT propagation of the
  CUDA path is checked against an independent construction.
* ``udt``: A = U D T with U orthogonal, D > 0 diagonal, T = D^-1 R P^T from a
  column-pivoted Householder QR (scipy/LAPACK geqp3): the QR stabilisation of
  the second implementation note of Sec. II.B.
* ``stable_green``: G = (1 + R L)^-1 from R = U_R D_R T_R and L^T = U_L D_L T_L,
  by the large/small scale split of Loh & Gubernatis (1992) as written out in
  Bauer, SciPost Phys. Core 2, 011 (2020).
"""
import numpy as np
import scipy.linalg as sla


def expm_taylor(A, tol=1e-17, max_terms=60):
    A = np.asarray(A)
    nrm = np.linalg.norm(A, 1)
    s = 0
    if nrm > 0.5:
        s = int(np.ceil(np.log2(nrm / 0.5)))
    As = A / (2.0 ** s)
    term = np.eye(A.shape[0], dtype=A.dtype)
    out = term.copy()
    for n in range(1, max_terms):
        term = term @ As / n
        out = out + term
        if np.linalg.norm(term, 1) <= tol * np.linalg.norm(out, 1):
            break
    for _ in range(s):
        out = out @ out
    return out


def udt(A):
    """A = U @ diag(D) @ T via QR with column pivoting; D is made positive by
    moving the sign (real) or phase (complex) of R's diagonal into U."""
    Q, R, piv = sla.qr(A, pivoting=True, mode="full")
    d = np.diag(R).copy()
    D = np.abs(d)
    ph = np.where(D > 0, d / np.where(D > 0, D, 1.0), 1.0)
    if not np.iscomplexobj(A):
        ph = np.where(d < 0, -1.0, 1.0)
    Q = Q * ph[None, :]
    R = R * np.conj(ph)[:, None]
    Tp = R / D[:, None]                    # upper triangular, unit diagonal, columns in pivot order
    T = np.empty_like(Tp)
    T[:, piv] = Tp                         # undo the column permutation: T = D^-1 R P^T
    return Q, D, T


def udt_identity(n):
    return np.eye(n), np.ones(n), np.eye(n)


def udt_left_multiply(C, udt_in):
    """UDT of C @ (U D T): decompose (C U) D with pivoted QR, then chain T."""
    U, D, T = udt_in
    U2, D2, T2 = udt((C @ U) * D[None, :])
    return U2, D2, T2 @ T


def stable_green(udt_R, udt_L):
    """G = (1 + R L)^-1 with R = U_R D_R T_R and L = (U_L D_L T_L)^T (plain
    transpose), U_R and U_L unitary:

    1 + R L = U_R Db_R [ Db_R^-1 U_R^H conj(U_L) Db_L^-1 + Ds_R T_R T_L^T Ds_L ] Db_L U_L^T,
    Db = max(D, 1), Ds = min(D, 1); for real matrices U^H = U^T and conj(U) = U.
    """
    UR, DR, TR = udt_R
    UL, DL, TL = udt_L
    DbR, DsR = np.maximum(DR, 1.0), np.minimum(DR, 1.0)
    DbL, DsL = np.maximum(DL, 1.0), np.minimum(DL, 1.0)
    URh = UR.conj().T
    ULc = UL.conj()
    Mmid = (URh @ ULc) / DbR[:, None] / DbL[None, :] + (DsR[:, None] * (TR @ TL.T)) * DsL[None, :]
    rhs = URh / DbR[:, None]
    X = np.linalg.solve(Mmid, rhs)
    return (ULc / DbL[None, :]) @ X
