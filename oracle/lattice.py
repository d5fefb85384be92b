"""Honeycomb lattice of Sec. II.A (Fig. 1, Eq. h0kMat) with the twisted boundary
phases of Sec. III.C (Eqs. VecATBC, PhaseFact, GaugeIPhase, kpoints).

Site order (Sec. III.A, below Eq. ExpLambda): all A sites first, then all B
sites.  Within a sublattice the unit cell r = n1 a1 + n2 a2 has index
n1 + L1 * n2.  Gauge-I (Sec. III.C): A and B of one cell share the coordinate
r, and A(r) bonds to B(r + delta) with delta in {0, a1 - a2, -a2}.
"""
import numpy as np

SQ3 = np.sqrt(3.0)
A1 = np.array([SQ3, 0.0])            # primitive vectors, Fig. 1(a)
A2 = np.array([SQ3 / 2.0, 1.5])
B1 = np.array([2.0 * np.pi / SQ3, -2.0 * np.pi / 3.0])   # reciprocal vectors, Sec. II.A
B2 = np.array([0.0, 4.0 * np.pi / 3.0])
# nearest-neighbour displacements of the B partner, in units of (a1, a2) (Sec. III.C, Gauge-I)
DELTAS = ((0, 0), (1, -1), (0, -1))


class Honeycomb:
    def __init__(self, L1, L2=None, t=1.0, theta=(0.0, 0.0)):
        self.L1 = int(L1)
        self.L2 = int(L1 if L2 is None else L2)
        self.t = float(t)
        self.theta = (float(theta[0]), float(theta[1]))
        self.Nc = self.L1 * self.L2
        self.N = 2 * self.Nc

    # ---- indexing -------------------------------------------------------
    def cell(self, n1, n2):
        return (n1 % self.L1) + self.L1 * (n2 % self.L2)

    def site(self, sub, n1, n2):
        return sub * self.Nc + self.cell(n1, n2)

    def cell_coords(self, c):
        return c % self.L1, c // self.L1

    def sublattice_sign(self):
        """(-1)^i of the partial particle-hole transform (Sec. II.B, 'Fourth'): +1 on A, -1 on B."""
        return np.concatenate([np.ones(self.Nc), -np.ones(self.Nc)])

    # ---- hopping --------------------------------------------------------
    def bond_phase(self, d1, d2):
        """Peierls phase Phi = A . delta with A . a_alpha = 2 pi theta_alpha / L_alpha (Eqs. VecATBC, GaugeIPhase)."""
        return 2.0 * np.pi * (self.theta[0] * d1 / self.L1 + self.theta[1] * d2 / self.L2)

    def bonds(self):
        """List of (i_A, j_B, Phi) for the three bonds leaving every A site."""
        out = []
        for n2 in range(self.L2):
            for n1 in range(self.L1):
                i = self.site(0, n1, n2)
                for d1, d2 in DELTAS:
                    out.append((i, self.site(1, n1 + d1, n2 + d2), self.bond_phase(d1, d2)))
        return out

    def hopping_matrix(self):
        """Dense N x N single-particle hopping matrix H0 of Eq. HubbModel.

        Reading (the twist sign): the bond A(r) -> B(r+delta) carries -t e^{+i Phi}
        so that the spectrum is +-|f(k + A)|, the shifted grid of Eq. kpoints.
        Real when theta = (0, 0).
        """
        K = np.zeros((self.N, self.N), dtype=complex)
        for i, j, phi in self.bonds():
            K[i, j] += -self.t * np.exp(1j * phi)
            K[j, i] += -self.t * np.exp(-1j * phi)
        if self.theta == (0.0, 0.0):
            return K.real.copy()
        return K

    # ---- momentum space -------------------------------------------------
    def kvectors(self):
        """k = ((l1+theta1)/L1) b1 + ((l2+theta2)/L2) b2, ordered l1 + L1*l2 (Eq. kpoints)."""
        ks = []
        for l2 in range(self.L2):
            for l1 in range(self.L1):
                ks.append((l1 + self.theta[0]) / self.L1 * B1 + (l2 + self.theta[1]) / self.L2 * B2)
        return np.array(ks)

    def qvectors(self):
        """The untwisted grid q = (l1/L1) b1 + (l2/L2) b2 of the DFT over cells.

        In Gauge-I the twist sits on the bonds, so K stays translation invariant:
        the cell DFT with these q block-diagonalises it, and block q carries the
        Bloch matrix at the shifted momentum k = q + A (kvectors)."""
        return np.array([(l1 / self.L1) * B1 + (l2 / self.L2) * B2
                         for l2 in range(self.L2) for l1 in range(self.L1)])

    def f_of_k(self, k):
        """f(k) = -t [1 + e^{i k.(a1-a2)} + e^{-i k.a2}] (below Eq. h0kMat)."""
        return -self.t * (1.0 + np.exp(1j * (k @ (A1 - A2))) + np.exp(-1j * (k @ A2)))

    def bravais_vector(self, d1, d2):
        return d1 * A1 + d2 * A2
