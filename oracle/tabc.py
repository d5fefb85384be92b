"""Twist-averaged boundary conditions (Sec. III.C, test infrastructure).

N_Theta independent twisted simulations, their observables averaged; the twist
angles (theta1, theta2) in [0, 1)^2 come from a 2D quasi-random sequence
(Sec. III.C; the paper does not name it).  Reading taken here: the Halton
sequence in bases 2 and 3, (phi_2(m), phi_3(m)) for m = start, start + 1, ...,
where phi_b(m) mirrors the base-b digits of m behind the point (the radical
inverse of van der Corput and Halton).  Computed as exact fractions and
rounded once to double.
"""
from fractions import Fraction

import numpy as np


def radical_inverse(m, b):
    """phi_b(m) as an exact Fraction: m = sum_k d_k b^k  ->  sum_k d_k b^-(k+1)."""
    out, scale = Fraction(0), Fraction(1, b)
    while m:
        m, d = divmod(m, b)
        out += d * scale
        scale /= b
    return out


def halton_twists(n, start=1):
    """(n, 2) float array of (phi_2(m), phi_3(m)), m = start .. start + n - 1."""
    return np.array([[float(radical_inverse(m, 2)), float(radical_inverse(m, 3))]
                     for m in range(start, start + n)], dtype=float).reshape(n, 2)


def twist_average(values):
    """TABC estimate: the plain mean over the twists (first axis)."""
    return np.mean(np.asarray(values, dtype=float), axis=0)
