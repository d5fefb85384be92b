"""Plain, slow FP64 CPU oracle for the finite-temperature AFQMC (DQMC) sweep of the
half-filled honeycomb Hubbard model.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline / reference arm
of ``bench.py`` may use it.  It shares no code with the CUDA path; the only
common module is ``synth`` (seeded input generators, no method arithmetic).

Every function states the passage of the paper it restates.  Dense linear
algebra (matrix products, determinants, LU solves, column-pivoted Householder
QR) comes from numpy/scipy as single library steps.

Modules
  lattice      honeycomb geometry, hopping matrix K, Bloch function f(k)   (Sec. II.A, III.C)
  linalg       Taylor matrix exponential, pivoted-QR UDT chains, stable (1+RL)^-1  (Sec. II.B)
  rng          counter-based SplitMix64 uniforms (not specified by the paper)
  dqmc         propagators, weights, ratios, local/delayed updates, the sweep, spin (Eq. SzHS)
               and charge (Eq. DensityHS) channel                      (Sec. II.B, III.A-B)
  observables  Wick-contracted equal-time observables (Sec. II.C, App. C)
  ed           Fock-space exact diagonalisation, continuum and Trotterised
  enumerate    exhaustive sum over Hubbard-Stratonovich fields for tiny systems
  tdgf         time-displaced Green's functions, C_{H_I}(tau), dD/dU, chi_F   (Eqs. DouOccDerive, fidelitysusp)
  learned      block-proposal network and exact block ratios (not in the paper)
  tabc         quasi-random twist sequence (Halton 2,3) and the twist average  (Sec. III.C)

Parity status: every function here is pinned by a test in tests/test_oracle_*.py
against closed forms, exact diagonalisation, brute-force determinants or
library routines; none is "parity unpinned".
"""
