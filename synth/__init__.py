"""Seeded synthetic inputs shared by the oracle-side tests, the CUDA-side tests and bench.py.

This module holds none of the method's arithmetic: it only defines the workload
shapes (lattice size, temperature, Trotter step, interaction, delay rank,
stabilisation period) and draws seeded random inputs (Ising field
configurations, dense test matrices).  Both the CPU oracle and the CUDA path
consume these inputs; neither side's numerics live here.
"""
import numpy as np

# Workload configurations (honeycomb Hubbard model, t = 1, half filling,
# periodic boundaries; spin-channel Ising Hubbard-Stratonovich field unless
# hs_channel = 1, the charge channel).
WORKLOADS = {
    # small case the oracle finishes in seconds
    "L3_beta3": dict(L=3, beta=3.0, dtau=0.1, U=3.73, n_delay=4, n_stab=10),
    # GPU plain FP64 case (three interaction strengths are run in the tests)
    "L6_beta6": dict(L=6, beta=6.0, dtau=0.1, U=3.73, n_delay=32, n_stab=10),
    # the headline sweep workload: N = 1152 sites, M = 240 slices
    "L24_beta24": dict(L=24, beta=24.0, dtau=0.1, U=3.73, n_delay=64, n_stab=8),
    # same N and kernels as the headline workload, 16 slices: small device
    # footprint for profiler captures
    "L24_beta1.6": dict(L=24, beta=1.6, dtau=0.1, U=3.73, n_delay=64, n_stab=8),
    # the charge-channel field (complex G held as its 2N x 2N real embedding,
    # hs_channel = 1) at the largest beta t = L lattice whose embedding fits the
    # column kernels (2N <= 2048), and the spin channel on the same lattice
    "L21_beta21_charge": dict(L=21, beta=21.0, dtau=0.1, U=3.73, n_delay=64, n_stab=7, hs_channel=1),
    "L21_beta21": dict(L=21, beta=21.0, dtau=0.1, U=3.73, n_delay=64, n_stab=7),
    # the headline lattice with the charge-channel field (device embedding 2304 x 2304)
    "L24_beta24_charge": dict(L=24, beta=24.0, dtau=0.1, U=3.73, n_delay=64, n_stab=8, hs_channel=1),
    # the learned-proposal lattice: N = 3528 sites, M = 420 slices (G: 99.6 MB)
    "L42_beta42": dict(L=42, beta=42.0, dtau=0.1, U=3.73, n_delay=64, n_stab=10),
}


# Batched twist-averaging workload: 64 independent chains of uneven size, each
# size on the uniform 4 x 4 grid of twist angles theta in {0, 1/4, 1/2, 3/4}^2
# (boundary phases 2 pi theta), beta t = L, U/t = 3.73, FP64.  64 chains over
# 3 sizes x 16 twists: 32 chains at L = 6 (two seeds per twist), 16 at L = 9,
# 16 at L = 12.
BATCHED = dict(sizes=((6, 2), (9, 1), (12, 1)), twists=4, dtau=0.1, U=3.73, n_stab=10)


# Learned block proposals, measured at the plain-GPU size (L = 6, beta t = 6):
# blocks of b x b cells x T slices, context h cells / ht slices, hidden width,
# training configurations taken one per sweep from a plain chain.
LEARNED = dict(L=6, beta=6.0, dtau=0.1, U=3.73, n_delay=32, n_stab=10, b=2, T=2, h=1, ht=1, hidden=64,
               n_cfg=600, train_steps=2000, batch=256, lr=3e-3)


# Reduced-precision study: the split-TF32 flush (precision 3: with the
# FP64-accurate tensor-core stabilisation products) against plain FP64
# (precision 0), independent seeds, equilibrium averages at L = 12, beta t = 12
# (and the headline L = 24 lattice); the drift profile uses n_stab in DRIFT_NS.
PRECISION_STUDY = dict(L12=dict(L=12, beta=12.0, dtau=0.1, U=3.73, n_delay=32, n_stab=8, chains=16, warm=60,
                                meas=200),
                       L24=dict(L=24, beta=24.0, dtau=0.1, U=3.73, n_delay=64, n_stab=8, chains=4, warm=30,
                                meas=30),
                       DRIFT_NS=(1, 2, 4, 8))


def batched_chains(twists=None):
    """(L, beta, theta, replica) of every chain of the batched workload.  twists:
    an explicit list of g*g twist angle pairs (e.g. a quasi-random sequence)
    replacing the uniform g x g grid."""
    out = []
    g = BATCHED["twists"]
    grid = [(a / g, b / g) for a in range(g) for b in range(g)] if twists is None else \
        [(float(t[0]), float(t[1])) for t in twists]
    if len(grid) != g * g:
        raise ValueError(f"the batched workload takes {g * g} twists per size")
    for L, reps in BATCHED["sizes"]:
        for th in grid:
            for r in range(reps):
                out.append((L, float(L), th, r))
    return out


def n_slices(beta, dtau):
    m = int(round(beta / dtau))
    if abs(m * dtau - beta) > 1e-9:
        raise ValueError("beta must be an integer multiple of dtau")
    return m


def random_field(M, N, seed):
    """Uniform i.i.d. Ising field s[l, i] in {+1, -1}, shape (M, N), int8."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.where(rng.random((M, N)) < 0.5, 1, -1).astype(np.int8)


def random_matrix(N, seed, scale=1.0):
    """Dense float64 N x N matrix with entries uniform in [-scale, scale)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return (2.0 * rng.random((N, N)) - 1.0) * scale
