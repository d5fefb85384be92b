"""Counter-based uniform random numbers for the Metropolis test (Eq. DetailBalance).

The paper does not specify a generator.  This project fixes one so that the
oracle and the CUDA path can be run in lockstep: each side implements it on
its own from its published definition.

SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): the n-th output (n >= 1) of the
stream seeded with s is mix64(s + n * GAMMA), with the finaliser
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
    z = (z ^ (z >> 27)) * 0x94D049BB133111EB
    z =  z ^ (z >> 31)
and a double in [0, 1) is (z >> 11) * 2^-53.

Stream of one Markov chain:  s_chain = mix64(seed ^ ((chain + 1) * 0xD1B54A32D192ED03)).
Counter of the proposal at site i of slice l (1-based) in pass p (0 forward,
1 backward) of sweep number w (0-based):  n = ((w*2 + p)*M + (l-1))*N + i + 1.
Initial field: s[l-1, i] = +1 if u(n = 2^62 + (l-1)*N + i + 1) < 0.5 else -1.
"""
MASK = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15
CHAIN_MUL = 0xD1B54A32D192ED03
INIT_BASE = 1 << 62


def mix64(z):
    z &= MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def chain_key(seed, chain):
    return mix64((seed ^ (((chain + 1) * CHAIN_MUL) & MASK)) & MASK)


def uniform(key, n):
    return (mix64((key + n * GAMMA) & MASK) >> 11) * (1.0 / 9007199254740992.0)


def proposal_counter(sweep, pas, l, i, M, N):
    return ((sweep * 2 + pas) * M + (l - 1)) * N + i + 1


def initial_field(seed, chain, M, N):
    import numpy as np
    key = chain_key(seed, chain)
    s = np.empty((M, N), dtype=np.int8)
    for l in range(M):
        for i in range(N):
            s[l, i] = 1 if uniform(key, INIT_BASE + l * N + i + 1) < 0.5 else -1
    return s
