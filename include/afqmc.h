/*
 * afqmc.h -- C ABI of libafqmc.so: the Monte Carlo sweep of finite-temperature
 * auxiliary-field QMC (DQMC) for the half-filled honeycomb Hubbard model on an
 * L1 x L2 two-sublattice lattice, run on one CUDA GPU (sm_103a).
 *
 * The method is the one of "Finite-temperature quantum Monte Carlo study of
 * Dirac quantum criticality: Algorithmic advances and comprehensive analysis":
 *   - model and Trotter/HS decomposition: Sec. II.A-B, Eqs. HubbModel, SzHS,
 *     coupling, ConfgWeight, GrFMat;
 *   - propagation G -> B G B^-1 with e^{-dtau K} applied in momentum space,
 *     one 2x2 Bloch block per k: Sec. III.A, Eqs. NewBlMat, ExpLambda,
 *     FourierMat, ColumnDem;
 *   - Metropolis updates with determinant ratios and the delayed rank-k
 *     Green's-function update: Sec. III.B, Eqs. DetailBalance, DRatio,
 *     rRatioLocal, DelayG0, DelayRatio, DelayRgenk, FinalDelay;
 *   - periodic QR stabilisation of the propagator chains: Sec. II.B (second note);
 *   - equal-time observables: Sec. II.C, App. C.
 *
 * Conventions shared by every entry point
 *   - Sites: N = 2*L1*L2.  Index i < Nc = L1*L2 is sublattice A, i >= Nc is B;
 *     within a sublattice the cell r = n1 a1 + n2 a2 has index n1 + L1*n2.
 *   - Slices l = 1..M, M = beta/dtau.  Field s[l-1][i] in {+1,-1}, int8,
 *     slice-major (M*N bytes).
 *   - Matrices are FP64, row-major, N*N, G[i][j] = <c_i c_j^+> of spin up.
 *   - Host pointers are owned by the caller and only read/written during the
 *     call; the library owns all device memory it allocates in afqmc_create.
 *   - All work is enqueued on the stream given to afqmc_create; calls that
 *     return host data synchronise that stream.
 *   - No C++ exception crosses this boundary.  A non-OK status leaves a message
 *     retrievable with afqmc_last_error(handle).  Numeric failures (NaN/Inf)
 *     and device-side wait timeouts return a status; nothing traps.
 *
 * Scope of this version: the spin-channel field (hs_channel = 0, Eq. SzHS) or
 * the charge-channel field (hs_channel = 1, Eq. DensityHS), one Markov chain
 * per handle, periodic (theta = 0) or twisted (theta != 0, Sec. III.C)
 * boundaries; FP64, optionally with tensor-core products (precision bits).
 *
 * Complex G (twisted boundaries, or the charge channel, whose propagator
 * e^{i alpha diag(s)} e^{-dtau K} is complex): every N x N matrix that crosses
 * this boundary (afqmc_get_G, afqmc_wrap_matrix, afqmc_update_slice,
 * afqmc_force_slice) is complex, row-major, interleaved (re, im): 2 N^2
 * doubles.  On the device it is held as its real 2N x 2N embedding
 * [[Re, -Im], [Im, Re]].  Only the spin channel with periodic boundaries has a
 * real G.
 */
#ifndef AFQMC_H
#define AFQMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct afqmc_handle afqmc_handle;

typedef enum {
    AFQMC_OK = 0,
    AFQMC_E_INVALID = 1,     /* bad argument or unsupported parameter combination */
    AFQMC_E_NOMEM = 2,       /* device or host allocation failed */
    AFQMC_E_CUDA = 3,        /* a CUDA runtime call failed */
    AFQMC_E_NUMERIC = 4,     /* NaN/Inf in G or in a ratio */
    AFQMC_E_TIMEOUT = 5,     /* a bounded device-side wait gave up */
    AFQMC_E_STATE = 6        /* handle unusable after an earlier error */
} afqmc_status;

/* Simulation parameters (Sec. II.A-B; Sec. III.B for n_delay). */
typedef struct {
    int32_t L1, L2;        /* unit cells along a1, a2 (>= 1) */
    double t;              /* hopping amplitude */
    double U;              /* Hubbard repulsion (>= 0) */
    double beta, dtau;     /* M = beta/dtau must be an integer (|M dtau - beta| < 1e-9) */
    double theta1, theta2; /* twist (Eq. kpoints: k = ((l + theta)/L) b), each in [0, 1);
                              any nonzero value selects the complex path */
    int32_t hs_channel;    /* 0 = spin channel HS-s^z (Eq. SzHS): B_l = e^{gamma_s diag(s)} e^{-dtau K},
                              flip ratio R = e^{2 gamma_s s} |r|^2.  1 = charge channel HS-n
                              (Eq. DensityHS): B_l = e^{i alpha diag(s)} e^{-dtau K} with
                              gamma_c = i alpha = i arccos(e^{-dtau U/2}) (Eq. coupling), R = |r|^2,
                              complex G.  Block proposals (afqmc_block_sweep) need 0 and theta = 0 */
    int32_t n_delay;       /* delay rank n_d >= 1; 1 is the local Sherman-Morrison update */
    int32_t n_stab;        /* slices between QR recomputations of G; M % n_stab == 0 */
    int32_t precision;     /* bit mask; 0 = FP64 everywhere.  Bit 0: delayed-update flush
                              G -= X Y as three TF32 tensor-core products (hi*hi + hi*lo + lo*hi,
                              FP32 accumulate) subtracted from the FP64 G.  Bit 1: the matrix
                              products of the stabilisation (stack extension, middle matrix and G
                              recomputation) on the BF16 tensor cores by the Ozaki scheme,
                              FP64-accurate (8 digits of 7 bits, exact FP32 class sums).  Bit 2
                              (needs bit 1): the triangular solves of the G recomputation blocked,
                              their couplings as bit-1 products and only diagonal blocks of at most
                              64 in FP64 (less latency for a chain alone; with several chains on one
                              GPU the many short tensor-core launches cost more than they save).
                              Ratios, x/y recursion, wraps, QR, LU and measurements stay FP64 */
    int32_t measure;       /* 1: accumulate observables at every recomputation of G in a sweep */
    int32_t chain;         /* chain index: selects the random stream */
    int32_t device;        /* CUDA device ordinal */
    int32_t update_ctas;   /* CTAs of the cooperative slice kernel; 0 = one per SM.  A tuning
                              knob only (results do not depend on it); see afqmc_batch_autotune */
    uint64_t seed;         /* random seed; also draws the initial field */
} afqmc_params;

/* Counters of the sweeps done by one afqmc_sweep call. */
typedef struct {
    uint64_t proposed;      /* single-site flips proposed (2*N*M per sweep) */
    uint64_t accepted;      /* flips accepted */
    double max_stab_drift;  /* max |G_wrapped - G_recomputed| over recomputations */
    uint64_t launches;      /* CUDA kernels launched by the call */
} afqmc_sweep_stats;

/* Per-kernel-family launch counts and device times (CUDA events on the
 * handle's stream), accumulated while timing is enabled. */
enum {
    AFQMC_K_PROPAGATE = 0,  /* momentum-space propagation rows (wrap, chain products, half step) */
    AFQMC_K_UPDATE = 1,     /* delayed-update slice kernel (proposals, x/y recursion, flush) */
    AFQMC_K_QR = 2,         /* Householder QR of the stack products */
    AFQMC_K_GEMM = 3,       /* FP64 GEMM */
    AFQMC_K_QRAUX = 4,      /* Q formation, pivoting, triangular solves of the middle matrix */
    AFQMC_K_MEASURE = 5,    /* observables */
    AFQMC_K_MISC = 6,       /* copies of identity, drift check, small helpers */
    AFQMC_K_LU = 7,         /* LU with partial pivoting of the middle matrix of G */
    AFQMC_K_COUNT = 8
};
typedef struct {
    uint64_t launches[AFQMC_K_COUNT];
    double ms[AFQMC_K_COUNT];
} afqmc_timing;

/* Equal-time observables (Sec. II.C; App. C).  Averages over n_samples measurements. */
typedef struct {
    double energy;      /* e = (<H0> + N U D) / N                          (App. C) */
    double double_occ;  /* D = N^-1 sum_i <n_i_up n_i_dn>                   (Sec. II.C) */
    double ekin;        /* <H0> / N */
    double density;     /* N^-1 sum_i <n_i> (1 at half filling) */
    double m2;          /* S_zz(Gamma) / (2 Nc)                             (Eq. SpinStrucF) */
    double S_af;        /* S_zz(Gamma) */
    double S_af_dk;     /* S_zz(Gamma + b1/L1) */
    double R_m2;        /* 1 - S_zz(Gamma + b1/L1) / S_zz(Gamma)            (Eq. CrfRatio) */
    double Czz_half;    /* C_zz(r = floor(L1/2) a1)                         (Eq. SzSzCrF) */
    double chi_e;       /* (beta / N) (<N^2> - <N>^2), charge compressibility (Eq. ChiCharge) */
    int64_t n_samples;
} afqmc_obs;

/* Create a chain: builds the lattice, the 2x2 Bloch propagator blocks
 * e^{-+dtau h(k)}, e^{-+dtau h(k)/2} (Eq. ExpLambda), draws the initial field
 * from (seed, chain), builds the QR-stabilised propagator stacks and G at
 * slice 0.  cuda_stream: a cudaStream_t (e.g. torch.cuda.Stream.cuda_stream) or
 * NULL for a stream owned by the handle.  *out is NULL on failure. */
afqmc_status afqmc_create(const afqmc_params* p, void* cuda_stream, afqmc_handle** out);

/* Release all device memory of the handle.  NULL is allowed. */
afqmc_status afqmc_destroy(afqmc_handle* h);

/* Replace the field (host, M*N int8, entries must be +1 or -1; otherwise
 * AFQMC_E_INVALID and the handle is unchanged), rebuild the stacks and G at
 * slice 0, reset the sweep counter to sweep_index. */
afqmc_status afqmc_set_field(afqmc_handle* h, const int8_t* s_host, uint64_t sweep_index);

/* Copy the current field to host (M*N int8). */
afqmc_status afqmc_get_field(afqmc_handle* h, int8_t* s_host);

/* Sanity limit on the stabilisation drift: at a recomputation of G, an element of
 * the wrapped G that differs from the recomputed one by more than
 * AFQMC_DRIFT_LIMIT * max(1, |G_ij|) makes the sweep fail with AFQMC_E_NUMERIC
 * (the chain no longer samples Eq. ConfgWeight).  The FP64 path drifts by ~1e-8
 * at L = 24, n_stab = 8; the split-TF32 flush by up to ~0.5 in the worst element
 * of long runs. */
#define AFQMC_DRIFT_LIMIT 10.0

/* Run n_sweeps sweeps (Sec. III.A: a forward pass l = 1..M and a backward pass
 * l = M..1; in each slice every site i = 0..N-1 is proposed once, accepted iff
 * u < R with R = e^{2 gamma s_i} |r|^2 (spin channel) or |r|^2 (charge channel),
 * r = 1 + Delta (1 - G_ii), Delta = e^{-2 gamma s_i} - 1 (gamma = gamma_s or
 * gamma_c), using the delayed update of rank n_delay; G recomputed every
 * n_stab slices).  stats may be NULL.  AFQMC_E_NUMERIC on a non-finite value
 * or a drift above AFQMC_DRIFT_LIMIT; AFQMC_E_TIMEOUT when a device wait runs
 * out. */
afqmc_status afqmc_sweep(afqmc_handle* h, int32_t n_sweeps, afqmc_sweep_stats* stats);

/* Measure the current G (the slice the chain is at: slice 0 between sweeps) now.
 * Czz (Nc doubles, order d1 + L1*d2) and nk (Nc*2*2 complex, interleaved
 * re,im, order (l1 + L1*l2)*4 + 2*a + b, n_ab(k) of Eq. nkMatrix) may be NULL. */
afqmc_status afqmc_measure(afqmc_handle* h, afqmc_obs* out, double* Czz, double* nk);

/* Averages of the measurements accumulated during sweeps since the last call
 * (params.measure = 1), then reset.  n_samples = 0 if none.  Arrays as above.
 * R_m2 here is the correlation ratio of the averages,
 * 1 - <S_zz(Gamma + b1/L1)> / <S_zz(Gamma)> (Eq. CrfRatio is defined on
 * expectation values), not the mean of per-field ratios. */
afqmc_status afqmc_get_obs(afqmc_handle* h, afqmc_obs* out, double* Czz, double* nk);

/* G at slice l (0 <= l <= M) recomputed from scratch for the current field by
 * QR-stabilised chains (Eq. GrFMat); written to out (host, N*N).  Observer path. */
afqmc_status afqmc_get_G(afqmc_handle* h, int32_t slice, double* out);

/* Propagate a host matrix with the current field (Sec. III.A): direction +1
 * computes B_l A B_l^-1, -1 computes B_l^-1 A B_l; 0 computes the half step
 * e^{-dtau K/2} A e^{+dtau K/2} used for measurements.  In place on A (N*N). */
afqmc_status afqmc_wrap_matrix(afqmc_handle* h, int32_t slice, int32_t direction, double* A);

/* Delayed update of slice l on a given G (host, N*N, in/out), pass 0 or 1, with
 * the random numbers of sweep number sweep_index; updates the handle's field
 * for slice l and returns the accepted count in *n_accepted (may be NULL). */
afqmc_status afqmc_update_slice(afqmc_handle* h, int32_t slice, int32_t pass,
                                uint64_t sweep_index, double* G, int32_t* n_accepted);

/* Weight ratio of flipping s[l-1][i] (Eqs. DRatio, rRatioLocal with the
 * particle-hole factor): out[0] = R = e^{2 gamma s} |r|^2 (spin channel) or
 * |r|^2 (charge channel), out[1] = Re r, out[2] = Im r (0 when G is real),
 * r = 1 + Delta (1 - G_ii), using G at slice l recomputed from scratch. */
afqmc_status afqmc_det_ratio(afqmc_handle* h, int32_t slice, int32_t site, double out[3]);

/* Time-displaced measurement of the current field (call between sweeps, the
 * chain at slice 0; M must be even): G(tau, 0), G(0, tau) and G(tau, tau) for
 * tau = l dtau, l = 0 .. M/2, from the QR-stabilised stacks every n_stab slices
 * and propagated in between, and the per-field estimator of
 * <H_I(tau) H_I(0)> (Wick; H_I = sum_i [n_up n_dn - (n_up + n_dn)/2]) on the
 * symmetric-split Green's functions, accumulated. */
afqmc_status afqmc_measure_td(afqmc_handle* h);

/* Averages since the last call, then reset: C[l] = <H_I(tau_l) H_I(0)> - <H_I>^2
 * for l = 0 .. M/2 (may be NULL), dD/dU = -(2/N) int_0^{beta/2} C dtau
 * (Eq. DouOccDerive) and chi_F = int_0^{beta/2} tau C dtau (Eq. fidelitysusp),
 * both by the trapezoidal rule over the slice times; n_samples = measurements. */
afqmc_status afqmc_get_td(afqmc_handle* h, double* C, double* dDdU, double* chiF, int64_t* n_samples);

/* Per-launch CUDA-event timing of the kernel families whose bit (1 << AFQMC_K_*)
 * is set in family_mask; 0 disables timing, AFQMC_TIMING_ALL times every
 * family.  Resets the totals.  Each timed launch records two events on the
 * handle's stream, so time only the families being studied when the
 * surrounding throughput matters.  Bits above AFQMC_TIMING_ALL: AFQMC_E_INVALID. */
#define AFQMC_TIMING_ALL ((1 << AFQMC_K_COUNT) - 1)
afqmc_status afqmc_set_timing(afqmc_handle* h, int32_t family_mask);

/* Totals since afqmc_set_timing (synchronises the stream); the launch counts
 * cover every family, the times only the timed ones (0 for the others). */
afqmc_status afqmc_get_timing(afqmc_handle* h, afqmc_timing* out);

/* Test hook for the failure paths (no counterpart in the paper): the limit, in
 * nanoseconds, of every device-side wait between CTAs of this handle's kernels
 * (grid barriers of the cooperative kernels, the column hand-offs of the QR and
 * LU).  0 restores the default of 2 s.  A wait that runs out sets the handle's
 * device error flag and its kernel returns; the next call that checks the
 * device returns AFQMC_E_TIMEOUT and every later call AFQMC_E_STATE.  Waits on
 * the tensor cores' own completion keep the 2 s limit.  Synchronises the
 * stream. */
afqmc_status afqmc_set_wait_limit(afqmc_handle* h, uint64_t wait_ns);

/* Largest sizes accepted by afqmc_update_slice_noalloc. */
#define AFQMC_NOALLOC_MAX_N 1152
#define AFQMC_NOALLOC_MAX_NDELAY 64

/* Allocation-free delayed update of one slice, for callers that cannot call
 * cudaMalloc: code running where the CUDA allocator is off limits (inside a
 * host allocator or a memory-pool callback, in a process whose device memory
 * is entirely owned by another framework's caching allocator, or under a
 * strict no-allocation policy for a real-time loop).  The paper has no
 * counterpart.  It covers one form only: the periodic, spin-channel chain
 * (real G, N = 2 L^2 physical sites) with the FP64 flush.  For that form it
 * computes what afqmc_update_slice computes on a handle created with
 * theta = (0, 0), hs_channel = 0 and precision 0 or 2; twisted,
 * charge-channel and split-TF32 (precision bit 0) handles compute something
 * else and have no allocation-free variant.
 *
 * The caller passes device pointers on the current device: G_dev (N*N FP64,
 * row-major, read and overwritten with the updated G) and s_dev (the N int8
 * field values of slice `slice`, +1/-1, flipped in place where accepted), plus
 * the sizes and physics parameters (N sites, M slices for the random-number
 * counter, U, dtau, n_delay) and the random stream (seed, chain, sweep_index,
 * pass).  All scratch lives in one file-scope __device__ array sized for
 * N <= AFQMC_NOALLOC_MAX_N and n_delay <= AFQMC_NOALLOC_MAX_NDELAY (about
 * 1.2 MB, held by every GPU that loads the library until the process exits);
 * larger sizes return AFQMC_E_INVALID with a message from
 * afqmc_last_error(NULL).  The call never allocates: no cudaMalloc/cudaFree
 * and no allocating library routine.
 *
 * The first call on a device does a one-time set-up on that device (looks up
 * the device address of the scratch array and sets the kernel's shared-memory
 * limit); that first call should come before any stream capture begins.
 * Every call shares the one scratch array, so calls that overlap on the GPU
 * (different streams or threads at the same time) race; serialise them.  The
 * call enqueues on cuda_stream (NULL = legacy default stream), copies the
 * status and the accepted count to host memory and synchronises the stream
 * before returning; *n_accepted (may be NULL) receives the number of accepted
 * flips. */
afqmc_status afqmc_update_slice_noalloc(double* G_dev, int8_t* s_dev, int32_t N, int32_t M, int32_t slice,
                                        int32_t pass, uint64_t sweep_index, double U, double dtau,
                                        int32_t n_delay, uint64_t seed, int32_t chain, void* cuda_stream,
                                        int32_t* n_accepted);

/* ---------------------------------------------------------------- batches
 * Independent chains (any mix of L, twist, seed; e.g. twist averaging over a
 * grid of boundary phases, Sec. III.C) run together on one device.  Each
 * chain keeps its own handle, stream and state; one sweep of the whole batch
 * is a single CUDA graph (captured on the first sweep: every chain's launch
 * sequence on its own branch), so the chains' kernels overlap on the GPU and
 * the host issues one launch per batched sweep.  Every chain computes exactly
 * what afqmc_sweep computes for it (same random numbers, same decisions). */
typedef struct afqmc_batch afqmc_batch;

/* Create n >= 1 chains from params[0..n-1] (all on params[0].device).
 * Per-launch timing is not available on batch chains. */
afqmc_status afqmc_batch_create(const afqmc_params* params, int32_t n, afqmc_batch** out);
afqmc_status afqmc_batch_destroy(afqmc_batch* b);

/* n_sweeps sweeps of every chain (one graph launch each); total (may be NULL)
 * sums proposed/accepted/launches over the chains, max_stab_drift is the max. */
afqmc_status afqmc_batch_sweep(afqmc_batch* b, int32_t n_sweeps, afqmc_sweep_stats* total);

/* Chain i of the batch (0 <= i < n), owned by the batch: use it for fields,
 * observables and G between batched sweeps; do not destroy it.  NULL if out of range. */
afqmc_handle* afqmc_batch_chain(afqmc_batch* b, int32_t i);

/* Autotuner: for the chains described by params[0..n-1], builds the batch for
 * every candidate (n_delays[a], ctas[c]) (ctas 0 = one CTA per SM), runs one
 * warm-up and n_timed timed batched sweeps, and returns the pair with the
 * highest total proposals per second (and that rate).  The delay rank and the
 * slice kernel's grid change only the speed, never the Markov chain (the
 * delayed update is exact algebra).  Errors from a candidate abort the search. */
afqmc_status afqmc_batch_autotune(const afqmc_params* params, int32_t n, const int32_t* n_delays, int32_t n_nd,
                                  const int32_t* ctas, int32_t n_ctas, int32_t n_timed, int32_t* best_n_delay,
                                  int32_t* best_ctas, double* best_rate);

/* Message of the last failed batch call on b (never NULL); b == NULL: the last
 * failure of afqmc_batch_create or afqmc_batch_autotune on this thread. */
const char* afqmc_batch_last_error(const afqmc_batch* b);

/* ---------------------------------------------------------------- learned block proposals
 * Not in the paper.  A small network proposes new values for a block of the
 * Ising field (b x b unit cells, both sublattices, T consecutive slices) from
 * the field around it (h cells and ht slices of context on every side, the
 * block itself masked); the chain accepts the proposal by Metropolis-Hastings
 * with the exact weight ratio W(X')/W(X) (the slice kernel flips the block's
 * changed sites one after the other and multiplies their ratios, Eq. DRatio)
 * and the proposal ratio q(s|x)/q(s'|x), so the stationary distribution stays
 * that of Eq. ConfgWeight whatever the network has learned.
 *
 * Network: z = W2 tanh(W1 x + b1) + b2 in FP32, x the context (+1/-1, 0 on the
 * block), one logit per block entry, q(s'|x) = prod_i sigmoid(s'_i z_i).
 * Orders: context ((t*W + w2)*W + w1)*2 + sub with W = b + 2h; block
 * ((t*b + c2)*b + c1)*2 + sub.  Parameters, one FP32 vector:
 * [W1 (H x Din, row-major) | b1 (H) | W2 (Dout x H) | b2 (Dout)]. */
typedef struct afqmc_net afqmc_net;

/* New network with seeded random weights on `device`. */
afqmc_status afqmc_net_create(int32_t b, int32_t T, int32_t h, int32_t ht, int32_t hidden, uint64_t seed,
                              int32_t device, afqmc_net** out);
afqmc_status afqmc_net_destroy(afqmc_net* net);

/* dims[0..3] = Din, H, Dout, number of parameters. */
afqmc_status afqmc_net_dims(const afqmc_net* net, int32_t dims[4]);
afqmc_status afqmc_net_get_params(afqmc_net* net, float* host);
afqmc_status afqmc_net_set_params(afqmc_net* net, const float* host);   /* also resets the Adam state */

/* Contexts X (B x Din) and block values S (B x Dout) of B blocks of host field
 * configurations (n_cfg x M x 2 L1 L2 int8) at pos[4q..4q+3] = (configuration,
 * l0, o1, o2), as the training and the block pass build them (test hook). */
afqmc_status afqmc_net_inputs(afqmc_net* net, const int8_t* fields, int32_t n_cfg, int32_t L1, int32_t L2, int32_t M,
                              const int32_t* pos, int32_t B, float* X, float* S);

/* Logits Z (B x Dout) of contexts X (B x Din), host buffers (test hook). */
afqmc_status afqmc_net_forward(afqmc_net* net, const float* X, int32_t B, float* Z);

/* Gradient (n_params, host) of the mean loss -sum_i log sigmoid(s_i z_i) over
 * the batch of contexts X (B x Din) and block values S (B x Dout, +1/-1), and
 * the loss (test hook; no update). */
afqmc_status afqmc_net_gradient(afqmc_net* net, const float* X, const float* S, int32_t B, float* grad, double* loss);

/* Train on the GPU: n_cfg field configurations (host, n_cfg x M x 2 L1 L2 int8,
 * e.g. taken from a chain of the plain sampler); each of n_steps Adam steps
 * (learning rate lr) uses `batch` blocks at random positions (configuration,
 * slice, cell offset) drawn from `seed`.  *loss: mean loss of the last step. */
afqmc_status afqmc_net_train(afqmc_net* net, const int8_t* fields, int32_t n_cfg, int32_t L1, int32_t L2, int32_t M,
                             int32_t n_steps, int32_t batch, float lr, uint64_t seed, double* loss);

typedef struct {
    uint64_t proposed;      /* block proposals */
    uint64_t accepted;      /* accepted block moves */
    uint64_t flipped;       /* field entries changed by accepted moves */
    double max_stab_drift;  /* max |G_wrapped - G_recomputed| over the pass */
} afqmc_block_stats;

/* One block pass of the chain: for every window of T slices (l0 = 1, 1+T, ...)
 * and every block offset (o1, o2 on the b-grid), propose with the network and
 * accept or reject (Metropolis-Hastings, exact ratios); G is recomputed from
 * the stacks every n_stab slices and at the end of the pass, where the chain
 * is back at slice 0 as after a sweep.  Requires a periodic (real) chain,
 * T | n_stab and b | L1, L2.  Random numbers: a stream of the chain's key
 * separate from the sweeps', indexed by the pass number. */
afqmc_status afqmc_block_sweep(afqmc_handle* h, afqmc_net* net, afqmc_block_stats* stats);

/* Slice update in forced mode (test hook): flip exactly the sites of slice l
 * with mask[i] != 0 (host, N int8) on a given G (host, N*N, in/out), updating
 * the handle's field; *logR = sum over the flips of log R = 2 gamma s + log |r|^2
 * (spin channel) or log |r|^2 (charge channel). */
afqmc_status afqmc_force_slice(afqmc_handle* h, int32_t slice, const int8_t* mask, double* G, double* logR);

/* Message of the last failed network call on net (never NULL); net == NULL:
 * the last failure of afqmc_net_create on this thread. */
const char* afqmc_net_last_error(const afqmc_net* net);

/* Twist angles for twist-averaged boundary conditions (Sec. III.C: N_Theta
 * independent twisted chains whose observables are averaged, the (theta1,
 * theta2) drawn from a 2D quasi-random sequence with the cumulative property).
 * The paper does not name the sequence; this library uses the Halton sequence
 * in bases 2 and 3: theta[2i] = phi_2(start + i), theta[2i+1] = phi_3(start + i),
 * phi_b the radical inverse (base-b digits mirrored behind the point), exact
 * fractions rounded once to double, each in [0, 1).  start = 1 skips the
 * periodic point (0, 0).  Any prefix of the sequence is evenly spread, so
 * N_Theta can grow without discarding chains.  theta: host, 2n doubles.
 * Host-only (no device work); AFQMC_E_INVALID if n < 0, start < 0 or
 * start + n >= 2^31, message in afqmc_last_error(NULL). */
afqmc_status afqmc_quasirandom_twists(int32_t n, int32_t start, double* theta);

/* Sizes of the handle: N (physical sites 2 Nc), M, Nc. */
afqmc_status afqmc_dims(const afqmc_handle* h, int32_t* N, int32_t* M, int32_t* Nc);

/* Message of the last failed call on h (never NULL).  With h == NULL: the last
 * failure of afqmc_create or afqmc_update_slice_noalloc on this thread. */
const char* afqmc_last_error(const afqmc_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* AFQMC_H */
