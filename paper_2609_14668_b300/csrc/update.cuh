// Delayed rank-k Green's-function update of one time slice (Sec. III.B).
//
// Every site i = 0..N-1 of slice l is proposed once, in ascending order.  The
// flip s_i -> -s_i has Delta = e^{-2 gamma s_i} - 1, r = 1 + Delta (1 - G_ii)
// (Eq. DelayRatio with the maintained diagonal) and weight ratio
// R = e^{2 gamma s_i} r^2 (the particle-hole factor of the spin channel); it is
// accepted iff u < R (Eq. DetailBalance).  Accepted moves add x_k, y_k of
// Eq. DelayRgenk; after n_delay accepted moves, and at the end of the slice,
// G <- G - X Y (Eq. FinalDelay).
//
// Charge channel (Eq. DensityHS, charge = 1, always on the embedding): Delta =
// e^{-2 i alpha s_i} - 1 is complex and R = |r|^2.  The complex rank-1 move
// G <- G - kappa G(:,p) (1 - G)(p,:), kappa = Delta / r, is in the embedding the
// sum of two real rank-1 moves taken together (not one after the other):
//   x1 = kappa_r z_p + kappa_i z_q,  x2 = -kappa_i z_p + kappa_r z_q,  y1 = w_p, y2 = w_q,
// with z_p, z_q the columns p, q = p + Np and w_p, w_q the rows p, q of the
// current G and 1 - G, so the window, the x/y recursion and the flush keep
// their real form; mcoef holds kappa_r at the first and kappa_i at the second.
//
// GPU schedule (one cooperative kernel per slice, all SMs):
//   B  CTA 0 proposes the sites of a window of W consecutive sites.  It holds
//      the W x W block of the current G on chip and keeps it current with the
//      rank-1 form of each accepted move, which makes its diagonal exactly the
//      maintained diagonal of the paper.  It stops early at the n_delay-th
//      pending move.
//   C  all CTAs: full N-vectors x_m, y_m of the window's accepted moves by the
//      recursion of Eq. DelayRgenk, one thread per vector index j.
//   F  all CTAs, when n_delay moves are pending or the slice is done: the
//      rank-k flush G -= X Y over tiles of G.
//   A  all CTAs, when moves are pending: the next window's block
//      G0(W,W) - X(W,:) Y(:,W) for phase B.
// Phases are separated by a bounded grid barrier.
#pragma once
#include "common.cuh"

namespace afq {

constexpr int UPD_WMAX = 32;      // maximum window width
constexpr int UPD_THREADS = 256;

struct UpdArgs {
    double* G; int N;
    double* Xs; double* Ys;       // n_delay x N: row m = x_m, y_m
    int* msite; double* mcoef;    // pending moves: site, Delta/r
    double* xw; double* yw;       // n_delay x W: x_m, y_m at the positions of the window
    double* Gw;                   // W x W staging block (phase A -> B)
    int* ctl;                     // [0] window start, [1] k before, [2] k after, [3] next start
    int8_t* s;                    // field of this slice (N entries)
    int nd, W;
    double dl_p, dl_m;            // Delta for s = +1, -1
    double ef_p, ef_m;            // e^{2 gamma s} for s = +1, -1
    uint64_t key, ctr0;           // random number of site i is u(key, ctr0 + sweep * ctr_stride + i)
    const unsigned long long* sweep_dev;   // device-resident sweep number (nullptr: 0)
    uint64_t ctr_stride;
    unsigned long long* n_acc;
    DevStatus* st;
    int precision;                // bit 0: split-TF32 tcgen05 flush (FP32 accumulate); else FP64 flush
    int pair;                     // 1: G is the real 2Np x 2Np embedding of a complex G (twist)
    int Np;                       // physical sites (field length); N = 2 Np when pair
    // forced mode (block moves): flip exactly the sites with force[i] != 0, no
    // random test, and add log R = 2 gamma s + log |r|^2 of every flip to *logR
    const int8_t* force;
    double* logR;
    double two_gamma;
    double dli_p, dli_m;          // Im Delta for s = +1, -1 (charge channel)
    // split-TF32 flush (precision bit 0): the TF32 hi and lo parts of x_m(i) and
    // y_m(i), written once by phase C, K-major: row i holds moves m = 0..ldt-1
    // (ldt = n_delay rounded up to 4, so every row starts on 16 bytes)
    uint32_t *xh, *xl, *yh, *yl;
    int ldt;
};

// Window of the proposals.  Plain: positions t = 0..nw-1 are the sites c0 + t.
// Pair mode: a physical flip of site p changes rows p and p + Np of the
// embedding (Delta is real), i.e. two rank-1 moves; positions 2q and 2q + 1 are
// the sites c0 + q and c0 + q + Np, so a window holds whole pairs and the
// positions stay in proposal order.
__device__ __forceinline__ int win_site(const UpdArgs& a, int c0, int t) {
    return a.pair ? c0 + (t >> 1) + (t & 1) * a.Np : c0 + t;
}
__device__ __forceinline__ int win_pos(const UpdArgs& a, int c0, int site) {
    if (!a.pair) return site - c0;
    return site < a.Np ? 2 * (site - c0) : 2 * (site - a.Np - c0) + 1;
}
__device__ __forceinline__ int win_len(const UpdArgs& a, int c0) {
    return a.pair ? 2 * min(a.W >> 1, a.Np - c0) : min(a.W, a.N - c0);
}
__device__ __forceinline__ int win_phys(const UpdArgs& a, int c0, int t) {   // physical site of position t
    return a.pair ? c0 + (t >> 1) : c0 + t;
}

// 1 / r: hardware reciprocal estimate refined by two Newton steps
__device__ __forceinline__ double recip_nr(double r) {
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(r));
    y = fma(y, fma(-r, y, 1.0), y);
    y = fma(y, fma(-r, y, 1.0), y);
    return y;
}

// ---------------------------------------------------------------------------
// Split-TF32 flush (precision 1): G -= X Y with X = Xh + Xl, Y = Yh + Yl (each
// part a TF32 number, from the FP32 rounding of the FP64 value), product
// Xh Yh + Xh Yl + Xl Yh on the tensor cores with FP32 accumulation (Ootomo &
// Yokota 2022), subtracted in FP64.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t f32_to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// x = hi + lo: hi the TF32 rounding of the FP32 rounding xf of x, lo the TF32
// rounding of xf - hi
__device__ __forceinline__ void split_tf32(double x, uint32_t& hi, uint32_t& lo) {
    const float xf = (float)x;
    hi = f32_to_tf32(xf);
    lo = f32_to_tf32(xf - __uint_as_float(hi));
}

// ---------------------------------------------------------------------------
// Split-TF32 flush tile on the 5th-generation tensor cores (tcgen05): one
// 128 x 128 tile of G per CTA iteration, accumulator in tensor memory (TMEM,
// 128 columns allocated per CTA for the kernel's lifetime), operands staged in
// shared memory in the canonical no-swizzle K-major layout (core matrices of
// 8 rows x 16 bytes; 16-byte steps along K inside a core matrix row, LBO =
// 128 B between the two K-adjacent core matrices of one MMA, SBO = kp*32 B
// between 8-row groups), 3 x kp/8 MMAs of m128n128k8 issued by one thread,
// completion signalled by tcgen05.commit on an mbarrier.
// K is staged in rounds of 32 (shared memory: 4 operands x 128 x 32 x 4 B = 64 KB),
// then the accumulator tile goes through shared memory (128 x 129 floats).
// ---------------------------------------------------------------------------
constexpr int TCT = 128;                  // tile edge
constexpr uint32_t IDESC_TF32_128x128 =   // kind::tf32 instruction descriptor
    (1u << 4)                             // D format: F32
    | (2u << 7) | (2u << 10)              // A, B format: TF32
    | ((uint32_t)(TCT >> 3) << 17)        // N / 8
    | ((uint32_t)(TCT >> 4) << 24);       // M / 16

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ void tc_mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n"
        :: "r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(IDESC_TF32_128x128), "r"(acc));
}

// Waits for the phase of an mbarrier, bounded by WAIT_LIMIT_NS.  Each try
// suspends the thread in hardware for up to ~1 us (woken when the phase
// completes), so waiting warps do not spin on the issue slots of the working ones.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, uint32_t phase) {
    const unsigned long long t0 = global_ns();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n" : "=r"(done) : "r"(mbar), "r"(phase), "r"(1000u) : "memory");
        if (done) return true;
        if (global_ns() - t0 > WAIT_LIMIT_NS) return false;
    }
}

// element (r, m) of a 128 x kp operand, byte offset in the canonical layout
__device__ __forceinline__ uint32_t tc_off(int r, int m, int kp) {
    return (uint32_t)((r >> 3) * (kp * 32) + (m >> 2) * 128 + (r & 7) * 16 + (m & 3) * 4);
}

constexpr int TCK = 32;                   // K staged per round (shared memory: 4 x 128 x 32 x 4 B = 64 KB)
static_assert((TCK & (TCK / 4 - 1)) == 0 && ((TCK / 4) & (TCK / 4 - 1)) == 0 && ((TCT / 8) & (TCT / 8 - 1)) == 0,
              "staging index arithmetic uses shifts");

// returns false on a wait timeout (error flagged)
__device__ bool flush_tile_tcgen05(const UpdArgs& a, int k, int i0, int j0, unsigned char* sm, uint32_t tmem,
                                   uint32_t mbar, uint32_t& phase) {
    const int N = a.N;
    unsigned char* Ah = sm;
    unsigned char* Al = sm + TCT * TCK * 4;
    unsigned char* Bh = sm + 2 * TCT * TCK * 4;
    unsigned char* Bl = sm + 3 * TCT * TCK * 4;
    for (int k0 = 0; k0 < k; k0 += TCK) {
        const int kc = min(TCK, k - k0);
        const int kp = TCK;                                // full rounds: moves kc..31 are zero
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        // The operands were split into TF32 parts once, by phase C: copy groups
        // of 4 moves (16 bytes) per row into the canonical layout, zero beyond
        // the pending moves and beyond N.  Vector v -> (operand, group of 8 rows,
        // group of 4 moves, row within the group) with the row fastest: a warp
        // reads 8 rows x 64 contiguous bytes and stores 4 x 128 contiguous bytes
        // of shared memory (no bank conflicts); all loads of a thread are issued
        // before its stores.
        constexpr int groups = TCK / 4;                    // 4 moves per 16 bytes
        constexpr int total = 4 * TCT * groups;
        constexpr int VB = 8;
        for (int v0 = threadIdx.x; v0 < total; v0 += VB * blockDim.x) {
            uint4 w[VB];
            uint32_t off[VB];
#pragma unroll
            for (int q = 0; q < VB; ++q) {
                const int v = v0 + q * blockDim.x;
                w[q] = make_uint4(0u, 0u, 0u, 0u);
                off[q] = 0xffffffffu;
                if (v >= total) continue;
                const int rl = v & 7;
                const int t = v >> 3;
                const int g4 = t & (groups - 1);
                const int t2 = t / groups;
                const int rg = t2 & (TCT / 8 - 1), op = t2 / (TCT / 8);   // 0 Ah, 1 Al, 2 Bh, 3 Bl
                const int r = 8 * rg + rl, m = 4 * g4;
                off[q] = (uint32_t)op * TCT * TCK * 4 + tc_off(r, m, kp);
                const int gi = (op < 2 ? i0 : j0) + r;
                if (gi < N && m < kc) {
                    const uint32_t* src = op == 0 ? a.xh : op == 1 ? a.xl : op == 2 ? a.yh : a.yl;
                    w[q] = __ldcg(reinterpret_cast<const uint4*>(src + (size_t)gi * a.ldt + k0 + m));
                    if (m + 1 >= kc) w[q].y = 0u;
                    if (m + 2 >= kc) w[q].z = 0u;
                    if (m + 3 >= kc) w[q].w = 0u;
                }
            }
#pragma unroll
            for (int q = 0; q < VB; ++q)
                if (off[q] != 0xffffffffu) *reinterpret_cast<uint4*>(sm + off[q]) = w[q];
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sbo = (uint32_t)(kp * 32);
            const uint32_t ah = smem_u32(Ah), al = smem_u32(Al), bh = smem_u32(Bh), bl = smem_u32(Bl);
            uint32_t acc = k0 > 0 ? 1u : 0u;
            for (int s = 0; s < kp / 8; ++s) {
                const uint32_t ko = (uint32_t)(s * 256);
                tc_mma_tf32(tmem, tc_desc(al + ko, 128, sbo), tc_desc(bh + ko, 128, sbo), acc); acc = 1;
                tc_mma_tf32(tmem, tc_desc(ah + ko, 128, sbo), tc_desc(bl + ko, 128, sbo), 1);
                tc_mma_tf32(tmem, tc_desc(ah + ko, 128, sbo), tc_desc(bh + ko, 128, sbo), 1);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(mbar) : "memory");
        }
        const bool ok = mbar_wait_bounded(mbar, phase);
        phase ^= 1u;
        if (!ok) { flag_error(a.st, DERR_TIMEOUT, 210); return false; }
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // warps w and w+4 share TMEM lanes 32*(w%4)..+31; they split the 128 columns.
    // The tile goes through shared memory (row-major, padded: conflict-free)
    // so that G is then read and written in warp-contiguous row segments.
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = 32 * (warp & 3) + lane;
    const int cbase = 64 * (warp >> 2);
    constexpr int CLD = TCT + 1;
    float* ct = reinterpret_cast<float*>(sm);          // operands are consumed: reuse
    for (int cc = 0; cc < 64; cc += 32) {
        uint32_t v[32];
        const uint32_t taddr = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(cbase + cc);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
            "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
              "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
              "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
              "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int q = 0; q < 32; ++q) ct[row * CLD + cbase + cc + q] = __uint_as_float(v[q]);
    }
    __syncthreads();
    // G -= tile: each warp takes rows r, r + 8, ...; the loads of RB rows are in
    // flight together before their subtractions and stores
    constexpr int RB = 4;
    for (int r0 = warp; r0 < TCT; r0 += 8 * RB) {
        double gv[RB][TCT / 32];
#pragma unroll
        for (int b = 0; b < RB; ++b) {
            const int gi = i0 + r0 + 8 * b;
#pragma unroll
            for (int q = 0; q < TCT / 32; ++q) {
                const int c = lane + 32 * q;
                gv[b][q] = (gi < N && j0 + c < N) ? __ldcg(a.G + (size_t)gi * N + j0 + c) : 0.0;
            }
        }
#pragma unroll
        for (int b = 0; b < RB; ++b) {
            const int r = r0 + 8 * b, gi = i0 + r;
            if (gi >= N) break;
#pragma unroll
            for (int q = 0; q < TCT / 32; ++q) {
                const int c = lane + 32 * q;
                if (j0 + c < N) a.G[(size_t)gi * N + j0 + c] = gv[b][q] - (double)ct[r * CLD + c];
            }
        }
    }
    return true;
}

// CHARGE = 1: charge-channel field (complex Delta, pair mode); a template
// parameter so that the spin-channel kernel carries none of its code.
template <int CHARGE>
// At most 85 registers (three CTAs per SM): several chains' cooperative slice
// grids must be resident together.
__global__ void __launch_bounds__(UPD_THREADS, 3) k_update_slice(UpdArgs a) {
    extern __shared__ double upd_smem[];
    const int N = a.N, W = a.W, nd = a.nd;
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const int gthreads = gridDim.x * blockDim.x;
    // tensor-memory accumulator and completion barrier of the tcgen05 flush
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_mbar;
    uint32_t tmem = 0, mbar = 0, phase = 0;
    if ((a.precision & 1)) {
        if (threadIdx.x < 32) {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                         :: "r"(smem_u32(&s_tmem)), "r"(TCT) : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        }
        if (threadIdx.x == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&s_mbar)), "r"(1) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        tmem = s_tmem;
        mbar = smem_u32(&s_mbar);
    }
    const uint64_t ctr0 = a.ctr0 + (a.sweep_dev ? (uint64_t)__ldcg(a.sweep_dev) * a.ctr_stride : 0ull);
    int cursor = 0, k = 0;
    for (;;) {
        // ------------------------------------------------------------ phase B
        // Thread 0 walks the window's sites and decides each one; the CTA syncs
        // only at accepted sites.  Warp 0 keeps the diagonal of the window block
        // current (one entry per lane, W <= 32; it is all the next decisions
        // read), the other warps update the off-diagonal part of the trailing block.
        if (blockIdx.x == 0) {
            double* Gw = upd_smem;                        // W x (W+1)
            double* vv = Gw + W * (W + 1);                // W thresholds on r^2: u e^{-2 gamma s}
            double* dd = vv + W;                          // W values of Delta
            double* od = dd + W;                          // W values of 1 + Delta (charge: Im Delta)
            double* xs = od + W;                          // W: x of the current move at the window positions
            int8_t* sw = reinterpret_cast<int8_t*>(xs + W); // W field values (W doubles reserved), then
                                                          // the second W x (W+1) block and a second x
                                                          // vector (W) of the spin-channel path
            __shared__ int s_found[2];
            __shared__ double s_c[2], s_c2[2];
            const int nw = win_len(a, cursor);
            const int ld = W + 1;
            {
                // W x W block: every load of a thread in flight before its stores
                constexpr int BL = (UPD_WMAX * UPD_WMAX + UPD_THREADS - 1) / UPD_THREADS;
                double v[BL];
#pragma unroll
                for (int q = 0; q < BL; ++q) {
                    const int o = threadIdx.x + q * blockDim.x;
                    v[q] = 0.0;
                    if (o < nw * nw) {
                        const int r = o / nw, c = o - r * nw;
                        v[q] = (k == 0) ? __ldcg(a.G + (size_t)win_site(a, cursor, r) * N + win_site(a, cursor, c))
                                        : __ldcg(a.Gw + r * W + c);
                    }
                }
#pragma unroll
                for (int q = 0; q < BL; ++q) {
                    const int o = threadIdx.x + q * blockDim.x;
                    if (o < nw * nw) Gw[(o / nw) * ld + o % nw] = v[q];
                }
            }
            for (int t = threadIdx.x; t < nw; t += blockDim.x) {
                const int ps = win_phys(a, cursor, t);
                const int sg = a.s[ps];
                if (a.force) {
                    // forced: threshold -1 accepts any real r, +inf accepts none
                    vv[t] = a.force[ps] ? -1.0 : __longlong_as_double(0x7ff0000000000000ll);
                } else {
                    const double u = sm64_uniform(a.key, ctr0 + ps);
                    // accept iff u < e^{2 gamma s} r^2  <=>  r^2 > u e^{-2 gamma s}
                    vv[t] = u * (sg > 0 ? a.ef_m : a.ef_p);
                }
                dd[t] = sg > 0 ? a.dl_p : a.dl_m;
                od[t] = CHARGE ? (sg > 0 ? a.dli_p : a.dli_m) : 1.0 + dd[t];
                sw[t] = (int8_t)sg;
            }
            __syncthreads();
            int kk = k, tstop = nw, t0 = 0, it = 0;
            double lacc = 0.0;                            // forced mode: sum of log R (thread 0)
            if (CHARGE == 0 && !a.pair && !a.force) {
                // Spin channel, real G: warp 0 holds window position q in lane q,
                // with the current diagonal entry g, the ratio r = 1 + Delta (1 - g),
                // its accept test and the coefficient Delta / r computed ahead of
                // time.  A ballot over the positions not yet visited names the next
                // accepted site at once, so no thread walks the rejected sites one
                // by one.
                // On this part every FP64 warp instruction holds its sub-partition's
                // FP64 unit for ~64 cycles whatever the number of active lanes, so
                // the decision chain is written with as few of them as possible:
                // lane q keeps rr = r / Delta, which an accepted move at tf changes
                // by -c G(q,tf) G(tf,q) (c = Delta / r of that move, the diagonal
                // change times Delta); the test r^2 > v reads rr^2 > v / Delta^2 and
                // the coefficient Delta / r of lane q is 1 / rr.  Delta = 0 (U = 0):
                // r = 1 and c = 0.  (The values follow the serial scan below up to
                // the rounding of these reformulations.)
                // Pipeline.  The block after a accepted moves, G^(a), lives in
                // buffer a & 1 (Gw, Gw2).  Warps 1-7 form G^(a+1) (the trailing
                // rank-1 update of move a, off the diagonal) into the other buffer
                // while warp 0 already decides the next move: it needs only column
                // and row t' of G^(a+1) for the next accepted site t', which it forms
                // itself from G^(a) and the rank-1 term of move a (the same FMAs as
                // the trailing update, so the values are identical).  So the
                // trailing update runs one move behind and leaves the decision chain.
                // Hand-offs are named barriers, each used on alternate moves so that
                // no barrier is arrived at twice before its phase completes:
                //   TF (2, 3): warp 0 publishes move a (site, c, and its x at the
                //     window positions; site -1 ends the window) and arrives; warps
                //     1-7 wait.  Warp 0 publishes move a+1 only after it has read G^(a)
                //     (which move a+1 overwrites).
                //   DONE (4, 5): warps 1-7 arrive when G^(a+1) is complete; warp 0
                //     waits before reading it (one move later), and once at the end.
                const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
                double* Gw2 = xs + 2 * W;                          // second block buffer, after sw
                double* xsb[2] = {xs, Gw2 + W * ld};               // x of move a at the window positions, by a & 1
                __shared__ int s_tf[2];
                __shared__ double s_cc[2];
                if (warp == 0) {
                    double rr = 0.0, sq = 0.0, cq = 0.0;
                    bool okq = false, dz = false;
                    auto test = [&]() {     // r^2 > v  <=>  |rr| > sqrt(v) / |Delta| = sq
                        if (dz) return;
                        if (!finite_bits(rr)) { flag_error(a.st, DERR_NUMERIC, 200); okq = false; cq = 0.0; return; }
                        okq = abs_gt(rr, sq);
                        cq = recip_fast(rr);
                    };
                    if (lane < nw) {
                        const double dq = dd[lane];
                        dz = dq == 0.0;
                        if (dz) {
                            okq = 1.0 > vv[lane];
                        } else {
                            const double inv = 1.0 / dq;
                            rr = fma(-dq, Gw[lane * ld + lane], od[lane]) * inv;
                            sq = sqrt(vv[lane]) * fabs(inv);
                            test();
                        }
                    }
                    // first accepted site, its column and row of G^(0)
                    unsigned m = __ballot_sync(0xffffffffu, okq && lane < nw);
                    int tf = m ? __ffs((int)m) - 1 : -1;
                    double c = __shfl_sync(0xffffffffu, cq, tf >= 0 ? tf : 0);
                    double col = 0.0, row = 0.0;
                    if (tf >= 0 && lane < nw) { col = Gw[lane * ld + tf]; row = Gw[tf * ld + lane]; }
                    double xq = c * col;                            // x of the move at position q
                    if (lane < nw) xsb[0][lane] = xq;
                    if (lane == 0) { s_tf[0] = tf; s_cc[0] = c; }
                    asm volatile("bar.arrive 2, %0;" :: "r"(UPD_THREADS) : "memory");
                    int na = 0;
                    while (tf >= 0) {
                        // move na at tf: the later diagonal entries, their tests
                        // (rr -= c G(q,tf) G(tf,q) as x_q G(tf,q), x_q = c G(q,tf))
                        if (lane > tf && lane < nw && !dz) {
                            rr = fma(-xq, row, rr);
                            test();
                        }
                        ++kk;
                        int tn = -1;
                        double cn = 0.0;
                        if (kk == nd) {
                            tstop = tf + 1;
                        } else {
                            m = __ballot_sync(0xffffffffu, okq && lane > tf && lane < nw);
                            tn = m ? __ffs((int)m) - 1 : -1;
                            cn = __shfl_sync(0xffffffffu, cq, tn >= 0 ? tn : 0);
                        }
                        // G^(na) complete (warps 1-7 finished move na-1)
                        if (na >= 1) {
                            if ((na - 1) & 1) asm volatile("bar.sync 5, %0;" :: "r"(UPD_THREADS) : "memory");
                            else asm volatile("bar.sync 4, %0;" :: "r"(UPD_THREADS) : "memory");
                        }
                        double coln = 0.0, rown = 0.0;
                        if (tn >= 0) {
                            // column and row tn of G^(na+1) = G^(na) + x (row tf of G^(na))
                            const double* B = (na & 1) ? Gw2 : Gw;
                            const double rtn = __shfl_sync(0xffffffffu, row, tn);   // G^(na)(tf, tn)
                            const double xtn = __shfl_sync(0xffffffffu, xq, tn);    // x at tn
                            if (lane < nw) {
                                coln = fma(xq, rtn, B[lane * ld + tn]);
                                rown = fma(xtn, row, B[tn * ld + lane]);
                            }
                        }
                        // publish move na+1 (or the end); G^(na) has been read
                        const int ns = (na + 1) & 1;
                        const double xn = cn * coln;
                        if (tn >= 0 && lane < nw) xsb[ns][lane] = xn;
                        if (lane == 0) { s_tf[ns] = tn; s_cc[ns] = cn; }
                        if (ns) asm volatile("bar.arrive 3, %0;" :: "r"(UPD_THREADS) : "memory");
                        else asm volatile("bar.arrive 2, %0;" :: "r"(UPD_THREADS) : "memory");
                        tf = tn;
                        c = cn;
                        col = coln;
                        row = rown;
                        xq = xn;
                        ++na;
                    }
                    if (na >= 1) {
                        if ((na - 1) & 1) asm volatile("bar.sync 5, %0;" :: "r"(UPD_THREADS) : "memory");
                        else asm volatile("bar.sync 4, %0;" :: "r"(UPD_THREADS) : "memory");
                    }
                } else {
                    for (int na = 0;; ++na) {
                        const int sl = na & 1;
                        if (sl) asm volatile("bar.sync 3, %0;" :: "r"(UPD_THREADS) : "memory");
                        else asm volatile("bar.sync 2, %0;" :: "r"(UPD_THREADS) : "memory");
                        const int tf = s_tf[sl];
                        if (tf < 0) break;
                        const double c = s_cc[sl];
                        const double* src = sl ? Gw2 : Gw;
                        double* dst = sl ? Gw : Gw2;
                        const double* xv = xsb[sl];
                        const int rest = nw - tf - 1;
                        if (warp == 4) {
                            // the move and its x, y at the later window positions, to
                            // the recursion of phase C (global stores, off the FP64 warps)
                            const int km = k + na;
                            if (lane == 0) {
                                a.msite[km] = cursor + tf;
                                a.mcoef[km] = c;
                                a.s[cursor + tf] = (int8_t)(-sw[tf]);
                            }
                            if (lane < rest) {
                                const int q = tf + 1 + lane;
                                a.xw[km * W + q] = xv[q];
                                a.yw[km * W + q] = -src[tf * ld + q];
                            }
                        } else {
                            // G^(na+1)(q,p) = G^(na)(q,p) + x_q G^(na)(tf,p) for q != p > tf,
                            // packed 32 entries per warp instruction over warps 1-3 and 5-7
                            // (warp 4 shares warp 0's sub-partition and stays off FP64)
                            const int wr = warp < 4 ? warp - 1 : warp - 2;      // 0..5
                            const int tot = rest * rest;
                            const float rinv = 1.0f / (float)max(rest, 1);
                            // entry e -> (e / rest, e % rest); the FP32 quotient is off
                            // by at most one for e < 1024 and is corrected
                            auto split = [&](int e, int& q, int& pp) {
                                int qi = __float2int_rz((float)e * rinv);
                                if (qi * rest > e) --qi;
                                else if ((qi + 1) * rest <= e) ++qi;
                                q = tf + 1 + qi;
                                pp = tf + 1 + (e - qi * rest);
                            };
                            for (int e0 = 32 * wr; e0 < tot; e0 += 2 * 6 * 32) {
                                const int e1 = e0 + lane, e2 = e0 + 6 * 32 + lane;
                                int q1 = 0, p1 = 0, q2 = 0, p2 = 0;
                                const bool h1 = e1 < tot, h2 = e2 < tot;
                                double x1 = 0.0, y1 = 0.0, g1 = 0.0, x2 = 0.0, y2 = 0.0, g2 = 0.0;
                                if (h1) { split(e1, q1, p1); x1 = xv[q1]; y1 = src[tf * ld + p1]; g1 = src[q1 * ld + p1]; }
                                if (h2) { split(e2, q2, p2); x2 = xv[q2]; y2 = src[tf * ld + p2]; g2 = src[q2 * ld + p2]; }
                                if (h1 && q1 != p1) dst[q1 * ld + p1] = fma(x1, y1, g1);
                                if (h2 && q2 != p2) dst[q2 * ld + p2] = fma(x2, y2, g2);
                            }
                        }
                        if (sl) asm volatile("bar.arrive 5, %0;" :: "r"(UPD_THREADS) : "memory");
                        else asm volatile("bar.arrive 4, %0;" :: "r"(UPD_THREADS) : "memory");
                    }
                }
            } else
            for (;; ++it) {
                const int slot = it & 1;
                if (threadIdx.x == 0) {
                    int found = -1;
                    double c = 0.0, c2 = 0.0;
                    for (; t0 < nw; ++t0) {
                        const double dl = dd[t0];
                        if constexpr (CHARGE != 0) {
                            // one complex flip per pair (t0 even): G_pp = Gw[t0][t0] + i Gw[t0+1][t0],
                            // r = 1 + Delta (1 - G_pp), R = |r|^2, kappa = Delta conj(r) / |r|^2
                            const double di = od[t0];
                            const double gr = Gw[t0 * ld + t0], gi = Gw[(t0 + 1) * ld + t0];
                            const double omg = 1.0 - gr;
                            const double rr = fma(dl, omg, fma(di, gi, 1.0));
                            const double ri = fma(di, omg, -dl * gi);
                            const double R2 = fma(rr, rr, ri * ri);
                            if (!isfinite(R2)) { flag_error(a.st, DERR_NUMERIC, 201); ++t0; continue; }
                            if (R2 > vv[t0]) {
                                const double inv = 1.0 / R2;
                                found = t0;
                                c = fma(dl, rr, di * ri) * inv;
                                c2 = fma(di, rr, -dl * ri) * inv;
                                if (a.force) lacc += log(R2);
                                break;
                            }
                            ++t0;                    // rejected: skip the partner too
                            continue;
                        }
                        const double r = fma(-dl, Gw[t0 * ld + t0], od[t0]);   // 1 + Delta (1 - G_ii)
                        if (!isfinite(r)) { flag_error(a.st, DERR_NUMERIC, 200); continue; }
                        if (a.pair) {
                            if (t0 & 1) {            // second half of an accepted pair
                                found = t0;
                                c = dl * recip_nr(r);
                                break;
                            }
                            // r1 r2 = |1 + Delta (1 - G_pp)|^2 of the complex G: r2 from the
                            // diagonal entry the first move leaves behind (same arithmetic as
                            // warp 0's update below)
                            const double c1 = dl * recip_nr(r);
                            const int q = t0 + 1;
                            const double g2 = fma(c1 * Gw[q * ld + t0], Gw[t0 * ld + q], Gw[q * ld + q]);
                            const double r2 = fma(-dl, g2, od[t0]);
                            if (r * r2 > vv[t0]) {
                                found = t0;
                                c = c1;
                                if (a.force) lacc += log(r * r2) + a.two_gamma * sw[t0];
                                break;
                            }
                            ++t0;                    // rejected: skip the partner too
                            continue;
                        }
                        if (r * r > vv[t0]) {
                            found = t0;
                            c = dl * recip_nr(r);
                            if (a.force) lacc += log(r * r) + a.two_gamma * sw[t0];
                            break;
                        }
                    }
                    if (found >= 0) t0 += CHARGE ? 2 : 1;
                    s_found[slot] = found;
                    s_c[slot] = c;
                    s_c2[slot] = c2;
                }
                __syncthreads();
                const int tf = s_found[slot];
                if (tf < 0) break;
                const double c = s_c[slot];
                if constexpr (CHARGE != 0) {
                    // the pair (tf, tg) as two simultaneous real moves (x1, y1), (x2, y2)
                    const double c2 = s_c2[slot];
                    const int tg = tf + 1;
                    if (threadIdx.x == 32) {
                        a.msite[kk] = win_site(a, cursor, tf);
                        a.msite[kk + 1] = win_site(a, cursor, tg);
                        a.mcoef[kk] = c;
                        a.mcoef[kk + 1] = c2;
                        a.s[win_phys(a, cursor, tf)] = (int8_t)(-sw[tf]);
                    }
                    const int rest = nw - tg - 1;
                    for (int p = (int)threadIdx.x - 32; p >= 0 && p < rest; p += blockDim.x - 32) {
                        const int q = tg + 1 + p;
                        const double zp = Gw[q * ld + tf], zq = Gw[q * ld + tg];
                        a.xw[kk * W + q] = fma(c, zp, c2 * zq);
                        a.xw[(kk + 1) * W + q] = fma(-c2, zp, c * zq);
                        a.yw[kk * W + q] = -Gw[tf * ld + q];
                        a.yw[(kk + 1) * W + q] = -Gw[tg * ld + q];
                    }
                    if (threadIdx.x < 32) {
                        // warp 0: the diagonal and the two entries inside each later pair
                        const int q = tg + 1 + (int)threadIdx.x;
                        if (q < nw) {
                            const double x1 = fma(c, Gw[q * ld + tf], c2 * Gw[q * ld + tg]);
                            const double x2 = fma(-c2, Gw[q * ld + tf], c * Gw[q * ld + tg]);
                            Gw[q * ld + q] = fma(x1, Gw[tf * ld + q], fma(x2, Gw[tg * ld + q], Gw[q * ld + q]));
                            if (!(q & 1) && q + 1 < nw) {
                                const int q1 = q + 1;
                                const double v1 = fma(c, Gw[q1 * ld + tf], c2 * Gw[q1 * ld + tg]);
                                const double v2 = fma(-c2, Gw[q1 * ld + tf], c * Gw[q1 * ld + tg]);
                                Gw[q1 * ld + q] = fma(v1, Gw[tf * ld + q], fma(v2, Gw[tg * ld + q], Gw[q1 * ld + q]));
                                Gw[q * ld + q1] = fma(x1, Gw[tf * ld + q1], fma(x2, Gw[tg * ld + q1], Gw[q * ld + q1]));
                            }
                        }
                        __syncwarp();
                    } else {
                        for (int o = threadIdx.x - 32; o < rest * rest; o += blockDim.x - 32) {
                            const int q = tg + 1 + o / rest, pp = tg + 1 + o % rest;
                            if ((q >> 1) == (pp >> 1)) continue;      // warp 0's entries
                            const double x1 = fma(c, Gw[q * ld + tf], c2 * Gw[q * ld + tg]);
                            const double x2 = fma(-c2, Gw[q * ld + tf], c * Gw[q * ld + tg]);
                            Gw[q * ld + pp] = fma(x1, Gw[tf * ld + pp], fma(x2, Gw[tg * ld + pp], Gw[q * ld + pp]));
                        }
                    }
                    kk += 2;
                    if (kk >= nd) { tstop = tg + 1; break; }
                    continue;
                }
                if (threadIdx.x == 32) {
                    a.msite[kk] = win_site(a, cursor, tf);
                    a.mcoef[kk] = c;
                    if (!a.pair || !(tf & 1)) a.s[win_phys(a, cursor, tf)] = (int8_t)(-sw[tf]);
                }
                const int rest = nw - tf - 1;
                for (int p = (int)threadIdx.x - 32; p >= 0 && p < rest; p += blockDim.x - 32) {
                    const int q = tf + 1 + p;
                    a.xw[kk * W + q] = c * Gw[q * ld + tf];
                    a.yw[kk * W + q] = -Gw[tf * ld + q];
                }
                if (threadIdx.x < 32) {
                    // warp 0: one diagonal entry per lane (and, in pair mode, the two
                    // off-diagonal entries inside the pair that starts there: the
                    // pair decision reads them), then hand back to thread 0
                    const int q = tf + 1 + (int)threadIdx.x;
                    if (q < nw) {
                        Gw[q * ld + q] = fma(c * Gw[q * ld + tf], Gw[tf * ld + q], Gw[q * ld + q]);
                        if (a.pair && !(q & 1) && q + 1 < nw) {
                            const int q1 = q + 1;
                            Gw[q1 * ld + q] = fma(c * Gw[q1 * ld + tf], Gw[tf * ld + q], Gw[q1 * ld + q]);
                            Gw[q * ld + q1] = fma(c * Gw[q * ld + tf], Gw[tf * ld + q1], Gw[q * ld + q1]);
                        }
                    }
                    __syncwarp();
                } else {
                    for (int o = threadIdx.x - 32; o < rest * rest; o += blockDim.x - 32) {
                        const int q = tf + 1 + o / rest, p = tf + 1 + o % rest;
                        if (q == p || (a.pair && (q >> 1) == (p >> 1))) continue;   // warp 0's entries
                        Gw[q * ld + p] = fma(c * Gw[q * ld + tf], Gw[tf * ld + p], Gw[q * ld + p]);
                    }
                }
                ++kk;
                if (kk == nd) { tstop = tf + 1; break; }
            }
            if (threadIdx.x == 0) {
                if (a.force) *a.logR += lacc;
                a.ctl[0] = cursor;
                a.ctl[1] = k;
                a.ctl[2] = kk;
                a.ctl[3] = cursor + (a.pair ? tstop >> 1 : tstop);
                if (kk > k) atomicAdd(a.n_acc, (unsigned long long)(kk - k));
            }
        }
        if (!grid_barrier(a.st, 1)) break;
        const int c0 = __ldcg(a.ctl + 0), kb = __ldcg(a.ctl + 1), ka = __ldcg(a.ctl + 2), c1 = __ldcg(a.ctl + 3);
        // ------------------------------------------------------------ phase C
        // CTA b owns the contiguous vector indices [b*JPB, (b+1)*JPB), one warp
        // per index, one lane per new move of the window (no FP64 cross-lane
        // reductions).  Everything the loops read is first staged in shared
        // memory: X, Y of the pending moves at the CTA's indices and at the
        // window's sites, and the window tables of the new moves.
        if (ka > kb) {
            const int nn = ka - kb;
            const int nw = c1 > c0 ? win_len(a, c0) : 0;
            const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
            const int JPB = (N + gridDim.x - 1) / gridDim.x;
            const int jb = blockIdx.x * JPB;
            const int nj = max(0, min(JPB, N - jb));
            double* sXj = upd_smem;                  // kb x JPB
            double* sYj = sXj + kb * JPB;            // kb x JPB
            double* sXw = sYj + kb * JPB;            // kb x W  (X at the window sites)
            double* sYw = sXw + kb * W;              // kb x W
            double* sxw = sYw + kb * W;              // nn x W  (new moves' x at window positions)
            double* syw = sxw + nn * W;              // nn x W
            if (nj > 0) {
                // issue all loads of a thread before its shared-memory stores
                // (the loads are independent; one L2 latency instead of many)
                constexpr int BATCH = 8;
                const int n1 = kb * JPB, n2 = kb * W, n3 = nn * W;
                const int tot = 2 * (n1 + n2 + n3);
                for (int o0 = threadIdx.x; o0 < tot; o0 += BATCH * blockDim.x) {
                    double v[BATCH];
                    int dst[BATCH];
#pragma unroll
                    for (int q = 0; q < BATCH; ++q) {
                        const int o = o0 + q * blockDim.x;
                        dst[q] = -1;
                        v[q] = 0.0;
                        if (o >= tot) continue;
                        const int half = o & 1, e = o >> 1;      // even: X, odd: Y
                        const double* srcm = half ? a.Ys : a.Xs;
                        if (e < n1) {
                            const int p = e / JPB, jj = e - p * JPB;
                            if (jj < nj) v[q] = __ldcg(srcm + (size_t)p * N + jb + jj);
                            dst[q] = (half ? (int)(sYj - upd_smem) : (int)(sXj - upd_smem)) + e;
                        } else if (e < n1 + n2) {
                            const int f = e - n1, p = f / W, t = f - p * W;
                            if (t < nw) v[q] = __ldcg(srcm + (size_t)p * N + win_site(a, c0, t));
                            dst[q] = (half ? (int)(sYw - upd_smem) : (int)(sXw - upd_smem)) + f;
                        } else {
                            const int f = e - n1 - n2;
                            v[q] = __ldcg((half ? a.yw : a.xw) + kb * W + f);
                            dst[q] = (half ? (int)(syw - upd_smem) : (int)(sxw - upd_smem)) + f;
                        }
                    }
#pragma unroll
                    for (int q = 0; q < BATCH; ++q)
                        if (dst[q] >= 0) upd_smem[dst[q]] = v[q];
                }
            }
            __syncthreads();
            const bool mine = lane < nn;
            const int mm = kb + lane;
            const int im = mine ? __ldcg(a.msite + mm) : c0;
            const int tm = win_pos(a, c0, im);
            const double cm = mine ? __ldcg(a.mcoef + mm) : 0.0;
            for (int jj = warp; jj < nj; jj += nwarp) {
                const int j = jb + jj;
                const double g_jm = mine ? __ldcg(a.G + (size_t)j * N + im) : 0.0;
                const double g_mj = mine ? __ldcg(a.G + (size_t)im * N + j) : 0.0;
                double ox0 = 0.0, ox1 = 0.0, oy0 = 0.0, oy1 = 0.0;
                if (mine) {
                    int p = 0;
                    for (; p + 1 < kb; p += 2) {
                        ox0 = fma(sXj[p * JPB + jj], sYw[p * W + tm], ox0);
                        oy0 = fma(sXw[p * W + tm], sYj[p * JPB + jj], oy0);
                        ox1 = fma(sXj[(p + 1) * JPB + jj], sYw[(p + 1) * W + tm], ox1);
                        oy1 = fma(sXw[(p + 1) * W + tm], sYj[(p + 1) * JPB + jj], oy1);
                    }
                    if (p < kb) {
                        ox0 = fma(sXj[p * JPB + jj], sYw[p * W + tm], ox0);
                        oy0 = fma(sXw[p * W + tm], sYj[p * JPB + jj], oy0);
                    }
                }
                // recursion over the new moves (Eq. DelayRgenk), lane m accumulates move m
                double ax = mine ? g_jm - (ox0 + ox1) : 0.0;
                double ay = mine ? (j == im ? 1.0 : 0.0) - g_mj + (oy0 + oy1) : 0.0;
                double xv = 0.0, yv = 0.0;
                if constexpr (CHARGE != 0) {
                    // moves come in pairs (q, q + 1) of one complex flip: both take the
                    // columns and rows as they were before the pair, x mixes them by kappa
                    for (int q = 0; q + 1 < nn; q += 2) {
                        const double axa = __shfl_sync(0xffffffffu, ax, q), axb = __shfl_sync(0xffffffffu, ax, q + 1);
                        const double kr = __shfl_sync(0xffffffffu, cm, q), ki = __shfl_sync(0xffffffffu, cm, q + 1);
                        if (lane == q) { xv = fma(kr, axa, ki * axb); yv = ay; }
                        if (lane == q + 1) { xv = fma(-ki, axa, kr * axb); yv = ay; }
                        const double x0 = __shfl_sync(0xffffffffu, xv, q), y0 = __shfl_sync(0xffffffffu, yv, q);
                        const double x1 = __shfl_sync(0xffffffffu, xv, q + 1), y1 = __shfl_sync(0xffffffffu, yv, q + 1);
                        if (mine && lane > q + 1) {
                            ax = fma(-x0, syw[q * W + tm], fma(-x1, syw[(q + 1) * W + tm], ax));
                            ay = fma(sxw[q * W + tm], y0, fma(sxw[(q + 1) * W + tm], y1, ay));
                        }
                    }
                } else {
                    for (int q = 0; q < nn; ++q) {
                        if (lane == q) { xv = cm * ax; yv = ay; }
                        const double xq = __shfl_sync(0xffffffffu, xv, q);
                        const double yq = __shfl_sync(0xffffffffu, yv, q);
                        if (mine && lane > q) {
                            ax = fma(-xq, syw[q * W + tm], ax);
                            ay = fma(sxw[q * W + tm], yq, ay);
                        }
                    }
                }
                if (mine) {
                    a.Xs[(size_t)mm * N + j] = xv;
                    a.Ys[(size_t)mm * N + j] = yv;
                    if (a.precision & 1) {
                        uint32_t h, l;
                        split_tf32(xv, h, l);
                        a.xh[(size_t)j * a.ldt + mm] = h;
                        a.xl[(size_t)j * a.ldt + mm] = l;
                        split_tf32(yv, h, l);
                        a.yh[(size_t)j * a.ldt + mm] = h;
                        a.yl[(size_t)j * a.ldt + mm] = l;
                    }
                }
            }
        }
        if (!grid_barrier(a.st, 2)) break;
        k = ka;
        const bool done = (c1 >= (a.pair ? a.Np : N));
        // ------------------------------------------------------------ phase F
        if (k > 0 && (k == nd || done)) {
            if ((a.precision & 1)) {
                const int nt = (N + TCT - 1) / TCT;
                for (int tile = blockIdx.x; tile < nt * nt; tile += gridDim.x)
                    if (!flush_tile_tcgen05(a, k, (tile / nt) * TCT, (tile % nt) * TCT,
                                            reinterpret_cast<unsigned char*>(upd_smem), tmem, mbar, phase))
                        break;
            } else {
                double* xs = upd_smem;               // k x 32
                double* ys = upd_smem + nd * 32;     // k x 32
                const int nt = (N + 31) / 32;
                for (int tile = blockIdx.x; tile < nt * nt; tile += gridDim.x) {
                    const int i0 = (tile / nt) * 32, j0 = (tile % nt) * 32;
                    __syncthreads();
                    for (int o = threadIdx.x; o < k * 32; o += blockDim.x) {
                        const int m = o / 32, q = o % 32;
                        xs[o] = (i0 + q < N) ? __ldcg(a.Xs + (size_t)m * N + i0 + q) : 0.0;
                        ys[o] = (j0 + q < N) ? __ldcg(a.Ys + (size_t)m * N + j0 + q) : 0.0;
                    }
                    __syncthreads();
                    for (int o = threadIdx.x; o < 32 * 32; o += blockDim.x) {
                        const int ii = o / 32, jj = o % 32;
                        if (i0 + ii >= N || j0 + jj >= N) continue;
                        double acc0 = 0.0, acc1 = 0.0;
                        int m = 0;
                        for (; m + 1 < k; m += 2) {
                            acc0 = fma(xs[m * 32 + ii], ys[m * 32 + jj], acc0);
                            acc1 = fma(xs[(m + 1) * 32 + ii], ys[(m + 1) * 32 + jj], acc1);
                        }
                        if (m < k) acc0 = fma(xs[m * 32 + ii], ys[m * 32 + jj], acc0);
                        double* gp = a.G + (size_t)(i0 + ii) * N + j0 + jj;
                        *gp = __ldcg(gp) - (acc0 + acc1);
                    }
                }
            }
            k = 0;
            if (!grid_barrier(a.st, 3)) break;
        }
        if (done) break;
        cursor = c1;
        // ------------------------------------------------------------ phase A
        if (k > 0) {
            const int nw = win_len(a, cursor);
            const int lane = threadIdx.x & 31;
            const int gwarp = gtid >> 5, nwarps = gthreads >> 5;
            for (int e = gwarp; e < nw * nw; e += nwarps) {
                const int r = e / nw, c = e - r * nw;
                const int sr = win_site(a, cursor, r), sc = win_site(a, cursor, c);
                double acc = 0.0;
                for (int m = lane; m < k; m += 32)
                    acc = fma(__ldcg(a.Xs + (size_t)m * N + sr), __ldcg(a.Ys + (size_t)m * N + sc), acc);
                acc = warp_sum(acc);
                if (lane == 0) a.Gw[r * W + c] = __ldcg(a.G + (size_t)sr * N + sc) - acc;
            }
            if (!grid_barrier(a.st, 4)) break;
        }
    }
    if ((a.precision & 1)) {
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (threadIdx.x < 32)
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(TCT) : "memory");
    }
}

}  // namespace afq
