// FP64-accurate matrix product on the BF16 tensor cores (Ozaki scheme: Ozaki,
// Ogita, Oishi & Rump, "Error-free transformations of matrix multiplication by
// using fast routines of matrix multiplication", Numer. Algorithms 59, 2012),
// for the stabilisation products (B300 FP64 runs at ~1/64 of FP32).
//
// Split.  Row i of op(A) is scaled by 2^-e_i (e_i from frexp of the row's
// largest magnitude, so |a| < 1), rounded to q = a 2^56 (an integer, |q| < 2^56)
// and cut into S = 8 balanced digits of 7 bits by integer shifts,
// q = sum_s d_s 2^(49 - 7s), |d_0| <= 128, |d_s>0| <= 64: every digit is an
// integer that BF16 holds exactly, and a = q 2^-56 up to 2^-57 (relative to the
// row's largest entry).  Columns of op(B) likewise.
//
// Product.  C_ij = 2^(e_i + f_j) sum_{s+t <= 7} 2^-7(s+t+2) (D^A_s D^B_t)_ij; the
// 36 digit products (pairs with s + t > 7 contribute below 2^-63 and are dropped)
// run as kind::f16 BF16 MMAs with FP32 accumulation in tensor memory, one
// accumulator per weight class w = s + t (8 x 64 columns = all 512).  Digit
// products are integers of at most 14 bits; summed over 320 values of k the
// class sums stay below 2^24 (class 0: 320 * 2^14; class w >= 1: 320 *
// (2 * 2^13 + (w-1) * 2^12) <= 1.4e7), so the FP32 accumulation is exact.  After
// every 320 values of k (10 chunks of 32) the classes are read out and added, scaled by their
// power of two, into FP64 registers: the only rounding is that of the final
// FP64 sums, as in an FP64 GEMM.
//
// Tile: 128 x 64 outputs per CTA (m128n64k16 MMAs), K staged 32 at a time for
// all 8 digits of both operands (64 KB + 32 KB), double-buffered so that the
// copies of chunk c+1 (cp.async) overlap the MMAs of chunk c; canonical
// no-swizzle K-major layout (8-row x 16-byte core matrices, LBO 128 B,
// SBO = 32 * 2 * 8 B); one thread issues the MMAs, completion on an mbarrier
// (bounded wait), tensor memory freed on every exit path.
#pragma once
#include <cuda_bf16.h>
#include "common.cuh"
#include "update.cuh"

namespace afq {

constexpr int OZ_S = 8;          // digits per operand
constexpr int OZ_BITS = 7;
constexpr int OZ_TM = 128, OZ_TN = 64, OZ_KC = 32, OZ_WIN = 10;  // tile, K chunk, chunks per exact window
constexpr int OZ_CLASSES = 8;    // w = s + t = 0..7
constexpr uint32_t IDESC_BF16_128x64 =
    (1u << 4)                             // D format: F32
    | (1u << 7) | (1u << 10)              // A, B format: BF16 (kind::f16)
    | ((uint32_t)(OZ_TN >> 3) << 17)      // N / 8
    | ((uint32_t)(OZ_TM >> 4) << 24);     // M / 16

constexpr size_t OZ_STAGE = (size_t)OZ_S * (OZ_TM + OZ_TN) * OZ_KC * 2;   // one K chunk of all digits

inline size_t oz_smem_bytes() { return 2 * OZ_STAGE + 1024; }   // double-buffered

// rows of X (rows x K, row-major, leading dimension ld) into OZ_S digit planes
// out[s][row][0..Kpad) (BF16, zero beyond K) and the row exponents ex[row];
// one warp per row.
__global__ void k_oz_split(const double* __restrict__ X, int rows, int K, int ld, __nv_bfloat16* out, int Kpad,
                           int* ex) {
    const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= rows) return;
    auto at = [&](int k) { return X[(size_t)row * ld + k]; };
    double mx = 0.0;
    for (int k = lane; k < K; k += 32) mx = fmax(mx, fabs(at(k)));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    int e = 0;
    if (mx > 0.0) frexp(mx, &e);          // mx = f 2^e, f in [0.5, 1): |x| 2^-e < 1
    if (lane == 0) ex[row] = e;
    const size_t plane = (size_t)rows * Kpad;
    constexpr int TOP = OZ_BITS * OZ_S;      // 56 fraction bits kept
    for (int k = lane; k < Kpad; k += 32) {
        // q = a 2^56 rounded to an integer (|q| < 2^56: exact in int64), then balanced
        // base-2^7 digits by integer shifts: d = round(q / 2^shift), q -= d 2^shift
        long long q = k < K ? __double2ll_rn(ldexp(at(k), TOP - e)) : 0ll;
#pragma unroll
        for (int s = 0; s < OZ_S; ++s) {
            const int shift = TOP - OZ_BITS * (s + 1);
            const long long d = shift > 0 ? (q + (1ll << (shift - 1))) >> shift : q;
            q -= d << shift;
            out[s * plane + (size_t)row * Kpad + k] = __float2bfloat16_rn((float)d);
        }
    }
}

struct OzArgs {
    const __nv_bfloat16* As;   // OZ_S x m x Kpad
    const __nv_bfloat16* Bs;   // OZ_S x n x Kpad (rows = columns of op(B))
    const int* ea;             // m
    const int* eb;             // n
    int m, n, Kpad;
    double* C; int ldc;
    double alpha, beta;
    const double* rs; const double* cs; int rs_inv, cs_inv;
    DevStatus* st;
};

// byte offset of element (r, k) of a staged operand with kp = OZ_KC columns of K
__device__ __forceinline__ uint32_t oz_off(int r, int k) {
    return (uint32_t)((r >> 3) * (OZ_KC * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ void tc_mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
        :: "r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(IDESC_BF16_128x64), "r"(acc));
}

constexpr int OZ_THREADS = 512;

__global__ void __launch_bounds__(OZ_THREADS, 1) k_oz_gemm(OzArgs g) {
    extern __shared__ __align__(1024) unsigned char oz_smem[];
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_mbar;
    __shared__ int s_fail;
    const int i0 = blockIdx.y * OZ_TM, j0 = blockIdx.x * OZ_TN;
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&s_tmem)), "r"(512) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        s_fail = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&s_mbar)), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem, mbar = smem_u32(&s_mbar);
    uint32_t phase = 0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = 32 * (warp & 3) + lane;          // TMEM lane = output row of the tile
    const int cbase = 16 * (warp >> 2);              // warps w, w+4, w+8, w+12 split the 64 columns
    // exact integer sums of classes 0..3 (each < 4 * 2^24 over K <= 1152... < 2^31 for K <= 40960)
    // and one FP32 sum of classes 4..7 weighted 2^-7(w-4) (its rounding is below 2^-52 of class 0)
    int iacc[4][16];
    float facc[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        iacc[0][q] = iacc[1][q] = iacc[2][q] = iacc[3][q] = 0;
        facc[q] = 0.0f;
    }
    const size_t planeA = (size_t)g.m * g.Kpad, planeB = (size_t)g.n * g.Kpad;
    const int nchunks = g.Kpad / OZ_KC;

    // stage chunk c of all digits into buffer c & 1: asynchronous 16-byte copies,
    // zero-filled outside the matrix
    auto stage = [&](int c) {
        unsigned char* Asm = oz_smem + (size_t)(c & 1) * OZ_STAGE;
        unsigned char* Bsm = Asm + (size_t)OZ_S * OZ_TM * OZ_KC * 2;
        const int k0 = c * OZ_KC;
        constexpr int VA = OZ_S * OZ_TM * (OZ_KC / 8), VB = OZ_S * OZ_TN * (OZ_KC / 8);
#pragma unroll 1
        for (int v = threadIdx.x; v < VA + VB; v += blockDim.x) {
            const bool isA = v < VA;
            const int u = isA ? v : v - VA;
            const int rows = isA ? OZ_TM : OZ_TN;
            const int k8 = u % (OZ_KC / 8);
            const int r = (u / (OZ_KC / 8)) % rows;
            const int s = u / ((OZ_KC / 8) * rows);
            const int gr = (isA ? i0 : j0) + r;
            const bool in = gr < (isA ? g.m : g.n);
            const __nv_bfloat16* src = (isA ? g.As + s * planeA : g.Bs + s * planeB) +
                                       (size_t)(in ? gr : 0) * g.Kpad + k0 + 8 * k8;
            unsigned char* dst = (isA ? Asm + (size_t)s * OZ_TM * OZ_KC * 2 : Bsm + (size_t)s * OZ_TN * OZ_KC * 2) +
                                 oz_off(r, 8 * k8);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;"
                         :: "r"(smem_u32(dst)), "l"(src), "r"(in ? 16 : 0) : "memory");
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };

    stage(0);
    bool pending = false;        // MMAs of the previous chunk not waited for yet
    for (int c = 0; c < nchunks; ++c) {
        // the buffer chunk c+1 will fill was read by the MMAs of chunk c-1
        if (pending) {
            if (!mbar_wait_bounded(mbar, phase)) { s_fail = 1; flag_error(g.st, DERR_TIMEOUT, 600); }
            phase ^= 1u;
            pending = false;
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (s_fail) break;
        if (c + 1 < nchunks) {
            stage(c + 1);
            asm volatile("cp.async.wait_group 1;" ::: "memory");     // chunk c has landed
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        // ---- 36 digit products of chunk c into the 8 class accumulators
        const int cw = c % OZ_WIN;          // chunk within the exact window
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sbo = (uint32_t)(OZ_KC * 16);
            const uint32_t abase = smem_u32(oz_smem + (size_t)(c & 1) * OZ_STAGE);
            const uint32_t bbase = abase + (uint32_t)(OZ_S * OZ_TM * OZ_KC * 2);
#pragma unroll 1
            for (int w = 0; w < OZ_CLASSES; ++w)
#pragma unroll 1
                for (int s = 0; s <= w; ++s) {
                    const uint32_t a0 = abase + (uint32_t)(s * OZ_TM * OZ_KC * 2);
                    const uint32_t b0 = bbase + (uint32_t)((w - s) * OZ_TN * OZ_KC * 2);
#pragma unroll
                    for (int kk = 0; kk < OZ_KC / 16; ++kk) {
                        const uint32_t ko = (uint32_t)(kk * 256);
                        const uint32_t accf = (cw > 0 || s > 0 || kk > 0) ? 1u : 0u;
                        tc_mma_bf16(tmem + (uint32_t)(w * OZ_TN), tc_desc(a0 + ko, 128, sbo), tc_desc(b0 + ko, 128, sbo),
                                    accf);
                    }
                }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(mbar) : "memory");
        }
        pending = true;
        // ---- end of an exact window: wait for the MMAs, read the classes out into FP64
        if (cw == OZ_WIN - 1 || c == nchunks - 1) {
            if (!mbar_wait_bounded(mbar, phase)) { s_fail = 1; flag_error(g.st, DERR_TIMEOUT, 601); }
            phase ^= 1u;
            pending = false;
            __syncthreads();
            if (s_fail) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int w = 0; w < OZ_CLASSES; ++w) {
                uint32_t v[16];
                const uint32_t taddr = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(w * OZ_TN + cbase);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                    "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                      "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                      "=r"(v[14]), "=r"(v[15])
                    : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (w < 4) {
#pragma unroll
                    for (int q = 0; q < 16; ++q) iacc[w][q] += __float2int_rn(__uint_as_float(v[q]));
                } else {
                    const float sc = ldexpf(1.0f, -OZ_BITS * (w - 4));
#pragma unroll
                    for (int q = 0; q < 16; ++q) facc[q] = fmaf(__uint_as_float(v[q]), sc, facc[q]);
                }
            }
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    // ---- epilogue through shared memory (coalesced rows of C)
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (!s_fail) {
        constexpr int CLD = OZ_TN + 1;
        double* ct = reinterpret_cast<double*>(oz_smem);
        const double s0 = ldexp(1.0, -2 * OZ_BITS), s1 = ldexp(1.0, -3 * OZ_BITS), s2 = ldexp(1.0, -4 * OZ_BITS),
                     s3 = ldexp(1.0, -5 * OZ_BITS), s4 = ldexp(1.0, -6 * OZ_BITS);
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            // smallest terms first
            double v = (double)facc[q] * s4;
            v = fma((double)iacc[3][q], s3, v);
            v = fma((double)iacc[2][q], s2, v);
            v = fma((double)iacc[1][q], s1, v);
            v = fma((double)iacc[0][q], s0, v);
            ct[row * CLD + cbase + q] = v;
        }
        __syncthreads();
        for (int r = warp; r < OZ_TM; r += OZ_THREADS / 32) {
            const int gi = i0 + r;
            if (gi >= g.m) break;
            double ri = g.alpha * ldexp(1.0, g.ea[gi]);
            if (g.rs) ri = g.rs_inv ? ri / g.rs[gi] : ri * g.rs[gi];
            for (int cc = lane; cc < OZ_TN; cc += 32) {
                const int gj = j0 + cc;
                if (gj >= g.n) continue;
                double v = ct[r * CLD + cc] * ri * ldexp(1.0, g.eb[gj]);
                if (g.cs) v = g.cs_inv ? v / g.cs[gj] : v * g.cs[gj];
                double* cp = g.C + (size_t)gi * g.ldc + gj;
                *cp = (g.beta == 0.0) ? v : fma(g.beta, *cp, v);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(512) : "memory");
}

}  // namespace afq
