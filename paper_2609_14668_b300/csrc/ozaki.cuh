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
// every 320 values of k (10 chunks of 32) the classes are read out: classes 0..3
// into one exact 64-bit integer (weights 2^21, 2^14, 2^7, 1), classes 4..7 into one
// FP32 sum; the final FP64 value rounds once, as in an FP64 GEMM.
//
// Tile: 128 x 64 outputs per CTA (m128n64k16 MMAs), K staged 32 at a time for
// all 8 digits of both operands (64 KB + 32 KB) by tensor-memory-access copies
// (cp.async.bulk.tensor, 3-D view k x row x digit of each digit-plane array,
// one copy per operand per group of 8 values of k) into two stages; a producer
// warp issues the copies, an MMA warp issues the 72 MMAs of a chunk (one
// elected thread) and commits them, and 16 read-out warps move the classes
// out of tensor memory at the end of every exact window.  Stages and tensor
// memory change hands through mbarriers (bounded waits); tensor memory is
// freed on every exit path, after the copies and MMAs in flight have landed.
#pragma once
#include <cuda.h>
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

// Stage layout: operand A, then B; inside an operand the K chunk is 4 groups
// of 8 values of k, a group holds all digits s, a digit all rows r, a row 16
// bytes (8 BF16 values of k): offset = kg * KGROUP + s * rows * 16 + r * 16.
// This is the canonical no-swizzle K-major layout with the 8 x 16-byte core
// matrices 128 bytes apart along M (SBO) and KGROUP bytes apart along K (LBO).
constexpr uint32_t OZ_A_KGROUP = OZ_S * OZ_TM * 16;      // 16 KB
constexpr uint32_t OZ_B_KGROUP = OZ_S * OZ_TN * 16;      // 8 KB
constexpr size_t OZ_STAGE = (size_t)(OZ_KC / 8) * (OZ_A_KGROUP + OZ_B_KGROUP);   // one K chunk of all digits
static_assert(OZ_STAGE == (size_t)OZ_S * (OZ_TM + OZ_TN) * OZ_KC * 2, "stage size");
constexpr int OZ_EPI_WARPS = 16;                          // tensor-memory read-out and epilogue
constexpr int OZ_PRODUCER_WARP = OZ_EPI_WARPS, OZ_MMA_WARP = OZ_EPI_WARPS + 1;
static_assert(sizeof(double) * (OZ_TM * (OZ_TN + 1) + OZ_TN) <= 2 * OZ_STAGE, "epilogue tile fits the staging buffers");

// 2^e from its bit pattern (no FP64 arithmetic) for an exponent in the normal
// range; outside it (not met by the stabilisation's matrices) the library ldexp
__device__ __forceinline__ double pow2i(int e) {
    return (e >= -1022 && e <= 1023) ? __longlong_as_double((long long)(e + 1023) << 52) : ldexp(1.0, e);
}

inline size_t oz_smem_bytes() { return 2 * OZ_STAGE + 1024; }   // two stages (+ alignment slack)

// rows of X (rows x K, row-major, leading dimension ld) into OZ_S digit planes
// out[s][row][0..Kw) (BF16, zero for K <= k < Kw) and the row exponents ex[row];
// one warp per row.  The planes are prows x Kpad (prows >= rows, Kpad >= Kw), the
// shape of the tensor map that stages them.
__global__ void k_oz_split(const double* __restrict__ X, int rows, int K, int ld, __nv_bfloat16* out, int prows,
                           int Kpad, int Kw, int* ex) {
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
    const size_t plane = (size_t)prows * Kpad;
    constexpr int TOP = OZ_BITS * OZ_S;      // 56 fraction bits kept
    for (int k = lane; k < Kw; k += 32) {
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

__device__ __forceinline__ void tc_mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
        :: "r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(IDESC_BF16_128x64), "r"(acc));
}

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_u32(b)) : "memory");
}
// 3-D tiled tensor copy global -> shared, completion counted on an mbarrier
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        :: "r"(smem_u32(dst)), "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* b) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(smem_u32(b)) : "memory");
}

constexpr int OZ_THREADS = (OZ_EPI_WARPS + 2) * 32;

// tmA, tmB: 3-D tensor maps (k, row, digit) of the digit planes of op(A) rows
// and op(B)^T rows, box 8 x OZ_TM (OZ_TN) x OZ_S.
__global__ void __launch_bounds__(OZ_THREADS, 1) k_oz_gemm(const __grid_constant__ CUtensorMap tmA,
                                                          const __grid_constant__ CUtensorMap tmB, OzArgs g) {
    extern __shared__ __align__(1024) unsigned char oz_smem_raw[];
    // stages on a 1024-byte boundary (the dynamic allocation carries 1 KB of slack)
    unsigned char* oz_smem = oz_smem_raw + ((1024u - (smem_u32(oz_smem_raw) & 1023u)) & 1023u);
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_full[2], s_empty[2], s_win, s_free;
    __shared__ int s_fail, s_mma_waited, s_prod_issued;
    const int i0 = blockIdx.y * OZ_TM, j0 = blockIdx.x * OZ_TN;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&s_tmem)), "r"(512) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        s_fail = 0;
        s_mma_waited = 0;
        s_prod_issued = 0;
        mbar_init(&s_full[0], 1); mbar_init(&s_full[1], 1);
        mbar_init(&s_empty[0], 1); mbar_init(&s_empty[1], 1);
        mbar_init(&s_win, 1); mbar_init(&s_free, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;
    const int nchunks = g.Kpad / OZ_KC;
    const int nwin = (nchunks + OZ_WIN - 1) / OZ_WIN;
    volatile int* vfail = &s_fail;
    auto fail = [&](int where) {
        *vfail = 1;
        flag_error(g.st, DERR_TIMEOUT, where);
    };
    auto stage_a = [&](int st) { return oz_smem + (size_t)st * OZ_STAGE; };
    auto stage_b = [&](int st) { return oz_smem + (size_t)st * OZ_STAGE + (OZ_KC / 8) * OZ_A_KGROUP; };

    long long iacc[16];
    float facc[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        iacc[q] = 0;
        facc[q] = 0.0f;
    }
    const int row = 32 * (warp & 3) + lane;          // TMEM lane = output row of the tile (read-out warps)
    const int cbase = 16 * (warp >> 2);              // read-out warps w, w+4, w+8, w+12 split the 64 columns

    if (warp == OZ_PRODUCER_WARP) {
        // ---- producer: one elected thread issues the tensor copies of every chunk
        if (lane == 0) {
            int c = 0;
            for (; c < nchunks && !*vfail; ++c) {
                const int st = c & 1;
                if (c >= 2 && !mbar_wait_bounded(smem_u32(&s_empty[st]), ((c - 2) >> 1) & 1)) { fail(602); break; }
                mbar_expect_tx(&s_full[st], (uint32_t)OZ_STAGE);
                const int k0 = c * OZ_KC;
#pragma unroll
                for (int kg = 0; kg < OZ_KC / 8; ++kg) {
                    tma_load_3d(stage_a(st) + kg * OZ_A_KGROUP, &tmA, k0 + 8 * kg, i0, 0, &s_full[st]);
                    tma_load_3d(stage_b(st) + kg * OZ_B_KGROUP, &tmB, k0 + 8 * kg, j0, 0, &s_full[st]);
                }
            }
            s_prod_issued = c;
        }
    } else if (warp == OZ_MMA_WARP) {
        // ---- MMA issue: 36 digit products of each chunk into the 8 class accumulators
        if (lane == 0) {
            int c = 0;
            for (; c < nchunks && !*vfail; ++c) {
                const int st = c & 1, cw = c % OZ_WIN, wi = c / OZ_WIN;
                // a new window restarts the accumulators: the read-out of the last one must be done
                if (cw == 0 && c > 0 && !mbar_wait_bounded(smem_u32(&s_free), (wi - 1) & 1)) { fail(603); break; }
                if (!mbar_wait_bounded(smem_u32(&s_full[st]), (c >> 1) & 1)) { fail(604); break; }
                s_mma_waited = c + 1;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t abase = smem_u32(stage_a(st)), bbase = smem_u32(stage_b(st));
#pragma unroll 1
                for (int w = 0; w < OZ_CLASSES; ++w)
#pragma unroll 1
                    for (int sd = 0; sd <= w; ++sd) {
                        const uint32_t a0 = abase + (uint32_t)(sd * OZ_TM * 16);
                        const uint32_t b0 = bbase + (uint32_t)((w - sd) * OZ_TN * 16);
#pragma unroll
                        for (int kk = 0; kk < OZ_KC / 16; ++kk) {
                            const uint32_t accf = (cw > 0 || sd > 0 || kk > 0) ? 1u : 0u;
                            tc_mma_bf16(tmem + (uint32_t)(w * OZ_TN),
                                        tc_desc(a0 + (uint32_t)(2 * kk) * OZ_A_KGROUP, OZ_A_KGROUP, 128),
                                        tc_desc(b0 + (uint32_t)(2 * kk) * OZ_B_KGROUP, OZ_B_KGROUP, 128), accf);
                        }
                    }
                tc_commit(&s_empty[st]);
                if (cw == OZ_WIN - 1 || c == nchunks - 1) tc_commit(&s_win);
            }
            // on a failure, let the MMAs already issued land before tensor memory is freed
            if (*vfail && c > 0) mbar_wait_bounded(smem_u32(&s_empty[(c - 1) & 1]), ((c - 1) >> 1) & 1);
        }
    } else {
        // ---- read-out warps: classes 0..3 into one exact 64-bit integer, 4..7 into one FP32 sum
        // Every read-out warp reaches both named barriers of every window, and
        // all of them leave together on the stop flag latched between the two
        // (bar.sync has no time limit: no warp may skip one that others wait at).
        __shared__ int s_stop;
        for (int wi = 0; wi < nwin; ++wi) {
            int ok = 0;
            if (lane == 0) ok = mbar_wait_bounded(smem_u32(&s_win), wi & 1) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok && lane == 0) fail(601);
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int w = 0; w < OZ_CLASSES && ok; ++w) {
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
                    for (int q = 0; q < 16; ++q)
                        iacc[q] += (long long)__float2int_rn(__uint_as_float(v[q])) << (OZ_BITS * (3 - w));
                } else {
                    const float sc = ldexpf(1.0f, -OZ_BITS * (w - 4));
#pragma unroll
                    for (int q = 0; q < 16; ++q) facc[q] = fmaf(__uint_as_float(v[q]), sc, facc[q]);
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            asm volatile("bar.sync 1, %0;" :: "r"(OZ_EPI_WARPS * 32) : "memory");
            if (threadIdx.x == 0) {
                s_stop = *vfail;
                if (!s_stop) mbar_arrive(&s_free);
            }
            asm volatile("bar.sync 1, %0;" :: "r"(OZ_EPI_WARPS * 32) : "memory");
            if (s_stop) break;
        }
    }
    // copies still in flight after a failure must land before the CTA leaves
    __syncthreads();
    if (*vfail && threadIdx.x == OZ_PRODUCER_WARP * 32)
        for (int c = s_mma_waited; c < s_prod_issued; ++c) mbar_wait_bounded(smem_u32(&s_full[c & 1]), (c >> 1) & 1);
    // ---- epilogue through shared memory (coalesced rows of C).  Every FP64
    // instruction holds a sub-partition's FP64 unit for ~64 cycles on this part,
    // so the epilogue uses few of them per element: classes 0..3 were combined
    // exactly in 64-bit integers (|sum| < 2^50, exact in one conversion), powers
    // of two are built from exponent bits, and the column factors (and
    // reciprocals) are computed once per tile.
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (!*vfail) {
        constexpr int CLD = OZ_TN + 1;
        double* ct = reinterpret_cast<double*>(oz_smem);
        double* cfac = ct + OZ_TM * CLD;                 // OZ_TN column factors
        if (threadIdx.x < OZ_TN) {
            const int gj = j0 + threadIdx.x;
            double f = 0.0;
            if (gj < g.n) {
                f = pow2i(g.eb[gj]);
                if (g.cs) f = g.cs_inv ? f / g.cs[gj] : f * g.cs[gj];
            }
            cfac[threadIdx.x] = f;
        }
        if (warp < OZ_EPI_WARPS) {
            const double s3 = pow2i(-5 * OZ_BITS), s4 = pow2i(-6 * OZ_BITS);
#pragma unroll
            for (int q = 0; q < 16; ++q) ct[row * CLD + cbase + q] = fma((double)facc[q], s4, (double)iacc[q] * s3);
        }
        __syncthreads();
        for (int r = warp; r < OZ_TM; r += OZ_THREADS / 32) {
            const int gi = i0 + r;
            if (gi >= g.m) break;
            double ri = g.alpha * pow2i(g.ea[gi]);
            if (g.rs) ri = g.rs_inv ? ri / g.rs[gi] : ri * g.rs[gi];
            for (int cc = lane; cc < OZ_TN; cc += 32) {
                const int gj = j0 + cc;
                if (gj >= g.n) continue;
                const double v = ct[r * CLD + cc] * ri * cfac[cc];
                double* cp = g.C + (size_t)gi * g.ldc + gj;
                *cp = (g.beta == 0.0) ? v : fma(g.beta, *cp, v);
            }
        }
    }
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(512) : "memory");
}

}  // namespace afq
