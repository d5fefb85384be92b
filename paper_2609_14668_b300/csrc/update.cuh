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
    uint64_t key, ctr0;           // random number of site i is u(key, ctr0 + i)
    unsigned long long* n_acc;
    DevStatus* st;
    int precision;                // 0: FP64 flush; 1: split-TF32 tensor-core flush, FP32 accumulate
};

// ---------------------------------------------------------------------------
// Split-TF32 flush tile (precision 1): G[i0:i0+64, j0:j0+64] -= X Y with
// X = Xh + Xl, Y = Yh + Yl (each part a TF32 number, from the FP32 rounding of
// the FP64 value), product Xh Yh + Xh Yl + Xl Yh on the tensor cores with
// FP32 accumulation (Ootomo & Yokota 2022), subtracted in FP64.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t f32_to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void mma_m16n8k8_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

constexpr int FT = 64;   // flush tile edge (precision 1)

// smem: 4 arrays of kp x FT uint32 (kp = k rounded up to 8): Xh, Xl, Yh, Yl.
__device__ void flush_tile_tf32(const UpdArgs& a, int k, int i0, int j0, uint32_t* sm) {
    const int N = a.N;
    const int kp = (k + 7) & ~7;
    uint32_t* xh = sm;
    uint32_t* xl = xh + kp * FT;
    uint32_t* yh = xl + kp * FT;
    uint32_t* yl = yh + kp * FT;
    __syncthreads();
    for (int o = threadIdx.x; o < kp * FT; o += blockDim.x) {
        const int m = o / FT, q = o - m * FT;
        double xv = 0.0, yv = 0.0;
        if (m < k) {
            if (i0 + q < N) xv = __ldcg(a.Xs + (size_t)m * N + i0 + q);
            if (j0 + q < N) yv = __ldcg(a.Ys + (size_t)m * N + j0 + q);
        }
        const float xf = (float)xv, yf = (float)yv;
        const uint32_t xhi = f32_to_tf32(xf), yhi = f32_to_tf32(yf);
        xh[o] = xhi; xl[o] = f32_to_tf32(xf - __uint_as_float(xhi));
        yh[o] = yhi; yl[o] = f32_to_tf32(yf - __uint_as_float(yhi));
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int r0 = 16 * (warp >> 1);          // 4 row blocks of 16
    const int c0 = 32 * (warp & 1);           // 2 column blocks of 32 (4 n8 tiles)
    float acc[4][4];
#pragma unroll
    for (int n = 0; n < 4; ++n)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[n][q] = 0.f;
    for (int k0 = 0; k0 < kp; k0 += 8) {
        const int ka = (k0 + t) * FT, kb = (k0 + t + 4) * FT;
        const uint32_t ah[4] = {xh[ka + r0 + g], xh[ka + r0 + g + 8], xh[kb + r0 + g], xh[kb + r0 + g + 8]};
        const uint32_t al[4] = {xl[ka + r0 + g], xl[ka + r0 + g + 8], xl[kb + r0 + g], xl[kb + r0 + g + 8]};
#pragma unroll
        for (int n = 0; n < 4; ++n) {
            const int cc = c0 + 8 * n + g;
            const uint32_t bh0 = yh[ka + cc], bh1 = yh[kb + cc];
            const uint32_t bl0 = yl[ka + cc], bl1 = yl[kb + cc];
            mma_m16n8k8_tf32(acc[n], al, bh0, bh1);
            mma_m16n8k8_tf32(acc[n], ah, bl0, bl1);
            mma_m16n8k8_tf32(acc[n], ah, bh0, bh1);
        }
    }
#pragma unroll
    for (int n = 0; n < 4; ++n) {
        const int col = j0 + c0 + 8 * n + 2 * t;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int row = i0 + r0 + g + 8 * h;
            if (row >= N) continue;
            double* gp = a.G + (size_t)row * N + col;
            if (col < N) gp[0] = __ldcg(gp) - (double)acc[n][2 * h];
            if (col + 1 < N) gp[1] = __ldcg(gp + 1) - (double)acc[n][2 * h + 1];
        }
    }
}

__global__ void __launch_bounds__(UPD_THREADS) k_update_slice(UpdArgs a) {
    extern __shared__ double upd_smem[];
    __shared__ int s_dec[4];
    __shared__ double s_coef;
    const int N = a.N, W = a.W, nd = a.nd;
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const int gthreads = gridDim.x * blockDim.x;
    int cursor = 0, k = 0;
    for (;;) {
        // ------------------------------------------------------------ phase B
        if (blockIdx.x == 0) {
            double* Gw = upd_smem;                        // W x (W+1)
            double* uu = Gw + W * (W + 1);                // W uniforms
            int8_t* sw = reinterpret_cast<int8_t*>(uu + W); // W field values
            const int nw = min(W, N - cursor);
            const int ld = W + 1;
            for (int o = threadIdx.x; o < nw * nw; o += blockDim.x) {
                const int r = o / nw, c = o - r * nw;
                Gw[r * ld + c] = (k == 0) ? __ldcg(a.G + (size_t)(cursor + r) * N + cursor + c)
                                          : __ldcg(a.Gw + r * W + c);
            }
            for (int t = threadIdx.x; t < nw; t += blockDim.x) {
                uu[t] = sm64_uniform(a.key, a.ctr0 + cursor + t);
                sw[t] = a.s[cursor + t];
            }
            __syncthreads();
            int kk = k, tstop = nw;
            for (int t = 0; t < nw; ++t) {
                if (threadIdx.x == 0) {
                    const int i = cursor + t;
                    const int sg = sw[t];
                    const double g = Gw[t * ld + t];
                    const double dl = sg > 0 ? a.dl_p : a.dl_m;
                    const double ef = sg > 0 ? a.ef_p : a.ef_m;
                    const double r = fma(dl, 1.0 - g, 1.0);
                    const double R = ef * r * r;
                    int acc = uu[t] < R;
                    if (!isfinite(r)) { flag_error(a.st, DERR_NUMERIC, 200); acc = 0; }
                    s_dec[0] = acc;
                    if (acc) {
                        s_coef = dl / r;
                        a.msite[kk] = i;
                        a.mcoef[kk] = dl / r;
                        a.s[i] = (int8_t)(-sg);
                    }
                }
                __syncthreads();
                if (s_dec[0]) {
                    const double c = s_coef;
                    const int rest = nw - t - 1;
                    // x, y of the new move at the later window positions
                    for (int p = threadIdx.x; p < rest; p += blockDim.x) {
                        const int q = t + 1 + p;
                        a.xw[kk * W + q] = c * Gw[q * ld + t];
                        a.yw[kk * W + q] = -Gw[t * ld + q];
                    }
                    // rank-1 update of the trailing block: Gw -= x y^T
                    for (int o = threadIdx.x; o < rest * rest; o += blockDim.x) {
                        const int q = t + 1 + o / rest, p = t + 1 + o % rest;
                        Gw[q * ld + p] = fma(c * Gw[q * ld + t], Gw[t * ld + p], Gw[q * ld + p]);
                    }
                    ++kk;
                    __syncthreads();
                    if (kk == nd) { tstop = t + 1; break; }
                }
            }
            if (threadIdx.x == 0) {
                a.ctl[0] = cursor;
                a.ctl[1] = k;
                a.ctl[2] = kk;
                a.ctl[3] = cursor + tstop;
                if (kk > k) atomicAdd(a.n_acc, (unsigned long long)(kk - k));
            }
        }
        if (!grid_barrier(a.st, 1)) return;
        const int c0 = __ldcg(a.ctl + 0), kb = __ldcg(a.ctl + 1), ka = __ldcg(a.ctl + 2), c1 = __ldcg(a.ctl + 3);
        // ------------------------------------------------------------ phase C
        // One warp per vector index j (spread over all CTAs); lane m owns the
        // window's m-th new move, so no FP64 cross-lane reductions are needed.
        if (ka > kb) {
            const int nn = ka - kb;
            const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
            const bool mine = lane < nn;
            const int mm = kb + lane;
            const int im = mine ? __ldcg(a.msite + mm) : 0;
            const int tm = im - c0;
            const double cm = mine ? __ldcg(a.mcoef + mm) : 0.0;
            for (int j = blockIdx.x + gridDim.x * warp; j < N; j += gridDim.x * nwarp) {
                // contributions of moves pending from earlier windows (4 partial sums for ILP)
                double ox0 = 0.0, ox1 = 0.0, oy0 = 0.0, oy1 = 0.0;
                if (mine) {
                    int p = 0;
                    for (; p + 1 < kb; p += 2) {
                        const double* X0 = a.Xs + (size_t)p * N;
                        const double* Y0 = a.Ys + (size_t)p * N;
                        ox0 = fma(__ldcg(X0 + j), __ldcg(Y0 + im), ox0);
                        oy0 = fma(__ldcg(X0 + im), __ldcg(Y0 + j), oy0);
                        ox1 = fma(__ldcg(X0 + N + j), __ldcg(Y0 + N + im), ox1);
                        oy1 = fma(__ldcg(X0 + N + im), __ldcg(Y0 + N + j), oy1);
                    }
                    if (p < kb) {
                        ox0 = fma(__ldcg(a.Xs + (size_t)p * N + j), __ldcg(a.Ys + (size_t)p * N + im), ox0);
                        oy0 = fma(__ldcg(a.Xs + (size_t)p * N + im), __ldcg(a.Ys + (size_t)p * N + j), oy0);
                    }
                }
                // recursion over the new moves (Eq. DelayRgenk), lane m accumulates move m
                double ax = mine ? __ldcg(a.G + (size_t)j * N + im) - (ox0 + ox1) : 0.0;
                double ay = mine ? (j == im ? 1.0 : 0.0) - __ldcg(a.G + (size_t)im * N + j) + (oy0 + oy1) : 0.0;
                double xv = 0.0, yv = 0.0;
                for (int q = 0; q < nn; ++q) {
                    if (lane == q) { xv = cm * ax; yv = ay; }
                    const double xq = __shfl_sync(0xffffffffu, xv, q);
                    const double yq = __shfl_sync(0xffffffffu, yv, q);
                    if (mine && lane > q) {
                        ax = fma(-xq, __ldcg(a.yw + (kb + q) * W + tm), ax);
                        ay = fma(__ldcg(a.xw + (kb + q) * W + tm), yq, ay);
                    }
                }
                if (mine) {
                    a.Xs[(size_t)mm * N + j] = xv;
                    a.Ys[(size_t)mm * N + j] = yv;
                }
            }
        }
        if (!grid_barrier(a.st, 2)) return;
        k = ka;
        const bool done = (c1 >= N);
        // ------------------------------------------------------------ phase F
        if (k > 0 && (k == nd || done)) {
            if (a.precision == 1) {
                const int nt = (N + FT - 1) / FT;
                for (int tile = blockIdx.x; tile < nt * nt; tile += gridDim.x)
                    flush_tile_tf32(a, k, (tile / nt) * FT, (tile % nt) * FT, reinterpret_cast<uint32_t*>(upd_smem));
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
            if (!grid_barrier(a.st, 3)) return;
        }
        if (done) return;
        cursor = c1;
        // ------------------------------------------------------------ phase A
        if (k > 0) {
            const int nw = min(W, N - cursor);
            const int lane = threadIdx.x & 31;
            const int gwarp = gtid >> 5, nwarps = gthreads >> 5;
            for (int e = gwarp; e < nw * nw; e += nwarps) {
                const int r = e / nw, c = e - r * nw;
                double acc = 0.0;
                for (int m = lane; m < k; m += 32)
                    acc = fma(__ldcg(a.Xs + (size_t)m * N + cursor + r), __ldcg(a.Ys + (size_t)m * N + cursor + c), acc);
                acc = warp_sum(acc);
                if (lane == 0) a.Gw[r * W + c] = __ldcg(a.G + (size_t)(cursor + r) * N + cursor + c) - acc;
            }
            if (!grid_barrier(a.st, 4)) return;
        }
    }
}

}  // namespace afq
