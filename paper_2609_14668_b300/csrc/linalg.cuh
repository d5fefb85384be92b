// FP64 dense linear algebra for the QR stabilisation of Sec. II.B (its second
// implementation note) and the recomputation of G = (1 + R L)^-1 (Eq. GrFMat).
//
// B300 design notes.  FP64 runs at ~1.1 TFLOP/s on this part (SIMT DFMA is a
// little faster than the FP64 tensor path, DMMA), so every kernel here is
// bound by the FP64 pipes, not by memory: the working matrices (10.6 MB at
// N = 1152) stay resident in the 126 MB L2.  The kernels therefore aim at
// keeping all 148 SMs' FP64 units busy:
//   * k_dgemm: SIMT GEMM on 32x32 output tiles with a row/column scaling epilogue;
//   * k_qr_cols, k_lu_cols: Householder QR and LU with partial pivoting as
//     cooperative kernels, columns owned cyclically by CTAs, column j handed on
//     through publication buffers (no flag, no fence) and applied by every CTA
//     to its own columns (one-column lookahead on the critical path);
//   * column-parallel kernels (one warp per column, no inter-CTA sync) for
//     forming Q and the triangular solves; the blocked solves' diagonal blocks
//     (k_trsm_leaf).
// Matrices are row-major; a "column-major" matrix X is stored as its
// transpose Xt (row c of Xt = column c of X).
#pragma once
#include "common.cuh"

namespace afq {

// C[i][j] = alpha * rs_i * (op(A) op(B))_ij * cs_j + beta * C[i][j]
// op(A) is m x k: A[i][p] (transA = 0, lda >= k) or A[p][i] (transA = 1, lda >= m).
// op(B) is k x n: B[p][j] (transB = 0) or B[j][p] (transB = 1).
struct GemmArgs {
    const double* A; const double* B; double* C;
    int m, n, k, lda, ldb, ldc, transA, transB;
    double alpha, beta;
    const double* rs; const double* cs;   // optional (nullptr = 1)
    int rs_inv, cs_inv;                   // 1: scale by the reciprocal
    int a_upper;                          // 1: op(A) is upper triangular, skip the zero blocks p < i
};

// 32 x 32 output tiles (1296 CTAs at N = 1152: 8.8 per SM, so the last wave is
// nearly full), 256 threads with 2 x 2 outputs each.  FP64 FMAs, not shared
// memory or L2 bandwidth, are the limit at this size.
constexpr int GT = 32, GK = 32;

__global__ void __launch_bounds__(256) k_dgemm(GemmArgs g) {
    __shared__ double As[GK][GT + 1];
    __shared__ double Bs[GK][GT + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int i0 = blockIdx.y * GT, j0 = blockIdx.x * GT;
    double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
    const int pstart = g.a_upper ? (i0 / GK) * GK : 0;
    for (int p0 = pstart; p0 < g.k; p0 += GK) {
        for (int o = threadIdx.x; o < GK * GT; o += 256) {
            int pp, ii;
            if (g.transA) { pp = o / GT; ii = o % GT; } else { ii = o / GK; pp = o % GK; }
            const int gi = i0 + ii, gp = p0 + pp;
            double v = 0.0;
            if (gi < g.m && gp < g.k) v = g.transA ? g.A[(size_t)gp * g.lda + gi] : g.A[(size_t)gi * g.lda + gp];
            As[pp][ii] = v;
            int jj;
            if (g.transB) { jj = o / GK; pp = o % GK; } else { pp = o / GT; jj = o % GT; }
            const int gj = j0 + jj, gq = p0 + pp;
            double w = 0.0;
            if (gj < g.n && gq < g.k) w = g.transB ? g.B[(size_t)gj * g.ldb + gq] : g.B[(size_t)gq * g.ldb + gj];
            Bs[pp][jj] = w;
        }
        __syncthreads();
#pragma unroll 8
        for (int p = 0; p < GK; ++p) {
            const double a0 = As[p][ty], a1 = As[p][ty + 16];
            const double b0 = Bs[p][tx], b1 = Bs[p][tx + 16];
            acc[0][0] = fma(a0, b0, acc[0][0]);
            acc[0][1] = fma(a0, b1, acc[0][1]);
            acc[1][0] = fma(a1, b0, acc[1][0]);
            acc[1][1] = fma(a1, b1, acc[1][1]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const int i = i0 + ty + 16 * a;
        if (i >= g.m) continue;
        double r = g.alpha;
        if (g.rs) r = g.rs_inv ? r / g.rs[i] : r * g.rs[i];
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int j = j0 + tx + 16 * b;
            if (j >= g.n) continue;
            double v = acc[a][b] * r;
            if (g.cs) v = g.cs_inv ? v / g.cs[j] : v * g.cs[j];
            double* c = g.C + (size_t)i * g.ldc + j;
            *c = (g.beta == 0.0) ? v : fma(g.beta, *c, v);
        }
    }
}

// out[j][i] = in[i][j] * (rs ? rs[i] : 1) * (cs ? cs[j] : 1)   (in: m x n, row-major)
__global__ void k_transpose_scale(const double* __restrict__ in, double* __restrict__ out, int m, int n,
                                  const double* rs, int rs_inv, const double* cs, int cs_inv) {
    __shared__ double tile[32][33];
    const int bi = blockIdx.y * 32, bj = blockIdx.x * 32;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int i = bi + y, j = bj + threadIdx.x;
        double v = 0.0;
        if (i < m && j < n) {
            v = in[(size_t)i * n + j];
            if (rs) v = rs_inv ? v / rs[i] : v * rs[i];
            if (cs) v = cs_inv ? v / cs[j] : v * cs[j];
        }
        tile[y][threadIdx.x] = v;
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int j = bj + y, i = bi + threadIdx.x;
        if (i < m && j < n) out[(size_t)j * m + i] = tile[threadIdx.x][y];
    }
}

// out[j][i] = in[perm[i]][j] * rs[perm[i]] (or / rs[perm[i]] with rs_inv), n x n
// row-major: the transpose of the row-permuted, row-scaled input (the right-hand
// sides P Y of the blocked solves, one per row of out).  perm must be a
// permutation of [0, n).
__global__ void k_transpose_perm(const double* __restrict__ in, double* __restrict__ out, int n,
                                 const int* __restrict__ perm, const double* rs, int rs_inv) {
    __shared__ double tile[32][33];
    const int bi = blockIdx.y * 32, bj = blockIdx.x * 32;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int i = bi + y, j = bj + threadIdx.x;
        double v = 0.0;
        if (i < n && j < n) {
            const int r = perm[i];
            v = in[(size_t)r * n + j];
            if (rs) v = rs_inv ? v / rs[r] : v * rs[r];
        }
        tile[y][threadIdx.x] = v;
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int j = bj + y, i = bi + threadIdx.x;
        if (i < n && j < n) out[(size_t)j * n + i] = tile[threadIdx.x][y];
    }
}

// Diagonal-block step of the blocked triangular solves.  Every row c of Yt (a
// right-hand side; one warp each) has its entries r0 .. r0+nb replaced by
// L_bb^-1 y (UPPER = 0: the unit lower triangle) or U_bb^-1 y (UPPER = 1: the
// upper triangle with its diagonal) of the block at (r0, r0) of the row-major LU
// factor Fr.  nb <= TRSM_LEAF: lane l holds entries l and l + 32.  The block
// is staged transposed in shared memory (Ls[j][i] = the coefficient of row i in
// step j) with zeros where a step must leave a row alone, so a step is one FMA
// instruction per group of 32 rows it can reach: the FP64 unit of this part
// takes a warp instruction per ~64 cycles however many lanes are busy.
constexpr int TRSM_LEAF = 64;
template <int UPPER>
__global__ void __launch_bounds__(256) k_trsm_leaf(const double* __restrict__ Fr, double* Yt, int n, int nrhs,
                                                   int r0, int nb) {
    __shared__ double Ls[TRSM_LEAF][TRSM_LEAF + 1];
    __shared__ double dinv[TRSM_LEAF];
    for (int idx = threadIdx.x; idx < TRSM_LEAF * TRSM_LEAF; idx += blockDim.x) {
        const int i = idx / TRSM_LEAF, j = idx % TRSM_LEAF;
        double v = 0.0;
        if (i < nb && j < nb && (UPPER ? i < j : i > j)) v = Fr[(size_t)(r0 + i) * n + r0 + j];
        Ls[j][i] = v;
    }
    if (UPPER)
        for (int j = threadIdx.x; j < nb; j += blockDim.x) dinv[j] = 1.0 / Fr[(size_t)(r0 + j) * n + r0 + j];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int c = blockIdx.x * nw + warp; c < nrhs; c += gridDim.x * nw) {
        double* y = Yt + (size_t)c * n + r0;
        double y0 = lane < nb ? y[lane] : 0.0;
        double y1 = lane + 32 < nb ? y[lane + 32] : 0.0;
        if (!UPPER) {
            // step j: y_i -= L_ij y_j for i > j
            for (int j = 0; j < nb - 1; ++j) {
                const double yj = __shfl_sync(0xffffffffu, j < 32 ? y0 : y1, j & 31);
                if (j < 31) y0 = fma(-Ls[j][lane], yj, y0);
                if (nb > 32) y1 = fma(-Ls[j][lane + 32], yj, y1);
            }
        } else {
            // step j (descending): x_j = y_j / U_jj, then y_i -= U_ij x_j for i < j
            for (int j = nb - 1; j >= 0; --j) {
                const double xj = __shfl_sync(0xffffffffu, j < 32 ? y0 : y1, j & 31) * dinv[j];
                if (lane == (j & 31)) {
                    if (j < 32) y0 = xj;
                    else y1 = xj;
                }
                if (j >= 1) y0 = fma(-Ls[j][lane], xj, y0);
                if (j >= 33) y1 = fma(-Ls[j][lane + 32], xj, y1);
            }
        }
        if (lane < nb) y[lane] = y0;
        if (lane + 32 < nb) y[lane + 32] = y1;
    }
}

// out[c][i] = in[c][i] / xs[i] (xs may be null: a copy), n x n; flags
// DERR_NUMERIC on a non-finite result (the end of the solves of G).
__global__ void k_div_cols_check(const double* __restrict__ in, double* out, int n, const double* __restrict__ xs,
                                 DevStatus* st) {
    bool bad = false;
    const size_t nn = (size_t)n * n;
    for (size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x; o < nn; o += (size_t)gridDim.x * blockDim.x) {
        double v = in[o];
        if (xs) v /= xs[o % n];
        if (!isfinite(v)) bad = true;
        out[o] = v;
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) flag_error(st, DERR_NUMERIC, 102);
}

// ---------------------------------------------------------------------------
// Column hand-off of the QR and LU kernels.  Step j of either factorisation
// needs column j as its owner finished it (the reflector, or the multipliers)
// and one scalar (tau_j, or the pivot row).  The owner stores them into
// publication buffers (column j at pub + j n, the scalar at pubx[j]) that were
// filled with the PUB_EMPTY pattern before the launch.  Every element is
// stored exactly once and 8-byte stores are single-copy atomic, so a reader
// knows an element is final as soon as it differs from the pattern: no flag,
// no memory fence, and readers stage the column while the owner is still
// writing it.  The scalar is stored first; while a CTA waits, only its thread
// 0 polls (the scalar), then every thread loads its elements once and polls
// again only those still empty.  The pattern is a signalling NaN (arithmetic
// never produces one).  Every wait is bounded by the wait limit.
// ---------------------------------------------------------------------------
constexpr unsigned long long PUB_EMPTY = 0x7FF4A5A55A5AA5A5ull;

__device__ __forceinline__ unsigned long long ld_relaxed_b64(const double* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_b64(double* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" :: "l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed_f64(double* p, double x) {
    st_relaxed_b64(p, (unsigned long long)__double_as_longlong(x));
}

// pub[0..len) and pubx[0..n) <- PUB_EMPTY (before every QR or LU launch).
__global__ void k_pub_clear(double* pub, size_t len, double* pubx, int n) {
    const double e = __longlong_as_double((long long)PUB_EMPTY);
    for (size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x; o < len; o += (size_t)gridDim.x * blockDim.x)
        pub[o] = e;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) pubx[i] = e;
}

// Wait until *p is published (its bits in v).  False on another CTA's failure,
// or on a timeout, which is flagged with site code `where`.
__device__ bool await_published(const double* p, unsigned long long& v, DevStatus* st, unsigned long long lim,
                                int where) {
    v = ld_relaxed_b64(p);
    if (v != PUB_EMPTY) return true;
    const unsigned long long t0 = global_ns();
    unsigned int ns = 8;
    for (;;) {
        __nanosleep(ns);
        v = ld_relaxed_b64(p);
        if (v != PUB_EMPTY) return true;
        if (*(volatile int*)&st->err) return false;
        if (global_ns() - t0 > lim) {
            flag_error(st, DERR_TIMEOUT, where);
            return false;
        }
        if (ns < 64) ns <<= 1;
    }
}

// dst[i - off] = src[i] for i in [lo, n) from a publication buffer (whole CTA),
// up to 8 loads per thread in flight.  False as await_published.
__device__ bool stage_published(const double* src, double* dst, int lo, int n, int off, DevStatus* st,
                                unsigned long long lim, int where) {
    constexpr int SB = 8;
    for (int i0 = lo + threadIdx.x; i0 < n; i0 += SB * blockDim.x) {
        unsigned long long v[SB];
#pragma unroll
        for (int q = 0; q < SB; ++q) {
            const int i = i0 + q * blockDim.x;
            v[q] = i < n ? ld_relaxed_b64(src + i) : 0ull;
        }
#pragma unroll
        for (int q = 0; q < SB; ++q) {
            const int i = i0 + q * blockDim.x;
            if (i < n) {
                if (v[q] == PUB_EMPTY && !await_published(src + i, v[q], st, lim, where)) return false;
                dst[i - off] = __longlong_as_double((long long)v[q]);
            }
        }
    }
    return true;
}

// ---------------------------------------------------------------------------
// Householder QR of a column-major n x n matrix A (array At, row c = column c).
// On exit: R in the upper triangle (At[c][i], i <= c), reflector j stored below
// the diagonal (At[j][i], i > j, implicit 1 at i = j), tau[j].
// H_j = I - tau_j v_j v_j^T,  A = H_0 H_1 ... H_{n-2} R.
// Cooperative launch; column c is owned by CTA c % gridDim.x; reflector j and
// tau_j are handed on through the publication buffers (pub: n x n, pubx: n).
// ---------------------------------------------------------------------------
struct QRArgs {
    double* At; double* tau; double* pub; double* pubx; int n;
    DevStatus* st;
};

// Householder reflector of column j (rows j..n-1), in place in `col`, and its
// publication (tau_j first, then v_j); whole CTA (256 threads).  The scalars
// (norm, beta, tau, 1/(alpha - beta)) are computed by one thread and shared:
// redundant FP64 square roots and reciprocals in every warp would each hold an
// FP64 unit.  red: >= 140 doubles.
__device__ void qr_make_reflector(const QRArgs& q, double* col, int j, double* red) {
    const int n = q.n;
    double s = 0.0;
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) { const double x = col[i]; s = fma(x, x, s); }
    s = block_sum256(s, red);
    if (threadIdx.x == 0) {
        const double alpha = col[j];
        double tau = 0.0, beta = alpha, scale = 0.0;
        if (s > 0.0) {
            const double nrm = sqrt(fma(alpha, alpha, s));
            beta = alpha <= 0.0 ? nrm : -nrm;
            tau = (beta - alpha) * recip_fast(beta);
            scale = recip_fast(alpha - beta);
        }
        col[j] = beta;
        q.tau[j] = tau;
        st_relaxed_f64(q.pubx + j, tau);
        red[138] = scale;
        if (!isfinite(beta) || !isfinite(tau)) flag_error(q.st, DERR_NUMERIC, 100);
    }
    __syncthreads();
    const double scale = red[138];
    double* pj = q.pub + (size_t)j * n;
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) {
        const double x = col[i] * scale;
        col[i] = x;
        st_relaxed_f64(pj + i, x);
    }
    __syncthreads();
}

// Apply H_j (v in shared memory, rows j..n-1, v[0] = 1) to a column; one warp.
__device__ __forceinline__ void qr_apply_warp(const double* __restrict__ v, double tau, double* col, int j, int n) {
    const int lane = threadIdx.x & 31;
    double w = 0.0;
    for (int i = j + lane; i < n; i += 32) w = fma(v[i - j], col[i], w);
    w = warp_sum(w) * tau;
    for (int i = j + lane; i < n; i += 32) col[i] = fma(-w, v[i - j], col[i]);
}

// Apply H_j to a column with the whole CTA (the lookahead column on the critical path).
__device__ void qr_apply_block(const double* __restrict__ v, double tau, double* col, int j, int n, double* red) {
    double w = 0.0;
    for (int i = j + threadIdx.x; i < n; i += blockDim.x) w = fma(v[i - j], col[i], w);
    w = block_sum256(w, red) * tau;
    for (int i = j + threadIdx.x; i < n; i += blockDim.x) col[i] = fma(-w, v[i - j], col[i]);
    __syncthreads();
}

// Dynamic shared memory: n doubles for the current reflector, plus (when
// cols_in_smem) ceil(n / gridDim.x) * n doubles holding this CTA's columns,
// which are copied to At once final.
__global__ void __launch_bounds__(256) k_qr_cols(QRArgs q, int cols_in_smem) {
    extern __shared__ double qr_smem[];
    __shared__ double red[140];
    __shared__ double s_tau;
    __shared__ int s_abort;
    const int n = q.n, G = gridDim.x, me = blockIdx.x;
    const int warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    double* v = qr_smem;
    double* cols = qr_smem + n;
    auto col = [&](int c) -> double* {
        return cols_in_smem ? cols + (size_t)((c - me) / G) * n : q.At + (size_t)c * n;
    };
    auto store_final = [&](int c) {
        if (cols_in_smem) {
            const double* src = col(c);
            double* g = q.At + (size_t)c * n;
            for (int i = threadIdx.x; i < n; i += blockDim.x) g[i] = src[i];
        }
    };
    if (threadIdx.x == 0) s_abort = 0;
    if (cols_in_smem)
        for (int c = me; c < n; c += G) {
            double* d = col(c);
            for (int i = threadIdx.x; i < n; i += blockDim.x) d[i] = q.At[(size_t)c * n + i];
        }
    __syncthreads();
    const unsigned long long lim = wait_limit(q.st);
    if (me == 0) {
        qr_make_reflector(q, col(0), 0, red);
        store_final(0);
    }
    for (int j = 0; j < n - 1; ++j) {
        if (threadIdx.x == 0) {
            unsigned long long t;
            if (await_published(q.pubx + j, t, q.st, lim, 101)) s_tau = __longlong_as_double((long long)t);
            else s_abort = 1;
        }
        __syncthreads();
        if (s_abort) return;
        const double tau = s_tau;
        if (!stage_published(q.pub + (size_t)j * n, v, j + 1, n, j, q.st, lim, 101)) s_abort = 1;
        if (threadIdx.x == 0) v[0] = 1.0;
        __syncthreads();
        if (s_abort) return;
        // lookahead: the owner of column j+1 finishes it first and publishes it
        if ((j + 1) % G == me) {
            double* c1 = col(j + 1);
            if (tau != 0.0) qr_apply_block(v, tau, c1, j, n, red);
            if (j + 1 < n - 1) qr_make_reflector(q, c1, j + 1, red);
            store_final(j + 1);
        }
        if (tau != 0.0) {
            int cnt = 0;
            for (int c = j + 2 + ((me - (j + 2)) % G + G) % G; c < n; c += G, ++cnt)
                if (cnt % nwarp == warp) qr_apply_warp(v, tau, col(c), j, n);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Column-parallel kernels on CPB_ columns per CTA (one warp each, 256 threads).
// The CPB_ columns stay in shared memory; the vector every column needs at
// step j (reflector v_j, or column i of R) is staged once per step in shared
// memory for all warps, with the next step's vector prefetched into registers
// (PRE_ per thread, so n <= 256 PRE_) while the current step computes.
// Dynamic shared memory: (CPB_ + 2) * n doubles.  Two shapes: <8, 8> for
// n <= 2048, and <4, 16> for n <= 4096 (the larger matrices leave room in
// shared memory for only four columns; the other four warps help staging).
// ---------------------------------------------------------------------------
constexpr int COL_MAX_N = 4096;   // largest matrix dimension of the column kernels

__device__ __forceinline__ double dot4(const double* __restrict__ a, const double* __restrict__ b, int lo, int hi) {
    const int lane = threadIdx.x & 31;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int i = lo + lane;
    for (; i + 96 < hi; i += 128) {
        s0 = fma(a[i], b[i], s0);
        s1 = fma(a[i + 32], b[i + 32], s1);
        s2 = fma(a[i + 64], b[i + 64], s2);
        s3 = fma(a[i + 96], b[i + 96], s3);
    }
    for (; i < hi; i += 32) s0 = fma(a[i], b[i], s0);
    return warp_sum((s0 + s1) + (s2 + s3));
}

// Stage vector src[lo..hi) into dst[lo..hi) (whole CTA), using per-thread
// prefetch registers: pre[q] holds src[lo + threadIdx.x + q*blockDim.x].
template <int PRE_>
__device__ __forceinline__ void prefetch_vec(const double* __restrict__ src, int lo, int hi, double (&pre)[PRE_]) {
#pragma unroll
    for (int q = 0; q < PRE_; ++q) {
        const int i = lo + threadIdx.x + q * blockDim.x;
        pre[q] = (i < hi) ? __ldg(src + i) : 0.0;
    }
}
template <int PRE_>
__device__ __forceinline__ void store_vec(double* dst, int lo, int hi, const double (&pre)[PRE_]) {
#pragma unroll
    for (int q = 0; q < PRE_; ++q) {
        const int i = lo + threadIdx.x + q * blockDim.x;
        if (i < hi) dst[i] = pre[q];
    }
}

// ---------------------------------------------------------------------------
// LU factorisation with partial pivoting of a column-major n x n matrix A
// (array At), P A = L U: on exit L (unit lower, below the diagonal) and U
// (upper, with the diagonal) overwrite At, piv[j] is the row swapped with row j
// at step j.  Cooperative launch, the same column ownership, shared-memory
// column storage and publication hand-off as k_qr_cols (the scalar of step j is
// the pivot row, stored as the bits of an integer); the critical path of a step
// holds one reduction (the pivot search) instead of the two of a Householder
// step.
// In At the multipliers of column j stay in the row order of step j (the
// column-step solves replay the swaps in turn).  With Fr set, the kernel also
// writes the factor row-major with every later swap applied to the earlier
// multipliers (P A = L U with P = P_{n-2} ... P_0 and the final L, as the
// blocked solves need it), and lperm (the combined row order: row i of P A is
// row lperm[i] of A): the owner of a finished column swaps its two entries in
// Fr at every later step, CTA 0 keeps lperm.  Neither is read during the
// factorisation.
// ---------------------------------------------------------------------------
struct LUArgs {
    double* At; int* piv; double* pub; double* pubx; int n;
    DevStatus* st;
    double* Fr; int* lperm;     // optional (both or neither)
};

// pivot search, swap, scaling and publication of column j (rows j..n-1), whole
// CTA (256 threads).  Magnitudes are compared as the integer images of |x| (ties
// to the smaller row, a NaN wins and is flagged), so the search uses no FP64
// instruction; one thread forms the pivot's reciprocal.
__device__ void lu_pivot_column(const LUArgs& q, double* col, int j, double* redv, int* redi) {
    const int n = q.n;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    long long best = -1;
    int bi = j;
    for (int i = j + threadIdx.x; i < n; i += blockDim.x) {
        const long long m = __double_as_longlong(col[i]) & 0x7fffffffffffffffll;
        if (m > best) { best = m; bi = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    long long* redb = reinterpret_cast<long long*>(redv);
    if (lane == 0) { redb[warp] = best; redi[warp] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < nwarp; ++w)
            if (redb[w] > best || (redb[w] == best && redi[w] < bi)) { best = redb[w]; bi = redi[w]; }
        const double t = col[j];
        col[j] = col[bi];
        col[bi] = t;
        const double pv = col[j];
        q.piv[j] = bi;
        st_relaxed_b64(q.pubx + j, (unsigned long long)bi);
        if (best <= 0 || !finite_bits(pv)) flag_error(q.st, DERR_NUMERIC, 110);
        redv[33] = recip_fast(pv);
    }
    __syncthreads();
    const double inv = redv[33];
    double* pj = q.pub + (size_t)j * n;
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) {
        const double x = col[i] * inv;
        col[i] = x;
        st_relaxed_f64(pj + i, x);
    }
    __syncthreads();
}

// apply step j (swap rows j, p; a_i -= l_ij a_j for i > j) to a column; one warp
__device__ __forceinline__ void lu_apply_warp(const double* __restrict__ l, int p, double* col, int j, int n) {
    const int lane = threadIdx.x & 31;
    double aj = 0.0;
    if (lane == 0) {
        aj = col[p];
        if (p != j) { col[p] = col[j]; col[j] = aj; }
    }
    aj = __shfl_sync(0xffffffffu, aj, 0);
    __syncwarp();
    for (int i = j + 1 + lane; i < n; i += 32) col[i] = fma(-l[i], aj, col[i]);
    __syncwarp();
}

__global__ void __launch_bounds__(256) k_lu_cols(LUArgs q, int cols_in_smem) {
    extern __shared__ double lu_smem[];
    __shared__ double redv[34];
    __shared__ int redi[33];
    __shared__ int s_abort, s_piv;
    const int n = q.n, G = gridDim.x, me = blockIdx.x;
    const int warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    double* l = lu_smem;                  // multipliers of the current step (rows j+1..n-1)
    double* cols = lu_smem + n;
    auto col = [&](int c) -> double* {
        return cols_in_smem ? cols + (size_t)((c - me) / G) * n : q.At + (size_t)c * n;
    };
    // a finished column: to At (when held in shared memory) and to the row-major factor
    auto store_final = [&](int c) {
        const double* src = col(c);
        if (cols_in_smem) {
            double* g = q.At + (size_t)c * n;
            for (int i = threadIdx.x; i < n; i += blockDim.x) g[i] = src[i];
        }
        if (q.Fr)
            for (int i = threadIdx.x; i < n; i += blockDim.x) q.Fr[(size_t)i * n + c] = src[i];
    };
    if (threadIdx.x == 0) s_abort = 0;
    if (cols_in_smem)
        for (int c = me; c < n; c += G) {
            double* d = col(c);
            for (int i = threadIdx.x; i < n; i += blockDim.x) d[i] = q.At[(size_t)c * n + i];
        }
    if (me == 0 && q.lperm)
        for (int i = threadIdx.x; i < n; i += blockDim.x) q.lperm[i] = i;
    __syncthreads();
    const unsigned long long lim = wait_limit(q.st);
    if (me == 0) {
        lu_pivot_column(q, col(0), 0, redv, redi);
        store_final(0);
    }
    for (int j = 0; j < n - 1; ++j) {
        if (threadIdx.x == 0) {
            unsigned long long t;
            if (await_published(q.pubx + j, t, q.st, lim, 111)) s_piv = (int)t;
            else s_abort = 1;
        }
        __syncthreads();
        if (s_abort) return;
        const int p = s_piv;
        if (q.Fr && p != j) {
            // step j's swap on the multipliers of this CTA's finished columns (c < j; warp 0,
            // whose memory latency the other warps' FP64 work covers), and on the row order
            for (int c = me + threadIdx.x * G; threadIdx.x < 32 && c < j; c += 32 * G) {
                double* f = q.Fr + c;
                const double a = f[(size_t)j * n], b = f[(size_t)p * n];
                f[(size_t)j * n] = b;
                f[(size_t)p * n] = a;
            }
            if (me == 0 && threadIdx.x == 32) {
                const int a = q.lperm[j], b = q.lperm[p];
                q.lperm[j] = b;
                q.lperm[p] = a;
            }
        }
        if (!stage_published(q.pub + (size_t)j * n, l, j + 1, n, 0, q.st, lim, 111)) s_abort = 1;
        __syncthreads();
        if (s_abort) return;
        // lookahead: the owner of column j+1 finishes it first and publishes it
        if ((j + 1) % G == me) {
            double* c1 = col(j + 1);
            if (threadIdx.x == 0) {
                const double t = c1[p];
                if (p != j) { c1[p] = c1[j]; c1[j] = t; }
                redv[32] = t;
            }
            __syncthreads();
            const double aj = redv[32];
            for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) c1[i] = fma(-l[i], aj, c1[i]);
            __syncthreads();
            if (j + 1 < n - 1) lu_pivot_column(q, c1, j + 1, redv, redi);
            else if (threadIdx.x == 0) q.piv[j + 1] = j + 1;
            store_final(j + 1);
        }
        int cnt = 0;
        for (int c = j + 2 + ((me - (j + 2)) % G + G) % G; c < n; c += G, ++cnt)
            if (cnt % nwarp == warp) lu_apply_warp(l, p, col(c), j, n);
        __syncthreads();
    }
}

// Y <- (L_{n-2} P_{n-2} ... L_0 P_0) Y for every column y (row of
// Yt): at step j the swap of rows j and piv[j], then elimination with column j
// of the unit lower triangle of the column-major Lt, as stored at step j.
// CPB_ columns per CTA in shared memory, column j of L staged once per step and
// prefetched one step ahead, the pivot list staged in shared memory.
template <int CPB_, int PRE_>
__global__ void __launch_bounds__(256) k_fwdsolve_perm(const double* __restrict__ Lt, const int* __restrict__ piv,
                                                       double* Yt, int n, int ncols) {
    extern __shared__ double cs_smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c0 = blockIdx.x * CPB_;
    double* lbuf = cs_smem;
    double* y = cs_smem + n + (size_t)(warp < CPB_ ? warp : 0) * n;
    int* spiv = reinterpret_cast<int*>(cs_smem + (size_t)(CPB_ + 1) * n);
    const int c = c0 + warp;
    const bool has = warp < CPB_ && c < ncols;
    if (has)
        for (int i = lane; i < n; i += 32) y[i] = Yt[(size_t)c * n + i];
    for (int i = threadIdx.x; i < n; i += blockDim.x) spiv[i] = piv[i];
    double pre[PRE_];
    prefetch_vec<PRE_>(Lt, 1, n, pre);
    for (int j = 0; j < n - 1; ++j) {
        __syncthreads();
        store_vec<PRE_>(lbuf, j + 1, n, pre);
        __syncthreads();
        if (j + 1 < n - 1) prefetch_vec<PRE_>(Lt + (size_t)(j + 1) * n, j + 2, n, pre);
        if (has) {
            // step j of P A = L U: swap rows j and piv[j], then eliminate with column j of L
            double yj = 0.0;
            if (lane == 0) {
                const int p = spiv[j];
                yj = y[p];
                if (p != j) { y[p] = y[j]; y[j] = yj; }
            }
            yj = __shfl_sync(0xffffffffu, yj, 0);
            __syncwarp();
            for (int i = j + 1 + lane; i < n; i += 32) y[i] = fma(-lbuf[i], yj, y[i]);
            __syncwarp();
        }
    }
    __syncthreads();
    if (has)
        for (int i = lane; i < n; i += 32) Yt[(size_t)c * n + i] = y[i];
}

// Form columns of Q = H_0 ... H_{n-2} (Qt rows), each multiplied by sgn[c]:
// column c starts as e_c and takes H_j for j = min(c, n-2) down to 0.  Column c
// needs about 2 c n FMAs, so the columns of a CTA are taken cyclically
// (b, b + G, b + 2G, ...) to give every CTA the same mix of short and long ones,
// and with eight columns warps w and w + 4 (which share a sub-partition and its
// FP64 unit) take columns k = w and k = 7 - w of that list: a short one with a
// long one on every sub-partition.
template <int CPB_, int PRE_>
__global__ void __launch_bounds__(256) k_form_q(const double* __restrict__ Vt, const double* __restrict__ tau,
                                                const double* __restrict__ sgn, double* Qt, int n) {
    extern __shared__ double cs_smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double* vbuf = cs_smem;
    double* col = cs_smem + n + (size_t)(warp < CPB_ ? warp : 0) * n;
    const int kk = (CPB_ == 8 && warp >= 4) ? 11 - warp : warp;
    const int c = blockIdx.x + gridDim.x * kk;
    const bool has = warp < CPB_ && c < n;
    if (warp < CPB_)
        for (int i = lane; i < n; i += 32) col[i] = (i == c) ? 1.0 : 0.0;
    int cmax = blockIdx.x;
    for (int w = 1; w < CPB_; ++w)
        if ((int)blockIdx.x + (int)gridDim.x * w < n) cmax = blockIdx.x + gridDim.x * w;
    const int jtop = min(cmax, n - 2);
    double pre[PRE_];
    if (jtop >= 0) prefetch_vec<PRE_>(Vt + (size_t)jtop * n, jtop + 1, n, pre);
    for (int j = jtop; j >= 0; --j) {
        __syncthreads();
        store_vec<PRE_>(vbuf, j + 1, n, pre);
        if (threadIdx.x == 0) vbuf[j] = 1.0;
        __syncthreads();
        if (j > 0) prefetch_vec<PRE_>(Vt + (size_t)(j - 1) * n, j, n, pre);
        const double tj = __ldg(tau + j);
        if (has && j <= c && tj != 0.0) {
            const double w = dot4(vbuf, col, j, n) * tj;
            for (int i = j + lane; i < n; i += 32) col[i] = fma(-w, vbuf[i], col[i]);
        }
    }
    __syncthreads();
    if (has) {
        const double s = sgn[c];
        for (int i = lane; i < n; i += 32) Qt[(size_t)c * n + i] = col[i] * s;
    }
}

// Back substitution: for every column y (row of Yt), solve R x = y with R the
// upper triangle of the column-major Rt (R[i][c] = Rt[c][i]); writes
// x_i * (xs ? 1/xs[i] : 1) into Xt.
template <int CPB_, int PRE_>
__global__ void __launch_bounds__(256) k_backsolve(const double* __restrict__ Rt, const double* __restrict__ Yt,
                                                   double* Xt, int n, int ncols, const double* xs, DevStatus* st) {
    extern __shared__ double cs_smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c0 = blockIdx.x * CPB_;
    double* rbuf = cs_smem;                      // column i of R, rows 0..i
    double* x = cs_smem + n + (size_t)(warp < CPB_ ? warp : 0) * n;
    double* rinv = cs_smem + (size_t)(CPB_ + 1) * n;   // 1 / R_ii
    const int c = c0 + warp;
    const bool has = warp < CPB_ && c < ncols;
    for (int i = threadIdx.x; i < n; i += blockDim.x) rinv[i] = 1.0 / __ldg(Rt + (size_t)i * n + i);
    if (has)
        for (int i = lane; i < n; i += 32) x[i] = Yt[(size_t)c * n + i];
    double pre[PRE_];
    prefetch_vec<PRE_>(Rt + (size_t)(n - 1) * n, 0, n, pre);
    for (int i = n - 1; i >= 0; --i) {
        __syncthreads();
        store_vec<PRE_>(rbuf, 0, i + 1, pre);
        __syncthreads();
        if (i > 0) prefetch_vec<PRE_>(Rt + (size_t)(i - 1) * n, 0, i, pre);
        if (has) {
            const double xi = x[i] * rinv[i];
            __syncwarp();
            if (lane == 0) x[i] = xi;
            for (int r = lane; r < i; r += 32) x[r] = fma(-rbuf[r], xi, x[r]);
            __syncwarp();
        }
    }
    if (has) {
        bool bad = false;
        for (int i = lane; i < n; i += 32) {
            double v = x[i];
            if (xs) v /= xs[i];
            if (!isfinite(v)) bad = true;
            Xt[(size_t)c * n + i] = v;
        }
        if (__any_sync(0xffffffffu, bad) && lane == 0) flag_error(st, DERR_NUMERIC, 102);
    }
}

// Column norms w_c = D_c * ||A_c|| of a column-major A (At); one warp per column.
__global__ void k_colnorm_scaled(const double* __restrict__ At, const double* __restrict__ D, double* w, int n,
                                 DevStatus* st) {
    const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (c >= n) return;
    double s = 0.0;
    for (int i = lane; i < n; i += 32) { const double x = At[(size_t)c * n + i]; s = fma(x, x, s); }
    s = warp_sum(s);
    if (lane == 0) {
        double v = sqrt(s) * D[c];
        if (!isfinite(v)) { flag_error(st, DERR_NUMERIC, 105); v = 0.0; }   // keeps the ranks a permutation
        w[c] = v;
    }
}

// Pre-pivoting (Bai, Lee, Li & Xu 2011): permutation sorting columns by w,
// descending, ties by index.  perm[rank] = c.
__global__ void k_rank_perm(const double* __restrict__ w, int* perm, int n) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const double wc = w[c];
    int rank = 0;
    for (int d = 0; d < n; ++d) {
        const double wd = w[d];
        rank += (wd > wc) || (wd == wc && d < c);
    }
    perm[rank] = c;
}

// Row gather: out[k][:] = in[perm[k]][:], and Dp[k] = D[perm[k]].
__global__ void k_gather_rows(const double* __restrict__ in, double* out, const int* __restrict__ perm,
                              const double* __restrict__ D, double* Dp, int n) {
    const int k = blockIdx.x;
    int src = perm[k];
    if (src < 0 || src >= n) src = k;   // defensive: perm is always a permutation of [0, n)
    for (int i = threadIdx.x; i < n; i += blockDim.x) out[(size_t)k * n + i] = in[(size_t)src * n + i];
    if (threadIdx.x == 0 && D) Dp[k] = D[src];
}

// From the QR of A P (R in the column-major Rt) and the permuted scales Dp:
// Dnew_i = |R_ii| Dp_i, sgn_i = sign(R_ii), F = Dnew^-1 S R Dp (unit upper
// triangular, row-major), so that (A D) P = (Q S) Dnew F.
__global__ void k_make_F(const double* __restrict__ Rt, const double* __restrict__ Dp, double* F,
                         double* Dnew, double* sgn, int n, DevStatus* st) {
    const int i = blockIdx.x;
    const double rii = Rt[(size_t)i * n + i];
    const double s = rii < 0.0 ? -1.0 : 1.0;
    const double dn = fabs(rii) * Dp[i];
    if (threadIdx.x == 0) {
        Dnew[i] = dn;
        sgn[i] = s;
        if (!(dn > 0.0) || !isfinite(dn)) flag_error(st, DERR_NUMERIC, 103);
    }
    const double f = s / dn;
    for (int j = threadIdx.x; j < n; j += blockDim.x)
        F[(size_t)i * n + j] = (j < i) ? 0.0 : (j == i ? 1.0 : Rt[(size_t)j * n + i] * Dp[j] * f);
}

// M = Db_R^-1 P1 Db_L^-1 + Ds_R P2 Ds_L is built by two GEMMs; these helpers
// split D into Db = max(D,1), Ds = min(D,1).
__global__ void k_split_scales(const double* __restrict__ D, double* Db, double* Ds, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) { const double d = D[i]; Db[i] = fmax(d, 1.0); Ds[i] = fmin(d, 1.0); }
}

__global__ void k_set_identity(double* A, int n) {
    const size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o < (size_t)n * n) A[o] = (o / n == o % n) ? 1.0 : 0.0;
}

__global__ void k_fill(double* a, double v, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = v;
}

// Flags DERR_NUMERIC if any of the len values is NaN or infinite.
__global__ void k_check_finite(const double* __restrict__ A, size_t len, DevStatus* st, int where) {
    bool bad = false;
    for (size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x; o < len; o += (size_t)gridDim.x * blockDim.x)
        if (!isfinite(A[o])) bad = true;
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) flag_error(st, DERR_NUMERIC, where);
}

// max |A - B| (elementwise) and NaN detection -> out[0] (atomic max on the bit pattern of a non-negative double).
// A is the recomputed G, B the wrapped one: an element with |A - B| > limit max(1, |A|)
// flags DERR_NUMERIC (site 107): the chain no longer samples its weight.
__global__ void k_maxabsdiff(const double* __restrict__ A, const double* __restrict__ B, size_t len,
                             unsigned long long* out, DevStatus* st, double limit) {
    double m = 0.0;
    bool bad = false, over = false;
    for (size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x; o < len; o += (size_t)gridDim.x * blockDim.x) {
        const double a = A[o];
        const double d = fabs(a - B[o]);
        if (!isfinite(a)) bad = true;
        if (d > limit * fmax(1.0, fabs(a))) over = true;
        m = fmax(m, d);
    }
    m = warp_max(m);
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) flag_error(st, DERR_NUMERIC, 104);
    if (__any_sync(0xffffffffu, over) && (threadIdx.x & 31) == 0) flag_error(st, DERR_NUMERIC, 107);
}

}  // namespace afq
