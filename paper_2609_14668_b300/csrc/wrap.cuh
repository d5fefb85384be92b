// Momentum-space application of the kinetic propagator (Sec. III.A).
//
// e^{-c dtau K} = U^+ e^{-c dtau Lambda} U (Eq. NewBlMat) with U = diag(U_A, U_B)
// the per-sublattice 2D Fourier transform (Eqs. FourierMat, ColumnDem) and
// e^{-c dtau Lambda} one 2x2 block per k (Eq. ExpLambda).  The kernel applies it
// to every row of a real matrix, optionally scaling by the diagonal e^{+-gamma s}
// before and/or after (step (iv) of Sec. III.A), and writes the result either in
// place or transposed.  Two transposed passes make one wrap B G B^-1.
//
// B300 design: FP64 arithmetic is the bound (the measured DFMA rate is ~1/62 of
// FP32), so the kernel minimises FP64 work: two real rows are packed into one
// complex vector (the operator is real, E(a+ib) = Ea + iEb), each 1D DFT of
// length n = a*b is one Cooley-Tukey split into two short naive passes, and the
// whole pipeline for a row pair stays in shared memory (one HBM/L2 read and one
// write per element).
#pragma once
#include "common.cuh"

namespace afq {

struct FFTPlan {
    int N, Nc, L1, L2;
    int a1, b1, a2, b2;          // L1 = a1*b1, L2 = a2*b2 (a <= b)
    const double2* tw1;          // e^{-2 pi i m / L1}, m < L1
    const double2* tw2;          // e^{-2 pi i m / L2}, m < L2
};

// Diagonal scaling d_i = s_i > 0 ? vp : vm, or 1 when s == nullptr.
struct DiagScale {
    const int8_t* s;
    double vp, vm;
    __device__ __forceinline__ double at(int i) const { return s ? (s[i] > 0 ? vp : vm) : 1.0; }
};

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {   // a*b + c
    return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}

// One naive DFT pass along dimension `dim` for all VP vectors and both
// sublattices.  Output element at line position e (0..n-1) is
//   mode 0 (full):   Y[e] = sum_{j<n} X[j] w^{j e}
//   mode 1 (inner):  e = k1*b + j2:  Y[e] = w^{j2 k1} sum_{j1<a} X[j1*b + j2] w^{b j1 k1}
//   mode 2 (outer):  e = k1 + a*k2:  Y[e] = sum_{j2<b} X[k1*b + j2] w^{a j2 k2}
// with w = e^{-+2 pi i / n} (conj for the inverse).
__device__ void dft_pass(const double2* __restrict__ src, double2* __restrict__ dst, int VP,
                         const FFTPlan& P, int dim, int mode, bool inverse) {
    const int Nc = P.Nc, L1 = P.L1;
    const int n = dim == 1 ? P.L1 : P.L2;
    const int a = dim == 1 ? P.a1 : P.a2;
    const int b = dim == 1 ? P.b1 : P.b2;
    const double2* tw = dim == 1 ? P.tw1 : P.tw2;
    const double sg = inverse ? -1.0 : 1.0;
    const int total = VP * 2 * Nc;
    for (int o = threadIdx.x; o < total; o += blockDim.x) {
        const int v = o / (2 * Nc);
        const int rem = o - v * 2 * Nc;
        const int sub = rem / Nc;
        const int c = rem - sub * Nc;
        int e, base, stride;
        if (dim == 1) { e = c % L1; base = sub * Nc + (c - e); stride = 1; }
        else          { e = c / L1; base = sub * Nc + (c - e * L1); stride = L1; }
        const double2* x = src + (size_t)v * P.N + base;
        double2 acc = make_double2(0.0, 0.0);
        if (mode == 0) {
            for (int j = 0; j < n; ++j) {
                double2 w = tw[(j * e) % n]; w.y *= sg;
                acc = cfma(x[j * stride], w, acc);
            }
        } else if (mode == 1) {
            const int k1 = e / b, j2 = e - k1 * b;
            for (int j1 = 0; j1 < a; ++j1) {
                double2 w = tw[(b * j1 * k1) % n]; w.y *= sg;
                acc = cfma(x[(j1 * b + j2) * stride], w, acc);
            }
            double2 w = tw[(j2 * k1) % n]; w.y *= sg;
            acc = cmul(acc, w);
        } else {
            const int k1 = e % a, k2 = e / a;
            for (int j2 = 0; j2 < b; ++j2) {
                double2 w = tw[(a * j2 * k2) % n]; w.y *= sg;
                acc = cfma(x[(k1 * b + j2) * stride], w, acc);
            }
        }
        dst[(size_t)v * P.N + sub * Nc + c] = acc;
    }
}

// 2D DFT (both sublattices) from buffer `z` using `t` as scratch; returns the
// buffer holding the result.
__device__ double2* dft2d(double2* z, double2* t, int VP, const FFTPlan& P, bool inverse) {
    double2* cur = z;
    double2* oth = t;
    for (int dim = 1; dim <= 2; ++dim) {
        const int a = dim == 1 ? P.a1 : P.a2;
        if (a == 1) {
            dft_pass(cur, oth, VP, P, dim, 0, inverse);
            __syncthreads();
            double2* s = cur; cur = oth; oth = s;
        } else {
            dft_pass(cur, oth, VP, P, dim, 1, inverse);
            __syncthreads();
            dft_pass(oth, cur, VP, P, dim, 2, inverse);
            __syncthreads();
        }
    }
    return cur;
}

// out_row = post .* ( Op (pre .* in_row) ) for rows [0, nrows) of a row-major
// matrix with N columns; Op = U^+ blk U.  blk: Nc entries of 4 double2
// (row-major 2x2 block per k, index l1 + L1*l2).  transpose_out: write
// out[j*ldo + r] instead of out[r*ldo + j] (then in != out is required).
__global__ void __launch_bounds__(256) k_rowop(const double* in, double* out,
                                               int nrows, int ldi, int ldo, FFTPlan P,
                                               const double2* __restrict__ blk,
                                               DiagScale pre, DiagScale post, int transpose_out, int VP) {
    extern __shared__ double2 smem_rowop[];
    const int N = P.N, Nc = P.Nc;
    double2* z = smem_rowop;
    double2* t = smem_rowop + (size_t)VP * N;
    const int r0 = blockIdx.x * 2 * VP;
    // load: vector v = row (r0+2v) + i row (r0+2v+1)
    for (int o = threadIdx.x; o < VP * N; o += blockDim.x) {
        const int v = o / N, j = o - v * N;
        const int ra = r0 + 2 * v, rb = ra + 1;
        const double d = pre.at(j);
        const double xa = ra < nrows ? in[(size_t)ra * ldi + j] * d : 0.0;
        const double xb = rb < nrows ? in[(size_t)rb * ldi + j] * d : 0.0;
        z[o] = make_double2(xa, xb);
    }
    __syncthreads();
    double2* y = dft2d(z, t, VP, P, false);
    // 2x2 block per k (Eq. ExpLambda)
    for (int o = threadIdx.x; o < VP * Nc; o += blockDim.x) {
        const int v = o / Nc, k = o - v * Nc;
        double2* yv = y + (size_t)v * N;
        const double2 qa = yv[k], qb = yv[Nc + k];
        const double2 b00 = blk[4 * k], b01 = blk[4 * k + 1], b10 = blk[4 * k + 2], b11 = blk[4 * k + 3];
        yv[k] = cfma(b00, qa, cmul(b01, qb));
        yv[Nc + k] = cfma(b10, qa, cmul(b11, qb));
    }
    __syncthreads();
    double2* w = (y == z) ? t : z;
    double2* res = dft2d(y, w, VP, P, true);
    const double inv = 1.0 / (double)Nc;
    if (!transpose_out) {
        for (int o = threadIdx.x; o < VP * N; o += blockDim.x) {
            const int v = o / N, j = o - v * N;
            const int ra = r0 + 2 * v, rb = ra + 1;
            const double d = post.at(j) * inv;
            const double2 q = res[o];
            if (ra < nrows) out[(size_t)ra * ldo + j] = q.x * d;
            if (rb < nrows) out[(size_t)rb * ldo + j] = q.y * d;
        }
    } else {
        const int R = 2 * VP;
        for (int o = threadIdx.x; o < R * N; o += blockDim.x) {
            const int j = o / R, rho = o - j * R;
            const int r = r0 + rho;
            if (r < nrows) {
                const double2 q = res[(size_t)(rho >> 1) * N + j];
                out[(size_t)j * ldo + r] = ((rho & 1) ? q.y : q.x) * post.at(j) * inv;
            }
        }
    }
}

}  // namespace afq
