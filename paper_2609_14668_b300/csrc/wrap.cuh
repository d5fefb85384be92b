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
// length L is a mixed-radix Stockham FFT (radix 4, 2, 3 butterflies, a plain
// small DFT for other primes such as 7), and the whole pipeline for a row pair
// stays in shared memory (one L2/HBM read and one write per element).
#pragma once
#include "common.cuh"

namespace afq {

constexpr int FFT_MAX_STAGES = 8;

struct FFTPlan {
    int N, Nc, L1, L2;
    int nr1, nr2;                         // number of radix stages per dimension
    int r1[FFT_MAX_STAGES], r2[FFT_MAX_STAGES];   // radices, product = L1 (L2)
    const double2* tw1;                   // e^{-2 pi i m / L1}, m < L1
    const double2* tw2;                   // e^{-2 pi i m / L2}, m < L2
};

// Diagonal scaling d_i = s_i > 0 ? vp : vm, or 1 when s == nullptr.  With
// phase != 0 (charge-channel field, complex operator path only) the factor is
// the complex number (vp, ip) or (vm, im) that multiplies each complex vector
// element of the embedding rows (see k_rowop).
struct DiagScale {
    const int8_t* s;
    double vp, vm;
    double ip = 0.0, im = 0.0;
    int phase = 0;
    __device__ __forceinline__ double at(int i) const { return s ? (s[i] > 0 ? vp : vm) : 1.0; }
    __device__ __forceinline__ double2 cat(int i) const {
        return s ? (s[i] > 0 ? make_double2(vp, ip) : make_double2(vm, im)) : make_double2(1.0, 0.0);
    }
};

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {   // a*b + c
    return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
// multiply by -i (forward) or +i (inverse)
__device__ __forceinline__ double2 cmul_mi(double2 a, bool inverse) {
    return inverse ? make_double2(-a.y, a.x) : make_double2(a.y, -a.x);
}

// One radix-R stage of a Stockham autosort FFT (Govindaraju et al., SC 2008)
// along dimension `dim` for all VP vectors and both sublattices: butterfly j
// (0 <= j < n/R) of a line reads R elements n/R apart, applies the twiddles
// w^{r (j mod Ns) n/(Ns R)}, does an R-point DFT and writes them Ns apart from
// (j / Ns) Ns R + j mod Ns.  w = e^{-2 pi i / n} (conjugate for the inverse).
__device__ void fft_stage(const double2* __restrict__ src, double2* __restrict__ dst, int VP, const FFTPlan& P,
                          int dim, int R, int Ns, bool inverse) {
    const int Nc = P.Nc, L1 = P.L1;
    const int n = dim == 1 ? P.L1 : P.L2;
    const double2* tw = dim == 1 ? P.tw1 : P.tw2;
    const double sg = inverse ? -1.0 : 1.0;
    const int nb = n / R;                        // butterflies per line
    const int lines = Nc / n;                    // lines per sublattice
    const int total = VP * 2 * lines * nb;
    const int tstep = n / (Ns * R);
    for (int o = threadIdx.x; o < total; o += blockDim.x) {
        const int j = o % nb;
        const int rem = o / nb;
        const int line = rem % lines;
        const int vs = rem / lines;              // v * 2 + sub
        const int v = vs >> 1, sub = vs & 1;
        int base, stride;
        if (dim == 1) { base = sub * Nc + line * L1; stride = 1; }
        else          { base = sub * Nc + line;      stride = L1; }
        const double2* x = src + (size_t)v * P.N + base;
        double2* y = dst + (size_t)v * P.N + base;
        const int jm = j % Ns;
        const int od = (j / Ns) * Ns * R + jm;
        double2 a[8];
        for (int r = 0; r < R; ++r) {
            double2 e = x[(j + r * nb) * stride];
            if (r > 0 && jm > 0) {
                double2 w = tw[(r * jm * tstep) % n];
                w.y *= sg;
                e = cmul(e, w);
            }
            a[r] = e;
        }
        if (R == 2) {
            y[od * stride] = cadd(a[0], a[1]);
            y[(od + Ns) * stride] = csub(a[0], a[1]);
        } else if (R == 4) {
            const double2 s02 = cadd(a[0], a[2]), d02 = csub(a[0], a[2]);
            const double2 s13 = cadd(a[1], a[3]), d13 = cmul_mi(csub(a[1], a[3]), inverse);
            y[od * stride] = cadd(s02, s13);
            y[(od + Ns) * stride] = cadd(d02, d13);
            y[(od + 2 * Ns) * stride] = csub(s02, s13);
            y[(od + 3 * Ns) * stride] = csub(d02, d13);
        } else if (R == 3) {
            const double c3 = 0.86602540378443864676;       // sqrt(3)/2
            const double2 t1 = cadd(a[1], a[2]), t2 = csub(a[1], a[2]);
            const double2 m = make_double2(fma(-0.5, t1.x, a[0].x), fma(-0.5, t1.y, a[0].y));
            const double2 it = cmul_mi(t2, inverse);        // -+ i t2
            y[od * stride] = cadd(a[0], t1);
            y[(od + Ns) * stride] = make_double2(fma(c3, it.x, m.x), fma(c3, it.y, m.y));
            y[(od + 2 * Ns) * stride] = make_double2(fma(-c3, it.x, m.x), fma(-c3, it.y, m.y));
        } else {
            // generic small radix: R-point DFT with roots from the same table
            for (int q = 0; q < R; ++q) {
                double2 acc = a[0];
                for (int r = 1; r < R; ++r) {
                    double2 w = tw[((q * r) % R) * nb];
                    w.y *= sg;
                    acc = cfma(a[r], w, acc);
                }
                y[(od + q * Ns) * stride] = acc;
            }
        }
    }
}

// 2D DFT (both sublattices) from buffer `z` using `t` as scratch; returns the
// buffer holding the result.
__device__ double2* dft2d(double2* z, double2* t, int VP, const FFTPlan& P, bool inverse) {
    double2* cur = z;
    double2* oth = t;
    for (int dim = 1; dim <= 2; ++dim) {
        const int ns = dim == 1 ? P.nr1 : P.nr2;
        const int* rr = dim == 1 ? P.r1 : P.r2;
        int Ns = 1;
        for (int st = 0; st < ns; ++st) {
            fft_stage(cur, oth, VP, P, dim, rr[st], Ns, inverse);
            __syncthreads();
            Ns *= rr[st];
            double2* sw = cur; cur = oth; oth = sw;
        }
    }
    return cur;
}

// out_row = post .* ( Op (pre .* in_row) ) for rows [0, nrows) of a row-major
// matrix with N columns; Op = U^+ blk U.  blk: Nc entries of 4 double2
// (row-major 2x2 block per k, index l1 + L1*l2).  transpose_out: write
// out[j*ldo + r] instead of out[r*ldo + j] (then in != out is required).
//
// emb != 0 (twisted boundaries, complex operator): the matrix is the real
// 2N x 2N embedding [[Re X, -Im X], [Im X, Re X]] of a complex X, and each row
// of length 2N is one complex vector z = row[0:N] + i row[N:2N]; the kernel
// writes [Re Op z, Im Op z].  For a column of the embedding this is the
// embedding of Op applied to the complex column; for a row it is the row
// times the embedding of Op, because every Op used here (e^{+-c dtau K}) is
// Hermitian.  The diagonal scalings act on both halves; a complex scaling
// (DiagScale::phase) multiplies z itself, so for a row z = conj(row) a factor
// c applies conj(c) to the row, and for a column it applies c.
__global__ void __launch_bounds__(256) k_rowop(const double* in, double* out,
                                               int nrows, int ldi, int ldo, FFTPlan P,
                                               const double2* __restrict__ blk,
                                               DiagScale pre, DiagScale post, int transpose_out, int VP, int emb) {
    extern __shared__ double2 smem_rowop[];
    const int N = P.N, Nc = P.Nc;
    double2* z = smem_rowop;
    double2* t = smem_rowop + (size_t)VP * N;
    const int r0 = blockIdx.x * (emb ? VP : 2 * VP);
    // load: vector v = row (r0+2v) + i row (r0+2v+1), or (emb) the two halves of row r0+v
    for (int o = threadIdx.x; o < VP * N; o += blockDim.x) {
        const int v = o / N, j = o - v * N;
        const double d = pre.at(j);
        if (emb) {
            const int r = r0 + v;
            const double* row = in + (size_t)r * ldi;
            if (r >= nrows) { z[o] = make_double2(0.0, 0.0); continue; }
            z[o] = pre.phase ? cmul(make_double2(row[j], row[N + j]), pre.cat(j))
                             : make_double2(row[j] * d, row[N + j] * d);
            continue;
        }
        const int ra = r0 + 2 * v, rb = ra + 1;
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
    if (emb) {
        if (!transpose_out) {
            for (int o = threadIdx.x; o < VP * N; o += blockDim.x) {
                const int v = o / N, j = o - v * N;
                const int r = r0 + v;
                if (r >= nrows) continue;
                if (post.phase) {
                    const double2 q = cmul(res[o], post.cat(j));
                    out[(size_t)r * ldo + j] = q.x * inv;
                    out[(size_t)r * ldo + N + j] = q.y * inv;
                    continue;
                }
                const double d = post.at(j) * inv;
                const double2 q = res[o];
                out[(size_t)r * ldo + j] = q.x * d;
                out[(size_t)r * ldo + N + j] = q.y * d;
            }
        } else {
            for (int o = threadIdx.x; o < VP * 2 * N; o += blockDim.x) {
                const int j2 = o / VP, v = o - j2 * VP;
                const int r = r0 + v;
                if (r >= nrows) continue;
                const int j = j2 < N ? j2 : j2 - N;
                const double2 q = res[(size_t)v * N + j];
                if (post.phase) {
                    const double2 qc = cmul(q, post.cat(j));
                    out[(size_t)j2 * ldo + r] = (j2 < N ? qc.x : qc.y) * inv;
                    continue;
                }
                out[(size_t)j2 * ldo + r] = (j2 < N ? q.x : q.y) * post.at(j) * inv;
            }
        }
        return;
    }
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
