// Time-displaced Green's functions and the interaction autocorrelation
// C_{H_I}(tau) (Eqs. DouOccDerive, fidelitysusp).
//
// For one field, at tau = l dtau with B(tau, 0) = U_R D_R T_R and
// B(beta, tau)^T = U_L D_L T_L (the QR-stabilised stacks), the three up-spin
// Green's functions share the middle matrix M of G = (1 + R L)^-1:
//   G(tau, tau) = U_L Db_L^-1 M^-1 Db_R^-1 U_R^T,
//   G(tau, 0)   = U_L Db_L^-1 M^-1 Ds_R T_R,
//   G(0, tau)   = -T_L^T Ds_L M^-1 Db_R^-1 U_R^T,
// M = Db_R^-1 U_R^T U_L Db_L^-1 + Ds_R T_R T_L^T Ds_L (one LU, three right or
// left factors).  Between stabilisations they are propagated:
// G(tau + dtau, 0) = B G(tau, 0), G(0, tau + dtau) = G(0, tau) B^-1 and the wrap.
//
// Wick, one field, spin up from G, spin down from the particle-hole relations
// (G_dn is built from the complex conjugate of G_up): with g = the symmetric
// split (e^{-dtau K/2} X e^{+dtau K/2}) of each Green's function,
//   a_up = 1 - g(t,t)_ii, a_dn = conj g(t,t)_ii, b_up = 1 - g(0,0)_jj, b_dn = conj g(0,0)_jj,
//   P = g(0,t)_ji g(t,0)_ij, X_up = a_up b_up - P, X_dn = a_dn b_dn - conj P,
//   <A_i(t) A_j(0)> = X_up X_dn - (X_up a_dn + a_up X_dn)/2 - (X_up b_dn + b_up X_dn)/2
//                     + (X_up + X_dn + a_up b_dn + a_dn b_up)/4,
// A = n_up n_dn - (n_up + n_dn)/2; the estimator is Re sum_ij <A_i(t) A_j(0)>.
#pragma once
#include "common.cuh"
#include "measure.cuh"
#include "wrap.cuh"

namespace afq {

// out[r][c] = in[r][c] * d[c]  (n x n)
__global__ void k_scale_cols(const double* __restrict__ in, double* out, int n, const double* __restrict__ d) {
    const size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o < (size_t)n * n) out[o] = in[o] * d[o % n];
}

// A -= I  (n x n)
__global__ void k_sub_identity(double* A, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) A[(size_t)i * n + i] -= 1.0;
}

__global__ void k_td_diag(GView gtt, GView g00, double2* dtt, double2* d00) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= gtt.N) return;
    dtt[i] = gtt.at(i, i);
    d00[i] = g00.at(i, i);
}

__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }

// One 32 x 32 tile (I, J) per CTA: g(t,0) tile (I, J) and g(0,t) tile (J, I)
// through shared memory; out[tile] = Re sum over the tile of <A_i(t) A_j(0)>.
__global__ void k_td_tiles(GView gt0, GView g0t, const double2* __restrict__ dtt, const double2* __restrict__ d00,
                           double* out) {
    __shared__ double2 a[32][33], b[32][33];
    __shared__ double red[33];
    const int N = gt0.N;
    const int nt = (N + 31) / 32;
    const int I = blockIdx.x / nt, J = blockIdx.x % nt;
    for (int o = threadIdx.x; o < 32 * 32; o += blockDim.x) {
        const int r = o / 32, c = o % 32;
        const int i = I * 32 + r, j = J * 32 + c;
        const int i2 = J * 32 + r, j2 = I * 32 + c;
        a[r][c] = (i < N && j < N) ? gt0.at(i, j) : make_double2(0.0, 0.0);
        b[r][c] = (i2 < N && j2 < N) ? g0t.at(i2, j2) : make_double2(0.0, 0.0);
    }
    __syncthreads();
    double acc = 0.0;
    for (int o = threadIdx.x; o < 32 * 32; o += blockDim.x) {
        const int r = o / 32, c = o % 32;
        const int i = I * 32 + r, j = J * 32 + c;
        if (i >= N || j >= N) continue;
        const double2 P = cmul(b[c][r], a[r][c]);          // g(0,t)_ji g(t,0)_ij
        const double2 gt = dtt[i], g0 = d00[j];
        const double2 au = make_double2(1.0 - gt.x, -gt.y), ad = cconj(gt);
        const double2 bu = make_double2(1.0 - g0.x, -g0.y), bd = cconj(g0);
        const double2 Xu = csub(cmul(au, bu), P);
        const double2 Xd = csub(cmul(ad, bd), cconj(P));
        double2 ab = cmul(Xu, Xd);
        ab = csub(ab, cscale(cadd(cmul(Xu, ad), cmul(au, Xd)), 0.5));
        ab = csub(ab, cscale(cadd(cmul(Xu, bd), cmul(bu, Xd)), 0.5));
        ab = cadd(ab, cscale(cadd(cadd(Xu, Xd), cadd(cmul(au, bd), cmul(ad, bu))), 0.25));
        acc += ab.x;
    }
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) out[blockIdx.x] = acc;
}

// hh[slot] += sum of the tile partials; with_h: h += Re sum_i [b_up b_dn - (b_up + b_dn)/2]
// (the equal-time <H_I> of the field).  One CTA, fixed summation order.
__global__ void k_td_reduce(const double* __restrict__ part, int nparts, const double2* __restrict__ d00, int N,
                            double* hh, int slot, double* h, int with_h, DevStatus* st) {
    __shared__ double red[33];
    double s = 0.0, e = 0.0;
    for (int q = threadIdx.x; q < nparts; q += blockDim.x) s += part[q];
    if (with_h)
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
            const double2 g0 = d00[i];
            const double2 bu = make_double2(1.0 - g0.x, -g0.y), bd = cconj(g0);
            e += cmul(bu, bd).x - 0.5 * (bu.x + bd.x);
        }
    s = block_sum(s, red);
    e = block_sum(e, red);
    if (threadIdx.x == 0) {
        if (!isfinite(s) || !isfinite(e)) flag_error(st, DERR_NUMERIC, 500);
        hh[slot] += s;
        if (with_h) *h += e;
    }
}

}  // namespace afq
