// Equal-time observables by Wick contraction (Sec. II.C; App. C) on the
// symmetric-split Green's function g = e^{-dtau K/2} G e^{+dtau K/2} of the spin
// up channel.  With the partial particle-hole transform,
// G_dn_ij = (-1)^{i+j} (delta_ij - conj(g_ji)), which gives
//   n_i_up = 1 - g_ii,  n_i_dn = conj(g_ii),  Re <n_i_up n_i_dn> = Re g_ii - |g_ii|^2,
//   <s_i s_j> = 1/4 [ m_i m_j + 2 Re(g_ij (delta_ij - g_ji)) ]  (i, j on one sublattice),
//   m_i = 1 - 2 Re g_ii,
//   <H0> = 2t sum_bonds [ Re(e^{i Phi} g_BA) + Re(e^{-i Phi} g_AB) ]
// for the bond A -> B with hopping -t e^{i Phi} (Phi = 0 without a twist, where
// all of this reduces to the real formulas).  A twisted G arrives as its real
// 2N x 2N embedding: Re g is the top-left block, Im g the bottom-left block.
#pragma once
#include "common.cuh"

namespace afq {

constexpr int OBS_SCALARS = 10;  // energy, D, ekin, density, m2, S_af, S_af_dk, R_m2, Czz_half, chi_e

// Read access to g (N x N physical sites): real, or the embedding of a complex g.
struct GView {
    const double* g;
    int N;          // physical sites
    int ld;         // row stride: N, or 2N for the embedding
    int cplx;
    __device__ __forceinline__ double2 at(int i, int j) const {
        return make_double2(g[(size_t)i * ld + j], cplx ? g[(size_t)(N + i) * ld + j] : 0.0);
    }
};

// One CTA per Bravais displacement d = d1 + L1*d2:
//   czz[d]  = (1 / 2Nc) sum_{sub, I} <s_{sub,I} s_{sub,I+d}>
//   h[2(4d + 2a + b)] (re, im) = sum_J <a^+_{J+d} b_J>  with <c_i^+ c_j> = delta_ij - g_ji
__global__ void k_measure_pairs(GView g, int L1, int L2, double* czz, double* h) {
    __shared__ double red[33];
    const int Nc = L1 * L2;
    const int d = blockIdx.x;
    const int d1 = d % L1, d2 = d / L1;
    double acc_s = 0.0, hre[4] = {0.0, 0.0, 0.0, 0.0}, him[4] = {0.0, 0.0, 0.0, 0.0};
    for (int I = threadIdx.x; I < Nc; I += blockDim.x) {
        const int n1 = I % L1, n2 = I / L1;
        const int J = ((n1 + d1) % L1) + L1 * ((n2 + d2) % L2);     // I + d
        for (int sub = 0; sub < 2; ++sub) {
            const int i = sub * Nc + I, j = sub * Nc + J;
            const double2 gii = g.at(i, i), gjj = g.at(j, j), gij = g.at(i, j), gji = g.at(j, i);
            const double ex = (i == j ? 1.0 : 0.0) - gji.x;
            // Re(g_ij (delta_ij - g_ji))
            const double x = fma(gij.x, ex, gij.y * gji.y);
            acc_s += 0.25 * ((1.0 - 2.0 * gii.x) * (1.0 - 2.0 * gjj.x) + 2.0 * x);
        }
        // <a^+_{K+d} b_K> summed over K: here K = I, K+d = J
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                const int ia = a * Nc + J, jb = b * Nc + I;
                const double2 v = g.at(jb, ia);
                hre[2 * a + b] += (ia == jb ? 1.0 : 0.0) - v.x;
                him[2 * a + b] -= v.y;
            }
    }
    acc_s = block_sum(acc_s, red);
    if (threadIdx.x == 0) czz[d] = acc_s / (2.0 * Nc);
    for (int q = 0; q < 4; ++q) {
        const double vr = block_sum(hre[q], red);
        const double vi = block_sum(him[q], red);
        if (threadIdx.x == 0) { h[2 * (4 * d + q)] = vr; h[2 * (4 * d + q) + 1] = vi; }
    }
}

// n_ab(k) = Nc^-1 sum_d e^{i q.d} h_ab(d) (Eq. nkMatrix); one thread per q of the
// cell-DFT grid (with a twist: the momentum q + A).  tw1[m] = e^{-2 pi i m/L1},
// tw2[m] = e^{-2 pi i m/L2}.  nk: interleaved complex, index (k*4 + 2a + b).
// acc != 0 adds into nk.
__global__ void k_measure_nk(const double* __restrict__ h, int L1, int L2, const double2* __restrict__ tw1,
                             const double2* __restrict__ tw2, double* nk, int acc) {
    const int Nc = L1 * L2;
    const int kq = blockIdx.x * blockDim.x + threadIdx.x;
    if (kq >= Nc) return;
    const int l1 = kq % L1, l2 = kq / L1;
    double re[4] = {0, 0, 0, 0}, im[4] = {0, 0, 0, 0};
    for (int d = 0; d < Nc; ++d) {
        const int d1 = d % L1, d2 = d / L1;
        const double2 w1 = tw1[(l1 * d1) % L1], w2 = tw2[(l2 * d2) % L2];
        // e^{+i k.d} = conj(w1 w2)
        const double cr = w1.x * w2.x - w1.y * w2.y;
        const double ci = -(w1.x * w2.y + w1.y * w2.x);
        for (int q = 0; q < 4; ++q) {
            const double vr = h[2 * (4 * d + q)], vi = h[2 * (4 * d + q) + 1];
            re[q] = fma(cr, vr, fma(-ci, vi, re[q]));
            im[q] = fma(ci, vr, fma(cr, vi, im[q]));
        }
    }
    for (int q = 0; q < 4; ++q) {
        double* o = nk + 2 * (4 * kq + q);
        if (acc) { o[0] += re[q] / Nc; o[1] += im[q] / Nc; }
        else     { o[0] = re[q] / Nc; o[1] = im[q] / Nc; }
    }
}

// Scalars (one CTA).  out[0..8] = energy, D, ekin, density, m2, S_af, S_af_dk,
// R_m2, Czz_half; czz_acc (optional) accumulates czz; acc != 0 adds into out;
// count (optional) is incremented.
// Re tr(g^2) = Re sum_ij g_ij g_ji, one 32 x 32 tile pair per CTA: tile (I, J)
// and tile (J, I) are read coalesced through shared memory; out[tile] is the
// tile's partial sum (summed in fixed order by k_measure_scalars).
__global__ void k_measure_tr2(GView g, double* out) {
    __shared__ double a_re[32][33], a_im[32][33], b_re[32][33], b_im[32][33];
    __shared__ double red[33];
    const int nt = (g.N + 31) / 32;
    const int I = blockIdx.x / nt, J = blockIdx.x % nt;
    for (int o = threadIdx.x; o < 32 * 32; o += blockDim.x) {
        const int r = o / 32, c = o % 32;
        const int i = I * 32 + r, j = J * 32 + c;
        const int i2 = J * 32 + r, j2 = I * 32 + c;
        double2 v = make_double2(0.0, 0.0), w = make_double2(0.0, 0.0);
        if (i < g.N && j < g.N) v = g.at(i, j);
        if (i2 < g.N && j2 < g.N) w = g.at(i2, j2);
        a_re[r][c] = v.x; a_im[r][c] = v.y;
        b_re[r][c] = w.x; b_im[r][c] = w.y;
    }
    __syncthreads();
    double acc = 0.0;
    for (int o = threadIdx.x; o < 32 * 32; o += blockDim.x) {
        const int r = o / 32, c = o % 32;
        // g_ij g_ji with i = I*32 + r, j = J*32 + c; g_ji sits at b[c][r]
        acc += a_re[r][c] * b_re[c][r] - a_im[r][c] * b_im[c][r];
    }
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) out[blockIdx.x] = acc;
}

// Bond phases e^{i Phi_e} of the three bonds A(r) -> B(r + delta_e) (Gauge-I, Sec. III.C).
struct BondPhases { double2 e[3]; };

__global__ void k_measure_scalars(GView g, const double* __restrict__ czz, const double* __restrict__ tr2, int ntr2,
                                  int L1, int L2, double t, double U, double beta, const double2* __restrict__ tw1,
                                  BondPhases ph, double* out, double* czz_acc, int acc, long long* count,
                                  DevStatus* st) {
    __shared__ double red[33];
    const int Nc = L1 * L2, N = 2 * Nc;
    double dsum = 0.0, dens = 0.0, kin = 0.0, s0 = 0.0, sdk = 0.0, trr = 0.0, tri = 0.0, t2 = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const double2 gii = g.at(i, i);
        dsum += gii.x - fma(gii.x, gii.x, gii.y * gii.y);     // Re((1 - g) conj(g))
        dens += (1.0 - gii.x) + gii.x;
        trr += gii.x;
        tri += gii.y;
    }
    for (int q = threadIdx.x; q < ntr2; q += blockDim.x) t2 += tr2[q];
    // bonds A(n1,n2) - B(n1+d1, n2+d2), d in {(0,0), (1,-1), (0,-1)} (Gauge-I, Sec. III.C)
    for (int I = threadIdx.x; I < Nc; I += blockDim.x) {
        const int n1 = I % L1, n2 = I / L1;
        const int dd1[3] = {0, 1, 0}, dd2[3] = {0, -1, -1};
        for (int e = 0; e < 3; ++e) {
            const int J = ((n1 + dd1[e] + L1) % L1) + L1 * ((n2 + dd2[e] + L2) % L2);
            const int i = I, j = Nc + J;
            const double2 gij = g.at(i, j), gji = g.at(j, i), w = ph.e[e];
            // Re(e^{i Phi} g_ji) + Re(e^{-i Phi} g_ij)
            kin += 2.0 * t * (fma(w.x, gji.x, -w.y * gji.y) + fma(w.x, gij.x, w.y * gij.y));
        }
    }
    for (int d = threadIdx.x; d < Nc; d += blockDim.x) {
        const double c = czz[d];
        const double2 w = tw1[d % L1];     // e^{-2 pi i d1 / L1}; S is real so Re e^{+i...} = w.x
        s0 += c;
        sdk += c * w.x;
        if (czz_acc) czz_acc[d] += c;
    }
    dsum = block_sum(dsum, red);
    dens = block_sum(dens, red);
    trr = block_sum(trr, red);
    tri = block_sum(tri, red);
    t2 = block_sum(t2, red);
    kin = block_sum(kin, red);
    s0 = block_sum(s0, red);
    sdk = block_sum(sdk, red);
    if (threadIdx.x == 0) {
        const double D = dsum / N;
        double v[OBS_SCALARS];
        v[0] = (kin + N * U * D) / N;
        v[1] = D;
        v[2] = kin / N;
        v[3] = dens / N;
        v[4] = s0 / (2.0 * Nc);
        v[5] = s0;
        v[6] = sdk;
        v[7] = 1.0 - sdk / s0;
        v[8] = czz[(L1 / 2)];
        // Eq. ChiCharge: sum_ij <n_i n_j> - N^2 = 2 Re(tr g - tr g^2) - 4 (Im tr g)^2 for one field
        v[9] = beta / N * (2.0 * (trr - t2) - 4.0 * tri * tri);
        bool bad = false;
        for (int q = 0; q < OBS_SCALARS; ++q) {
            if (!isfinite(v[q]) && q != 7) bad = true;
            out[q] = acc ? out[q] + v[q] : v[q];
        }
        if (bad) flag_error(st, DERR_NUMERIC, 300);
        if (count) *count += 1;
    }
}

// Weight ratio of flipping site i given G (test hook): out = {R, Re r, Im r},
// R = e^{2 gamma s} |r|^2 (spin channel) or |r|^2 (charge channel, ef = 1),
// r = 1 + Delta (1 - G_ii) with Delta = dl + i dli.
__global__ void k_ratio(GView G, int i, int s, double dl_p, double dl_m, double dli_p, double dli_m, double ef_p,
                        double ef_m, double* out) {
    const double2 g = G.at(i, i);
    const double dl = s > 0 ? dl_p : dl_m, di = s > 0 ? dli_p : dli_m, ef = s > 0 ? ef_p : ef_m;
    const double rr = fma(di, g.y, fma(dl, 1.0 - g.x, 1.0)), ri = fma(di, 1.0 - g.x, -dl * g.y);
    out[0] = ef * fma(rr, rr, ri * ri);
    out[1] = rr;
    out[2] = ri;
}

// Real 2N x 2N embedding E = [[Re X, -Im X], [Im X, Re X]] of a complex N x N
// matrix X (interleaved re, im, row-major), and back (top-left and
// bottom-left blocks).  One thread per element of X.
__global__ void k_embed(const double2* __restrict__ X, double* E, int N) {
    const size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= (size_t)N * N) return;
    const int i = (int)(o / N), j = (int)(o % N);
    const double2 v = X[o];
    const size_t ld = 2 * (size_t)N;
    E[i * ld + j] = v.x;
    E[i * ld + N + j] = -v.y;
    E[(N + i) * ld + j] = v.y;
    E[(N + i) * ld + N + j] = v.x;
}
__global__ void k_extract(const double* __restrict__ E, double2* X, int N) {
    const size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= (size_t)N * N) return;
    const int i = (int)(o / N), j = (int)(o % N);
    const size_t ld = 2 * (size_t)N;
    X[o] = make_double2(E[i * ld + j], E[(N + i) * ld + j]);
}

// *p += v (a device-resident counter advanced inside the launch sequence)
__global__ void k_add_u64(unsigned long long* p, unsigned long long v) { *p += v; }

// Initial field from the counter-based stream: s = +1 iff u(key, 2^62 + l*N + i + 1) < 1/2.
__global__ void k_init_field(int8_t* s, int M, int N, uint64_t key) {
    const size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o < (size_t)M * N) s[o] = sm64_uniform(key, (1ull << 62) + o + 1) < 0.5 ? 1 : -1;
}

}  // namespace afq
