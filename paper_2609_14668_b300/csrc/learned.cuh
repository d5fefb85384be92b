// Learned block proposals (not in the paper): a small MLP proposes new values
// for a block of the Ising field from the field around it; every proposal is
// accepted by Metropolis-Hastings with the exact weight ratio, computed by
// the slice kernel in forced mode (update.cuh).
//
// Geometry (shared with the oracle): block = b x b unit cells, both
// sublattices, slices l0 .. l0+T-1 (1-based); context = cells
// [o1-h, o1+b+h) x [o2-h, o2+b+h) (periodic), slices [l0-ht, l0+T+ht)
// (periodic in imaginary time), block entries set to 0.  Context index
// ((t * W + w2) * W + w1) * 2 + sub, W = b + 2h; block index
// ((t * b + c2) * b + c1) * 2 + sub.
//
// Network: z = W2 tanh(W1 x + b1) + b2 (FP32), parameters contiguous as
// [W1 (H x Din) | b1 (H) | W2 (Dout x H) | b2 (Dout)]; proposal
// q(s'|x) = prod_i sigmoid(s'_i z_i); training loss: mean over the batch of
// -sum_i log sigmoid(s_i z_i).  The sizes are small (Din <= a few thousand,
// H <= 256, batch <= 1024), so the kernels are plain FP32 SIMT loops.
#pragma once
#include "common.cuh"

namespace afq {

struct BlockGeom {
    int L1, L2, Nc, Np, M;     // lattice of the chain / configurations
    int b, T, h, ht, W;        // block and context shape, W = b + 2h
    int d_in, d_out, d_hid;
};

__device__ __forceinline__ int pmod(int x, int n) { return ((x % n) + n) % n; }

// x (and the block's values s, if S != nullptr) of block instance n:
// pos[4n .. 4n+3] = (configuration, l0, o1, o2), or, with pos == nullptr, the
// single block (0, l0s, o1s, o2s); one CTA per instance.
__global__ void k_block_inputs(const int8_t* __restrict__ fields, size_t cfg_stride, const int* __restrict__ pos,
                               BlockGeom g, float* X, float* S, int l0s = 1, int o1s = 0, int o2s = 0) {
    const int n = blockIdx.x;
    const int cfg = pos ? pos[4 * n] : 0;
    const int l0 = pos ? pos[4 * n + 1] : l0s, o1 = pos ? pos[4 * n + 2] : o1s, o2 = pos ? pos[4 * n + 3] : o2s;
    const int8_t* f = fields + (size_t)cfg * cfg_stride;
    for (int idx = threadIdx.x; idx < g.d_in; idx += blockDim.x) {
        const int sub = idx & 1;
        int rest = idx >> 1;
        const int w1 = rest % g.W;
        rest /= g.W;
        const int w2 = rest % g.W;
        const int t = rest / g.W;
        const int c1 = w1 - g.h, c2 = w2 - g.h;
        const bool inside = t >= g.ht && t < g.ht + g.T && c1 >= 0 && c1 < g.b && c2 >= 0 && c2 < g.b;
        const int l = pmod(l0 - 1 - g.ht + t, g.M);
        const int cell = pmod(o1 + c1, g.L1) + g.L1 * pmod(o2 + c2, g.L2);
        X[(size_t)n * g.d_in + idx] = inside ? 0.0f : (float)f[(size_t)l * g.Np + sub * g.Nc + cell];
    }
    if (S)
        for (int idx = threadIdx.x; idx < g.d_out; idx += blockDim.x) {
            const int sub = idx & 1;
            int rest = idx >> 1;
            const int c1 = rest % g.b;
            rest /= g.b;
            const int c2 = rest % g.b;
            const int t = rest / g.b;
            const int cell = pmod(o1 + c1, g.L1) + g.L1 * pmod(o2 + c2, g.L2);
            S[(size_t)n * g.d_out + idx] = (float)f[(size_t)(l0 - 1 + t) * g.Np + sub * g.Nc + cell];
        }
}

// hidden layer: Hd[n][j] = tanh(b1[j] + sum_i W1[j][i] X[n][i]); one thread per (n, j)
__global__ void k_mlp_hidden(const float* __restrict__ P, const float* __restrict__ X, int B, int din, int dh,
                             float* Hd) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= B * dh) return;
    const int n = o / dh, j = o - n * dh;
    const float* w = P + (size_t)j * din;
    const float* x = X + (size_t)n * din;
    float acc = P[(size_t)dh * din + j];
    for (int i = 0; i < din; ++i) acc = fmaf(w[i], x[i], acc);
    Hd[o] = tanhf(acc);
}

// output layer: Z[n][k] = b2[k] + sum_j W2[k][j] Hd[n][j]
__global__ void k_mlp_out(const float* __restrict__ P, const float* __restrict__ Hd, int B, int din, int dh,
                          int dout, float* Z) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= B * dout) return;
    const int n = o / dout, k = o - n * dout;
    const float* W2 = P + (size_t)dh * din + dh;
    const float* w = W2 + (size_t)k * dh;
    const float* hn = Hd + (size_t)n * dh;
    float acc = W2[(size_t)dout * dh + k];
    for (int j = 0; j < dh; ++j) acc = fmaf(w[j], hn[j], acc);
    Z[o] = acc;
}

__device__ __forceinline__ double log_sigmoid(double x) { return x >= 0.0 ? -log1p(exp(-x)) : x - log1p(exp(x)); }

// dZ = d(loss)/dZ = -s sigmoid(-s z) / B; loss += -sum log sigmoid(s z) / B
__global__ void k_mlp_dz(const float* __restrict__ Z, const float* __restrict__ S, int B, int dout, float* dZ,
                         double* loss) {
    __shared__ double red[33];
    double l = 0.0;
    for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < B * dout; o += gridDim.x * blockDim.x) {
        const double s = S[o], z = Z[o];
        const double sz = s * z;
        const double sig_m = sz >= 0.0 ? exp(-sz) / (1.0 + exp(-sz)) : 1.0 / (1.0 + exp(sz));   // sigmoid(-s z)
        dZ[o] = (float)(-s * sig_m / B);
        l -= log_sigmoid(sz);
    }
    l = block_sum(l, red);
    if (threadIdx.x == 0) atomicAdd(loss, l / B);
}

// gradients of the output layer: G_W2[k][j] = sum_n dZ[n][k] Hd[n][j], G_b2[k] = sum_n dZ[n][k]
__global__ void k_mlp_grad_out(const float* __restrict__ dZ, const float* __restrict__ Hd, int B, int din, int dh,
                               int dout, float* G) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    float* GW2 = G + (size_t)dh * din + dh;
    if (o < dout * dh) {
        const int k = o / dh, j = o - k * dh;
        float acc = 0.0f;
        for (int n = 0; n < B; ++n) acc = fmaf(dZ[(size_t)n * dout + k], Hd[(size_t)n * dh + j], acc);
        GW2[o] = acc;
    } else if (o < dout * dh + dout) {
        const int k = o - dout * dh;
        float acc = 0.0f;
        for (int n = 0; n < B; ++n) acc += dZ[(size_t)n * dout + k];
        GW2[(size_t)dout * dh + k] = acc;
    }
}

// back through the output layer and tanh: dA[n][j] = (sum_k dZ[n][k] W2[k][j]) (1 - Hd^2)
__global__ void k_mlp_dA(const float* __restrict__ P, const float* __restrict__ dZ, const float* __restrict__ Hd,
                         int B, int din, int dh, int dout, float* dA) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= B * dh) return;
    const int n = o / dh, j = o - n * dh;
    const float* W2 = P + (size_t)dh * din + dh;
    float acc = 0.0f;
    for (int k = 0; k < dout; ++k) acc = fmaf(dZ[(size_t)n * dout + k], W2[(size_t)k * dh + j], acc);
    const float hv = Hd[o];
    dA[o] = acc * (1.0f - hv * hv);
}

// gradients of the hidden layer: G_W1[j][i] = sum_n dA[n][j] X[n][i], G_b1[j] = sum_n dA[n][j]
__global__ void k_mlp_grad_hidden(const float* __restrict__ dA, const float* __restrict__ X, int B, int din, int dh,
                                  float* G) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o < dh * din) {
        const int j = o / din, i = o - j * din;
        float acc = 0.0f;
        for (int n = 0; n < B; ++n) acc = fmaf(dA[(size_t)n * dh + j], X[(size_t)n * din + i], acc);
        G[o] = acc;
    } else if (o < dh * din + dh) {
        const int j = o - dh * din;
        float acc = 0.0f;
        for (int n = 0; n < B; ++n) acc += dA[(size_t)n * dh + j];
        G[(size_t)dh * din + j] = acc;
    }
}

// Adam (Kingma & Ba 2015) with bias correction; bc1 = 1 - beta1^step, bc2 = 1 - beta2^step
__global__ void k_adam(float* P, const float* __restrict__ G, float* m, float* v, int n, float lr, float bc1,
                       float bc2) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n) return;
    const float g = G[o];
    const float mo = 0.9f * m[o] + 0.1f * g;
    const float vo = 0.999f * v[o] + 0.001f * g * g;
    m[o] = mo;
    v[o] = vo;
    P[o] -= lr * (mo / bc1) / (sqrtf(vo / bc2) + 1e-8f);
}

// One proposal from the logits z of a block at (l0, o1, o2): s'_i = +1 iff
// u_i < sigmoid(z_i); mask (T x Np, zero outside the block on entry) gets 1
// where s' differs from the current field; lq[0] = log q(s'|x),
// lq[1] = log q(s|x).  One CTA.
__global__ void k_block_propose(const float* __restrict__ Z, const int8_t* __restrict__ field, BlockGeom g, int l0,
                                int o1, int o2, uint64_t key, uint64_t ctr, int8_t* mask, double* lq) {
    __shared__ double red[33];
    double ln = 0.0, lo = 0.0;
    for (int idx = threadIdx.x; idx < g.d_out; idx += blockDim.x) {
        const int sub = idx & 1;
        int rest = idx >> 1;
        const int c1 = rest % g.b;
        rest /= g.b;
        const int c2 = rest % g.b;
        const int t = rest / g.b;
        const int site = sub * g.Nc + pmod(o1 + c1, g.L1) + g.L1 * pmod(o2 + c2, g.L2);
        const double z = Z[idx];
        const int s_old = field[(size_t)(l0 - 1 + t) * g.Np + site];
        // P(s' = +1) = sigmoid(z) = e^{log_sigmoid(z)}
        const int s_new = log(sm64_uniform(key, ctr + idx)) < log_sigmoid(z) ? 1 : -1;
        ln += log_sigmoid(s_new * z);
        lo += log_sigmoid(s_old * z);
        mask[(size_t)t * g.Np + site] = (int8_t)(s_new != s_old);
    }
    ln = block_sum(ln, red);
    lo = block_sum(lo, red);
    if (threadIdx.x == 0) { lq[0] = ln; lq[1] = lo; }
}

// Metropolis-Hastings: accept iff u < e^{logR} q(s|x) / q(s'|x).
// stats[0] proposals, stats[1] accepted, stats[2] flipped sites of accepted moves
__global__ void k_block_accept(const double* __restrict__ logR, const double* __restrict__ lq,
                               const int8_t* __restrict__ mask, int nmask, uint64_t key, uint64_t ctr, int* flag,
                               unsigned long long* stats, DevStatus* st) {
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    int c = 0;
    for (int o = threadIdx.x; o < nmask; o += blockDim.x) c += mask[o];
    atomicAdd(&cnt, c);
    __syncthreads();
    if (threadIdx.x == 0) {
        const double la = *logR + lq[1] - lq[0];
        if (isnan(la)) flag_error(st, DERR_NUMERIC, 400);
        const int acc = log(sm64_uniform(key, ctr)) < la ? 1 : 0;
        *flag = acc;
        stats[0] += 1;
        stats[1] += acc;
        if (acc) stats[2] += cnt;
    }
}

// rejected move: put back the saved G and field slices
__global__ void k_block_restore(const int* __restrict__ flag, const double* __restrict__ Gs, double* G, size_t nn,
                                const int8_t* __restrict__ fs, int8_t* f, size_t nf) {
    if (*flag) return;
    for (size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x; o < nn; o += (size_t)gridDim.x * blockDim.x) {
        G[o] = Gs[o];
        if (o < nf) f[o] = fs[o];
    }
}

}  // namespace afq
