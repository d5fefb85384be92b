// libafqmc.so: host orchestration of the DQMC sweep and the C ABI of afqmc.h.
//
// Host side: parameter checks, the lattice set-up (Sec. II.A: Bloch function
// f(k), Eq. h0kMat; the 2x2 propagator blocks of Eq. ExpLambda in closed form),
// device memory, and the launch schedule of a sweep.  Every step of the Monte
// Carlo path runs in the kernels of wrap.cuh, update.cuh, linalg.cuh and
// measure.cuh.
#include <cmath>
#include <cstddef>
#include <complex>
#include <cstdio>
#include <cstring>
#include <map>
#include <random>
#include <mutex>
#include <string>
#include <vector>

#include "afqmc.h"
#include "common.cuh"
#include "learned.cuh"
#include "linalg.cuh"
#include "measure.cuh"
#include "ozaki.cuh"
#include "tdgf.cuh"
#include "update.cuh"
#include "wrap.cuh"

using namespace afq;

namespace {

thread_local std::string g_create_error;

struct UDTe {            // U D T of a propagator chain
    double* Ut = nullptr;  // U stored column-major (row c = column c)
    double* D = nullptr;
    double* T = nullptr;   // row-major
};

struct CudaFail {
    afqmc_status code;
    std::string msg;
};

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            throw CudaFail{AFQMC_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)}; \
    } while (0)

enum Op { OP_E = 0, OP_EINV = 1, OP_EH = 2, OP_EHINV = 3 };

}  // namespace

struct afqmc_handle {
    afqmc_params p{};
    // Np = 2 Nc physical sites; N = dimension of the device matrices: Np, or 2 Np
    // for twisted boundaries or the charge-channel field, where every complex
    // N x N matrix is held as its real embedding [[Re, -Im], [Im, Re]] (cplx = 1)
    int N = 0, Np = 0, Nc = 0, L1 = 0, L2 = 0, M = 0, ns = 0, nc = 0, nd = 0, W = UPD_WMAX;
    int cplx = 0;
    int charge = 0;                // 1: charge-channel field (Eq. DensityHS), B_l = e^{i alpha diag(s)} E
    BondPhases bond_ph{};          // e^{i Phi} of the three bonds (measurements)
    double gamma = 0.0, egp = 1.0, egm = 1.0;      // e^{gamma}, e^{-gamma}
    double alpha = 0.0, ca = 1.0, sa = 0.0;        // charge channel: alpha = arccos(e^{-dtau U/2}), cos, sin
    double dl_p = 0.0, dl_m = 0.0, ef_p = 1.0, ef_m = 1.0;
    double dli_p = 0.0, dli_m = 0.0;               // Im Delta (charge channel)
    uint64_t key = 0, sweep_index = 0;
    unsigned long long* d_sweep = nullptr;   // device copy of sweep_index (read by the slice kernel)
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int sms = 0;
    int upd_grid = 0;              // CTAs of the cooperative slice kernel
    // precision bit 1: digit planes and exponents of the Ozaki products, and the
    // tensor maps of the two digit-plane arrays (tensor-memory-access staging)
    CUtensorMap oz_tmA{}, oz_tmB{};
    __nv_bfloat16 *ozA = nullptr, *ozB = nullptr;
    int *ozea = nullptr, *ozeb = nullptr;
    int ozKpad = 0;
    bool in_batch = false;         // owned by an afqmc_batch (no per-launch timing)
    bool broken = false;
    std::string err;
    // device memory
    std::vector<void*> allocs;
    int8_t* field = nullptr;
    double* G = nullptr;
    double* Wk[6] = {};
    double *Xs = nullptr, *Ys = nullptr, *mcoef = nullptr, *xw = nullptr, *yw = nullptr, *Gw = nullptr;
    uint32_t *tf_xh = nullptr, *tf_xl = nullptr, *tf_yh = nullptr, *tf_yl = nullptr;   // split-TF32 operands
    int tf_ld = 0;
    int *msite = nullptr, *ctl = nullptr, *perm = nullptr;
    double *vtmp = nullptr, *Dp = nullptr, *sgn = nullptr, *tau = nullptr, *DbR = nullptr, *DsR = nullptr,
           *DbL = nullptr, *DsL = nullptr;
    double* pubx = nullptr;        // scalar of each column hand-off of the QR and LU kernels
    int* piv = nullptr;            // LU pivots of the middle matrix of G
    int* lperm = nullptr;          // precision bit 2: combined LU row order (blocked solves)
    double2* blocks = nullptr;     // 4 operators x Nc x 4
    double2 *tw1 = nullptr, *tw2 = nullptr;
    DevStatus* st = nullptr;
    unsigned long long* n_acc = nullptr;
    unsigned long long* drift = nullptr;
    double *czz = nullptr, *hab = nullptr, *tr2 = nullptr;     // per-measurement scratch
    double *obs_now = nullptr, *czz_now = nullptr, *nk_now = nullptr;
    double *obs_acc = nullptr, *czz_acc = nullptr, *nk_acc = nullptr;
    // block moves (allocated on the first block pass)
    double* Gsave = nullptr;
    int8_t *fsave = nullptr, *bmask = nullptr;
    double *logR = nullptr, *lq = nullptr;
    int* bflag = nullptr;
    unsigned long long* bstats = nullptr;
    float *bX = nullptr, *bH = nullptr, *bZ = nullptr;
    int* bpos = nullptr;
    size_t bcap_in = 0, bcap_hid = 0, bcap_out = 0, bcap_T = 0;
    uint64_t block_passes = 0;
    // time-displaced measurement (allocated on first use)
    double *td_t0 = nullptr, *td_0t = nullptr, *td_tt = nullptr, *td_s[4] = {}, *td_tmp = nullptr;
    double2 *td_dtt = nullptr, *td_d00 = nullptr;
    double *td_part = nullptr, *td_hh = nullptr, *td_h = nullptr;
    long long td_count = 0;
    long long* obs_count = nullptr;
    std::vector<UDTe> Rst, Lst;
    UDTe tmpA, tmpB;               // scratch entries for get_G
    FFTPlan plan{};
    int vp = 1;
    size_t rowop_smem = 0;
    bool qr_smem_cols = false;     // QR keeps each CTA's columns in shared memory
    // launch accounting and optional per-launch event timing
    uint64_t launches = 0;
    int timing = 0;                // bit mask of the timed kernel families
    uint64_t cat_launches[AFQMC_K_COUNT] = {};
    double cat_ms[AFQMC_K_COUNT] = {};
    std::vector<cudaEvent_t> ev_free;
    struct Pending { cudaEvent_t a, b; int cat; };
    std::vector<Pending> pending;

    template <class T>
    T* dalloc(size_t n) {
        void* ptr = nullptr;
        cudaError_t e = cudaMalloc(&ptr, n * sizeof(T) > 0 ? n * sizeof(T) : 16);
        if (e != cudaSuccess) throw CudaFail{AFQMC_E_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e)};
        allocs.push_back(ptr);
        return static_cast<T*>(ptr);
    }
};

namespace {

// ------------------------------------------------------------------ set-up
// radices of an L-point FFT: 4s first, then 2, 3, then the remaining primes
int radices(int n, int* r) {
    int k = 0;
    while (n % 4 == 0 && k < FFT_MAX_STAGES) { r[k++] = 4; n /= 4; }
    for (int p = 2; n > 1 && k < FFT_MAX_STAGES; ++p)
        while (n % p == 0 && k < FFT_MAX_STAGES) { r[k++] = p; n /= p; }
    return n == 1 ? k : -1;
}

// f(k) = -t [1 + e^{i k.(a1-a2)} + e^{-i k.a2}] (below Eq. h0kMat) at
// k = ((l1 + theta1)/L1) b1 + ((l2 + theta2)/L2) b2 (Eq. kpoints), so
// k.a_alpha = 2 pi (l_alpha + theta_alpha) / L_alpha.  In Gauge-I (Sec. III.C)
// the twist sits on the bonds and K stays translation invariant: block l of
// the untwisted cell DFT is the Bloch matrix at this shifted k.
std::complex<double> bloch_f(double t, int l1, int l2, int L1, int L2, double th1, double th2) {
    const double p1 = 2.0 * M_PI * (l1 + th1) / L1, p2 = 2.0 * M_PI * (l2 + th2) / L2;
    const std::complex<double> I(0.0, 1.0);
    return -t * (1.0 + std::exp(I * (p1 - p2)) + std::exp(-I * p2));
}

// e^{-c h(k)} = cosh(c|f|) 1 - sinh(c|f|)/|f| h(k),  h = [[0, f], [f*, 0]]  (Eq. ExpLambda)
void block_exp(std::complex<double> f, double c, double2 out[4]) {
    const double af = std::abs(f);
    const double ch = std::cosh(c * af);
    const std::complex<double> sf = af > 0.0 ? -std::sinh(c * af) / af * f : std::complex<double>(0.0, 0.0);
    out[0] = make_double2(ch, 0.0);
    out[1] = make_double2(sf.real(), sf.imag());
    out[2] = make_double2(sf.real(), -sf.imag());
    out[3] = make_double2(ch, 0.0);
}

// The dynamic shared-memory limit of a kernel is process-wide state of the
// device: only ever raise it, so handles of different sizes can coexist.
std::mutex g_attr_mutex;
std::map<std::pair<int, const void*>, size_t> g_attr_max;

cudaError_t raise_smem_limit(const void* func, size_t bytes) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_attr_mutex);
    size_t& cur = g_attr_max[{dev, func}];
    if (bytes <= cur) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) cur = bytes;
    return e;
}

void set_error(afqmc_handle* h, afqmc_status code, const std::string& msg) {
    h->err = msg;
    if (code == AFQMC_E_CUDA || code == AFQMC_E_TIMEOUT || code == AFQMC_E_NUMERIC) h->broken = true;
}

// ------------------------------------------------------------------ launches
cudaEvent_t take_event(afqmc_handle* h) {
    if (!h->ev_free.empty()) { cudaEvent_t e = h->ev_free.back(); h->ev_free.pop_back(); return e; }
    cudaEvent_t e;
    CK(cudaEventCreate(&e));
    return e;
}

void flush_timing(afqmc_handle* h) {
    if (h->pending.empty()) return;
    CK(cudaStreamSynchronize(h->stream));
    for (auto& q : h->pending) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, q.a, q.b));
        h->cat_ms[q.cat] += ms;
        h->ev_free.push_back(q.a);
        h->ev_free.push_back(q.b);
    }
    h->pending.clear();
}

// Counts one kernel launch of family `cat`; brackets it with events when timing.
struct Scope {
    afqmc_handle* h;
    int cat;
    cudaEvent_t a = nullptr;
    Scope(afqmc_handle* h_, int c) : h(h_), cat(c) {
        h->launches += 1;
        h->cat_launches[c] += 1;
        if (h->timing & (1 << c)) {
            if (h->pending.size() > 50000) flush_timing(h);
            a = take_event(h);
            CK(cudaEventRecord(a, h->stream));
        }
    }
    ~Scope() {
        if (!a) return;
        cudaEvent_t b = nullptr;
        if (!h->ev_free.empty()) { b = h->ev_free.back(); h->ev_free.pop_back(); }
        else if (cudaEventCreate(&b) != cudaSuccess) { h->ev_free.push_back(a); return; }
        if (cudaEventRecord(b, h->stream) != cudaSuccess) { h->ev_free.push_back(a); h->ev_free.push_back(b); return; }
        h->pending.push_back({a, b, cat});
    }
};
void launch_rowop(afqmc_handle* h, const double* in, double* out, int nrows, Op op, DiagScale pre, DiagScale post,
                  bool transpose) {
    const int per = h->cplx ? h->vp : 2 * h->vp;
    const int grid = (nrows + per - 1) / per;
    Scope sc(h, AFQMC_K_PROPAGATE);
    k_rowop<<<grid, 256, h->rowop_smem, h->stream>>>(in, out, nrows, h->N, h->N, h->plan,
                                                     h->blocks + (size_t)op * h->Nc * 4, pre, post,
                                                     transpose ? 1 : 0, h->vp, h->cplx);
    CK(cudaGetLastError());
}

// The slice kernel of the handle's field: spin channel (0) or charge channel (1).
const void* upd_kernel(int charge) {
    return charge ? (const void*)k_update_slice<1> : (const void*)k_update_slice<0>;
}

DiagScale no_scale() { return DiagScale{nullptr, 1.0, 1.0}; }
// The diagonal factor of B_l.  Spin channel: e^{spin_sign gamma s_l} (real).
// Charge channel: the complex factor e^{charge_sign i alpha s_l} by which the
// row kernel multiplies the complex vectors of the embedding; each call site
// states which one it needs (for a row of the embedding the kernel's vector is
// the conjugate row, for a column it is the column itself).
DiagScale vdiag(afqmc_handle* h, int l, int spin_sign, int charge_sign) {
    const int8_t* s = h->field + (size_t)(l - 1) * h->Np;
    if (h->charge) {
        DiagScale d{s, h->ca, h->ca};
        d.ip = charge_sign > 0 ? h->sa : -h->sa;      // s = +1: e^{+-i alpha}
        d.im = -d.ip;                                  // s = -1: the conjugate
        d.phase = 1;
        return d;
    }
    return spin_sign > 0 ? DiagScale{s, h->egp, h->egm} : DiagScale{s, h->egm, h->egp};
}

// cuTensorMapEncodeTiled from the driver (through the runtime's entry-point query,
// so the library needs no link against the driver library)
using TensorMapEncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                       const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                       CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
std::mutex g_tmap_mutex;

TensorMapEncodeFn tensor_map_encoder() {
    static TensorMapEncodeFn fn = nullptr;
    std::lock_guard<std::mutex> lock(g_tmap_mutex);
    if (!fn) {
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<TensorMapEncodeFn>(ptr);
    }
    return fn;
}

// 3-D tensor map (k, row, digit) of OZ_S BF16 digit planes [digit][row][Kpad],
// box 8 x box_rows x OZ_S: one copy stages 8 values of k of all digits of a tile
void encode_digit_planes(CUtensorMap* map, void* base, int rows, int Kpad, int box_rows) {
    TensorMapEncodeFn enc = tensor_map_encoder();
    if (!enc) throw CudaFail{AFQMC_E_CUDA, "cuTensorMapEncodeTiled is not available from the driver"};
    const cuuint64_t dims[3] = {(cuuint64_t)Kpad, (cuuint64_t)rows, (cuuint64_t)OZ_S};
    const cuuint64_t strides[2] = {(cuuint64_t)Kpad * 2, (cuuint64_t)rows * Kpad * 2};
    const cuuint32_t box[3] = {8, (cuuint32_t)box_rows, (cuuint32_t)OZ_S};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) throw CudaFail{AFQMC_E_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r)};
}

// C = alpha rs .* (op(A) op(B)) .* cs + beta C on the BF16 tensor cores, FP64-accurate (ozaki.cuh)
void gemm_oz(afqmc_handle* h, const double* A, int transA, const double* B, int transB, double* C, double alpha,
             double beta, const double* rs, int rs_inv, const double* cs, int cs_inv) {
    const int n = h->N, Kp = h->ozKpad;
    // the digits are cut from rows: op(A) rows, and op(B)^T rows (= B rows when transB);
    // the other cases go through a transposed copy in the scratch matrix Wk[4]
    auto split = [&](const double* X, bool transpose, __nv_bfloat16* out, int* ex) {
        const double* src = X;
        if (transpose) {
            dim3 b(32, 8), gr((n + 31) / 32, (n + 31) / 32);
            Scope sc(h, AFQMC_K_GEMM);
            k_transpose_scale<<<gr, b, 0, h->stream>>>(X, h->Wk[4], n, n, nullptr, 0, nullptr, 0);
            src = h->Wk[4];
        }
        Scope sc(h, AFQMC_K_GEMM);
        k_oz_split<<<(n * 32 + 255) / 256, 256, 0, h->stream>>>(src, n, n, n, out, n, Kp, Kp, ex);
    };
    split(A, transA != 0, h->ozA, h->ozea);
    split(B, transB == 0, h->ozB, h->ozeb);
    OzArgs g{h->ozA, h->ozB, h->ozea, h->ozeb, n, n, Kp, C, n, alpha, beta, rs, cs, rs_inv, cs_inv, h->st};
    dim3 grid((n + OZ_TN - 1) / OZ_TN, (n + OZ_TM - 1) / OZ_TM);
    Scope sc(h, AFQMC_K_GEMM);
    k_oz_gemm<<<grid, OZ_THREADS, oz_smem_bytes(), h->stream>>>(h->oz_tmA, h->oz_tmB, g);
    CK(cudaGetLastError());
}

// C[i][j] = alpha sum_k A[i][k] B[j][k] + beta C[i][j] for i < m, j < n, k < K, on
// row segments (leading dimensions lda, ldb, ldc <= N): the Ozaki product of the
// blocked solves, FP64-accurate, counted in kernel family `cat`.
void gemm_rows_oz(afqmc_handle* h, const double* A, int lda, int m, const double* B, int ldb, int n, int K,
                  double* C, int ldc, double alpha, double beta, int cat) {
    const int Kp = h->ozKpad, Kw = (K + OZ_KC - 1) / OZ_KC * OZ_KC;
    { Scope sc(h, cat); k_oz_split<<<(m * 32 + 255) / 256, 256, 0, h->stream>>>(A, m, K, lda, h->ozA, h->N, Kp, Kw, h->ozea); }
    { Scope sc(h, cat); k_oz_split<<<(n * 32 + 255) / 256, 256, 0, h->stream>>>(B, n, K, ldb, h->ozB, h->N, Kp, Kw, h->ozeb); }
    OzArgs g{h->ozA, h->ozB, h->ozea, h->ozeb, m, n, Kw, C, ldc, alpha, beta, nullptr, nullptr, 0, 0, h->st};
    dim3 grid((n + OZ_TN - 1) / OZ_TN, (m + OZ_TM - 1) / OZ_TM);
    Scope sc(h, cat);
    k_oz_gemm<<<grid, OZ_THREADS, oz_smem_bytes(), h->stream>>>(h->oz_tmA, h->oz_tmB, g);
    CK(cudaGetLastError());
}

void gemm(afqmc_handle* h, const double* A, int transA, const double* B, int transB, double* C, double alpha,
          double beta, const double* rs, int rs_inv, const double* cs, int cs_inv, int a_upper = 0) {
    if (h->p.precision & 2) {
        gemm_oz(h, A, transA, B, transB, C, alpha, beta, rs, rs_inv, cs, cs_inv);
        return;
    }
    const int n = h->N;
    GemmArgs g{A, B, C, n, n, n, n, n, n, transA, transB, alpha, beta, rs, cs, rs_inv, cs_inv, a_upper};
    dim3 grid((n + GT - 1) / GT, (n + GT - 1) / GT);
    Scope sc(h, AFQMC_K_GEMM);
    k_dgemm<<<grid, 256, 0, h->stream>>>(g);
    CK(cudaGetLastError());
}

// the publication buffers of the QR and LU column hand-off (Wk[2] is free
// during both factorisations), filled with the empty pattern
double* pub_clear(afqmc_handle* h) {
    const size_t nn = (size_t)h->N * h->N;
    double* pub = h->Wk[2];
    Scope sc(h, AFQMC_K_MISC);
    k_pub_clear<<<(unsigned)std::min<size_t>((nn + 255) / 256, 4u * h->sms), 256, 0, h->stream>>>(pub, nn, h->pubx,
                                                                                                  h->N);
    CK(cudaGetLastError());
    return pub;
}

void qr(afqmc_handle* h, double* At) {
    const int n = h->N;
    double* pub = pub_clear(h);
    QRArgs q{At, h->tau, pub, h->pubx, n, h->st};
    const int grid = std::min(h->sms, n);
    int in_smem = h->qr_smem_cols ? 1 : 0;
    const size_t smem = sizeof(double) * (size_t)n * (in_smem ? 1 + (n + grid - 1) / grid : 1);
    void* args[] = {&q, &in_smem};
    Scope sc(h, AFQMC_K_QR);
    CK(cudaLaunchCooperativeKernel((void*)k_qr_cols, grid, 256, args, smem, h->stream));
}

// P A = L U of the column-major A (At) in place, pivots in h->piv; with Fr also the
// row-major factor with the swaps applied to L, and the row order in h->lperm.
void lu(afqmc_handle* h, double* At, double* Fr = nullptr) {
    const int n = h->N;
    double* pub = pub_clear(h);
    LUArgs q{At, h->piv, pub, h->pubx, n, h->st, Fr, Fr ? h->lperm : nullptr};
    const int grid = std::min(h->sms, n);
    int in_smem = h->qr_smem_cols ? 1 : 0;
    const size_t smem = sizeof(double) * (size_t)n * (in_smem ? 1 + (n + grid - 1) / grid : 1);
    void* args[] = {&q, &in_smem};
    Scope sc(h, AFQMC_K_LU);
    CK(cudaLaunchCooperativeKernel((void*)k_lu_cols, grid, 256, args, smem, h->stream));
}

int warp_grid(int ncols) { return (ncols * 32 + 255) / 256; }
// shape of the column-parallel kernels for matrix dimension n: <8 columns per
// CTA, 8 prefetch registers> up to n = 2048, <4, 16> up to COL_MAX_N
bool col_small(int n) { return n <= 2048; }
int col_cpb(int n) { return col_small(n) ? 8 : 4; }
int cpb_grid(int ncols, int n) { return (ncols + col_cpb(n) - 1) / col_cpb(n); }
size_t cpb_smem(int n) { return sizeof(double) * (size_t)(col_cpb(n) + 2) * n; }

void launch_form_q(afqmc_handle* h, const double* Vt, const double* tau, const double* sgn, double* Qt, int n) {
    Scope sc(h, AFQMC_K_QRAUX);
    if (col_small(n)) k_form_q<8, 8><<<cpb_grid(n, n), 256, cpb_smem(n), h->stream>>>(Vt, tau, sgn, Qt, n);
    else k_form_q<4, 16><<<cpb_grid(n, n), 256, cpb_smem(n), h->stream>>>(Vt, tau, sgn, Qt, n);
    CK(cudaGetLastError());
}
void launch_fwdsolve(afqmc_handle* h, const double* Lt, const int* piv, double* Yt, int n) {
    Scope sc(h, AFQMC_K_QRAUX);
    if (col_small(n)) k_fwdsolve_perm<8, 8><<<cpb_grid(n, n), 256, cpb_smem(n), h->stream>>>(Lt, piv, Yt, n, n);
    else k_fwdsolve_perm<4, 16><<<cpb_grid(n, n), 256, cpb_smem(n), h->stream>>>(Lt, piv, Yt, n, n);
    CK(cudaGetLastError());
}
void launch_backsolve(afqmc_handle* h, const double* Rt, const double* Yt, double* Xt, int n, const double* xs) {
    Scope sc(h, AFQMC_K_QRAUX);
    if (col_small(n)) k_backsolve<8, 8><<<cpb_grid(n, n), 256, cpb_smem(n), h->stream>>>(Rt, Yt, Xt, n, n, xs, h->st);
    else k_backsolve<4, 16><<<cpb_grid(n, n), 256, cpb_smem(n), h->stream>>>(Rt, Yt, Xt, n, n, xs, h->st);
    CK(cudaGetLastError());
}

// Blocked triangular solves on the rows of Yt (each row one right-hand side),
// columns r0 .. r1 of the system: with the row-major LU factor Fr, lower (unit
// L, forward) or upper (U, backward).  The range is halved (in units of 32)
// down to blocks of at most TRSM_LEAF, which k_trsm_leaf solves in FP64; the
// coupling between the halves is one Ozaki product per split:
//   forward:  Y[:, I2] -= Y[:, I1] L[I2, I1]^T   after solving I1,
//   backward: Y[:, I1] -= Y[:, I2] U[I1, I2]^T   after solving I2,
// so nearly all of the n^3 flops of a solve with n right-hand sides run on the
// tensor cores.  Both operands of a product are row segments (rows of Yt and of
// Fr), as the digit split wants them.
void trsm_blocked(afqmc_handle* h, const double* Fr, double* Yt, int r0, int r1, bool upper) {
    const int n = h->N, nb = r1 - r0;
    if (nb <= TRSM_LEAF) {
        const int grid = (n + 7) / 8;
        Scope sc(h, AFQMC_K_QRAUX);
        if (upper) k_trsm_leaf<1><<<grid, 256, 0, h->stream>>>(Fr, Yt, n, n, r0, nb);
        else k_trsm_leaf<0><<<grid, 256, 0, h->stream>>>(Fr, Yt, n, n, r0, nb);
        CK(cudaGetLastError());
        return;
    }
    const int mid = r0 + ((nb + 31) / 32 / 2) * 32;
    if (!upper) {
        trsm_blocked(h, Fr, Yt, r0, mid, false);
        gemm_rows_oz(h, Yt + r0, n, n, Fr + (size_t)mid * n + r0, n, r1 - mid, mid - r0, Yt + mid, n, -1.0, 1.0,
                     AFQMC_K_QRAUX);
        trsm_blocked(h, Fr, Yt, mid, r1, false);
    } else {
        trsm_blocked(h, Fr, Yt, mid, r1, true);
        gemm_rows_oz(h, Yt + mid, n, n, Fr + (size_t)r0 * n + mid, n, mid - r0, r1 - mid, Yt + r0, n, -1.0, 1.0,
                     AFQMC_K_QRAUX);
        trsm_blocked(h, Fr, Yt, r0, mid, true);
    }
}

// X = Db_L^-1 M^-1 rhs (rows of Xt), with P M = L U from lu(h, Mt, Fr) and the
// right-hand sides the columns of (rows of `in` scaled by rs): P (rs .* in) is
// gathered and transposed into Yt, solved in place by the blocked solves, and
// divided by Db_L into Xt.
void solve_blocked(afqmc_handle* h, const double* Fr, const double* in, const double* rs, int rs_inv, double* Yt,
                   double* Xt) {
    const int n = h->N;
    {
        dim3 b(32, 8), g((n + 31) / 32, (n + 31) / 32);
        Scope sc(h, AFQMC_K_QRAUX);
        k_transpose_perm<<<g, b, 0, h->stream>>>(in, Yt, n, h->lperm, rs, rs_inv);
    }
    CK(cudaGetLastError());
    trsm_blocked(h, Fr, Yt, 0, n, false);
    trsm_blocked(h, Fr, Yt, 0, n, true);
    const size_t nn = (size_t)n * n;
    { Scope sc(h, AFQMC_K_QRAUX); k_div_cols_check<<<(unsigned)std::min<size_t>((nn + 255) / 256, 4u * h->sms), 256, 0, h->stream>>>(Yt, Xt, n, h->DbL, h->st); }
    CK(cudaGetLastError());
}

// dynamic shared memory of k_update_slice: window block (phase B) or flush tiles (phase F)
size_t update_smem(int W, int nd, int precision, int N = AFQMC_NOALLOC_MAX_N, int grid = 148) {
    size_t b = sizeof(double) * (2 * (size_t)W * (W + 1) + 6 * W);
    const size_t jpb = (size_t)((N + grid - 1) / grid);
    b = std::max(b, sizeof(double) * (2 * (size_t)nd * jpb + 2 * (size_t)nd * W + 2 * (size_t)W * W));   // phase C staging
    size_t f = sizeof(double) * 2 * (size_t)nd * 32;
    if (precision & 1) {
        f = std::max(f, sizeof(uint32_t) * 4 * (size_t)TCK * TCT);     // TF32 operands of one K round
        f = std::max(f, sizeof(float) * (size_t)TCT * (TCT + 1));      // accumulator tile
    }
    return std::max(b, f);
}

// out = UDT of (chain of slices lo..hi) applied to `in`:
//   left  (R chain):  B_hi ... B_lo U D T
//   !left (L chain):  (B_hi ... B_lo)^T U D T
void udt_extend(afqmc_handle* h, const UDTe& in, const UDTe& out, int lo, int hi, bool left) {
    const int n = h->N;
    double* A = h->Wk[0];
    CK(cudaMemcpyAsync(A, in.Ut, sizeof(double) * n * n, cudaMemcpyDeviceToDevice, h->stream));
    // rows of A = U^T are the columns of U: B U = V E U (left), B^+ U = E V^+ U (L chain,
    // the real transpose of the embedding is the embedding of the adjoint)
    if (left) {
        for (int l = lo; l <= hi; ++l) launch_rowop(h, A, A, n, OP_E, no_scale(), vdiag(h, l, +1, +1), false);
    } else {
        for (int l = hi; l >= lo; --l) launch_rowop(h, A, A, n, OP_E, vdiag(h, l, +1, -1), no_scale(), false);
    }
    // pre-pivoting by scaled column norms, unpivoted Householder QR of A P
    double* AP = h->Wk[1];
    { Scope sc(h, AFQMC_K_QRAUX); k_colnorm_scaled<<<warp_grid(n), 256, 0, h->stream>>>(A, in.D, h->vtmp, n, h->st); }
    { Scope sc(h, AFQMC_K_QRAUX); k_rank_perm<<<(n + 255) / 256, 256, 0, h->stream>>>(h->vtmp, h->perm, n); }
    { Scope sc(h, AFQMC_K_QRAUX); k_gather_rows<<<n, 256, 0, h->stream>>>(A, AP, h->perm, in.D, h->Dp, n); }
    CK(cudaGetLastError());
    qr(h, AP);
    double* F = h->Wk[2];
    { Scope sc(h, AFQMC_K_QRAUX); k_make_F<<<n, 256, 0, h->stream>>>(AP, h->Dp, F, out.D, h->sgn, n, h->st); }
    launch_form_q(h, AP, h->tau, h->sgn, out.Ut, n);
    double* Tp = h->Wk[3];
    { Scope sc(h, AFQMC_K_QRAUX); k_gather_rows<<<n, 256, 0, h->stream>>>(in.T, Tp, h->perm, nullptr, nullptr, n); }
    CK(cudaGetLastError());
    gemm(h, F, 0, Tp, 0, out.T, 1.0, 0.0, nullptr, 0, nullptr, 0, /*a_upper=*/1);
}

// G = (1 + R L)^-1 with R = U_R D_R T_R, L^T = U_L D_L T_L (Loh-Gubernatis split);
// the well-conditioned middle matrix is solved by LU with partial pivoting.
// Optionally also the time-displaced G(tau, 0) = U_L Db_L^-1 M^-1 Ds_R T_R and
// G(0, tau) = -T_L^T Ds_L M^-1 Db_R^-1 U_R^T with the same LU (R = B(tau, 0),
// L = B(beta, tau)).
void form_green(afqmc_handle* h, const UDTe& R, const UDTe& Lt, double* Gout, double* Gt0 = nullptr,
                double* G0t = nullptr) {
    const int n = h->N;
    { Scope sc(h, AFQMC_K_MISC); k_split_scales<<<(n + 255) / 256, 256, 0, h->stream>>>(R.D, h->DbR, h->DsR, n); }
    { Scope sc(h, AFQMC_K_MISC); k_split_scales<<<(n + 255) / 256, 256, 0, h->stream>>>(Lt.D, h->DbL, h->DsL, n); }
    CK(cudaGetLastError());
    double* Mt = h->Wk[0];   // M column-major = M^T row-major
    gemm(h, Lt.Ut, 0, R.Ut, 1, Mt, 1.0, 0.0, h->DbL, 1, h->DbR, 1);
    gemm(h, Lt.T, 0, R.T, 1, Mt, 1.0, 1.0, h->DsL, 0, h->DsR, 0);
    // precision bit 2: blocked solves with their couplings on the tensor cores,
    // from the row-major factor Fr; otherwise the column-step FP64 solves
    const bool blocked = (h->p.precision & 4) != 0;
    double* Fr = blocked ? h->Wk[3] : nullptr;
    lu(h, Mt, Fr);
    double* Yt = h->Wk[1];   // Y = Db_R^-1 U_R^T, column-major
    double* Wt = h->Wk[2];
    if (blocked) {
        solve_blocked(h, Fr, R.Ut, h->DbR, 1, Yt, Wt);
    } else {
        {
            dim3 b(32, 8), g((n + 31) / 32, (n + 31) / 32);
            Scope sc(h, AFQMC_K_QRAUX);
            k_transpose_scale<<<g, b, 0, h->stream>>>(R.Ut, Yt, n, n, h->DbR, 1, nullptr, 0);
        }
        launch_fwdsolve(h, Mt, h->piv, Yt, n);
        launch_backsolve(h, Mt, Yt, Wt, n, h->DbL);
    }
    gemm(h, Lt.Ut, 1, Wt, 1, Gout, 1.0, 0.0, nullptr, 0, nullptr, 0);
    const size_t nn = (size_t)n * n;
    if (G0t) {
        // Wt holds (Db_L^-1 M^-1 Db_R^-1 U_R^T)^T: scale by D_L = Ds_L Db_L, then -T_L^T (.)
        { Scope sc(h, AFQMC_K_MISC); k_scale_cols<<<(unsigned)((nn + 255) / 256), 256, 0, h->stream>>>(Wt, Yt, n, Lt.D); }
        CK(cudaGetLastError());
        gemm(h, Lt.T, 1, Yt, 1, G0t, -1.0, 0.0, nullptr, 0, nullptr, 0);
    }
    if (Gt0) {
        if (blocked) {
            solve_blocked(h, Fr, R.T, h->DsR, 0, Yt, Wt);
        } else {
            {
                dim3 b(32, 8), g((n + 31) / 32, (n + 31) / 32);
                Scope sc(h, AFQMC_K_QRAUX);
                k_transpose_scale<<<g, b, 0, h->stream>>>(R.T, Yt, n, n, h->DsR, 0, nullptr, 0);
            }
            launch_fwdsolve(h, Mt, h->piv, Yt, n);
            launch_backsolve(h, Mt, Yt, Wt, n, h->DbL);
        }
        gemm(h, Lt.Ut, 1, Wt, 1, Gt0, 1.0, 0.0, nullptr, 0, nullptr, 0);
    }
}

void set_identity(afqmc_handle* h, const UDTe& e) {
    const int n = h->N;
    const size_t nn = (size_t)n * n;
    { Scope sc(h, AFQMC_K_MISC); k_set_identity<<<(unsigned)((nn + 255) / 256), 256, 0, h->stream>>>(e.Ut, n); }
    { Scope sc(h, AFQMC_K_MISC); k_set_identity<<<(unsigned)((nn + 255) / 256), 256, 0, h->stream>>>(e.T, n); }
    { Scope sc(h, AFQMC_K_MISC); k_fill<<<(n + 255) / 256, 256, 0, h->stream>>>(e.D, 1.0, n); }
    CK(cudaGetLastError());
}

// G <- B_l G B_l^-1 (dir +1) or B_l^-1 G B_l (dir -1), two transposed row passes.
void wrap(afqmc_handle* h, double* A, int l, int dir) {
    const int n = h->N;
    double* T = h->Wk[4];
    // pass 1 right-multiplies the rows (A E^-1 V^-1, or A V E); pass 2 acts on the rows
    // of the adjoint, i.e. left-multiplies (V E ., or E^-1 V^-1 .)
    if (dir > 0) {
        launch_rowop(h, A, T, n, OP_EINV, no_scale(), vdiag(h, l, -1, +1), true);
        launch_rowop(h, T, A, n, OP_E, no_scale(), vdiag(h, l, +1, +1), true);
    } else {
        launch_rowop(h, A, T, n, OP_E, vdiag(h, l, +1, -1), no_scale(), true);
        launch_rowop(h, T, A, n, OP_EINV, vdiag(h, l, -1, -1), no_scale(), true);
    }
}

// half step g = e^{-dtau K/2} A e^{+dtau K/2} into out
void half_step(afqmc_handle* h, const double* A, double* out) {
    double* T = h->Wk[4];
    launch_rowop(h, A, T, h->N, OP_EHINV, no_scale(), no_scale(), true);
    launch_rowop(h, T, out, h->N, OP_EH, no_scale(), no_scale(), true);
}

// sweep < 0: the sweep number is the device-resident one (sweep path, graph
// replays); otherwise the given number (test hooks).
void update_slice(afqmc_handle* h, double* G, int l, int pass, int64_t sweep, const int8_t* force = nullptr,
                  double* logR = nullptr) {
    UpdArgs a{};
    a.G = G; a.N = h->N; a.Xs = h->Xs; a.Ys = h->Ys; a.msite = h->msite; a.mcoef = h->mcoef;
    a.xw = h->xw; a.yw = h->yw; a.Gw = h->Gw; a.ctl = h->ctl;
    a.s = h->field + (size_t)(l - 1) * h->Np;
    a.nd = h->nd; a.W = h->W;
    a.pair = h->cplx; a.Np = h->Np;
    a.force = force; a.logR = logR; a.two_gamma = h->charge ? 0.0 : 2.0 * h->gamma;
    a.dl_p = h->dl_p; a.dl_m = h->dl_m; a.ef_p = h->ef_p; a.ef_m = h->ef_m;
    a.dli_p = h->dli_p; a.dli_m = h->dli_m;
    a.key = h->key;
    a.ctr_stride = 2ull * (uint64_t)h->M * (uint64_t)h->Np;
    a.ctr0 = ((uint64_t)pass * (uint64_t)h->M + (uint64_t)(l - 1)) * (uint64_t)h->Np + 1;
    if (sweep < 0) a.sweep_dev = h->d_sweep;
    else a.ctr0 += (uint64_t)sweep * a.ctr_stride;
    a.n_acc = h->n_acc; a.st = h->st;
    a.precision = h->p.precision;
    a.xh = h->tf_xh; a.xl = h->tf_xl; a.yh = h->tf_yh; a.yl = h->tf_yl; a.ldt = h->tf_ld;
    const size_t smem = update_smem(h->W, h->nd, h->p.precision, h->N, h->upd_grid);
    void* args[] = {&a};
    Scope sc(h, AFQMC_K_UPDATE);
    CK(cudaLaunchCooperativeKernel(upd_kernel(h->charge), h->upd_grid, UPD_THREADS, args, smem, h->stream));
}

void measure(afqmc_handle* h, const double* G, bool accumulate) {
    double* g = h->Wk[5];
    half_step(h, G, g);
    const GView gv{g, h->Np, h->N, h->cplx};
    { Scope sc(h, AFQMC_K_MEASURE); k_measure_pairs<<<h->Nc, 128, 0, h->stream>>>(gv, h->L1, h->L2, h->czz, h->hab); }
    const int nt = (h->Np + 31) / 32;
    { Scope sc(h, AFQMC_K_MEASURE); k_measure_tr2<<<nt * nt, 256, 0, h->stream>>>(gv, h->tr2); }
    CK(cudaGetLastError());
    if (accumulate) {
        { Scope sc(h, AFQMC_K_MEASURE); k_measure_nk<<<(h->Nc + 127) / 128, 128, 0, h->stream>>>(h->hab, h->L1, h->L2, h->tw1, h->tw2, h->nk_acc, 1); }
        { Scope sc(h, AFQMC_K_MEASURE); k_measure_scalars<<<1, 256, 0, h->stream>>>(gv, h->czz, h->tr2, nt * nt, h->L1, h->L2, h->p.t, h->p.U,
                                                    h->p.beta, h->tw1, h->bond_ph, h->obs_acc, h->czz_acc, 1,
                                                    h->obs_count, h->st); }
    } else {
        { Scope sc(h, AFQMC_K_MEASURE); k_measure_nk<<<(h->Nc + 127) / 128, 128, 0, h->stream>>>(h->hab, h->L1, h->L2, h->tw1, h->tw2, h->nk_now, 0); }
        { Scope sc(h, AFQMC_K_MEASURE); k_measure_scalars<<<1, 256, 0, h->stream>>>(gv, h->czz, h->tr2, nt * nt, h->L1, h->L2, h->p.t, h->p.U,
                                                    h->p.beta, h->tw1, h->bond_ph, h->obs_now, nullptr, 0,
                                                    nullptr, h->st); }
        CK(cudaMemcpyAsync(h->czz_now, h->czz, sizeof(double) * h->Nc, cudaMemcpyDeviceToDevice, h->stream));
    }
    CK(cudaGetLastError());
}

// recompute G at a stack boundary, recording the drift from the wrapped G
void recompute(afqmc_handle* h, int c) {
    const size_t nn = (size_t)h->N * h->N;
    double* saved = h->Wk[5];
    CK(cudaMemcpyAsync(saved, h->G, sizeof(double) * nn, cudaMemcpyDeviceToDevice, h->stream));
    form_green(h, h->Rst[c], h->Lst[c], h->G);
    { Scope sc(h, AFQMC_K_MISC); k_maxabsdiff<<<h->sms * 2, 256, 0, h->stream>>>(h->G, saved, nn, h->drift, h->st, AFQMC_DRIFT_LIMIT); }
    CK(cudaGetLastError());
    if (h->p.measure) measure(h, h->G, true);
}

void init_chain(afqmc_handle* h) {
    set_identity(h, h->Rst[0]);
    set_identity(h, h->Lst[h->nc]);
    for (int c = h->nc - 1; c >= 0; --c) udt_extend(h, h->Lst[c + 1], h->Lst[c], c * h->ns + 1, (c + 1) * h->ns, false);
    form_green(h, h->Rst[0], h->Lst[0], h->G);
}

afqmc_status check_device(afqmc_handle* h) {
    CK(cudaStreamSynchronize(h->stream));
    DevStatus st;
    CK(cudaMemcpy(&st, h->st, sizeof(st), cudaMemcpyDeviceToHost));
    if (st.err == DERR_NUMERIC && st.where == 107) {
        set_error(h, AFQMC_E_NUMERIC, "stabilisation drift above the limit: an element of the wrapped G differs from "
                                      "the recomputed one by more than AFQMC_DRIFT_LIMIT max(1, |G_ij|) (site code 107)");
        return AFQMC_E_NUMERIC;
    }
    if (st.err == DERR_NUMERIC) {
        set_error(h, AFQMC_E_NUMERIC, "non-finite value in device computation (site code " + std::to_string(st.where) + ")");
        return AFQMC_E_NUMERIC;
    }
    if (st.err == DERR_TIMEOUT) {
        set_error(h, AFQMC_E_TIMEOUT, "device-side wait timed out (site code " + std::to_string(st.where) + ")");
        return AFQMC_E_TIMEOUT;
    }
    if (st.err != 0) {
        set_error(h, AFQMC_E_CUDA, "device error " + std::to_string(st.err));
        return AFQMC_E_CUDA;
    }
    return AFQMC_OK;
}

void sweep_once(afqmc_handle* h) {
    const int M = h->M, ns = h->ns;
    for (int l = 1; l <= M; ++l) {
        wrap(h, h->G, l, +1);
        update_slice(h, h->G, l, 0, -1);
        if (l % ns == 0) {
            const int c = l / ns;
            udt_extend(h, h->Rst[c - 1], h->Rst[c], (c - 1) * ns + 1, c * ns, true);
            recompute(h, c);
        }
    }
    for (int l = M; l >= 1; --l) {
        update_slice(h, h->G, l, 1, -1);
        wrap(h, h->G, l, -1);
        if ((l - 1) % ns == 0) {
            const int c = (l - 1) / ns;
            udt_extend(h, h->Lst[c + 1], h->Lst[c], c * ns + 1, (c + 1) * ns, false);
            recompute(h, c);
        }
    }
    { Scope sc(h, AFQMC_K_MISC); k_add_u64<<<1, 1, 0, h->stream>>>(h->d_sweep, 1ull); }
    CK(cudaGetLastError());
    h->sweep_index += 1;
}

// fresh G at slice l into out (device): R chain in tmpA/tmpB, L chain in the
// spare last entries of the two stacks (the sweep state is not touched).
void green_at(afqmc_handle* h, int l, double* out) {
    const int ns = h->ns;
    UDTe cur = h->tmpA, nxt = h->tmpB;
    set_identity(h, cur);
    for (int lo = 1; lo <= l; lo += ns) {
        const int hi = std::min(lo + ns - 1, l);
        udt_extend(h, cur, nxt, lo, hi, true);
        std::swap(cur, nxt);
    }
    UDTe a = h->Rst[h->nc + 1], b = h->Lst[h->nc + 1];
    set_identity(h, a);
    for (int hi = h->M; hi > l; hi -= ns) {
        const int lo = std::max(hi - ns + 1, l + 1);
        udt_extend(h, a, b, lo, hi, false);
        std::swap(a, b);
    }
    form_green(h, cur, a, out);
}

// Host <-> device matrix transfer of the API: real N x N, or (twisted) a complex
// Np x Np host matrix (interleaved re, im) to and from the device embedding,
// through the staging buffer `stage` (>= 2 Np^2 doubles).
void from_host(afqmc_handle* h, const double* host, double* dev, double* stage) {
    if (!h->cplx) {
        CK(cudaMemcpyAsync(dev, host, sizeof(double) * h->N * h->N, cudaMemcpyHostToDevice, h->stream));
        return;
    }
    const size_t n2 = (size_t)h->Np * h->Np;
    CK(cudaMemcpyAsync(stage, host, sizeof(double2) * n2, cudaMemcpyHostToDevice, h->stream));
    { Scope sc(h, AFQMC_K_MISC); k_embed<<<(unsigned)((n2 + 255) / 256), 256, 0, h->stream>>>((const double2*)stage, dev, h->Np); }
    CK(cudaGetLastError());
}
void to_host(afqmc_handle* h, const double* dev, double* host, double* stage) {
    if (!h->cplx) {
        CK(cudaMemcpyAsync(host, dev, sizeof(double) * h->N * h->N, cudaMemcpyDeviceToHost, h->stream));
        return;
    }
    const size_t n2 = (size_t)h->Np * h->Np;
    { Scope sc(h, AFQMC_K_MISC); k_extract<<<(unsigned)((n2 + 255) / 256), 256, 0, h->stream>>>(dev, (double2*)stage, h->Np); }
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(host, stage, sizeof(double2) * n2, cudaMemcpyDeviceToHost, h->stream));
}

// ------------------------------------------------------------------ time-displaced measurement
void td_reserve(afqmc_handle* h) {
    if (h->td_t0) return;
    const size_t nn = (size_t)h->N * h->N;
    h->td_t0 = h->dalloc<double>(nn);
    h->td_0t = h->dalloc<double>(nn);
    h->td_tt = h->dalloc<double>(nn);
    h->td_tmp = h->dalloc<double>(nn);
    for (auto& b : h->td_s) b = h->dalloc<double>(nn);
    h->td_dtt = h->dalloc<double2>(h->Np);
    h->td_d00 = h->dalloc<double2>(h->Np);
    const int nt = (h->Np + 31) / 32;
    h->td_part = h->dalloc<double>((size_t)nt * nt);
    h->td_hh = h->dalloc<double>(h->M / 2 + 1);
    h->td_h = h->dalloc<double>(1);
    CK(cudaMemsetAsync(h->td_hh, 0, sizeof(double) * (h->M / 2 + 1), h->stream));
    CK(cudaMemsetAsync(h->td_h, 0, sizeof(double), h->stream));
}

// accumulate Re sum_ij <A_i(tau_l) A_j(0)> of the current symmetrised matrices
void td_accumulate(afqmc_handle* h, int l) {
    const int n = h->N;
    half_step(h, h->td_tt, h->td_s[1]);
    half_step(h, h->td_t0, h->td_s[2]);
    half_step(h, h->td_0t, h->td_s[3]);
    const GView tt{h->td_s[1], h->Np, n, h->cplx}, t0{h->td_s[2], h->Np, n, h->cplx}, ot{h->td_s[3], h->Np, n, h->cplx};
    const GView g00{h->td_s[0], h->Np, n, h->cplx};
    const int nt = (h->Np + 31) / 32;
    { Scope sc(h, AFQMC_K_MEASURE); k_td_diag<<<(h->Np + 255) / 256, 256, 0, h->stream>>>(tt, g00, h->td_dtt, h->td_d00); }
    { Scope sc(h, AFQMC_K_MEASURE); k_td_tiles<<<nt * nt, 256, 0, h->stream>>>(t0, ot, h->td_dtt, h->td_d00, h->td_part); }
    { Scope sc(h, AFQMC_K_MEASURE); k_td_reduce<<<1, 256, 0, h->stream>>>(h->td_part, nt * nt, h->td_d00, h->Np, h->td_hh, l,
                                                                       h->td_h, l == 0 ? 1 : 0, h->st); }
    CK(cudaGetLastError());
}

// One time-displaced measurement of the current field from slice 0 (between
// sweeps): G(tau, 0), G(0, tau), G(tau, tau) for tau = 0 .. beta/2, recomputed
// from the stacks every n_stab slices (the R stack is rebuilt on the way, the
// L stack is the one the last backward pass left), propagated in between.
void td_measure(afqmc_handle* h) {
    td_reserve(h);
    const int n = h->N;
    const size_t nn = (size_t)n * n;
    CK(cudaMemcpyAsync(h->td_tt, h->G, sizeof(double) * nn, cudaMemcpyDeviceToDevice, h->stream));
    CK(cudaMemcpyAsync(h->td_t0, h->G, sizeof(double) * nn, cudaMemcpyDeviceToDevice, h->stream));
    CK(cudaMemcpyAsync(h->td_0t, h->G, sizeof(double) * nn, cudaMemcpyDeviceToDevice, h->stream));
    { Scope sc(h, AFQMC_K_MISC); k_sub_identity<<<(n + 255) / 256, 256, 0, h->stream>>>(h->td_0t, n); }   // G(0, 0+) = G - 1
    CK(cudaGetLastError());
    half_step(h, h->G, h->td_s[0]);
    td_accumulate(h, 0);
    for (int l = 1; l <= h->M / 2; ++l) {
        if (l % h->ns == 0) {
            const int c = l / h->ns;
            udt_extend(h, h->Rst[c - 1], h->Rst[c], (c - 1) * h->ns + 1, c * h->ns, true);
            form_green(h, h->Rst[c], h->Lst[c], h->td_tt, h->td_t0, h->td_0t);
        } else {
            wrap(h, h->td_tt, l, +1);
            {
                dim3 b(32, 8), g((n + 31) / 32, (n + 31) / 32);
                Scope sc(h, AFQMC_K_MISC);
                k_transpose_scale<<<g, b, 0, h->stream>>>(h->td_t0, h->td_tmp, n, n, nullptr, 0, nullptr, 0);
            }
            CK(cudaGetLastError());
            launch_rowop(h, h->td_tmp, h->td_t0, n, OP_E, no_scale(), vdiag(h, l, +1, +1), true);     // B_l G(tau, 0)
            launch_rowop(h, h->td_0t, h->td_0t, n, OP_EINV, no_scale(), vdiag(h, l, -1, +1), false);  // G(0, tau) B_l^-1
        }
        td_accumulate(h, l);
    }
    h->td_count += 1;
}

// ------------------------------------------------------------------ allocation-free slice update
// One file-scope scratch array for afqmc_update_slice_noalloc (callers that
// cannot allocate device memory).  Layout, in bytes from the start:
//   DevStatus | n_acc | ctl[8] | msite[ND] | mcoef[ND] | Gw[W*W] | xw[ND*W] | yw[ND*W] | Xs[ND*N] | Ys[ND*N]
constexpr size_t NA_ND = AFQMC_NOALLOC_MAX_NDELAY, NA_N = AFQMC_NOALLOC_MAX_N, NA_W = UPD_WMAX;
constexpr size_t na_align(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t NA_OFF_STATUS = 0;
constexpr size_t NA_OFF_ACC = na_align(NA_OFF_STATUS + sizeof(DevStatus));
constexpr size_t NA_OFF_CTL = na_align(NA_OFF_ACC + sizeof(unsigned long long));
constexpr size_t NA_OFF_SITE = na_align(NA_OFF_CTL + 8 * sizeof(int));
constexpr size_t NA_OFF_COEF = na_align(NA_OFF_SITE + NA_ND * sizeof(int));
constexpr size_t NA_OFF_GW = na_align(NA_OFF_COEF + NA_ND * sizeof(double));
constexpr size_t NA_OFF_XW = na_align(NA_OFF_GW + NA_W * NA_W * sizeof(double));
constexpr size_t NA_OFF_YW = na_align(NA_OFF_XW + NA_ND * NA_W * sizeof(double));
constexpr size_t NA_OFF_XS = na_align(NA_OFF_YW + NA_ND * NA_W * sizeof(double));
constexpr size_t NA_OFF_YS = na_align(NA_OFF_XS + NA_ND * NA_N * sizeof(double));
constexpr size_t NA_BYTES = na_align(NA_OFF_YS + NA_ND * NA_N * sizeof(double));

static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_noalloc_mutex;
unsigned char* g_noalloc_addr[NA_MAX_DEVICES] = {};   // device address of the scratch, per device
int g_noalloc_sms[NA_MAX_DEVICES] = {};

// One-time set-up on the current device: the device address of the scratch
// array (the host-side symbol is only a stand-in and must never reach a
// kernel) and the update kernel's shared-memory limit.
afqmc_status noalloc_setup(int dev, size_t smem) {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (g_noalloc_addr[dev]) return AFQMC_OK;
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr) {
        g_create_error = std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e);
        return AFQMC_E_CUDA;
    }
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = raise_smem_limit(upd_kernel(0), smem);
    int occ = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, upd_kernel(0), UPD_THREADS, smem);
    if (e != cudaSuccess || occ < 1) {
        g_create_error = std::string("update kernel set-up failed: ") + cudaGetErrorString(e);
        return AFQMC_E_CUDA;
    }
    g_noalloc_sms[dev] = sms;
    g_noalloc_addr[dev] = static_cast<unsigned char*>(ptr);
    return AFQMC_OK;
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

afqmc_status afqmc_create(const afqmc_params* p, void* cuda_stream, afqmc_handle** out) {
    if (out) *out = nullptr;
    if (!p || !out) { g_create_error = "null argument"; return AFQMC_E_INVALID; }
    const afqmc_params P = *p;
    auto bad = [&](const char* m) { g_create_error = m; return AFQMC_E_INVALID; };
    if (P.L1 < 1 || P.L2 < 1 || P.L1 > 64 || P.L2 > 64) return bad("L1, L2 must be in [1, 64]");
    if (!(P.beta > 0) || !(P.dtau > 0)) return bad("beta and dtau must be positive");
    if (!(P.U >= 0)) return bad("U must be >= 0");
    if (!(P.theta1 >= 0.0 && P.theta1 < 1.0 && P.theta2 >= 0.0 && P.theta2 < 1.0))
        return bad("twist angles theta1, theta2 must be in [0, 1)");
    if (P.hs_channel != 0 && P.hs_channel != 1)
        return bad("hs_channel must be 0 (spin channel, Eq. SzHS) or 1 (charge channel, Eq. DensityHS)");
    if (P.precision < 0 || P.precision > 7 || ((P.precision & 4) && !(P.precision & 2)))
        return bad("precision must be 0..7 (bit 0: split-TF32 flush, bit 1: tensor-core FP64-accurate stabilisation "
                   "products, bit 2: blocked solves of G on them, needs bit 1)");
    const double Mr = P.beta / P.dtau;
    const int M = (int)std::llround(Mr);
    if (M < 1 || std::fabs(M * P.dtau - P.beta) > 1e-9) return bad("beta must be an integer multiple of dtau");
    if (P.n_stab < 1 || M % P.n_stab) return bad("n_stab must divide M = beta/dtau");
    if (P.n_delay < 1 || P.n_delay > 256) return bad("n_delay must be in [1, 256]");
    if (P.update_ctas < 0) return bad("update_ctas must be >= 0");
    auto* h = new afqmc_handle();
    try {
        h->p = P;
        h->L1 = P.L1; h->L2 = P.L2; h->Nc = P.L1 * P.L2; h->Np = 2 * h->Nc; h->M = M;
        h->charge = P.hs_channel == 1 ? 1 : 0;
        h->cplx = (P.theta1 != 0.0 || P.theta2 != 0.0 || h->charge) ? 1 : 0;
        h->N = h->cplx ? 2 * h->Np : h->Np;
        h->ns = P.n_stab; h->nc = M / P.n_stab;
        // a physical flip is two rank-1 moves of the embedding when twisted
        h->nd = h->cplx ? 2 * P.n_delay : P.n_delay;
        {
            const int dd1[3] = {0, 1, 0}, dd2[3] = {0, -1, -1};   // bond displacements (Gauge-I)
            for (int e = 0; e < 3; ++e) {
                const double phi = 2.0 * M_PI * (P.theta1 * dd1[e] / P.L1 + P.theta2 * dd2[e] / P.L2);
                h->bond_ph.e[e] = make_double2(std::cos(phi), std::sin(phi));
            }
        }
        h->W = std::min(UPD_WMAX, h->N);
        h->gamma = std::acosh(std::exp(P.dtau * P.U / 2.0));     // Eq. coupling
        h->egp = std::exp(h->gamma); h->egm = std::exp(-h->gamma);
        h->dl_p = std::exp(-2.0 * h->gamma) - 1.0;  h->dl_m = std::exp(2.0 * h->gamma) - 1.0;
        h->ef_p = std::exp(2.0 * h->gamma);         h->ef_m = std::exp(-2.0 * h->gamma);
        if (h->charge) {
            // Eq. coupling, charge channel: gamma_c = i alpha, alpha = arccos(e^{-dtau U/2});
            // Delta = e^{-2 i alpha s} - 1, and the weight ratio is |r|^2 (no scalar factor)
            h->alpha = std::acos(std::exp(-P.dtau * P.U / 2.0));
            h->ca = std::cos(h->alpha); h->sa = std::sin(h->alpha);
            const double c2 = std::cos(2.0 * h->alpha), s2 = std::sin(2.0 * h->alpha);
            h->dl_p = c2 - 1.0; h->dli_p = -s2;
            h->dl_m = c2 - 1.0; h->dli_m = s2;
            h->ef_p = h->ef_m = 1.0;
        }
        h->key = sm64_mix(P.seed ^ ((uint64_t)(P.chain + 1) * 0xD1B54A32D192ED03ull));
        CK(cudaSetDevice(P.device));
        CK(cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, P.device));
        if (cuda_stream) h->stream = (cudaStream_t)cuda_stream;
        else { CK(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking)); h->own_stream = true; }
        const int N = h->N, Np = h->Np, Nc = h->Nc;
        const size_t nn = (size_t)N * N;
        // FFT plan, twiddles, propagator blocks
        FFTPlan& pl = h->plan;
        pl.N = Np; pl.Nc = Nc; pl.L1 = h->L1; pl.L2 = h->L2;
        pl.nr1 = radices(h->L1, pl.r1);
        pl.nr2 = radices(h->L2, pl.r2);
        for (int q = 0; q < pl.nr1; ++q) if (pl.r1[q] > 8) pl.nr1 = -1;
        for (int q = 0; q < pl.nr2; ++q) if (pl.r2[q] > 8) pl.nr2 = -1;
        if (pl.nr1 < 0 || pl.nr2 < 0) throw CudaFail{AFQMC_E_INVALID, "L1 and L2 must factor into primes <= 7"};
        std::vector<double2> t1(h->L1), t2(h->L2);
        for (int m = 0; m < h->L1; ++m) t1[m] = make_double2(std::cos(2 * M_PI * m / h->L1), -std::sin(2 * M_PI * m / h->L1));
        for (int m = 0; m < h->L2; ++m) t2[m] = make_double2(std::cos(2 * M_PI * m / h->L2), -std::sin(2 * M_PI * m / h->L2));
        h->tw1 = h->dalloc<double2>(h->L1);
        h->tw2 = h->dalloc<double2>(h->L2);
        CK(cudaMemcpy(h->tw1, t1.data(), sizeof(double2) * h->L1, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(h->tw2, t2.data(), sizeof(double2) * h->L2, cudaMemcpyHostToDevice));
        pl.tw1 = h->tw1; pl.tw2 = h->tw2;
        std::vector<double2> blk((size_t)4 * Nc * 4);
        const double cs[4] = {P.dtau, -P.dtau, 0.5 * P.dtau, -0.5 * P.dtau};   // e^{-c h(k)}
        for (int op = 0; op < 4; ++op)
            for (int l2 = 0; l2 < h->L2; ++l2)
                for (int l1 = 0; l1 < h->L1; ++l1) {
                    const int q = l1 + h->L1 * l2;
                    block_exp(bloch_f(P.t, l1, l2, h->L1, h->L2, P.theta1, P.theta2), cs[op],
                              &blk[((size_t)op * Nc + q) * 4]);
                }
        h->blocks = h->dalloc<double2>(blk.size());
        CK(cudaMemcpy(h->blocks, blk.data(), sizeof(double2) * blk.size(), cudaMemcpyHostToDevice));
        h->vp = std::max(1, std::min(4, (int)(48000 / (sizeof(double2) * 2 * (size_t)Np))));
        h->rowop_smem = sizeof(double2) * 2 * (size_t)h->vp * Np;
        if (h->rowop_smem > 200 * 1024) throw CudaFail{AFQMC_E_INVALID, "lattice too large for the row kernel"};
        CK(raise_smem_limit((const void*)k_rowop, h->rowop_smem));
        if (N > COL_MAX_N)
            throw CudaFail{AFQMC_E_INVALID, "matrix dimension " + std::to_string(N) + " above the column kernels' " +
                                                std::to_string(COL_MAX_N) + " (2 L1 L2, doubled with a twist or the charge channel)"};
        if (col_small(N)) {
            for (const void* f : {(const void*)k_form_q<8, 8>, (const void*)k_backsolve<8, 8>,
                                  (const void*)k_fwdsolve_perm<8, 8>})
                CK(raise_smem_limit(f, cpb_smem(N)));
        } else {
            for (const void* f : {(const void*)k_form_q<4, 16>, (const void*)k_backsolve<4, 16>,
                                  (const void*)k_fwdsolve_perm<4, 16>})
                CK(raise_smem_limit(f, cpb_smem(N)));
        }
        h->upd_grid = P.update_ctas > 0 ? P.update_ctas : h->sms;
        const size_t usmem = update_smem(h->W, h->nd, P.precision, N, h->upd_grid);
        CK(raise_smem_limit(upd_kernel(h->charge), usmem));
        int occ = 0;
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, upd_kernel(h->charge), UPD_THREADS, usmem));
        if (occ < 1) throw CudaFail{AFQMC_E_INVALID, "update kernel does not fit on an SM"};
        if (h->upd_grid > occ * h->sms) throw CudaFail{AFQMC_E_INVALID, "update_ctas exceeds the co-resident CTAs of the device"};
        {
            const int qg = std::min(h->sms, N);
            const size_t qs = sizeof(double) * (size_t)N * (1 + (N + qg - 1) / qg);
            h->qr_smem_cols = qs <= 200 * 1024;
            const size_t qsm = h->qr_smem_cols ? qs : sizeof(double) * N;
            CK(raise_smem_limit((const void*)k_qr_cols, qsm));
            CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_qr_cols, 256, qsm));
            if (occ < 1) throw CudaFail{AFQMC_E_INVALID, "QR kernel does not fit on an SM"};
            CK(raise_smem_limit((const void*)k_lu_cols, qsm));
            CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_lu_cols, 256, qsm));
            if (occ < 1) throw CudaFail{AFQMC_E_INVALID, "LU kernel does not fit on an SM"};
        }
        // state
        h->field = h->dalloc<int8_t>((size_t)M * Np);
        h->G = h->dalloc<double>(nn);
        for (auto& w : h->Wk) w = h->dalloc<double>(nn);
        h->Xs = h->dalloc<double>((size_t)h->nd * N);
        h->Ys = h->dalloc<double>((size_t)h->nd * N);
        if (P.precision & 1) {
            // K-major TF32 parts of X and Y; rows padded to a multiple of 8 moves
            // (the flush reads whole groups of 8 past the last pending move)
            h->tf_ld = (h->nd + 7) & ~7;
            for (uint32_t** t : {&h->tf_xh, &h->tf_xl, &h->tf_yh, &h->tf_yl}) {
                *t = h->dalloc<uint32_t>((size_t)N * h->tf_ld);
                CK(cudaMemset(*t, 0, sizeof(uint32_t) * (size_t)N * h->tf_ld));
            }
        }
        h->msite = h->dalloc<int>(h->nd);
        h->mcoef = h->dalloc<double>(h->nd);
        h->xw = h->dalloc<double>((size_t)h->nd * h->W);
        h->yw = h->dalloc<double>((size_t)h->nd * h->W);
        h->Gw = h->dalloc<double>((size_t)h->W * h->W);
        h->ctl = h->dalloc<int>(8);
        h->perm = h->dalloc<int>(N);
        h->vtmp = h->dalloc<double>(N);
        h->Dp = h->dalloc<double>(N);
        h->sgn = h->dalloc<double>(N);
        h->tau = h->dalloc<double>(N);
        if (P.precision & 2) {
            // the 64-bit integer sum of classes 0..3 of the product kernel adds below 2^46 per
            // exact window of K and must stay exact in FP64 (2^53) for K <= COL_MAX_N
            static_assert(((COL_MAX_N + OZ_KC * OZ_WIN - 1) / (OZ_KC * OZ_WIN)) * (1ll << 46) <= (1ll << 53),
                          "class sums of the largest lattice exceed 2^53");
            h->ozKpad = (N + OZ_KC - 1) / OZ_KC * OZ_KC;
            h->ozA = h->dalloc<__nv_bfloat16>((size_t)OZ_S * N * h->ozKpad);
            h->ozB = h->dalloc<__nv_bfloat16>((size_t)OZ_S * N * h->ozKpad);
            h->ozea = h->dalloc<int>(N);
            h->ozeb = h->dalloc<int>(N);
            if (P.precision & 4) h->lperm = h->dalloc<int>(N);
            encode_digit_planes(&h->oz_tmA, h->ozA, N, h->ozKpad, OZ_TM);
            encode_digit_planes(&h->oz_tmB, h->ozB, N, h->ozKpad, OZ_TN);
            CK(raise_smem_limit((const void*)k_oz_gemm, oz_smem_bytes()));
            int occ_oz = 0;
            CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_oz, k_oz_gemm, OZ_THREADS, oz_smem_bytes()));
            if (occ_oz < 1) throw CudaFail{AFQMC_E_INVALID, "tensor-core product kernel does not fit on an SM"};
        }
        h->DbR = h->dalloc<double>(N); h->DsR = h->dalloc<double>(N);
        h->DbL = h->dalloc<double>(N); h->DsL = h->dalloc<double>(N);
        h->pubx = h->dalloc<double>(N);
        h->piv = h->dalloc<int>(N);
        h->st = h->dalloc<DevStatus>(1);
        CK(cudaMemset(h->st, 0, sizeof(DevStatus)));
        h->n_acc = h->dalloc<unsigned long long>(1);
        h->drift = h->dalloc<unsigned long long>(1);
        h->d_sweep = h->dalloc<unsigned long long>(1);
        CK(cudaMemset(h->d_sweep, 0, sizeof(unsigned long long)));
        h->czz = h->dalloc<double>(Nc);
        h->tr2 = h->dalloc<double>((size_t)((Np + 31) / 32) * ((Np + 31) / 32));
        h->hab = h->dalloc<double>((size_t)8 * Nc);
        h->obs_now = h->dalloc<double>(OBS_SCALARS);
        h->czz_now = h->dalloc<double>(Nc);
        h->nk_now = h->dalloc<double>((size_t)8 * Nc);
        h->obs_acc = h->dalloc<double>(OBS_SCALARS);
        h->czz_acc = h->dalloc<double>(Nc);
        h->nk_acc = h->dalloc<double>((size_t)8 * Nc);
        h->obs_count = h->dalloc<long long>(1);
        CK(cudaMemset(h->obs_acc, 0, sizeof(double) * OBS_SCALARS));
        CK(cudaMemset(h->czz_acc, 0, sizeof(double) * Nc));
        CK(cudaMemset(h->nk_acc, 0, sizeof(double) * 8 * Nc));
        CK(cudaMemset(h->obs_count, 0, sizeof(long long)));
        // stacks: nc+1 entries each, plus one spare per stack for green_at
        h->Rst.resize(h->nc + 2);
        h->Lst.resize(h->nc + 2);
        for (auto* st : {&h->Rst, &h->Lst})
            for (auto& e : *st) { e.Ut = h->dalloc<double>(nn); e.T = h->dalloc<double>(nn); e.D = h->dalloc<double>(N); }
        for (auto* e : {&h->tmpA, &h->tmpB}) { e->Ut = h->dalloc<double>(nn); e->T = h->dalloc<double>(nn); e->D = h->dalloc<double>(N); }
        // initial field from the counter-based stream, then stacks and G
        { Scope sc(h, AFQMC_K_MISC); k_init_field<<<(unsigned)(((size_t)M * Np + 255) / 256), 256, 0, h->stream>>>(h->field, M, Np, h->key); }
        CK(cudaGetLastError());
        init_chain(h);
        afqmc_status s = check_device(h);
        if (s != AFQMC_OK) { g_create_error = h->err; afqmc_destroy(h); return s; }
    } catch (const CudaFail& f) {
        g_create_error = f.msg;
        afqmc_destroy(h);
        return f.code;
    } catch (const std::exception& e) {
        g_create_error = e.what();
        afqmc_destroy(h);
        return AFQMC_E_NOMEM;
    }
    *out = h;
    return AFQMC_OK;
}

afqmc_status afqmc_destroy(afqmc_handle* h) {
    if (!h) return AFQMC_OK;
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (auto& q : h->pending) { cudaEventDestroy(q.a); cudaEventDestroy(q.b); }
    for (auto e : h->ev_free) cudaEventDestroy(e);
    for (void* ptr : h->allocs) cudaFree(ptr);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
    return AFQMC_OK;
}

#define API_BEGIN(h)                                                          \
    if (!(h)) return AFQMC_E_INVALID;                                         \
    if ((h)->broken) { (h)->err = "handle unusable after an earlier CUDA, numeric or timeout error"; return AFQMC_E_STATE; } \
    try {
#define API_END(h)                                    \
    } catch (const CudaFail& f) {                     \
        set_error((h), f.code, f.msg);                \
        return f.code;                                \
    } catch (const std::exception& e) {               \
        set_error((h), AFQMC_E_NOMEM, e.what());      \
        return AFQMC_E_NOMEM;                         \
    }

afqmc_status afqmc_set_field(afqmc_handle* h, const int8_t* s, uint64_t sweep_index) {
    API_BEGIN(h)
    if (!s) { h->err = "null field"; return AFQMC_E_INVALID; }
    const size_t len = (size_t)h->M * h->Np;
    for (size_t o = 0; o < len; ++o)
        if (s[o] != 1 && s[o] != -1) { h->err = "field entries must be +1 or -1"; return AFQMC_E_INVALID; }
    CK(cudaMemcpyAsync(h->field, s, len, cudaMemcpyHostToDevice, h->stream));
    h->sweep_index = sweep_index;
    CK(cudaMemcpyAsync(h->d_sweep, &h->sweep_index, sizeof(unsigned long long), cudaMemcpyHostToDevice, h->stream));
    init_chain(h);
    return check_device(h);
    API_END(h)
}

afqmc_status afqmc_get_field(afqmc_handle* h, int8_t* s) {
    API_BEGIN(h)
    if (!s) { h->err = "null field"; return AFQMC_E_INVALID; }
    CK(cudaMemcpyAsync(s, h->field, (size_t)h->M * h->Np, cudaMemcpyDeviceToHost, h->stream));
    return check_device(h);
    API_END(h)
}

afqmc_status afqmc_sweep(afqmc_handle* h, int32_t n_sweeps, afqmc_sweep_stats* stats) {
    API_BEGIN(h)
    if (n_sweeps < 0) { h->err = "n_sweeps < 0"; return AFQMC_E_INVALID; }
    CK(cudaMemsetAsync(h->n_acc, 0, sizeof(unsigned long long), h->stream));
    CK(cudaMemsetAsync(h->drift, 0, sizeof(unsigned long long), h->stream));
    const uint64_t l0 = h->launches;
    for (int w = 0; w < n_sweeps; ++w) sweep_once(h);
    if (stats) {
        unsigned long long acc = 0, dr = 0;
        CK(cudaMemcpyAsync(&acc, h->n_acc, sizeof(acc), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaMemcpyAsync(&dr, h->drift, sizeof(dr), cudaMemcpyDeviceToHost, h->stream));
        afqmc_status s = check_device(h);
        stats->proposed = (uint64_t)n_sweeps * 2ull * (uint64_t)h->Np * (uint64_t)h->M;
        stats->accepted = h->cplx ? acc / 2 : acc;       // two moves per flip when twisted
        double d;
        std::memcpy(&d, &dr, sizeof(d));
        stats->max_stab_drift = d;
        stats->launches = h->launches - l0;
        return s;
    }
    return check_device(h);
    API_END(h)
}

static void fill_obs(const double* v, long long n, afqmc_obs* out) {
    out->energy = v[0]; out->double_occ = v[1]; out->ekin = v[2]; out->density = v[3];
    out->m2 = v[4]; out->S_af = v[5]; out->S_af_dk = v[6]; out->R_m2 = v[7]; out->Czz_half = v[8];
    out->chi_e = v[9];
    out->n_samples = n;
}

afqmc_status afqmc_measure(afqmc_handle* h, afqmc_obs* out, double* Czz, double* nk) {
    API_BEGIN(h)
    if (!out) { h->err = "null output"; return AFQMC_E_INVALID; }
    measure(h, h->G, false);
    double v[OBS_SCALARS];
    CK(cudaMemcpyAsync(v, h->obs_now, sizeof(v), cudaMemcpyDeviceToHost, h->stream));
    if (Czz) CK(cudaMemcpyAsync(Czz, h->czz_now, sizeof(double) * h->Nc, cudaMemcpyDeviceToHost, h->stream));
    if (nk) CK(cudaMemcpyAsync(nk, h->nk_now, sizeof(double) * 8 * h->Nc, cudaMemcpyDeviceToHost, h->stream));
    afqmc_status s = check_device(h);
    fill_obs(v, 1, out);
    return s;
    API_END(h)
}

afqmc_status afqmc_get_obs(afqmc_handle* h, afqmc_obs* out, double* Czz, double* nk) {
    API_BEGIN(h)
    if (!out) { h->err = "null output"; return AFQMC_E_INVALID; }
    double v[OBS_SCALARS];
    long long n = 0;
    std::vector<double> cz(h->Nc), nkv((size_t)8 * h->Nc);
    CK(cudaMemcpyAsync(v, h->obs_acc, sizeof(v), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(&n, h->obs_count, sizeof(n), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(cz.data(), h->czz_acc, sizeof(double) * h->Nc, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(nkv.data(), h->nk_acc, sizeof(double) * 8 * h->Nc, cudaMemcpyDeviceToHost, h->stream));
    afqmc_status s = check_device(h);
    if (s != AFQMC_OK) return s;
    const double inv = n > 0 ? 1.0 / (double)n : 0.0;
    for (double& x : v) x *= inv;
    // Eq. CrfRatio on expectation values: the ratio of the averaged structure factors
    v[7] = (n > 0 && v[5] != 0.0) ? 1.0 - v[6] / v[5] : 0.0;
    fill_obs(v, n, out);
    if (Czz) for (int d = 0; d < h->Nc; ++d) Czz[d] = cz[d] * inv;
    if (nk) for (size_t q = 0; q < nkv.size(); ++q) nk[q] = nkv[q] * inv;
    CK(cudaMemsetAsync(h->obs_acc, 0, sizeof(double) * OBS_SCALARS, h->stream));
    CK(cudaMemsetAsync(h->czz_acc, 0, sizeof(double) * h->Nc, h->stream));
    CK(cudaMemsetAsync(h->nk_acc, 0, sizeof(double) * 8 * h->Nc, h->stream));
    CK(cudaMemsetAsync(h->obs_count, 0, sizeof(long long), h->stream));
    return check_device(h);
    API_END(h)
}

afqmc_status afqmc_get_G(afqmc_handle* h, int32_t slice, double* out) {
    API_BEGIN(h)
    if (!out || slice < 0 || slice > h->M) { h->err = "bad slice or null output"; return AFQMC_E_INVALID; }
    double* dst = h->Wk[5];
    green_at(h, slice, dst);
    to_host(h, dst, out, h->Wk[4]);
    return check_device(h);
    API_END(h)
}

afqmc_status afqmc_wrap_matrix(afqmc_handle* h, int32_t slice, int32_t direction, double* A) {
    API_BEGIN(h)
    if (!A || slice < 1 || slice > h->M || direction < -1 || direction > 1) { h->err = "bad arguments"; return AFQMC_E_INVALID; }
    double* d = h->Wk[3];
    from_host(h, A, d, h->Wk[2]);
    double* res = d;
    if (direction == 0) {
        half_step(h, d, h->Wk[5]);
        res = h->Wk[5];
    } else {
        wrap(h, d, slice, direction);
    }
    // a non-finite input propagates through the transforms: report it
    { Scope sc(h, AFQMC_K_MISC); k_check_finite<<<h->sms * 2, 256, 0, h->stream>>>(res, (size_t)h->N * h->N, h->st, 106); }
    CK(cudaGetLastError());
    to_host(h, res, A, h->Wk[2]);
    return check_device(h);
    API_END(h)
}

afqmc_status afqmc_update_slice(afqmc_handle* h, int32_t slice, int32_t pass, uint64_t sweep_index, double* G,
                                int32_t* n_accepted) {
    API_BEGIN(h)
    if (!G || slice < 1 || slice > h->M || (pass != 0 && pass != 1)) { h->err = "bad arguments"; return AFQMC_E_INVALID; }
    double* d = h->Wk[5];
    from_host(h, G, d, h->Wk[4]);
    CK(cudaMemsetAsync(h->n_acc, 0, sizeof(unsigned long long), h->stream));
    update_slice(h, d, slice, pass, (int64_t)sweep_index);
    unsigned long long acc = 0;
    to_host(h, d, G, h->Wk[4]);
    CK(cudaMemcpyAsync(&acc, h->n_acc, sizeof(acc), cudaMemcpyDeviceToHost, h->stream));
    afqmc_status s = check_device(h);
    if (n_accepted) *n_accepted = (int32_t)(h->cplx ? acc / 2 : acc);
    return s;
    API_END(h)
}

afqmc_status afqmc_det_ratio(afqmc_handle* h, int32_t slice, int32_t site, double out[3]) {
    API_BEGIN(h)
    if (!out || slice < 1 || slice > h->M || site < 0 || site >= h->Np) { h->err = "bad arguments"; return AFQMC_E_INVALID; }
    double* g = h->Wk[5];
    green_at(h, slice, g);
    int8_t sv = 0;
    CK(cudaMemcpyAsync(&sv, h->field + (size_t)(slice - 1) * h->Np + site, 1, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    double* o = h->vtmp;
    const GView gv{g, h->Np, h->N, h->cplx};
    { Scope sc(h, AFQMC_K_MISC); k_ratio<<<1, 1, 0, h->stream>>>(gv, site, sv, h->dl_p, h->dl_m, h->dli_p, h->dli_m, h->ef_p, h->ef_m, o); }
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(out, o, 3 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    return check_device(h);
    API_END(h)
}

afqmc_status afqmc_measure_td(afqmc_handle* h) {
    API_BEGIN(h)
    if (h->M % 2) { h->err = "the time-displaced measurement needs an even number of slices (tau up to beta/2)"; return AFQMC_E_INVALID; }
    td_measure(h);
    return check_device(h);
    API_END(h)
}

afqmc_status afqmc_get_td(afqmc_handle* h, double* C, double* dDdU, double* chiF, int64_t* n_samples) {
    API_BEGIN(h)
    const int nl = h->M / 2 + 1;
    std::vector<double> hh(nl, 0.0);
    double h1 = 0.0;
    const long long n = h->td_count;
    if (h->td_hh && n > 0) {
        CK(cudaMemcpyAsync(hh.data(), h->td_hh, sizeof(double) * nl, cudaMemcpyDeviceToHost, h->stream));
        CK(cudaMemcpyAsync(&h1, h->td_h, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        afqmc_status s = check_device(h);
        if (s != AFQMC_OK) return s;
    }
    // C(tau) = <H_I(tau) H_I(0)> - <H_I>^2 over the measured fields; trapezoidal integrals
    // dD/dU = -(2/N) int_0^{beta/2} C, chi_F = int_0^{beta/2} tau C (Eqs. DouOccDerive, fidelitysusp)
    const double inv = n > 0 ? 1.0 / (double)n : 0.0, hm = h1 * inv;
    double i0 = 0.0, i1 = 0.0;
    for (int l = 0; l < nl; ++l) {
        const double c = hh[l] * inv - hm * hm;
        if (C) C[l] = c;
        const double w = (l == 0 || l == nl - 1) ? 0.5 : 1.0;
        i0 += w * c;
        i1 += w * c * (l * h->p.dtau);
    }
    if (dDdU) *dDdU = -2.0 / h->Np * h->p.dtau * i0;
    if (chiF) *chiF = h->p.dtau * i1;
    if (n_samples) *n_samples = n;
    if (h->td_hh) {
        CK(cudaMemsetAsync(h->td_hh, 0, sizeof(double) * nl, h->stream));
        CK(cudaMemsetAsync(h->td_h, 0, sizeof(double), h->stream));
    }
    h->td_count = 0;
    return check_device(h);
    API_END(h)
}

afqmc_status afqmc_set_wait_limit(afqmc_handle* h, uint64_t wait_ns) {
    API_BEGIN(h)
    unsigned long long w = wait_ns;
    CK(cudaMemcpyAsync(reinterpret_cast<char*>(h->st) + offsetof(DevStatus, wait_ns), &w, sizeof(w),
                       cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return AFQMC_OK;
    API_END(h)
}

afqmc_status afqmc_set_timing(afqmc_handle* h, int32_t family_mask) {
    API_BEGIN(h)
    if (h->in_batch && family_mask) { h->err = "per-launch timing is not available on batch chains"; return AFQMC_E_INVALID; }
    if (family_mask < 0 || family_mask > AFQMC_TIMING_ALL) { h->err = "timing mask outside the kernel families"; return AFQMC_E_INVALID; }
    flush_timing(h);
    h->timing = family_mask;
    for (int c = 0; c < AFQMC_K_COUNT; ++c) { h->cat_launches[c] = 0; h->cat_ms[c] = 0.0; }
    return AFQMC_OK;
    API_END(h)
}

afqmc_status afqmc_get_timing(afqmc_handle* h, afqmc_timing* out) {
    API_BEGIN(h)
    if (!out) { h->err = "null output"; return AFQMC_E_INVALID; }
    flush_timing(h);
    for (int c = 0; c < AFQMC_K_COUNT; ++c) { out->launches[c] = h->cat_launches[c]; out->ms[c] = h->cat_ms[c]; }
    return check_device(h);
    API_END(h)
}

afqmc_status afqmc_update_slice_noalloc(double* G_dev, int8_t* s_dev, int32_t N, int32_t M, int32_t slice,
                                        int32_t pass, uint64_t sweep_index, double U, double dtau,
                                        int32_t n_delay, uint64_t seed, int32_t chain, void* cuda_stream,
                                        int32_t* n_accepted) {
    if (n_accepted) *n_accepted = 0;
    auto bad = [](const std::string& m) { g_create_error = m; return AFQMC_E_INVALID; };
    if (!G_dev || !s_dev) return bad("afqmc_update_slice_noalloc: null device pointer");
    if (N < 2 || N > (int32_t)NA_N)
        return bad("afqmc_update_slice_noalloc: N = " + std::to_string(N) + " outside [2, " + std::to_string(NA_N) + "]");
    if (n_delay < 1 || n_delay > (int32_t)NA_ND)
        return bad("afqmc_update_slice_noalloc: n_delay = " + std::to_string(n_delay) + " outside [1, " +
                   std::to_string(NA_ND) + "]");
    if (M < 1 || slice < 1 || slice > M || (pass != 0 && pass != 1) || !(dtau > 0) || !(U >= 0))
        return bad("afqmc_update_slice_noalloc: bad slice, pass, M, U or dtau");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) {
        g_create_error = std::string("afqmc_update_slice_noalloc: cudaGetDevice: ") + cudaGetErrorString(e);
        return AFQMC_E_CUDA;
    }
    const int W = std::min<int>(UPD_WMAX, N);
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess || sms < 1) {
        g_create_error = std::string("afqmc_update_slice_noalloc: SM count: ") + cudaGetErrorString(e);
        return AFQMC_E_CUDA;
    }
    const size_t smem = update_smem(W, n_delay, 0, N, sms);
    const size_t smem_max = update_smem((int)NA_W, (int)NA_ND, 0, (int)NA_N, sms);
    afqmc_status st0 = noalloc_setup(dev, smem_max);
    if (st0 != AFQMC_OK) return st0;
    unsigned char* base = g_noalloc_addr[dev];
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    const double gamma = std::acosh(std::exp(dtau * U / 2.0));
    UpdArgs a{};
    a.G = G_dev; a.N = N; a.Np = N; a.pair = 0;
    a.Xs = reinterpret_cast<double*>(base + NA_OFF_XS);
    a.Ys = reinterpret_cast<double*>(base + NA_OFF_YS);
    a.msite = reinterpret_cast<int*>(base + NA_OFF_SITE);
    a.mcoef = reinterpret_cast<double*>(base + NA_OFF_COEF);
    a.xw = reinterpret_cast<double*>(base + NA_OFF_XW);
    a.yw = reinterpret_cast<double*>(base + NA_OFF_YW);
    a.Gw = reinterpret_cast<double*>(base + NA_OFF_GW);
    a.ctl = reinterpret_cast<int*>(base + NA_OFF_CTL);
    a.s = s_dev;
    a.nd = n_delay; a.W = W;
    a.dl_p = std::exp(-2.0 * gamma) - 1.0; a.dl_m = std::exp(2.0 * gamma) - 1.0;
    a.ef_p = std::exp(2.0 * gamma);        a.ef_m = std::exp(-2.0 * gamma);
    a.key = sm64_mix(seed ^ ((uint64_t)(chain + 1) * 0xD1B54A32D192ED03ull));
    a.ctr0 = ((sweep_index * 2 + (uint64_t)pass) * (uint64_t)M + (uint64_t)(slice - 1)) * (uint64_t)N + 1;
    a.n_acc = reinterpret_cast<unsigned long long*>(base + NA_OFF_ACC);
    a.st = reinterpret_cast<DevStatus*>(base + NA_OFF_STATUS);
    // the scratch keeps the previous call's contents: clear the status, the
    // grid-barrier counter and the accepted count (everything else is written
    // before it is read within a call)
    e = cudaMemsetAsync(base, 0, NA_OFF_CTL, stream);
    void* args[] = {&a};
    if (e == cudaSuccess)
        e = cudaLaunchCooperativeKernel(upd_kernel(0), g_noalloc_sms[dev], UPD_THREADS, args, smem, stream);
    DevStatus ds{};
    unsigned long long acc = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ds, a.st, sizeof(ds), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&acc, a.n_acc, sizeof(acc), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
        g_create_error = std::string("afqmc_update_slice_noalloc: ") + cudaGetErrorString(e);
        return AFQMC_E_CUDA;
    }
    if (ds.err == DERR_NUMERIC) { g_create_error = "afqmc_update_slice_noalloc: non-finite ratio"; return AFQMC_E_NUMERIC; }
    if (ds.err == DERR_TIMEOUT) { g_create_error = "afqmc_update_slice_noalloc: device wait timed out"; return AFQMC_E_TIMEOUT; }
    if (ds.err != 0) { g_create_error = "afqmc_update_slice_noalloc: device error"; return AFQMC_E_CUDA; }
    if (n_accepted) *n_accepted = (int32_t)acc;
    return AFQMC_OK;
}

}  // extern "C"

// ====================================================================== batches
struct afqmc_batch {
    std::vector<afqmc_handle*> chains;
    cudaStream_t stream = nullptr;          // the graph is launched here
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint64_t launches_per_sweep = 0;
    std::string err;
};

namespace {

thread_local std::string g_batch_error;

void batch_free(afqmc_batch* b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (auto e : b->join) if (e) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    for (auto* h : b->chains) afqmc_destroy(h);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

// One sweep of every chain captured into one graph: fork from the batch
// stream to every chain's stream, each chain's launch sequence on its own
// branch, join back.
void batch_capture(afqmc_batch* b) {
    CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    uint64_t l0 = 0;
    try {
        CK(cudaEventRecord(b->fork, b->stream));
        for (size_t i = 0; i < b->chains.size(); ++i) {
            afqmc_handle* h = b->chains[i];
            CK(cudaStreamWaitEvent(h->stream, b->fork, 0));
            l0 = h->launches;
            sweep_once(h);
            b->launches_per_sweep += h->launches - l0;
            h->sweep_index -= 1;              // advanced on every replay instead
            CK(cudaEventRecord(b->join[i], h->stream));
            CK(cudaStreamWaitEvent(b->stream, b->join[i], 0));
        }
    } catch (...) {
        cudaGraph_t g = nullptr;
        cudaStreamEndCapture(b->stream, &g);
        if (g) cudaGraphDestroy(g);
        b->launches_per_sweep = 0;
        throw;
    }
    CK(cudaStreamEndCapture(b->stream, &b->graph));
    CK(cudaGraphInstantiate(&b->exec, b->graph, 0));
}

afqmc_status batch_sweep_impl(afqmc_batch* b, int32_t n_sweeps, afqmc_sweep_stats* total) {
    for (auto* h : b->chains) {
        if (h->broken) { b->err = "chain unusable after an earlier error: " + h->err; return AFQMC_E_STATE; }
        CK(cudaStreamSynchronize(h->stream));     // work issued on the chain's own stream comes first
        CK(cudaMemsetAsync(h->n_acc, 0, sizeof(unsigned long long), b->stream));
        CK(cudaMemsetAsync(h->drift, 0, sizeof(unsigned long long), b->stream));
    }
    if (!b->exec && n_sweeps > 0) batch_capture(b);
    for (int w = 0; w < n_sweeps; ++w) {
        CK(cudaGraphLaunch(b->exec, b->stream));
        for (auto* h : b->chains) h->sweep_index += 1;
    }
    std::vector<unsigned long long> acc(b->chains.size()), dr(b->chains.size());
    for (size_t i = 0; i < b->chains.size(); ++i) {
        CK(cudaMemcpyAsync(&acc[i], b->chains[i]->n_acc, sizeof(unsigned long long), cudaMemcpyDeviceToHost, b->stream));
        CK(cudaMemcpyAsync(&dr[i], b->chains[i]->drift, sizeof(unsigned long long), cudaMemcpyDeviceToHost, b->stream));
    }
    CK(cudaStreamSynchronize(b->stream));
    afqmc_status worst = AFQMC_OK;
    afqmc_sweep_stats t{};
    for (size_t i = 0; i < b->chains.size(); ++i) {
        afqmc_handle* h = b->chains[i];
        afqmc_status s = check_device(h);
        if (s != AFQMC_OK && worst == AFQMC_OK) { worst = s; b->err = "chain " + std::to_string(i) + ": " + h->err; }
        t.proposed += (uint64_t)n_sweeps * 2ull * (uint64_t)h->Np * (uint64_t)h->M;
        t.accepted += h->cplx ? acc[i] / 2 : acc[i];
        double d;
        std::memcpy(&d, &dr[i], sizeof(d));
        t.max_stab_drift = std::max(t.max_stab_drift, d);
    }
    t.launches = (uint64_t)n_sweeps * b->launches_per_sweep;
    if (total) *total = t;
    return worst;
}

}  // namespace

extern "C" {

afqmc_status afqmc_batch_create(const afqmc_params* params, int32_t n, afqmc_batch** out) {
    if (out) *out = nullptr;
    if (!params || !out || n < 1) { g_batch_error = "null argument or n < 1"; return AFQMC_E_INVALID; }
    for (int i = 1; i < n; ++i)
        if (params[i].device != params[0].device) { g_batch_error = "all chains of a batch must use one device"; return AFQMC_E_INVALID; }
    auto* b = new afqmc_batch();
    try {
        CK(cudaSetDevice(params[0].device));
        CK(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
        for (int i = 0; i < n; ++i) {
            afqmc_handle* h = nullptr;
            afqmc_status s = afqmc_create(&params[i], nullptr, &h);
            if (s != AFQMC_OK) {
                g_batch_error = "chain " + std::to_string(i) + ": " + g_create_error;
                batch_free(b);
                return s;
            }
            h->in_batch = true;
            b->chains.push_back(h);
            cudaEvent_t e;
            CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            b->join.push_back(e);
        }
    } catch (const CudaFail& f) {
        g_batch_error = f.msg;
        batch_free(b);
        return f.code;
    }
    *out = b;
    return AFQMC_OK;
}

afqmc_status afqmc_batch_destroy(afqmc_batch* b) {
    batch_free(b);
    return AFQMC_OK;
}

afqmc_status afqmc_batch_sweep(afqmc_batch* b, int32_t n_sweeps, afqmc_sweep_stats* total) {
    if (!b) return AFQMC_E_INVALID;
    if (n_sweeps < 0) { b->err = "n_sweeps < 0"; return AFQMC_E_INVALID; }
    try {
        return batch_sweep_impl(b, n_sweeps, total);
    } catch (const CudaFail& f) {
        b->err = f.msg;
        for (auto* h : b->chains) set_error(h, f.code, f.msg);
        return f.code;
    }
}

afqmc_handle* afqmc_batch_chain(afqmc_batch* b, int32_t i) {
    if (!b || i < 0 || i >= (int32_t)b->chains.size()) return nullptr;
    return b->chains[i];
}

afqmc_status afqmc_batch_autotune(const afqmc_params* params, int32_t n, const int32_t* n_delays, int32_t n_nd,
                                  const int32_t* ctas, int32_t n_ctas, int32_t n_timed, int32_t* best_n_delay,
                                  int32_t* best_ctas, double* best_rate) {
    if (!params || n < 1 || !n_delays || n_nd < 1 || !ctas || n_ctas < 1 || n_timed < 1) {
        g_batch_error = "bad autotune arguments";
        return AFQMC_E_INVALID;
    }
    std::vector<afqmc_params> ps(params, params + n);
    double best = -1.0;
    int bn = 0, bc = 0;
    for (int a = 0; a < n_nd; ++a)
        for (int c = 0; c < n_ctas; ++c) {
            for (auto& p : ps) { p.n_delay = n_delays[a]; p.update_ctas = ctas[c]; }
            afqmc_batch* b = nullptr;
            afqmc_status s = afqmc_batch_create(ps.data(), n, &b);
            if (s != AFQMC_OK) return s;
            afqmc_sweep_stats st{};
            s = afqmc_batch_sweep(b, 1, &st);
            cudaEvent_t e0 = nullptr, e1 = nullptr;
            float ms = 0.0f;
            if (s == AFQMC_OK) {
                cudaEventCreate(&e0);
                cudaEventCreate(&e1);
                cudaEventRecord(e0, b->stream);
                s = afqmc_batch_sweep(b, n_timed, &st);
                cudaEventRecord(e1, b->stream);
                cudaEventSynchronize(e1);
                cudaEventElapsedTime(&ms, e0, e1);
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
            }
            if (s != AFQMC_OK) {
                g_batch_error = "candidate (n_delay " + std::to_string(n_delays[a]) + ", ctas " +
                                std::to_string(ctas[c]) + "): " + b->err;
                batch_free(b);
                return s;
            }
            const double rate = (double)st.proposed / (ms * 1e-3);
            if (rate > best) { best = rate; bn = n_delays[a]; bc = ctas[c]; }
            batch_free(b);
        }
    if (best_n_delay) *best_n_delay = bn;
    if (best_ctas) *best_ctas = bc;
    if (best_rate) *best_rate = best;
    return AFQMC_OK;
}

const char* afqmc_batch_last_error(const afqmc_batch* b) {
    return b ? b->err.c_str() : g_batch_error.c_str();
}

}  // extern "C"

// ====================================================================== learned block proposals
struct afqmc_net {
    int device = 0;
    int b = 0, T = 0, h = 0, ht = 0, W = 0;
    int d_in = 0, d_hid = 0, d_out = 0, n_par = 0;
    float *P = nullptr, *m = nullptr, *v = nullptr, *G = nullptr;
    int step = 0;
    cudaStream_t stream = nullptr;
    // training scratch (grown on demand)
    float *X = nullptr, *S = nullptr, *Hd = nullptr, *Z = nullptr, *dZ = nullptr, *dA = nullptr;
    int* pos = nullptr;
    double* loss = nullptr;
    int cap_B = 0;
    int8_t* fields = nullptr;
    size_t cap_fields = 0;
    std::string err;
    std::vector<void*> allocs;
    template <class T_>
    T_* dalloc(size_t n) {
        void* ptr = nullptr;
        cudaError_t e = cudaMalloc(&ptr, n * sizeof(T_) > 0 ? n * sizeof(T_) : 16);
        if (e != cudaSuccess) throw CudaFail{AFQMC_E_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e)};
        allocs.push_back(ptr);
        return static_cast<T_*>(ptr);
    }
    void dfree(void* ptr) {
        for (auto& a : allocs) if (a == ptr) { cudaFree(a); a = nullptr; }
    }
};

namespace {

thread_local std::string g_net_error;

BlockGeom geom_of(const afqmc_net* n, int L1, int L2, int M) {
    BlockGeom g{};
    g.L1 = L1; g.L2 = L2; g.Nc = L1 * L2; g.Np = 2 * L1 * L2; g.M = M;
    g.b = n->b; g.T = n->T; g.h = n->h; g.ht = n->ht; g.W = n->W;
    g.d_in = n->d_in; g.d_out = n->d_out; g.d_hid = n->d_hid;
    return g;
}

void net_reserve(afqmc_net* n, int B) {
    if (B <= n->cap_B) return;
    for (void* ptr : {(void*)n->X, (void*)n->S, (void*)n->Hd, (void*)n->Z, (void*)n->dZ, (void*)n->dA, (void*)n->pos})
        if (ptr) n->dfree(ptr);
    n->X = n->dalloc<float>((size_t)B * n->d_in);
    n->S = n->dalloc<float>((size_t)B * n->d_out);
    n->Hd = n->dalloc<float>((size_t)B * n->d_hid);
    n->Z = n->dalloc<float>((size_t)B * n->d_out);
    n->dZ = n->dalloc<float>((size_t)B * n->d_out);
    n->dA = n->dalloc<float>((size_t)B * n->d_hid);
    n->pos = n->dalloc<int>((size_t)4 * B);
    n->cap_B = B;
}

unsigned grid_of(size_t work, int threads = 256) { return (unsigned)((work + threads - 1) / threads); }

// Z = net(X) for B contexts already on the device (stream s)
void net_forward_dev(afqmc_net* n, const float* X, int B, float* Hd, float* Z, cudaStream_t s) {
    k_mlp_hidden<<<grid_of((size_t)B * n->d_hid), 256, 0, s>>>(n->P, X, B, n->d_in, n->d_hid, Hd);
    k_mlp_out<<<grid_of((size_t)B * n->d_out), 256, 0, s>>>(n->P, Hd, B, n->d_in, n->d_hid, n->d_out, Z);
    CK(cudaGetLastError());
}

// gradient of the mean loss into n->G, loss added to n->loss (n->X, n->S hold the batch)
void net_gradient_dev(afqmc_net* n, int B) {
    cudaStream_t s = n->stream;
    net_forward_dev(n, n->X, B, n->Hd, n->Z, s);
    k_mlp_dz<<<std::min(grid_of((size_t)B * n->d_out), 1024u), 256, 0, s>>>(n->Z, n->S, B, n->d_out, n->dZ, n->loss);
    k_mlp_grad_out<<<grid_of((size_t)n->d_out * n->d_hid + n->d_out), 256, 0, s>>>(n->dZ, n->Hd, B, n->d_in, n->d_hid,
                                                                                  n->d_out, n->G);
    k_mlp_dA<<<grid_of((size_t)B * n->d_hid), 256, 0, s>>>(n->P, n->dZ, n->Hd, B, n->d_in, n->d_hid, n->d_out, n->dA);
    k_mlp_grad_hidden<<<grid_of((size_t)n->d_hid * n->d_in + n->d_hid), 256, 0, s>>>(n->dA, n->X, B, n->d_in,
                                                                                     n->d_hid, n->G);
    CK(cudaGetLastError());
}

// Per-handle buffers of the block pass, sized for this network.
void block_reserve(afqmc_handle* h, const afqmc_net* n) {
    if (!h->Gsave) {
        h->Gsave = h->dalloc<double>((size_t)h->N * h->N);
        h->logR = h->dalloc<double>(1);
        h->lq = h->dalloc<double>(2);
        h->bflag = h->dalloc<int>(1);
        h->bstats = h->dalloc<unsigned long long>(3);
        h->bpos = h->dalloc<int>(4);
    }
    if ((size_t)n->T > h->bcap_T) {
        h->fsave = h->dalloc<int8_t>((size_t)n->T * h->Np);
        h->bmask = h->dalloc<int8_t>((size_t)n->T * h->Np);
        h->bcap_T = n->T;
    }
    if ((size_t)n->d_in > h->bcap_in) { h->bX = h->dalloc<float>(n->d_in); h->bcap_in = n->d_in; }
    if ((size_t)n->d_hid > h->bcap_hid) { h->bH = h->dalloc<float>(n->d_hid); h->bcap_hid = n->d_hid; }
    if ((size_t)n->d_out > h->bcap_out) { h->bZ = h->dalloc<float>(n->d_out); h->bcap_out = n->d_out; }
}

// One block move at window l0, offset (o1, o2); G enters and leaves at slice l0 - 1.
void block_move(afqmc_handle* h, afqmc_net* n, const BlockGeom& g, int l0, int o1, int o2, uint64_t ctr) {
    const size_t nn = (size_t)h->N * h->N, nf = (size_t)n->T * h->Np;
    int8_t* fwin = h->field + (size_t)(l0 - 1) * h->Np;
    CK(cudaMemcpyAsync(h->Gsave, h->G, sizeof(double) * nn, cudaMemcpyDeviceToDevice, h->stream));
    CK(cudaMemcpyAsync(h->fsave, fwin, nf, cudaMemcpyDeviceToDevice, h->stream));
    CK(cudaMemsetAsync(h->bmask, 0, nf, h->stream));
    CK(cudaMemsetAsync(h->logR, 0, sizeof(double), h->stream));
    {
        Scope sc(h, AFQMC_K_MISC);
        k_block_inputs<<<1, 256, 0, h->stream>>>(h->field, 0, nullptr, g, h->bX, nullptr, l0, o1, o2);
        net_forward_dev(n, h->bX, 1, h->bH, h->bZ, h->stream);
        k_block_propose<<<1, 256, 0, h->stream>>>(h->bZ, h->field, g, l0, o1, o2, h->key, ctr, h->bmask, h->lq);
    }
    CK(cudaGetLastError());
    h->launches += 3;                                   // inputs + two network layers + proposal in one scope
    h->cat_launches[AFQMC_K_MISC] += 3;
    for (int t = 0; t < n->T; ++t) {
        wrap(h, h->G, l0 + t, +1);
        update_slice(h, h->G, l0 + t, 0, 0, h->bmask + (size_t)t * h->Np, h->logR);
    }
    { Scope sc(h, AFQMC_K_MISC);
      k_block_accept<<<1, 256, 0, h->stream>>>(h->logR, h->lq, h->bmask, (int)nf, h->key, ctr + n->d_out, h->bflag,
                                                h->bstats, h->st); }
    CK(cudaGetLastError());
    for (int t = n->T - 1; t >= 0; --t) wrap(h, h->G, l0 + t, -1);
    { Scope sc(h, AFQMC_K_MISC);
      k_block_restore<<<h->sms * 2, 256, 0, h->stream>>>(h->bflag, h->Gsave, h->G, nn, h->fsave, fwin, nf); }
    CK(cudaGetLastError());
}

void block_pass(afqmc_handle* h, afqmc_net* n) {
    const BlockGeom g = geom_of(n, h->L1, h->L2, h->M);
    const int nwin = h->M / n->T, np1 = h->L1 / n->b, np2 = h->L2 / n->b;
    const uint64_t base = (3ull << 62) + h->block_passes * (uint64_t)nwin * np1 * np2 * (uint64_t)(n->d_out + 1);
    for (int w = 0; w < nwin; ++w) {
        const int l0 = w * n->T + 1;
        for (int p2 = 0; p2 < np2; ++p2)
            for (int p1 = 0; p1 < np1; ++p1) {
                const uint64_t ctr = base + ((uint64_t)(w * np2 + p2) * np1 + p1) * (uint64_t)(n->d_out + 1);
                block_move(h, n, g, l0, p1 * n->b, p2 * n->b, ctr);
            }
        for (int t = 0; t < n->T; ++t) wrap(h, h->G, l0 + t, +1);
        const int lend = l0 + n->T - 1;
        if (lend % h->ns == 0) {
            const int c = lend / h->ns;
            udt_extend(h, h->Rst[c - 1], h->Rst[c], (c - 1) * h->ns + 1, c * h->ns, true);
            recompute(h, c);
        }
    }
    // the fields changed: rebuild the L stacks and G at slice 0
    init_chain(h);
    h->block_passes += 1;
}

}  // namespace

extern "C" {

afqmc_status afqmc_net_create(int32_t b, int32_t T, int32_t hc, int32_t ht, int32_t hidden, uint64_t seed,
                              int32_t device, afqmc_net** out) {
    if (out) *out = nullptr;
    if (!out || b < 1 || T < 1 || hc < 0 || ht < 0 || hidden < 1 || hidden > 4096) {
        g_net_error = "bad network shape";
        return AFQMC_E_INVALID;
    }
    auto* n = new afqmc_net();
    try {
        n->device = device;
        n->b = b; n->T = T; n->h = hc; n->ht = ht; n->W = b + 2 * hc;
        n->d_in = (T + 2 * ht) * n->W * n->W * 2;
        n->d_hid = hidden;
        n->d_out = T * b * b * 2;
        n->n_par = n->d_hid * n->d_in + n->d_hid + n->d_out * n->d_hid + n->d_out;
        CK(cudaSetDevice(device));
        CK(cudaStreamCreateWithFlags(&n->stream, cudaStreamNonBlocking));
        n->P = n->dalloc<float>(n->n_par);
        n->m = n->dalloc<float>(n->n_par);
        n->v = n->dalloc<float>(n->n_par);
        n->G = n->dalloc<float>(n->n_par);
        n->loss = n->dalloc<double>(1);
        // W1 ~ N(0, 1/Din), W2 ~ N(0, 0.01/H), biases 0 (seeded host generator)
        std::mt19937_64 gen(seed);
        std::normal_distribution<float> nd(0.0f, 1.0f);
        std::vector<float> p(n->n_par, 0.0f);
        const float s1 = 1.0f / std::sqrt((float)n->d_in), s2 = 0.1f / std::sqrt((float)n->d_hid);
        for (int o = 0; o < n->d_hid * n->d_in; ++o) p[o] = nd(gen) * s1;
        const int w2 = n->d_hid * n->d_in + n->d_hid;
        for (int o = 0; o < n->d_out * n->d_hid; ++o) p[w2 + o] = nd(gen) * s2;
        CK(cudaMemcpy(n->P, p.data(), sizeof(float) * n->n_par, cudaMemcpyHostToDevice));
        CK(cudaMemset(n->m, 0, sizeof(float) * n->n_par));
        CK(cudaMemset(n->v, 0, sizeof(float) * n->n_par));
    } catch (const CudaFail& f) {
        g_net_error = f.msg;
        afqmc_net_destroy(n);
        return f.code;
    }
    *out = n;
    return AFQMC_OK;
}

afqmc_status afqmc_net_destroy(afqmc_net* n) {
    if (!n) return AFQMC_OK;
    if (n->stream) cudaStreamSynchronize(n->stream);
    for (void* ptr : n->allocs) if (ptr) cudaFree(ptr);
    if (n->stream) cudaStreamDestroy(n->stream);
    delete n;
    return AFQMC_OK;
}

afqmc_status afqmc_net_dims(const afqmc_net* n, int32_t dims[4]) {
    if (!n || !dims) return AFQMC_E_INVALID;
    dims[0] = n->d_in; dims[1] = n->d_hid; dims[2] = n->d_out; dims[3] = n->n_par;
    return AFQMC_OK;
}

#define NET_BEGIN(n)   if (!(n)) return AFQMC_E_INVALID; try {
#define NET_END(n)     } catch (const CudaFail& f) { (n)->err = f.msg; return f.code; }

afqmc_status afqmc_net_get_params(afqmc_net* n, float* host) {
    NET_BEGIN(n)
    if (!host) { n->err = "null output"; return AFQMC_E_INVALID; }
    CK(cudaMemcpyAsync(host, n->P, sizeof(float) * n->n_par, cudaMemcpyDeviceToHost, n->stream));
    CK(cudaStreamSynchronize(n->stream));
    return AFQMC_OK;
    NET_END(n)
}

afqmc_status afqmc_net_set_params(afqmc_net* n, const float* host) {
    NET_BEGIN(n)
    if (!host) { n->err = "null input"; return AFQMC_E_INVALID; }
    CK(cudaMemcpyAsync(n->P, host, sizeof(float) * n->n_par, cudaMemcpyHostToDevice, n->stream));
    CK(cudaMemsetAsync(n->m, 0, sizeof(float) * n->n_par, n->stream));
    CK(cudaMemsetAsync(n->v, 0, sizeof(float) * n->n_par, n->stream));
    n->step = 0;
    CK(cudaStreamSynchronize(n->stream));
    return AFQMC_OK;
    NET_END(n)
}

afqmc_status afqmc_net_inputs(afqmc_net* n, const int8_t* fields, int32_t n_cfg, int32_t L1, int32_t L2, int32_t M,
                              const int32_t* pos, int32_t B, float* X, float* S) {
    NET_BEGIN(n)
    if (!fields || !pos || !X || n_cfg < 1 || L1 < 1 || L2 < 1 || M < 1 || B < 1) { n->err = "bad arguments"; return AFQMC_E_INVALID; }
    for (int q = 0; q < B; ++q)
        if (pos[4 * q] < 0 || pos[4 * q] >= n_cfg || pos[4 * q + 1] < 1 || pos[4 * q + 1] + n->T - 1 > M) {
            n->err = "block position outside the configurations";
            return AFQMC_E_INVALID;
        }
    const size_t stride = (size_t)M * 2 * L1 * L2;
    net_reserve(n, B);
    int8_t* f = n->dalloc<int8_t>((size_t)n_cfg * stride);
    CK(cudaMemcpyAsync(f, fields, (size_t)n_cfg * stride, cudaMemcpyHostToDevice, n->stream));
    CK(cudaMemcpyAsync(n->pos, pos, sizeof(int) * 4 * B, cudaMemcpyHostToDevice, n->stream));
    k_block_inputs<<<B, 256, 0, n->stream>>>(f, stride, n->pos, geom_of(n, L1, L2, M), n->X, S ? n->S : nullptr);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(X, n->X, sizeof(float) * B * n->d_in, cudaMemcpyDeviceToHost, n->stream));
    if (S) CK(cudaMemcpyAsync(S, n->S, sizeof(float) * B * n->d_out, cudaMemcpyDeviceToHost, n->stream));
    CK(cudaStreamSynchronize(n->stream));
    n->dfree(f);
    return AFQMC_OK;
    NET_END(n)
}

afqmc_status afqmc_net_forward(afqmc_net* n, const float* X, int32_t B, float* Z) {
    NET_BEGIN(n)
    if (!X || !Z || B < 1) { n->err = "bad arguments"; return AFQMC_E_INVALID; }
    net_reserve(n, B);
    CK(cudaMemcpyAsync(n->X, X, sizeof(float) * B * n->d_in, cudaMemcpyHostToDevice, n->stream));
    net_forward_dev(n, n->X, B, n->Hd, n->Z, n->stream);
    CK(cudaMemcpyAsync(Z, n->Z, sizeof(float) * B * n->d_out, cudaMemcpyDeviceToHost, n->stream));
    CK(cudaStreamSynchronize(n->stream));
    return AFQMC_OK;
    NET_END(n)
}

afqmc_status afqmc_net_gradient(afqmc_net* n, const float* X, const float* S, int32_t B, float* grad, double* loss) {
    NET_BEGIN(n)
    if (!X || !S || !grad || B < 1) { n->err = "bad arguments"; return AFQMC_E_INVALID; }
    net_reserve(n, B);
    CK(cudaMemcpyAsync(n->X, X, sizeof(float) * B * n->d_in, cudaMemcpyHostToDevice, n->stream));
    CK(cudaMemcpyAsync(n->S, S, sizeof(float) * B * n->d_out, cudaMemcpyHostToDevice, n->stream));
    CK(cudaMemsetAsync(n->loss, 0, sizeof(double), n->stream));
    net_gradient_dev(n, B);
    CK(cudaMemcpyAsync(grad, n->G, sizeof(float) * n->n_par, cudaMemcpyDeviceToHost, n->stream));
    double l = 0.0;
    CK(cudaMemcpyAsync(&l, n->loss, sizeof(double), cudaMemcpyDeviceToHost, n->stream));
    CK(cudaStreamSynchronize(n->stream));
    if (loss) *loss = l;
    return AFQMC_OK;
    NET_END(n)
}

afqmc_status afqmc_net_train(afqmc_net* n, const int8_t* fields, int32_t n_cfg, int32_t L1, int32_t L2, int32_t M,
                             int32_t n_steps, int32_t batch, float lr, uint64_t seed, double* loss) {
    NET_BEGIN(n)
    if (!fields || n_cfg < 1 || L1 < 1 || L2 < 1 || M < n->T || n_steps < 0 || batch < 1 || batch > 65536 ||
        L1 % n->b || L2 % n->b) {
        n->err = "bad training arguments (sizes, or b must divide L1 and L2, T <= M)";
        return AFQMC_E_INVALID;
    }
    const size_t stride = (size_t)M * 2 * L1 * L2;
    if ((size_t)n_cfg * stride > n->cap_fields) {
        if (n->fields) n->dfree(n->fields);
        n->fields = n->dalloc<int8_t>((size_t)n_cfg * stride);
        n->cap_fields = (size_t)n_cfg * stride;
    }
    CK(cudaMemcpyAsync(n->fields, fields, (size_t)n_cfg * stride, cudaMemcpyHostToDevice, n->stream));
    net_reserve(n, batch);
    const BlockGeom g = geom_of(n, L1, L2, M);
    std::mt19937_64 gen(seed);
    std::vector<int> pos((size_t)4 * batch);
    double l = 0.0;
    for (int it = 0; it < n_steps; ++it) {
        for (int q = 0; q < batch; ++q) {
            pos[4 * q] = (int)(gen() % (uint64_t)n_cfg);
            pos[4 * q + 1] = 1 + (int)(gen() % (uint64_t)(M - n->T + 1));
            pos[4 * q + 2] = (int)(gen() % (uint64_t)L1);
            pos[4 * q + 3] = (int)(gen() % (uint64_t)L2);
        }
        CK(cudaMemcpyAsync(n->pos, pos.data(), sizeof(int) * 4 * batch, cudaMemcpyHostToDevice, n->stream));
        CK(cudaStreamSynchronize(n->stream));     // pos is reused by the next step
        CK(cudaMemsetAsync(n->loss, 0, sizeof(double), n->stream));
        k_block_inputs<<<batch, 256, 0, n->stream>>>(n->fields, stride, n->pos, g, n->X, n->S);
        CK(cudaGetLastError());
        net_gradient_dev(n, batch);
        n->step += 1;
        const float bc1 = 1.0f - std::pow(0.9f, (float)n->step), bc2 = 1.0f - std::pow(0.999f, (float)n->step);
        k_adam<<<grid_of(n->n_par), 256, 0, n->stream>>>(n->P, n->G, n->m, n->v, n->n_par, lr, bc1, bc2);
        CK(cudaGetLastError());
    }
    if (n_steps > 0) CK(cudaMemcpyAsync(&l, n->loss, sizeof(double), cudaMemcpyDeviceToHost, n->stream));
    CK(cudaStreamSynchronize(n->stream));
    if (loss) *loss = l;
    return AFQMC_OK;
    NET_END(n)
}

const char* afqmc_net_last_error(const afqmc_net* n) { return n ? n->err.c_str() : g_net_error.c_str(); }

afqmc_status afqmc_block_sweep(afqmc_handle* h, afqmc_net* n, afqmc_block_stats* stats) {
    API_BEGIN(h)
    if (!n) { h->err = "null network"; return AFQMC_E_INVALID; }
    if (h->cplx) { h->err = "block moves need a periodic (real) chain"; return AFQMC_E_INVALID; }
    if (h->ns % n->T || h->L1 % n->b || h->L2 % n->b || n->device != h->p.device) {
        h->err = "block shape does not fit the chain (T | n_stab, b | L1, b | L2, same device)";
        return AFQMC_E_INVALID;
    }
    block_reserve(h, n);
    CK(cudaStreamSynchronize(n->stream));       // parameters written on the network's stream
    CK(cudaMemsetAsync(h->bstats, 0, sizeof(unsigned long long) * 3, h->stream));
    CK(cudaMemsetAsync(h->drift, 0, sizeof(unsigned long long), h->stream));
    block_pass(h, n);
    unsigned long long bs[3] = {0, 0, 0}, dr = 0;
    CK(cudaMemcpyAsync(bs, h->bstats, sizeof(bs), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(&dr, h->drift, sizeof(dr), cudaMemcpyDeviceToHost, h->stream));
    afqmc_status s = check_device(h);
    if (stats) {
        stats->proposed = bs[0];
        stats->accepted = bs[1];
        stats->flipped = bs[2];
        std::memcpy(&stats->max_stab_drift, &dr, sizeof(double));
    }
    return s;
    API_END(h)
}

afqmc_status afqmc_force_slice(afqmc_handle* h, int32_t slice, const int8_t* mask, double* G, double* logR) {
    API_BEGIN(h)
    if (!mask || !G || slice < 1 || slice > h->M) { h->err = "bad arguments"; return AFQMC_E_INVALID; }
    if (!h->Gsave) {
        h->Gsave = h->dalloc<double>((size_t)h->N * h->N);
        h->logR = h->dalloc<double>(1);
        h->lq = h->dalloc<double>(2);
        h->bflag = h->dalloc<int>(1);
        h->bstats = h->dalloc<unsigned long long>(3);
        h->bpos = h->dalloc<int>(4);
    }
    if (!h->bmask || h->bcap_T < 1) {
        h->bmask = h->dalloc<int8_t>(h->Np);
        h->fsave = h->dalloc<int8_t>(h->Np);
        h->bcap_T = 1;
    }
    double* d = h->Wk[5];
    from_host(h, G, d, h->Wk[4]);
    CK(cudaMemcpyAsync(h->bmask, mask, h->Np, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemsetAsync(h->logR, 0, sizeof(double), h->stream));
    update_slice(h, d, slice, 0, 0, h->bmask, h->logR);
    to_host(h, d, G, h->Wk[4]);
    double lr = 0.0;
    CK(cudaMemcpyAsync(&lr, h->logR, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    afqmc_status s = check_device(h);
    if (logR) *logR = lr;
    return s;
    API_END(h)
}

afqmc_status afqmc_dims(const afqmc_handle* h, int32_t* N, int32_t* M, int32_t* Nc) {
    if (!h) return AFQMC_E_INVALID;
    if (N) *N = h->Np;
    if (M) *M = h->M;
    if (Nc) *Nc = h->Nc;
    return AFQMC_OK;
}

const char* afqmc_last_error(const afqmc_handle* h) {
    if (!h) return g_create_error.c_str();
    return h->err.c_str();
}

// Radical inverse of n in base b as the exact fraction r / b^k (digits of n
// reversed behind the point), converted by one correctly rounded division.
static double radical_inverse(uint64_t n, uint64_t b) {
    uint64_t r = 0, d = 1;
    for (; n; n /= b) {
        r = r * b + n % b;
        d *= b;
    }
    return (double)r / (double)d;
}

afqmc_status afqmc_quasirandom_twists(int32_t n, int32_t start, double* theta) {
    if (n < 0 || start < 0 || (int64_t)start + n > 2147483647ll || (n > 0 && !theta)) {
        g_create_error = "afqmc_quasirandom_twists: need n >= 0, start >= 0, start + n < 2^31 and a buffer";
        return AFQMC_E_INVALID;
    }
    for (int32_t i = 0; i < n; ++i) {
        const uint64_t m = (uint64_t)start + (uint64_t)i;
        theta[2 * i] = radical_inverse(m, 2);
        theta[2 * i + 1] = radical_inverse(m, 3);
    }
    return AFQMC_OK;
}

}  // extern "C"
