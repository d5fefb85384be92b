// Shared device helpers: counter-based random numbers, bounded grid barrier,
// global-timer timeouts, small reductions.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace afq {

// Error codes written into DevStatus::err by device code (mirrors afqmc_status).
enum : int { DERR_OK = 0, DERR_NUMERIC = 4, DERR_TIMEOUT = 5 };

// Default wall-clock limit of any single device-side wait (nanoseconds).
constexpr unsigned long long WAIT_LIMIT_NS = 2000000000ull;

struct DevStatus {
    int err;            // first error seen (0 = none)
    int where;          // code of the wait that timed out
    unsigned int bar_count, bar_gen;   // grid barrier state
    // limit of the waits between CTAs (grid barriers, column hand-offs of the
    // QR and LU); 0 = WAIT_LIMIT_NS.  A test hook can shorten it to make a
    // wait run out on purpose.  Waits on the tensor cores' own completion
    // (mbarriers with asynchronous copies or MMAs in flight) keep the fixed
    // limit: their kernel must not release shared or tensor memory while such
    // work may still be running.
    unsigned long long wait_ns;
};

__device__ __forceinline__ unsigned long long wait_limit(const DevStatus* st) {
    const unsigned long long w = *(const volatile unsigned long long*)&st->wait_ns;
    return w ? w : WAIT_LIMIT_NS;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// SplitMix64 (Steele, Lea & Flood 2014): n-th output of the stream with seed k
// is mix(k + n*0x9E3779B97F4A7C15); finaliser constants of the published generator.
__host__ __device__ __forceinline__ uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ double sm64_uniform(uint64_t key, uint64_t n) {
    return (double)(sm64_mix(key + n * 0x9E3779B97F4A7C15ull) >> 11) * (1.0 / 9007199254740992.0);
}

// Grid-wide barrier for cooperative launches.  Every CTA must call it.  The
// wait is bounded by wait_limit(st); on timeout the error flag is set and the
// function returns false, as it does when any CTA has flagged an error.
// Thread 0 of a CTA arrives with an acquire-release add on the counter (it
// publishes the CTA's writes, made visible to it by the bar.sync before); the
// last one to arrive resets the counter and publishes the next generation with
// a release store; the others poll the generation with acquire loads.
__device__ __forceinline__ bool grid_barrier(DevStatus* st, int where) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int* cnt = &st->bar_count;
        unsigned int* genp = &st->bar_gen;
        unsigned int gen, arrived;
        asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(gen) : "l"(genp) : "memory");
        asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(arrived) : "l"(cnt) : "memory");
        if (arrived == gridDim.x - 1) {
            asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" :: "l"(cnt), "r"(0u) : "memory");
            asm volatile("st.release.gpu.global.u32 [%0], %1;" :: "l"(genp), "r"(gen + 1u) : "memory");
        } else {
            const unsigned long long t0 = global_ns(), lim = wait_limit(st);
            unsigned int nap = 32;     // back-off: the waiting CTAs poll one L2 line while
                                       // the working ones need the memory system; capped
                                       // at 128 ns (147 CTAs polling at that rate are ~1e9
                                       // loads/s, while each wait at the cap costs ~64 ns
                                       // of latency on average after the last arrival)
            for (;;) {
                unsigned int g;
                asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(g) : "l"(genp) : "memory");
                if (g != gen) break;
                if (*(volatile int*)&st->err) break;
                if (global_ns() - t0 > lim) {
                    if (atomicCAS(&st->err, 0, DERR_TIMEOUT) == 0) st->where = where;
                    break;
                }
                __nanosleep(nap);
                if (nap < 128) nap <<= 1;
            }
        }
        s_ok = (*(volatile int*)&st->err) == 0;
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ __forceinline__ void flag_error(DevStatus* st, int code, int where) {
    if (atomicCAS(&st->err, 0, code) == 0) st->where = where;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block-wide sum (blockDim.x a multiple of 32, <= 1024); result valid in all threads.
__device__ __forceinline__ double block_sum(double v, double* scratch /* >= 33 doubles */) {
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) scratch[w] = v;
    __syncthreads();
    if (w == 0) {
        double x = lane < nw ? scratch[lane] : 0.0;
        x = warp_sum(x);
        if (lane == 0) scratch[32] = x;
    }
    __syncthreads();
    return scratch[32];
}

// Sum over a 256-thread block with few FP64 instructions per sub-partition (on
// this part each FP64 warp instruction holds its sub-partition's unit for ~64
// cycles): warps w and w + 4 share a sub-partition, so they are folded first (one
// add), then four warp sums run on the four sub-partitions, then one warp adds
// the four.  Result valid in all threads.  scratch: >= 140 doubles.
__device__ __forceinline__ double block_sum256(double v, double* scratch) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();                              // scratch free
    if (w >= 4) scratch[threadIdx.x - 128] = v;
    __syncthreads();
    if (w < 4) {
        v += scratch[threadIdx.x];
        v = warp_sum(v);
        if (lane == 0) scratch[128 + w] = v;
    }
    __syncthreads();
    if (w == 0) {
        double x = lane < 4 ? scratch[128 + lane] : 0.0;
        x += __shfl_xor_sync(0xffffffffu, x, 1);
        x += __shfl_xor_sync(0xffffffffu, x, 2);
        if (lane == 0) scratch[136] = x;
    }
    __syncthreads();
    return scratch[136];
}

// 1 / r from the hardware estimate y0 (relative error below 2^-19.9 on this
// part, measured) by one cubic step y0 (1 + e + e^2), e = 1 - r y0: the error
// e^3 < 2^-59 is below FP64 rounding, in three dependent FP64 operations
__device__ __forceinline__ double recip_fast(double r) {
    double y0;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y0) : "d"(r));
    const double e = fma(-r, y0, 1.0);
    return fma(y0, fma(e, e, e), y0);
}

// |x| > t for t >= 0 (not NaN), on the bit patterns (non-negative doubles order
// as their integer images): keeps the comparison off the FP64 unit
__device__ __forceinline__ bool abs_gt(double x, double t) {
    return (__double_as_longlong(x) & 0x7fffffffffffffffll) > __double_as_longlong(t);
}
__device__ __forceinline__ bool finite_bits(double x) {
    return ((__double_as_longlong(x) >> 52) & 0x7ff) != 0x7ff;
}

}  // namespace afq
