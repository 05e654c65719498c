// Device-side helpers shared by the DSG-NLM / linearized PnP-ADMM kernels.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace dsg {

// Checked build (-DDSGNLM_CHECKED): the index checks below set a bit in a device word
// and skip the access instead of letting it leave its buffer; the word is read back
// by dsgnlm_check_word.  Every translation unit has its own word (no relocatable device
// code), and DSG_CHECK_WORD_ACCESSOR names the host function that reads and clears
// it.  In the normal build a check is the constant true and costs nothing.
enum : unsigned {
    kChkPlanes = 1u,      // a weight-plane store of the build
    kChkPartials = 2u,    // a phase-1 partial-region read or write
    kChkPixels = 4u,      // a per-pixel store of an epilogue
    kChkAdjPlanes = 8u,   // a G-plane store of pair pass G
    kChkAdjWindows = 16u, // a window-partial read or write of the adjoint
    kChkSelfTest = 0x80000000u,
};
#ifdef DSGNLM_CHECKED
static __device__ unsigned g_dsg_check_word;
__device__ __forceinline__ bool dsg_in_range(long long i, long long n, unsigned bit) {
    if (i >= 0 && i < n) return true;
    atomicOr(&g_dsg_check_word, bit);
    return false;
}
#define DSG_IN_RANGE(i, n, bit) ::dsg::dsg_in_range((long long)(i), (long long)(n), (bit))
#define DSG_CHECK_WORD_ACCESSOR(name)                                                   \
    unsigned name(bool clear) {                                                         \
        unsigned w = 0;                                                                 \
        if (cudaMemcpyFromSymbol(&w, g_dsg_check_word, sizeof w) != cudaSuccess) w = 0; \
        if (clear) {                                                                    \
            const unsigned z = 0;                                                       \
            cudaMemcpyToSymbol(g_dsg_check_word, &z, sizeof z);                         \
        }                                                                               \
        return w;                                                                       \
    }
#else
#define DSG_IN_RANGE(i, n, bit) true
#define DSG_CHECK_WORD_ACCESSOR(name) \
    unsigned name(bool) { return 0u; }
#endif

// Index of the half-window offset o = (oy, ox): first the oy = 0 row with
// ox = 1..rs, then the rows oy = 1..rs with ox = -rs..rs.  n_h = 2 rs (rs + 1).
__host__ __device__ __forceinline__ int num_half_offsets(int rs) { return 2 * rs * (rs + 1); }

__host__ __device__ __forceinline__ void half_offset(int k, int rs, int& oy, int& ox) {
    if (k < rs) {
        oy = 0;
        ox = k + 1;
    } else {
        const int kk = k - rs;
        const int w = 2 * rs + 1;
        oy = 1 + kk / w;
        ox = kk % w - rs;
    }
}

// first half-offset index of row oy and the ox it starts with
__host__ __device__ __forceinline__ int row_first_k(int oy, int rs) {
    return oy == 0 ? 0 : rs + (oy - 1) * (2 * rs + 1);
}

// half-sample symmetric extension of an index into [0, n)
__device__ __forceinline__ int sym_index(int i, int n) {
    const int p = 2 * n;
    int m = i % p;
    if (m < 0) m += p;
    return m < n ? m : p - 1 - m;
}

__device__ __forceinline__ int wrap_index(int i, int n) {
    int m = i % n;
    return m < 0 ? m + n : m;
}

// weight storage conversions (arithmetic is always FP32)
template <typename T> __device__ __forceinline__ float to_f32(T v);
template <> __device__ __forceinline__ float to_f32<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f32<__half>(__half v) { return __half2float(v); }
template <> __device__ __forceinline__ float to_f32<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename T> __device__ __forceinline__ T from_f32(float v);
template <> __device__ __forceinline__ float from_f32<float>(float v) { return v; }
template <> __device__ __forceinline__ __half from_f32<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 from_f32<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

// Error-free addition (Knuth's TwoSum): s + e == a + b exactly.  Used to add the
// per-row partial sums of a stencil so that the row sums entering the balancing
// residual are not limited by the length of the FP32 accumulation chain.
struct CompSum {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float b) {
        const float t = __fadd_rn(s, b);
        const float bb = __fsub_rn(t, s);
        const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bb)), __fsub_rn(b, bb));
        s = t;
        c = __fadd_rn(c, err);
    }
    __device__ __forceinline__ float value() const { return __fadd_rn(s, c); }
};

// Order-independent max of non-negative doubles through their bit patterns.
__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* addr, double v) {
    atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Wait until the grids this one depends on have completed and their writes are visible
// (a no-op without a programmatic dependency).  A kernel launched with programmatic
// stream serialization may start while its predecessor drains; it calls this before it
// reads or writes any memory the predecessor uses.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// A kernel's entry: wait for its predecessors, then let the next kernel of the stream
// (if launched with programmatic stream serialization) be scheduled as soon as every
// block of this one has started; that kernel waits in turn before touching memory, so
// only launch latency and the last wave's idle SMs are overlapped.
__device__ __forceinline__ void griddep_enter() {
    griddep_wait();
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum of one float per thread of a block of NW warps (256 threads by default): FP32
// within each warp (a fixed tree), the warp sums added in FP64 in warp order.  The result is valid in
// thread 0; every thread must call it, and a second call in the same kernel must be
// separated from the first by a barrier.  (FP64 arithmetic runs at a small fraction of
// the FP32 rate on this GPU, so per-element terms stay in FP32.)
template <int NW = 8>
__device__ __forceinline__ double block_sum(float v, int tid) {
    v = warp_sum_f(v);
    __shared__ float ws[NW];
    if ((tid & 31) == 0) ws[tid >> 5] = v;
    __syncthreads();
    double acc = 0.0;
    if (tid == 0)
        for (int w = 0; w < NW; ++w) acc += (double)ws[w];
    return acc;
}
__device__ __forceinline__ double block_sum_256(float v, int tid) { return block_sum<8>(v, tid); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace dsg
