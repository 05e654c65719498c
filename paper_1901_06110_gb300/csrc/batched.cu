// Batched form of Algorithm 1: many images of uneven sizes advance together, one
// launch per step of the iteration over a work-list of (image, tile) items, with
// the same per-image arithmetic as the single-image solve:
//   SR gradient A^T(A x - y)           batched_grad_kernel (32 x 32 tiles)
//   x-update of iteration 0            batched_xupdate0_kernel (per pixel)
//   per iteration: phase-1 gather      launch_tma_gather_batched (stencil_tma.cu)
//                  combine + x-update  batched_combine_kernel (per pixel)
// Each image keeps its own DSG-NLM weights (any storage type; the arithmetic is
// FP32), scaling, closure and iterates; the work-list only flattens the tiles of
// all images into one grid, so the GPU scheduler balances small and large images.
#include "combine.cuh"
#include "common.cuh"
#include "epilogue.cuh"
#include "grad.cuh"
#include "internal.h"
#include "xupdate.cuh"

namespace dsg {

namespace {

// elementwise single-photon x-update on the tile at (y0, x0)
__device__ __forceinline__ void spi_xupdate_tile(const EpilogueArgs& a, int y0, int x0) {
    const int pj = x0 + threadIdx.x;
    for (int py = threadIdx.y; py < kXH; py += 8) {
        const int pi = y0 + py;
        if (pi >= a.H || pj >= a.W) continue;
        const size_t q = (size_t)pi * a.W + pj;
        const float xv = a.x_in[q];
        const float g = spi_hprime(xv, a.counts[q], a.K, a.eta, a.eps);
        const float up = a.u[q];
        const float xn = project(a.mu * (a.alpha * xv + a.rho * (a.v[q] - up) - g), a.constraint);
        a.x_out[q] = xn;
        a.z[q] = xn + up;
    }
}

// x-update of iteration 0 on the 16 x 32 tile of the work item, per pixel: SR with
// the gradient formed beforehand (a.g), single-photon with h' in place
template <int KIND>
__global__ void __launch_bounds__(256)
batched_xupdate0_kernel(const BatchEpi* __restrict__ insts, const int4* __restrict__ work) {
    const int4 w = work[blockIdx.x];  // (instance, tile row, tile column, -)
    const EpilogueArgs& a = insts[w.x].a;
    const int y0 = w.y * kXH, x0 = w.z * kXW;
    if (KIND == 1) {
        spi_xupdate_tile(a, y0, x0);
        return;
    }
    const int pj = x0 + threadIdx.x;
    for (int py = threadIdx.y; py < kXH; py += 8) {
        const int pi = y0 + py;
        if (pi >= a.H || pj >= a.W) continue;
        const size_t q = (size_t)pi * a.W + pj;
        const float up = a.u[q];
        const float xn = project(a.mu * (a.alpha * a.x_in[q] + a.rho * (a.v[q] - up) - a.g[q]), a.constraint);
        a.x_out[q] = xn;
        a.z[q] = xn + up;
    }
}

// g = A^T (A x - y) of one image on the 32 x 32 tile of the work item
template <int R>
__global__ void __launch_bounds__(256)
batched_grad_kernel(const BatchEpi* __restrict__ insts, const int4* __restrict__ work) {
    __shared__ GradSmem<R> sm;
    const int4 w = work[blockIdx.x];  // (instance, tile row, tile column, -)
    const EpilogueArgs& a = insts[w.x].a;
    const BlurTaps taps = a.taps;
    sr_grad_tile<R>(sm, a.x_in, a.y, a.H, a.W, taps, a.g, w.y * kGT, w.z * kGT);
}

// finish v and u of iteration `it` and perform the next x-update, per pixel
template <int KIND>
__global__ void __launch_bounds__(256, 4)
batched_combine_kernel(const BatchEpi* __restrict__ insts, const int4* __restrict__ work, int it, int last) {
    const int4 w = work[blockIdx.x];
    const BatchEpi& e = insts[w.x];
    double* partials = e.partials + 2 * ((size_t)it * e.nblocks + (size_t)w.y * e.gx + w.z);
    combine_update_body<KIND>(e.cv, e.a, !last, w.y * kXH, w.z * kXW, partials);
}

// hist of (image, iteration) = fixed-order sums of that image's per-block residual partials
__global__ void __launch_bounds__(256)
batched_reduce_kernel(const BatchEpi* __restrict__ insts, double* __restrict__ hist, int iters) {
    const int it = blockIdx.x, inst = blockIdx.y, t = threadIdx.x;
    const BatchEpi& e = insts[inst];
    const double* p = e.partials + 2 * (size_t)it * e.nblocks;
    double a = 0.0, b = 0.0;
    for (int q = t; q < e.nblocks; q += 256) {
        a += p[2 * q];
        b += p[2 * q + 1];
    }
    __shared__ double ra[256], rb[256];
    ra[t] = a;
    rb[t] = b;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (t < s) {
            ra[t] += ra[t + s];
            rb[t] += rb[t + s];
        }
        __syncthreads();
    }
    if (t == 0) {
        hist[2 * ((size_t)inst * iters + it)] = ra[0];
        hist[2 * ((size_t)inst * iters + it) + 1] = rb[0];
    }
}

// One epilogue block of a batched balancing pass: t, the next scaling and the block's
// maxima (balance_pixels, as the single-image epilogue); the image's last block
// applies its stopping rule and, when the image stops, counts it in *stopped.
// Images that stopped in an earlier pass are skipped.
__global__ void __launch_bounds__(256)
batched_balance_epilogue_kernel(const BatchBal* __restrict__ bb, const int4* __restrict__ work, int parity,
                                unsigned* __restrict__ stopped) {
    const int4 w = work[blockIdx.x];  // (image, block row, block column, -)
    const BatchBal& b = bb[w.x];
    BalanceCtl* ctl = b.ctl;
    if (*(volatile const int*)&ctl->done) return;
    const int t = threadIdx.y * 32 + threadIdx.x;
    float e = 0.f, m = 0.f;
    const PassRule rule = pass_rule(ctl);
    balance_pixels(b.cv, b.H, b.W, b.d[parity], b.d[parity ^ 1], b.t[parity], w.y * kXH, w.z * kXW, threadIdx.x,
                   threadIdx.y, rule, e, m);
    e = warp_max(e);
    m = warp_max(m);
    __shared__ float se[8], sm[8];
    __shared__ int s_last;
    if ((t & 31) == 0) {
        se[t >> 5] = e;
        sm[t >> 5] = m;
    }
    __syncthreads();
    if (t == 0) {
        for (int k = 0; k < 8; ++k) {
            e = fmaxf(e, se[k]);
            m = fmaxf(m, sm[k]);
        }
        b.part[(size_t)w.y * b.nbx + w.z] = make_float2(e, m);
        __threadfence();  // the pair is visible before the arrival is counted
        s_last = atomicAdd(&ctl->arrive, 1u) == (unsigned)(b.nblocks - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    e = 0.f;
    m = 0.f;
    for (int q = t; q < b.nblocks; q += 256) {
        const float2 v = __ldcg(b.part + q);
        e = fmaxf(e, v.x);
        m = fmaxf(m, v.y);
    }
    e = warp_max(e);
    m = warp_max(m);
    __syncthreads();
    if ((t & 31) == 0) {
        se[t >> 5] = e;
        sm[t >> 5] = m;
    }
    __syncthreads();
    if (t != 0) return;
    for (int k = 0; k < 8; ++k) {
        e = fmaxf(e, se[k]);
        m = fmaxf(m, sm[k]);
    }
    ctl->arrive = 0u;
    balance_decide(ctl, e, m, 0, 0);
    if (ctl->done) atomicAdd(stopped, 1u);
}

}  // namespace

cudaError_t launch_batched_balance_epilogue(const BatchBal* bb, const int4* work, int nwork, int parity,
                                            unsigned* stopped, cudaStream_t st) {
    if (nwork <= 0) return cudaSuccess;
    batched_balance_epilogue_kernel<<<nwork, dim3(32, 8), 0, st>>>(bb, work, parity, stopped);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_batched_xupdate0(int kind, const BatchEpi* insts, const int4* work, int nwork, cudaStream_t st) {
    if (nwork <= 0) return cudaSuccess;
    if (kind == 0)
        batched_xupdate0_kernel<0><<<nwork, dim3(32, 8), 0, st>>>(insts, work);
    else
        batched_xupdate0_kernel<1><<<nwork, dim3(32, 8), 0, st>>>(insts, work);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_batched_grad(int blur_r, const BatchEpi* insts, const int4* work, int nwork, cudaStream_t st) {
    if (nwork <= 0) return cudaSuccess;
    switch (blur_r) {
        case 0: batched_grad_kernel<0><<<nwork, 256, 0, st>>>(insts, work); break;
        case 1: batched_grad_kernel<1><<<nwork, 256, 0, st>>>(insts, work); break;
        case 2: batched_grad_kernel<2><<<nwork, 256, 0, st>>>(insts, work); break;
        case 3: batched_grad_kernel<3><<<nwork, 256, 0, st>>>(insts, work); break;
        case 4: batched_grad_kernel<4><<<nwork, 256, 0, st>>>(insts, work); break;
        case 5: batched_grad_kernel<5><<<nwork, 256, 0, st>>>(insts, work); break;
        case 6: batched_grad_kernel<6><<<nwork, 256, 0, st>>>(insts, work); break;
        case 7: batched_grad_kernel<7><<<nwork, 256, 0, st>>>(insts, work); break;
        case 8: batched_grad_kernel<8><<<nwork, 256, 0, st>>>(insts, work); break;
        default: return cudaErrorInvalidValue;
    }
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_batched_combine(int kind, const BatchEpi* insts, const int4* work, int nwork, int it, int last,
                                   cudaStream_t st) {
    if (nwork <= 0) return cudaSuccess;
    if (kind == 0)
        batched_combine_kernel<0><<<nwork, dim3(32, 8), 0, st>>>(insts, work, it, last);
    else
        batched_combine_kernel<1><<<nwork, dim3(32, 8), 0, st>>>(insts, work, it, last);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_batched_reduce(const BatchEpi* insts, int count, double* hist, int iters, cudaStream_t st) {
    if (count <= 0 || iters <= 0) return cudaSuccess;
    batched_reduce_kernel<<<dim3(iters, count), 256, 0, st>>>(insts, hist, iters);
    count_launches(1);
    return cudaGetLastError();
}

DSG_CHECK_WORD_ACCESSOR(check_word_batched)

}  // namespace dsg
