// Epilogues of the TMA stencil passes.
//
// Balance (Eq. S2 iterated, Eq. S3): balance_combine_kernel finishes t = K1 d for
// every pixel, writes the next scaling sqrt(d / t) and t, and leaves one
// (max |d t - 1|, max d t) pair per block; balance_decide_kernel (one block)
// reduces the pairs, decides whether to stop (tolerance, maxit or a stalled
// residual), advances the pass counter and, inside a CUDA graph, sets the WHILE
// condition that repeats the balancing passes on the device without host
// round trips.
//
// Algorithm 1: combine_xupdate_kernel finishes v = W (x + u) and u <- u + x - v
// for iteration k (the third aggregation of Algorithm 2 with the closure of
// Eq. S3) and, in the same pass over the pixels, performs the linearized
// x-update of iteration k + 1, which needs v and u only at its own pixel.
#include "combine.cuh"
#include "common.cuh"
#include "epilogue.cuh"
#include "internal.h"
#include "xupdate.cuh"

namespace dsg {

namespace {

__global__ void __launch_bounds__(256)
balance_combine_kernel(Cover cv, int H, int W, const float* __restrict__ d_in, float* __restrict__ d_out,
                       float* __restrict__ t_out, float2* __restrict__ part, const BalanceCtl* __restrict__ ctl) {
    if (*(volatile const int*)&ctl->done) return;
    const int j = blockIdx.x * 32 + threadIdx.x;
    const int i = blockIdx.y * 8 + threadIdx.y;
    const int t = threadIdx.y * 32 + threadIdx.x;
    float e = 0.f, m = 0.f;
    if (i < H && j < W) {
        const size_t s = (size_t)i * W + j;
        const float ds = d_in[s];
        const float tt = ds + gather_partials(cv, i, j);  // (K1 d)_s with K1(s, s) = 1
        d_out[s] = sqrtf(ds / tt);
        t_out[s] = tt;
        e = fabsf(fmaf(ds, tt, -1.f));  // |d_s t_s - 1| with a single rounding
        m = ds * tt;
    }
    e = warp_max(e);
    m = warp_max(m);
    __shared__ float se[8], sm[8];
    if ((t & 31) == 0) {
        se[t >> 5] = e;
        sm[t >> 5] = m;
    }
    __syncthreads();
    if (t == 0) {
        for (int w = 0; w < 8; ++w) {
            e = fmaxf(e, se[w]);
            m = fmaxf(m, sm[w]);
        }
        part[blockIdx.y * gridDim.x + blockIdx.x] = make_float2(e, m);
    }
}

__global__ void __launch_bounds__(256)
balance_decide_kernel(const float2* __restrict__ part, int nblocks, BalanceCtl* __restrict__ ctl,
                      cudaGraphConditionalHandle cond, int use_cond) {
    const int t = threadIdx.x;
    if (*(volatile int*)&ctl->done) {
        if (t == 0 && use_cond) cudaGraphSetConditional(cond, 0u);
        return;
    }
    float e = 0.f, m = 0.f;
    for (int q = t; q < nblocks; q += 256) {
        const float2 v = part[q];
        e = fmaxf(e, v.x);
        m = fmaxf(m, v.y);
    }
    e = warp_max(e);
    m = warp_max(m);
    __shared__ float se[8], sm[8];
    if ((t & 31) == 0) {
        se[t >> 5] = e;
        sm[t >> 5] = m;
    }
    __syncthreads();
    if (t != 0) return;
    for (int w = 0; w < 8; ++w) {
        e = fmaxf(e, se[w]);
        m = fmaxf(m, sm[w]);
    }
    const int pass = ctl->pass;
    const double ed = (double)e;
    ctl->eps = ed;
    ctl->m = (double)m;
    int done = 0, status = 0;
    if (ed <= ctl->tol) {
        done = 1;
    } else if (pass >= ctl->maxit) {
        done = 1;
        status = 6;
    } else if (ed < 0.99 * ctl->best) {
        ctl->best = ed;
        ctl->since_best = 0;
    } else if (++ctl->since_best >= 3) {
        done = 1;
        status = 7;
    }
    if (done) {
        ctl->final_pass = pass;
        ctl->status = status;
        *(volatile int*)&ctl->done = 1;
    } else {
        ctl->pass = pass + 1;
    }
    if (use_cond) cudaGraphSetConditional(cond, done ? 0u : 1u);
}

template <int KIND>
__global__ void __launch_bounds__(256, 3)
combine_xupdate_kernel(Cover cv, EpilogueArgs a) {
    __shared__ SrTile tile;
    const size_t bid = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
    combine_xupdate_body<KIND>(tile, cv, a, blockIdx.y * kXH, blockIdx.x * kXW, a.partials + 2 * bid);
}

Cover cover(const TmaPlan& plan, int rs) {
    return Cover{plan.partials, plan.tiles_x, plan.tiles_y, plan.splits.n, rs};
}

}  // namespace

int balance_combine_blocks(int H, int W) { return ((W + 31) / 32) * ((H + 7) / 8); }

cudaError_t launch_balance_combine(const TmaPlan& plan, int H, int W, int rs, const float* d_in,
                                   float* d_out, float* t_out, float2* part, const BalanceCtl* ctl,
                                   cudaStream_t st) {
    balance_combine_kernel<<<dim3((W + 31) / 32, (H + 7) / 8), dim3(32, 8), 0, st>>>(
        cover(plan, rs), H, W, d_in, d_out, t_out, part, ctl);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_balance_decide(const float2* part, int nblocks, BalanceCtl* ctl,
                                  cudaGraphConditionalHandle cond, int use_cond, cudaStream_t st) {
    balance_decide_kernel<<<1, 256, 0, st>>>(part, nblocks, ctl, cond, use_cond);
    count_launches(1);
    return cudaGetLastError();
}

int combine_xupdate_blocks(int H, int W) { return ((W + kXW - 1) / kXW) * ((H + kXH - 1) / kXH); }

cudaError_t launch_combine_xupdate(int kind, const TmaPlan& plan, int rs, const EpilogueArgs& args,
                                   cudaStream_t st) {
    if (kind == 0 && args.do_x && args.taps.r > kMaxBlurR) return cudaErrorInvalidValue;
    dim3 grid((args.W + kXW - 1) / kXW, (args.H + kXH - 1) / kXH);
    if (kind == 0)
        combine_xupdate_kernel<0><<<grid, dim3(32, 8), 0, st>>>(cover(plan, rs), args);
    else
        combine_xupdate_kernel<1><<<grid, dim3(32, 8), 0, st>>>(cover(plan, rs), args);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace dsg
