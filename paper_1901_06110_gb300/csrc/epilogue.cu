// Epilogues of the TMA stencil passes.
//
// Balance (Eq. S2 iterated, Eq. S3): balance_epilogue_kernel finishes t = K1 d
// for every pixel, writes the next scaling sqrt(d / t) and t, and leaves one
// (max |d t - 1|, max d t) pair per block; the last block to finish reduces the
// pairs, decides whether to stop (tolerance, maxit or a stalled residual),
// advances the pass counter and, inside a CUDA graph, sets the WHILE condition
// that repeats the balancing passes on the device without host round trips.
//
// Algorithm 1: combine_update_kernel finishes v = W (x + u) and u <- u + x - v
// for iteration k (the third aggregation of Algorithm 2 with the closure of
// Eq. S3) and, in the same pass over the pixels, performs the linearized
// x-update of iteration k + 1, which needs v, u and the gradient only at its own
// pixel (the SR gradient is computed beforehand by sr_grad_tile_kernel).
#include <type_traits>

#include "combine.cuh"
#include "common.cuh"
#include "epilogue.cuh"
#include "internal.h"
#include "launch.h"
#include "xupdate.cuh"

namespace dsg {

namespace {

// Epilogue of one balancing pass on the kXH x kXW tile of each block: t = K1 d,
// the next scaling sqrt(d / t), and the block's (max |d t - 1|, max d t).  With
// `decide`, the last block to finish reduces the pairs of all blocks and applies
// the stopping rule; a pass launched after the deciding one returns at once.
template <int SL>
__global__ void __launch_bounds__(256)
balance_epilogue_kernel(Cover cv, int H, int W, const float* __restrict__ d_in, float* __restrict__ d_out,
                        float* __restrict__ t_out, float2* __restrict__ part, BalanceCtl* __restrict__ ctl,
                        int decide, cudaGraphConditionalHandle cond, int use_cond) {
    const int t = threadIdx.y * 32 + threadIdx.x;
    const int nblocks = gridDim.x * gridDim.y;
    const int bid = blockIdx.y * gridDim.x + blockIdx.x;
    if (decide && *(volatile const int*)&ctl->done) {
        if (use_cond && bid == 0 && t == 0) cudaGraphSetConditional(cond, 0u);
        return;
    }
    float e = 0.f, m = 0.f;
    const PassRule rule = pass_rule(ctl);
    balance_pixels<SL>(cv, H, W, d_in, d_out, t_out, blockIdx.y * kXH, blockIdx.x * kXW, threadIdx.x, threadIdx.y,
                       rule, e, m);
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
        for (int w = 0; w < 8; ++w) {
            e = fmaxf(e, se[w]);
            m = fmaxf(m, sm[w]);
        }
        part[bid] = make_float2(e, m);
        if (decide) {
            __threadfence();  // the pair is visible before the arrival is counted
            s_last = atomicAdd(&ctl->arrive, 1u) == (unsigned)(nblocks - 1);
        }
    }
    if (!decide) return;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    e = 0.f;
    m = 0.f;
    for (int q = t; q < nblocks; q += 256) {
        const float2 v = __ldcg(part + q);
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
    for (int w = 0; w < 8; ++w) {
        e = fmaxf(e, se[w]);
        m = fmaxf(m, sm[w]);
    }
    ctl->arrive = 0u;
    balance_decide(ctl, e, m, cond, use_cond);
}

template <int KIND, int SL>
__global__ void __launch_bounds__(256, SL > 0 ? 4 : 3)
combine_update_kernel(Cover cv, EpilogueArgs a) {
    griddep_enter();  // may be launched with programmatic stream serialization
    const size_t bid = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
    combine_update_body<KIND, SL>(cv, a, a.do_x, blockIdx.y * kXH, blockIdx.x * kXW, a.partials + 2 * bid);
}

// Kernels specialised for the common slice counts; SL = 0 takes any count.
template <typename F>
cudaError_t by_slices(int slices, F&& f) {
    switch (slices) {
        case 1: return f(std::integral_constant<int, 1>{});
        case 2: return f(std::integral_constant<int, 2>{});
        case 3: return f(std::integral_constant<int, 3>{});
        case 4: return f(std::integral_constant<int, 4>{});
        default: return f(std::integral_constant<int, 0>{});
    }
}

Cover cover(const TmaPlan& plan, int rs) {
    return Cover{plan.partials, plan.tiles_x, plan.tiles_y, plan.splits.n, rs, plan.part_cap};
}

}  // namespace

int balance_combine_blocks(int H, int W) { return ((W + kXW - 1) / kXW) * ((H + kXH - 1) / kXH); }

cudaError_t launch_balance_epilogue(const TmaPlan& plan, int H, int W, int rs, const float* d_in, float* d_out,
                                    float* t_out, float2* part, BalanceCtl* ctl, int decide,
                                    cudaGraphConditionalHandle cond, int use_cond, cudaStream_t st) {
    const dim3 grid((W + kXW - 1) / kXW, (H + kXH - 1) / kXH);
    const Cover cv = cover(plan, rs);
    return by_slices(plan.splits.n, [&](auto sl) {
        balance_epilogue_kernel<decltype(sl)::value><<<grid, dim3(32, 8), 0, st>>>(cv, H, W, d_in, d_out, t_out,
                                                                                   part, ctl, decide, cond, use_cond);
        count_launches(1);
        return cudaGetLastError();
    });
}

int combine_xupdate_blocks(int H, int W) { return ((W + kXW - 1) / kXW) * ((H + kXH - 1) / kXH); }

cudaError_t launch_combine_update(int kind, const TmaPlan& plan, int rs, const EpilogueArgs& args,
                                  cudaStream_t st, bool pdl) {
    if (kind == 0 && args.do_x && !args.g) return cudaErrorInvalidValue;
    const dim3 grid((args.W + kXW - 1) / kXW, (args.H + kXH - 1) / kXH);
    const Cover cv = cover(plan, rs);
    return by_slices(plan.splits.n, [&](auto sl) {
        constexpr int SL = decltype(sl)::value;
        count_launches(1);
        if (pdl)
            return kind == 0 ? launch_pdl(combine_update_kernel<0, SL>, grid, dim3(32, 8), 0, st, cv, args)
                             : launch_pdl(combine_update_kernel<1, SL>, grid, dim3(32, 8), 0, st, cv, args);
        if (kind == 0)
            combine_update_kernel<0, SL><<<grid, dim3(32, 8), 0, st>>>(cv, args);
        else
            combine_update_kernel<1, SL><<<grid, dim3(32, 8), 0, st>>>(cv, args);
        return cudaGetLastError();
    });
}

DSG_CHECK_WORD_ACCESSOR(check_word_epilogue)

}  // namespace dsg
