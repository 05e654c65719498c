// TMA-pipelined stencil pass over the half-window weight planes (the aggregation
// loops of Algorithm 2): A(s) = sum_{r != s} K1(s, r) q(r) for a per-pixel field q
// (q = d for a balancing pass, q = d z for an application of W).
//
// Each weight K1(s, s + o) is read from HBM exactly once and used twice: for the
// forward term K1(s, s+o) q(s+o) of pixel s and for the mirrored term
// K1(s, s+o) q(s) of pixel s + o (symmetry of K1).
//
// Phase 1 (one CTA per spatial tile of kTH x kTW pixels and per slice of the
// offsets): a producer warp streams the tile of every plane of the slice into a
// ring of shared-memory stages with cp.async.bulk.tensor (TMA) and mbarriers.
// Consumer thread c owns column c of the tile (kTH pixels).  Offsets are visited
// column-offset first (fixed o_x, then o_y = 0..N_s), so that for one o_x
//   - the forward neighbours q(i + o_y, j + o_x) of the thread's pixels form one
//     column strip of kTH + N_s values held in registers, and
//   - the mirrored contributions land in one column strip (column j + o_x) of
//     kTH + N_s register accumulators,
// which makes every weight cost one shared-memory load and two FMAs.  After each
// o_x the strips are added, with an error-free transformation, into a shared
// accumulator covering the tile plus the halo its mirrored terms reach (N_s rows
// below, N_s columns either side); consumers synchronise once per o_x, so no two
// threads update the same column at once.  The accumulator (tile + halo) is
// written to a per-CTA partial region.
//
// Phase 2 (one thread per pixel) adds, in a fixed order, the partial regions of
// the up to six tiles and every offset slice that cover the pixel, then applies
// the pass's epilogue: the balancing update and residual reduction, W z with the
// diagonal closure of Eq. S3, or W z fused with the dual update of Algorithm 1.
// Results do not depend on scheduling: every sum has a fixed order.
#include <cuda.h>

#include "combine.cuh"
#include "common.cuh"
#include "internal.h"
#include "launch.h"
#include "tma.cuh"

namespace dsg {

namespace {

constexpr int kTH = kTmaTH;              // tile rows (= pixels per consumer thread)
constexpr int kTW = kTmaTW;              // tile columns (= consumer threads)
constexpr int kConsumers = kTW;
constexpr int kConsumerWarps = kConsumers / 32;
constexpr int kThreads = kConsumers + 32;  // + one producer warp
constexpr long long kWaitBudget = kDefaultWaitBudget;  // cycles (about 2 s) before a wait gives up

// Wait for the phase with the given parity to complete; false after the budget.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > kWaitBudget) return false;
    }
    return true;
}

// The producer's wait for a free stage: ends early once the consumers have given
// up (they release no more stages), otherwise after kWaitBudget.
__device__ __forceinline__ bool mbar_wait_or_abort(uint64_t* bar, unsigned parity, const int* abort_flag) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (*(const volatile int*)abort_flag) return false;
        if (clock64() - t0 > kWaitBudget) return false;
    }
    return true;
}

__device__ __forceinline__ void consumer_sync() {
    asm volatile("bar.sync 1, %0;" ::"n"(kConsumers) : "memory");
}

__device__ __forceinline__ void two_sum_into(float& hi, float& lo, float b) {
    const float s = __fadd_rn(hi, b);
    const float bb = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    hi = s;
    lo = __fadd_rn(lo, e);
}

__host__ __device__ __forceinline__ int plane_index(int oy, int ox, int rs) {
    return oy == 0 ? ox - 1 : rs + (oy - 1) * (2 * rs + 1) + ox + rs;
}

// FP32 weights: the strips are flushed into the shared accumulator with an
// error-free transformation (hi + lo), so the pass sums are as accurate as the
// weights themselves and the balance can reach tolerances near 1e-8.  16-bit
// weights carry a rounding error of 2^-11 (FP16) or 2^-8 (BF16) already; their
// strips are added in plain FP32, which drops the lo half of the accumulator and
// the separate per-offset forward sum, so that four CTAs fit on an SM instead of two.
template <typename WT> struct P1Traits {
    static constexpr bool kComp = true;
    static constexpr int kMinBlocks = 2;
};
#ifndef DSG_P1_HALF_BLOCKS
#define DSG_P1_HALF_BLOCKS 4
#endif
template <> struct P1Traits<__half> {
    static constexpr bool kComp = false;
    static constexpr int kMinBlocks = DSG_P1_HALF_BLOCKS;
};
template <> struct P1Traits<__nv_bfloat16> {
    static constexpr bool kComp = false;
    static constexpr int kMinBlocks = DSG_P1_HALF_BLOCKS;
};

// Pipeline stages of the weight ring: 8 at two CTAs per SM; four CTAs per SM
// share the shared memory with fewer stages each.
template <typename WT, int RS> constexpr int p1_stages() {
    return P1Traits<WT>::kMinBlocks >= 4 ? (RS <= 10 ? 6 : 5) : 8;
}

// Phase 1 for one tile at (x0, y0) and the column offsets oxa..oxb: writes the
// tile's partial region (kTH + RS rows, kTW + 2 RS columns) to `out`.
template <int RS, typename WT>
__device__ __forceinline__ void p1_body(const CUtensorMap* tmap, int H, int W, const float* __restrict__ d,
                                        const float* __restrict__ z, int oxa, int oxb, int x0, int y0,
                                        float* __restrict__ out, unsigned* __restrict__ err, long long cbudget) {
    constexpr bool kComp = P1Traits<WT>::kComp;
    constexpr int kStages = p1_stages<WT, RS>();
    constexpr int RH = kTH + RS;
    constexpr int RW = kTW + 2 * RS;
    constexpr int kStageElems = kTH * kTW;

    extern __shared__ __align__(128) unsigned char smem_raw[];
    WT* stages = reinterpret_cast<WT*>(smem_raw);
    float* qt = reinterpret_cast<float*>(smem_raw + kStages * kStageElems * sizeof(WT));
    float* acc_hi = qt + RH * RW;
    float* acc_lo = acc_hi + RH * RW;  // used with kComp only
    uint64_t* full = reinterpret_cast<uint64_t*>(acc_hi + (kComp ? 2 : 1) * RH * RW);
    uint64_t* empty = full + kStages;
    __shared__ int s_abort;

    const int tid = threadIdx.x;

    if (tid == 0) {
        s_abort = 0;
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kConsumerWarps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();

    if (tid >= kConsumers) {
        // producer: one elected thread streams the plane tiles in consumption order;
        // the first kStages loads overlap the consumers' staging of q below
        if (tid == kConsumers) {
            const uint64_t policy = evict_first_policy();
            int q = 0, s = 0;
            unsigned ph = 0;  // parity of the ring pass of plane q
            bool ok = true;
            for (int ox = oxa; ox <= oxb && ok; ++ox) {
                for (int oy = ox > 0 ? 0 : 1; oy <= RS; ++oy, ++q) {
                    if (q >= kStages && !mbar_wait_or_abort(&empty[s], ph ^ 1u, &s_abort)) {
                        ok = false;
                        break;
                    }
                    if (*(volatile int*)&s_abort) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(&full[s], kStageElems * sizeof(WT));
                    tma_load_3d(stages + s * kStageElems, tmap, &full[s], x0, y0, plane_index(oy, ox, RS),
                                policy);
                    if (++s == kStages) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
            }
            if (!ok) {
                *(volatile int*)&s_abort = 1;
                atomicOr(err, 1u);
            }
            // do not leave while copies into this CTA's shared memory are in flight
            for (int back = 1; back <= kStages && q - back >= 0; ++back) {
                const int qq = q - back;
                mbar_wait(&full[qq % kStages], (qq / kStages) & 1);
            }
        }
        return;
    }

    // q over the tile + halo (zero outside the image); accumulators cleared.  The
    // loads of kStageBatch cells per thread (all of them for search radii up to 10)
    // are issued before their stores, so the round trips to L2 overlap instead of
    // following one another.
    constexpr int kCells = RH * RW;
    constexpr int kStageBatch = 32;
    for (int base = tid; base < kCells; base += kStageBatch * kConsumers) {
        float v[kStageBatch];
#pragma unroll
        for (int k = 0; k < kStageBatch; ++k) {
            const int idx = base + k * kConsumers;
            const int a = idx / RW, b = idx - a * RW;
            const int i = y0 + a, j = x0 - RS + b;
            const bool in = idx < kCells && i < H && j >= 0 && j < W;
            const size_t p = (size_t)i * W + j;
            const float dv = in ? d[p] : 0.f;
            const float zv = (in && z) ? z[p] : 1.f;
            v[k] = z ? dv * zv : dv;
        }
#pragma unroll
        for (int k = 0; k < kStageBatch; ++k) {
            const int idx = base + k * kConsumers;
            if (idx < kCells) {
                qt[idx] = v[k];
                acc_hi[idx] = 0.f;
                if (kComp) acc_lo[idx] = 0.f;
            }
        }
    }
    consumer_sync();

    // consumers
    const int c = tid;
    const int lane = tid & 31;
    bool ok = true;
    // wait for the next plane, copy this thread's column of it to registers and
    // release the stage
    int cs = 0;
    unsigned cph = 0;  // stage and ring-pass parity of the next plane
    auto fetch = [&](float (&dst)[kTH]) {
        const int s = cs;
        const unsigned ph = cph;
        if (++cs == kStages) {
            cs = 0;
            cph ^= 1u;
        }
        if (ok && (!mbar_wait_consumer(&full[s], ph, cbudget) || *(volatile int*)&s_abort)) {
            ok = false;
            *(volatile int*)&s_abort = 1;
            atomicOr(err, 2u);
        }
        if (!ok) {
#pragma unroll
            for (int r = 0; r < kTH; ++r) dst[r] = 0.f;
            return;
        }
        const WT* st = stages + s * kStageElems;
#pragma unroll
        for (int r = 0; r < kTH; ++r) dst[r] = to_f32(st[r * kTW + c]);
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
    };
    float qo[kTH], tot[kTH], comp[kTH];
#pragma unroll
    for (int r = 0; r < kTH; ++r) {
        qo[r] = qt[r * RW + c + RS];
        tot[r] = 0.f;
        comp[r] = 0.f;
    }
    for (int ox = oxa; ox <= oxb; ++ox) {
        const int col = c + RS + ox;
        float strip[RH], bacc[RH], fw[kTH];
#pragma unroll
        for (int a = 0; a < RH; ++a) {
            strip[a] = qt[a * RW + col];
            bacc[a] = 0.f;
        }
#pragma unroll
        for (int r = 0; r < kTH; ++r) fw[r] = 0.f;
#pragma unroll
        for (int oy = 0; oy <= RS; ++oy) {
            if (oy == 0 && ox <= 0) continue;
            float w[kTH];
            fetch(w);
            // with kComp the forward terms of one o_x are summed apart and added to
            // the total with an error-free transformation; otherwise straight into it
#pragma unroll
            for (int r = 0; r < kTH; ++r) {
                float& f = kComp ? fw[r] : tot[r];
                f = fmaf(w[r], strip[r + oy], f);
                bacc[r + oy] = fmaf(w[r], qo[r], bacc[r + oy]);
            }
        }
        if (kComp) {
#pragma unroll
            for (int r = 0; r < kTH; ++r) two_sum_into(tot[r], comp[r], fw[r]);
        }
        // one o_x at a time: column `col` is updated by this thread only
        consumer_sync();
#pragma unroll
        for (int a = 0; a < RH; ++a) {
            if (kComp)
                two_sum_into(acc_hi[a * RW + col], acc_lo[a * RW + col], bacc[a]);
            else
                acc_hi[a * RW + col] += bacc[a];
        }
    }
    consumer_sync();
#pragma unroll
    for (int r = 0; r < kTH; ++r) {
        if (kComp) {
            two_sum_into(acc_hi[r * RW + c + RS], acc_lo[r * RW + c + RS], tot[r]);
            acc_lo[r * RW + c + RS] += comp[r];
        } else {
            acc_hi[r * RW + c + RS] += tot[r];
        }
    }
    consumer_sync();
    for (int idx = c; idx < RH * RW; idx += kConsumers) out[idx] = kComp ? acc_hi[idx] + acc_lo[idx] : acc_hi[idx];
}


template <int RS, typename WT>
__global__ void __launch_bounds__(kThreads, P1Traits<WT>::kMinBlocks)
stencil_p1_kernel(const __grid_constant__ CUtensorMap tmap, int H, int W, const float* __restrict__ d,
                  const float* __restrict__ z, TmaSplits splits, float* __restrict__ part,
                  unsigned* __restrict__ err, const int* __restrict__ skip, long long cbudget, long long cap) {
    griddep_enter();
    if (skip && *(volatile const int*)skip) return;
    const int slice = blockIdx.z;
    const size_t region = (size_t)(kTH + RS) * (kTW + 2 * RS);
    const size_t roff = ((size_t)(slice * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x) * region;
    if (!DSG_IN_RANGE(roff + region - 1, cap, kChkPartials)) return;  // before any copy is issued
    float* out = part + roff;
    p1_body<RS, WT>(&tmap, H, W, d, z, splits.ox_lo[slice], splits.ox_hi[slice], blockIdx.x * kTW,
                    blockIdx.y * kTH, out, err, cbudget);
}

// One launch over the (instance, tile, slice) work items of a batch of images.
template <int RS, typename WT>
__global__ void __launch_bounds__(kThreads, P1Traits<WT>::kMinBlocks)
stencil_p1_batched_kernel(const __grid_constant__ BatchMaps maps, const BatchInst* __restrict__ insts,
                          const int4* __restrict__ work, unsigned* __restrict__ err) {
    griddep_enter();
    const int4 w = work[blockIdx.x];  // (instance, tile row, tile column, slice)
    const BatchInst& in = insts[w.x];
    if (in.done && *(volatile const int*)in.done) return;
    const size_t region = (size_t)(kTH + RS) * (kTW + 2 * RS);
    const size_t roff = ((size_t)(w.w * in.tiles_y + w.y) * in.tiles_x + w.z) * region;
    if (!DSG_IN_RANGE(roff + region - 1, in.part_cap, kChkPartials)) return;  // before any copy is issued
    float* out = in.part + roff;
    p1_body<RS, WT>(reinterpret_cast<const CUtensorMap*>(maps.m[w.x]), in.H, in.W, in.d, in.z, in.splits.ox_lo[w.w],
                    in.splits.ox_hi[w.w], w.z * kTW, w.y * kTH, out, err, kWaitBudget);
}

// --------------------------------------------------------------------------- phase 2

// W z = c_s z_s + (d_s / m) sum_{r != s} K1 d_r z_r with c_s = 1 - (d_s / m)(t_s - d_s):
// the third aggregation of Algorithm 2 with the diagonal closure of Eq. S3
__global__ void __launch_bounds__(256)
apply_finish_kernel(Cover cv, int H, int W, const float* __restrict__ d, const float* __restrict__ t_fin,
                    float inv_m, const float* __restrict__ z, float* __restrict__ y) {
    griddep_enter();
    const int j = blockIdx.x * 32 + threadIdx.x;
    const int i = blockIdx.y * 8 + threadIdx.y;
    if (i >= H || j >= W) return;
    const size_t s = (size_t)i * W + j;
    const float A = gather_partials(cv, i, j);
    const float ds = d[s];
    const float dm = ds * inv_m;
    const float cs = 1.f - dm * (t_fin[s] - ds);
    y[s] = fmaf(dm, A, cs * z[s]);
}

// hist[k] = fixed-order sums of the per-block residual partials of iteration k
__global__ void __launch_bounds__(256)
reduce_residuals_kernel(SolveRed red, int nblocks) {
    griddep_enter();
    const int iter = blockIdx.x, t = threadIdx.x;
    double a = 0.0, b = 0.0;
    for (int q = t; q < nblocks; q += 256) {
        a += red.partials[2 * ((size_t)iter * nblocks + q)];
        b += red.partials[2 * ((size_t)iter * nblocks + q) + 1];
    }
    __shared__ double ra[256], rb[256];
    ra[t] = a;
    rb[t] = b;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (t < w) {
            ra[t] += ra[t + w];
            rb[t] += rb[t + w];
        }
        __syncthreads();
    }
    if (t == 0) {
        red.hist[2 * iter] = ra[0];
        red.hist[2 * iter + 1] = rb[0];
    }
}

template <int RS, typename WT>
size_t p1_smem_bytes() {
    constexpr int kStages = p1_stages<WT, RS>();
    const int regions = P1Traits<WT>::kComp ? 3 : 2;  // q, acc_hi (, acc_lo)
    return (size_t)kStages * kTH * kTW * sizeof(WT) + regions * sizeof(float) * (size_t)(kTH + RS) * (kTW + 2 * RS) +
           2 * kStages * sizeof(uint64_t);
}

template <int RS, typename WT>
cudaError_t p1_launch(const TmaPlan& plan, int H, int W, const float* d, const float* z, unsigned* err,
                      const int* skip, cudaStream_t st, long long cbudget, bool pdl) {
    const size_t smem = p1_smem_bytes<RS, WT>();
    // set once per instantiation (a thread-safe static initialisation)
    static const cudaError_t configured =
        cudaFuncSetAttribute(stencil_p1_kernel<RS, WT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (configured != cudaSuccess) return configured;
    dim3 grid(plan.tiles_x, plan.tiles_y, plan.splits.n);
    count_launches(1);
    if (pdl)
        return launch_pdl(stencil_p1_kernel<RS, WT>, grid, dim3(kThreads), smem, st, *(const CUtensorMap*)plan.tmap, H,
                          W, d, z, plan.splits, plan.partials, err, skip, cbudget, plan.part_cap);
    stencil_p1_kernel<RS, WT><<<grid, kThreads, smem, st>>>(*(const CUtensorMap*)plan.tmap, H, W, d, z,
                                                            plan.splits, plan.partials, err, skip, cbudget,
                                                            plan.part_cap);
    return cudaGetLastError();
}

template <int RS, typename WT>
cudaError_t p1b_launch(const BatchMaps& maps, const BatchInst* insts, const int4* work, int nwork, unsigned* err,
                       cudaStream_t st) {
    const size_t smem = p1_smem_bytes<RS, WT>();
    static const cudaError_t configured = cudaFuncSetAttribute(
        stencil_p1_batched_kernel<RS, WT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (configured != cudaSuccess) return configured;
    if (nwork <= 0) return cudaSuccess;
    // programmatic stream serialization: the blocks may be scheduled while the previous
    // kernel drains (the kernel waits for it before touching memory)
    const cudaError_t e =
        launch_pdl(stencil_p1_batched_kernel<RS, WT>, dim3(nwork), dim3(kThreads), smem, st, maps, insts, work, err);
    count_launches(1);
    return e;
}

template <typename WT>
cudaError_t p1b_dispatch(int rs, const BatchMaps& maps, const BatchInst* insts, const int4* work, int nwork,
                         unsigned* err, cudaStream_t st) {
    switch (rs) {
        case 1: return p1b_launch<1, WT>(maps, insts, work, nwork, err, st);
        case 2: return p1b_launch<2, WT>(maps, insts, work, nwork, err, st);
        case 3: return p1b_launch<3, WT>(maps, insts, work, nwork, err, st);
        case 4: return p1b_launch<4, WT>(maps, insts, work, nwork, err, st);
        case 5: return p1b_launch<5, WT>(maps, insts, work, nwork, err, st);
        case 6: return p1b_launch<6, WT>(maps, insts, work, nwork, err, st);
        case 7: return p1b_launch<7, WT>(maps, insts, work, nwork, err, st);
        case 8: return p1b_launch<8, WT>(maps, insts, work, nwork, err, st);
        case 10: return p1b_launch<10, WT>(maps, insts, work, nwork, err, st);
        case 12: return p1b_launch<12, WT>(maps, insts, work, nwork, err, st);
        default: return cudaErrorInvalidValue;
    }
}

template <typename WT>
cudaError_t p1_dispatch(int rs, const TmaPlan& plan, int H, int W, const float* d, const float* z,
                        unsigned* err, const int* skip, cudaStream_t st, long long cbudget, bool pdl) {
    switch (rs) {
        case 1: return p1_launch<1, WT>(plan, H, W, d, z, err, skip, st, cbudget, pdl);
        case 2: return p1_launch<2, WT>(plan, H, W, d, z, err, skip, st, cbudget, pdl);
        case 3: return p1_launch<3, WT>(plan, H, W, d, z, err, skip, st, cbudget, pdl);
        case 4: return p1_launch<4, WT>(plan, H, W, d, z, err, skip, st, cbudget, pdl);
        case 5: return p1_launch<5, WT>(plan, H, W, d, z, err, skip, st, cbudget, pdl);
        case 6: return p1_launch<6, WT>(plan, H, W, d, z, err, skip, st, cbudget, pdl);
        case 7: return p1_launch<7, WT>(plan, H, W, d, z, err, skip, st, cbudget, pdl);
        case 8: return p1_launch<8, WT>(plan, H, W, d, z, err, skip, st, cbudget, pdl);
        case 10: return p1_launch<10, WT>(plan, H, W, d, z, err, skip, st, cbudget, pdl);
        case 12: return p1_launch<12, WT>(plan, H, W, d, z, err, skip, st, cbudget, pdl);
        default: return cudaErrorInvalidValue;
    }
}

Cover cover_of(const TmaPlan& plan, int rs) {
    return Cover{plan.partials, plan.tiles_x, plan.tiles_y, plan.splits.n, rs, plan.part_cap};
}

dim3 p2_grid(int H, int W) { return dim3((W + 31) / 32, (H + 7) / 8); }

}  // namespace

DSG_CHECK_WORD_ACCESSOR(check_word_stencil_tma)

bool tma_path_supports(int rs) {
    return rs == 1 || rs == 2 || rs == 3 || rs == 4 || rs == 5 || rs == 6 || rs == 7 || rs == 8 || rs == 10 ||
           rs == 12;
}

int tma_tile_w() { return kTW; }
int tma_ctas_per_sm(int dtype) {
    return dtype == 0 ? P1Traits<float>::kMinBlocks : P1Traits<__half>::kMinBlocks;
}
int tma_tile_h() { return kTH; }
size_t tma_region_floats(int rs) { return (size_t)(kTH + rs) * (kTW + 2 * rs); }
int tma_p2_blocks(int H, int W) {
    const dim3 g = p2_grid(H, W);
    return (int)(g.x * g.y);
}

cudaError_t launch_tma_gather(int dtype, const TmaPlan& plan, int H, int W, int rs, const float* d,
                              const float* z, unsigned* err, const int* skip, cudaStream_t st,
                              long long wait_budget, bool pdl) {
    switch (dtype) {
        case 0: return p1_dispatch<float>(rs, plan, H, W, d, z, err, skip, st, wait_budget, pdl);
        case 1: return p1_dispatch<__half>(rs, plan, H, W, d, z, err, skip, st, wait_budget, pdl);
        default: return p1_dispatch<__nv_bfloat16>(rs, plan, H, W, d, z, err, skip, st, wait_budget, pdl);
    }
}

cudaError_t launch_tma_gather_batched(int dtype, int rs, const BatchMaps& maps, const BatchInst* insts,
                                      const int4* work, int nwork, unsigned* err, cudaStream_t st) {
    switch (dtype) {
        case 0: return p1b_dispatch<float>(rs, maps, insts, work, nwork, err, st);
        case 1: return p1b_dispatch<__half>(rs, maps, insts, work, nwork, err, st);
        default: return p1b_dispatch<__nv_bfloat16>(rs, maps, insts, work, nwork, err, st);
    }
}

cudaError_t launch_tma_apply_finish(const TmaPlan& plan, int H, int W, int rs, const float* d, const float* t,
                                    float inv_m, const float* z, float* y, cudaStream_t st) {
    apply_finish_kernel<<<p2_grid(H, W), dim3(32, 8), 0, st>>>(cover_of(plan, rs), H, W, d, t, inv_m, z, y);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_reduce_residuals(SolveRed red, int iters, int nblocks, cudaStream_t st) {
    if (iters <= 0) return cudaSuccess;
    reduce_residuals_kernel<<<iters, 256, 0, st>>>(red, nblocks);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace dsg
