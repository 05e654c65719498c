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

// Sum of the phase-1 partial regions at pixel (i, j) for an epilogue tile that
// lies inside one phase-1 tile (ty, tx): the candidate tiles are the same for the
// whole block; per pixel only the halo tests differ.  Fixed order: own tile, the
// tile above, left, upper left, right, upper right; slices innermost.
struct TileCover {
    const float* own;  // region of (ty, tx), slice 0
    size_t region, slice_stride;
    int RW, rs, slices;
    bool up_ok, left_ok, right_ok;
    long long up_d, left_d, right_d;  // region offsets (in floats) of the neighbours
};

__device__ __forceinline__ TileCover tile_cover(const Cover& cv, int y0, int x0) {
    TileCover c;
    const int ty = y0 / kTmaTH, tx = x0 / kTmaTW;
    c.rs = cv.rs;
    c.RW = kTmaTW + 2 * cv.rs;
    c.region = (size_t)(kTmaTH + cv.rs) * c.RW;
    c.slice_stride = (size_t)cv.tiles_y * cv.tiles_x * c.region;
    c.slices = cv.slices;
    c.own = cv.part + ((size_t)ty * cv.tiles_x + tx) * c.region;
    c.up_ok = ty > 0;
    c.left_ok = tx > 0;
    c.right_ok = tx + 1 < cv.tiles_x;
    c.up_d = -(long long)cv.tiles_x * (long long)c.region;
    c.left_d = -(long long)c.region;
    c.right_d = (long long)c.region;
    return c;
}

__device__ __forceinline__ float tile_gather(const TileCover& c, int li, int lj) {
    const int rs = c.rs, RW = c.RW;
    const bool up = c.up_ok && li < rs;
    const bool left = c.left_ok && lj < rs;
    const bool right = c.right_ok && lj >= kTmaTW - rs;
    const size_t own_cell = (size_t)li * RW + lj + rs;
    const size_t up_cell = (size_t)(li + kTmaTH) * RW + lj + rs;
    float acc = 0.f;
    const float* base = c.own;
    for (int sl = 0; sl < c.slices; ++sl, base += c.slice_stride) {
        acc += __ldcg(base + own_cell);
        if (up) acc += __ldcg(base + c.up_d + up_cell);
        if (left) {
            acc += __ldcg(base + c.left_d + own_cell + kTmaTW);
            if (up) acc += __ldcg(base + c.up_d + c.left_d + up_cell + kTmaTW);
        }
        if (right) {
            acc += __ldcg(base + c.right_d + own_cell - kTmaTW);
            if (up) acc += __ldcg(base + c.up_d + c.right_d + up_cell - kTmaTW);
        }
    }
    return acc;
}

template <int KIND>  // 0 super-resolution, 1 single-photon
__global__ void __launch_bounds__(256, 3)
combine_xupdate_kernel(Cover cv, EpilogueArgs a) {
    __shared__ SrTile tile;
    const int y0 = blockIdx.y * kXH, x0 = blockIdx.x * kXW;
    const int H = a.H, W = a.W;
    const bool sr_x = KIND == 0 && a.do_x;
    SrTileRegs rg;
    if (sr_x) {
        sr_tile_index(tile, H, W, a.taps, y0, x0);
        sr_tile_load(tile, a.x_in, a.y, W, rg);
    }
    // per-pixel inputs of the combine, issued before the tile's shared-memory phases
    const TileCover tc = tile_cover(cv, y0, x0);
    const int pj = x0 + threadIdx.x;
    const int lj = pj - (x0 / kTmaTW) * kTmaTW;
    float A[2], zs[2], ds[2], ts[2], vo[2], uo[2], xs[2];
    int k1[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int py = threadIdx.y + 8 * r;
        const int pi = y0 + py;
        const bool ok = pi < H && pj < W;
        const size_t q = (size_t)pi * W + pj;
        A[r] = ok ? tile_gather(tc, py, lj) : 0.f;
        zs[r] = ok ? a.z[q] : 0.f;
        ds[r] = ok ? a.d[q] : 0.f;
        ts[r] = ok ? a.t[q] : 0.f;
        vo[r] = ok ? a.v[q] : 0.f;
        uo[r] = ok ? a.u[q] : 0.f;
        xs[r] = (ok && KIND == 1 && a.do_x) ? a.x_in[q] : 0.f;
        k1[r] = (ok && KIND == 1 && a.do_x) ? (int)a.counts[q] : 0;
    }
    if (sr_x) sr_tile_compute(tile, rg, a.taps.r);
    float sp = 0.f, sd = 0.f;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int py = threadIdx.y + 8 * r;
        const int pi = y0 + py;
        if (pi >= H || pj >= W) continue;
        const size_t q = (size_t)pi * W + pj;
        // v = W z with z = x + u: c_s z_s + (d_s / m) sum_{r != s} K1 d_r z_r
        const float dm = ds[r] * a.inv_m;
        const float cs = 1.f - dm * (ts[r] - ds[r]);
        const float vn = fmaf(dm, A[r], cs * zs[r]);
        const float un = zs[r] - vn;  // u + x - v
        a.v[q] = vn;
        a.u[q] = un;
        const float dp = un - uo[r], dd = vn - vo[r];  // x - v and v - v_prev
        sp = fmaf(dp, dp, sp);
        sd = fmaf(dd, dd, sd);
        if (a.do_x) {
            float xv, g;
            if (KIND == 0) {
                xv = sr_tile_x(tile, pi, pj);
                g = sr_tile_grad(tile, a.taps.r, py, pj);
            } else {
                xv = xs[r];
                g = spi_hprime(xv, k1[r], a.K, a.eta, a.eps);
            }
            const float xn = project(a.mu * (a.alpha * xv + a.rho * (vn - un) - g), a.constraint);
            a.x_out[q] = xn;
            a.z[q] = xn + un;
        }
    }
    sp = warp_sum_f(sp);
    sd = warp_sum_f(sd);
    __shared__ float s0[8], s1[8];
    const int t = threadIdx.y * 32 + threadIdx.x;
    if ((t & 31) == 0) {
        s0[t >> 5] = sp;
        s1[t >> 5] = sd;
    }
    __syncthreads();
    if (t == 0) {
        double pa = 0.0, pb = 0.0;
        for (int w = 0; w < 8; ++w) {
            pa += (double)s0[w];
            pb += (double)s1[w];
        }
        const size_t bid = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
        a.partials[2 * bid] = pa;
        a.partials[2 * bid + 1] = pb;
    }
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
