// Device body of the kernel that finishes one application of W inside
// Algorithm 1 (v, u and residual sums) and performs the next linearized
// x-update on the same pixels, per pixel; shared by the single-image and batched
// kernels.
#pragma once

#include "combine.cuh"
#include "common.cuh"
#include "internal.h"
#include "xupdate.cuh"

namespace dsg {

// Sum of the phase-1 partial regions at pixel (i, j) for an epilogue tile that
// lies inside one phase-1 tile (ty, tx): the candidate tiles are the same for the
// whole block; per pixel only the halo tests differ.  Fixed order: own tile, the
// tile above, left, upper left, right, upper right; slices innermost.
constexpr int kGatherGroup = 4;  // slices whose partial-region loads are issued together

struct TileCover {
    const float* part0;  // the partial regions (slice 0, tile 0) and the floats allocated there
    long long cap;
    const float* own;  // region of (ty, tx), slice 0
    size_t region, slice_stride;
    int RW, rs, slices;
    bool up_ok, left_ok, right_ok;
    int up_d, left_d, right_d;  // region offsets (in floats) of the neighbours
};

__device__ __forceinline__ TileCover tile_cover(const Cover& cv, int y0, int x0) {
    TileCover c;
    const int ty = y0 / kTmaTH, tx = x0 / kTmaTW;
    c.rs = cv.rs;
    c.RW = kTmaTW + 2 * cv.rs;
    c.region = (size_t)(kTmaTH + cv.rs) * c.RW;
    c.slice_stride = (size_t)cv.tiles_y * cv.tiles_x * c.region;
    c.slices = cv.slices;
    c.part0 = cv.part;
    c.cap = cv.cap;
    c.own = cv.part + ((size_t)ty * cv.tiles_x + tx) * c.region;
    c.up_ok = ty > 0;
    c.left_ok = tx > 0;
    c.right_ok = tx + 1 < cv.tiles_x;
    c.up_d = -cv.tiles_x * (int)c.region;
    c.left_d = -(int)c.region;
    c.right_d = (int)c.region;
    return c;
}

// One partial-sum load of a gather (checked build: only inside the allocation)
__device__ __forceinline__ float ld_part(const TileCover& c, const float* p) {
    return DSG_IN_RANGE(p - c.part0, c.cap, kChkPartials) ? __ldcg(p) : 0.f;
}

// Stopping rule of the balance (Eq. S2 iterated): stop at max |d t - 1| <= tol, at
// maxit (not converged), or when three passes bring no 1% improvement (stalled).
__device__ __forceinline__ void balance_decide(BalanceCtl* ctl, float e, float m, cudaGraphConditionalHandle cond,
                                               int use_cond) {
    const int pass = ctl->pass;
    const double ed = (double)e;
    ctl->eps = ed;
    ctl->m = (double)m;
    ctl->inv_m = (float)(1.0 / (double)m);
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

// Sum of the regions that cover pixel (li, lj) of the tile, per slice in the order
// own, up, left, upper left, right, upper right.  SL > 0: the slice count known at
// compile time, so that the whole sum unrolls and its loads are issued together
// with the caller's other loads (a region that does not cover the pixel adds an
// exact zero).  SL = 0: any slice count, in groups of kGatherGroup slices whose
// loads are issued before their sums.
template <int SL = 0>
__device__ __forceinline__ float tile_gather(const TileCover& c, int li, int lj) {
    const int rs = c.rs, RW = c.RW;
    const bool up = c.up_ok && li < rs;
    const bool left = c.left_ok && lj < rs;
    const bool right = c.right_ok && lj >= kTmaTW - rs;
    const int own_cell = li * RW + lj + rs;
    const int up_cell = (li + kTmaTH) * RW + lj + rs;
    float acc = 0.f;
    const float* base = c.own;
    if constexpr (SL > 0) {
#pragma unroll
        for (int sl = 0; sl < SL; ++sl, base += c.slice_stride) {
            const float v0 = ld_part(c, base + own_cell);
            const float v1 = up ? ld_part(c, base + c.up_d + up_cell) : 0.f;
            const float v2 = left ? ld_part(c, base + c.left_d + own_cell + kTmaTW) : 0.f;
            const float v3 = (left && up) ? ld_part(c, base + c.up_d + c.left_d + up_cell + kTmaTW) : 0.f;
            const float v4 = right ? ld_part(c, base + c.right_d + own_cell - kTmaTW) : 0.f;
            const float v5 = (right && up) ? ld_part(c, base + c.up_d + c.right_d + up_cell - kTmaTW) : 0.f;
            acc += v0;
            acc += v1;
            acc += v2;
            acc += v3;
            acc += v4;
            acc += v5;
        }
    } else {
        // the counts of the common plans take their unrolled forms
        switch (c.slices) {
            case 1: return tile_gather<1>(c, li, lj);
            case 2: return tile_gather<2>(c, li, lj);
            case 3: return tile_gather<3>(c, li, lj);
            case 4: return tile_gather<4>(c, li, lj);
            default: break;
        }
        for (int s0 = 0; s0 < c.slices; s0 += kGatherGroup) {
            float v[kGatherGroup][6];
#pragma unroll
            for (int k = 0; k < kGatherGroup; ++k) {
                const bool ok = s0 + k < c.slices;
                const float* b = base + (ok ? (size_t)(s0 + k) * c.slice_stride : 0);
                v[k][0] = ok ? ld_part(c, b + own_cell) : 0.f;
                v[k][1] = (ok && up) ? ld_part(c, b + c.up_d + up_cell) : 0.f;
                v[k][2] = (ok && left) ? ld_part(c, b + c.left_d + own_cell + kTmaTW) : 0.f;
                v[k][3] = (ok && left && up) ? ld_part(c, b + c.up_d + c.left_d + up_cell + kTmaTW) : 0.f;
                v[k][4] = (ok && right) ? ld_part(c, b + c.right_d + own_cell - kTmaTW) : 0.f;
                v[k][5] = (ok && right && up) ? ld_part(c, b + c.up_d + c.right_d + up_cell - kTmaTW) : 0.f;
            }
#pragma unroll
            for (int k = 0; k < kGatherGroup; ++k) {
                if (s0 + k >= c.slices) break;
                acc += v[k][0];
                if (up) acc += v[k][1];
                if (left) {
                    acc += v[k][2];
                    if (up) acc += v[k][3];
                }
                if (right) {
                    acc += v[k][4];
                    if (up) acc += v[k][5];
                }
            }
        }
    }
    return acc;
}

// The same sum with TwoSum compensation, in the fixed order of gather_partials
// (per slice: upper left, up, upper right, left, own, right); a region that does
// not cover the pixel contributes an exact zero, which leaves the sum unchanged.
// SL > 0: every slice's loads at once; SL = 0: groups of kGatherGroup slices.
template <int SL = 0>
__device__ __forceinline__ float tile_gather_comp(const TileCover& c, int li, int lj) {
    const int rs = c.rs, RW = c.RW;
    const bool up = c.up_ok && li < rs;
    const bool left = c.left_ok && lj < rs;
    const bool right = c.right_ok && lj >= kTmaTW - rs;
    const int own_cell = li * RW + lj + rs;
    const int up_cell = (li + kTmaTH) * RW + lj + rs;
    if constexpr (SL == 0) {  // the counts of the common plans take their unrolled forms
        switch (c.slices) {
            case 1: return tile_gather_comp<1>(c, li, lj);
            case 2: return tile_gather_comp<2>(c, li, lj);
            case 3: return tile_gather_comp<3>(c, li, lj);
            case 4: return tile_gather_comp<4>(c, li, lj);
            default: break;
        }
    }
    CompSum acc;
    const float* base = c.own;
    constexpr int kG = SL > 0 ? SL : kGatherGroup;
    const int ns = SL > 0 ? SL : c.slices;
    for (int s0 = 0; s0 < ns; s0 += kG) {
        float v[kG][6];
#pragma unroll
        for (int k = 0; k < kG; ++k) {
            const bool ok = s0 + k < ns;
            const float* b = base + (ok ? (size_t)(s0 + k) * c.slice_stride : 0);
            v[k][0] = (ok && up && left) ? ld_part(c, b + c.up_d + c.left_d + up_cell + kTmaTW) : 0.f;
            v[k][1] = (ok && up) ? ld_part(c, b + c.up_d + up_cell) : 0.f;
            v[k][2] = (ok && up && right) ? ld_part(c, b + c.up_d + c.right_d + up_cell - kTmaTW) : 0.f;
            v[k][3] = (ok && left) ? ld_part(c, b + c.left_d + own_cell + kTmaTW) : 0.f;
            v[k][4] = ok ? ld_part(c, b + own_cell) : 0.f;
            v[k][5] = (ok && right) ? ld_part(c, b + c.right_d + own_cell - kTmaTW) : 0.f;
        }
#pragma unroll
        for (int k = 0; k < kG; ++k) {
            if (s0 + k >= ns) break;
#pragma unroll
            for (int q = 0; q < 6; ++q) acc.add(v[k][q]);
        }
    }
    return acc.value();
}

// Finish v and u of one iteration on the kXH x kXW tile at (y0, x0) and, when
// do_x, perform the next x-update there from the gradient at each pixel alone:
// SR reads g = A^T(A x - y) computed beforehand (a.g), SPI evaluates h' in place.
// x_in and x_out may be the same buffer.  Stores the tile's residual sums at
// `partials` (two doubles; not when null).  All threads of a (32, 8) block must call it.
template <int KIND, int SL = 0>  // KIND 0 super-resolution, 1 single-photon; SL as tile_gather
__device__ __forceinline__ void combine_update_body(const Cover& cv, const EpilogueArgs& a, int do_x, int y0, int x0,
                                                    double* partials) {
    const int H = a.H, W = a.W;
    const float inv_m = a.inv_m_dev ? __ldg(a.inv_m_dev) : a.inv_m;
    const TileCover tc = tile_cover(cv, y0, x0);
    const int pj = x0 + threadIdx.x;
    const int lj = pj - (x0 / kTmaTW) * kTmaTW;
    float A[2], zs[2], ds[2], ts[2], vo[2], uo[2], xs[2], gs[2];
    int k1[2];
    // per-pixel loads first, then the partial sums: with SL > 0 in the same unrolled
    // loop, so that every load is issued before the first use; with SL = 0 after it
    // (the compiler does not hoist loads across the runtime slice loop)
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int pi = y0 + threadIdx.y + 8 * r;
        const bool ok = pi < H && pj < W;
        const size_t q = (size_t)pi * W + pj;
        zs[r] = ok ? a.z[q] : 0.f;
        ds[r] = ok ? a.d[q] : 0.f;
        ts[r] = ok ? a.t[q] : 0.f;
        vo[r] = ok ? a.v[q] : 0.f;
        uo[r] = ok ? a.u[q] : 0.f;
        xs[r] = (ok && do_x) ? a.x_in[q] : 0.f;
        gs[r] = (ok && KIND == 0 && do_x) ? a.g[q] : 0.f;
        k1[r] = (ok && KIND == 1 && do_x) ? (int)a.counts[q] : 0;
        if constexpr (SL > 0) A[r] = ok ? tile_gather<SL>(tc, threadIdx.y + 8 * r, lj) : 0.f;
    }
    if constexpr (SL == 0) {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int py = threadIdx.y + 8 * r;
            A[r] = (y0 + py < H && pj < W) ? tile_gather(tc, py, lj) : 0.f;
        }
    }
    float sp = 0.f, sd = 0.f;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int pi = y0 + threadIdx.y + 8 * r;
        if (pi >= H || pj >= W) continue;
        const size_t q = (size_t)pi * W + pj;
        // v = W z with z = x + u: c_s z_s + (d_s / m) sum_{r != s} K1 d_r z_r
        const float dm = ds[r] * inv_m;
        const float cs = 1.f - dm * (ts[r] - ds[r]);
        const float vn = fmaf(dm, A[r], cs * zs[r]);
        const float un = zs[r] - vn;  // u + x - v
        a.v[q] = vn;
        a.u[q] = un;
        const float dp = un - uo[r], dd = vn - vo[r];  // x - v and v - v_prev
        sp = fmaf(dp, dp, sp);
        sd = fmaf(dd, dd, sd);
        if (do_x) {
            const float g = KIND == 0 ? gs[r] : spi_hprime(xs[r], k1[r], a.K, a.eta, a.eps);
            const float xn = project(a.mu * (a.alpha * xs[r] + a.rho * (vn - un) - g), a.constraint);
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
    if (t == 0 && partials) {
        double pa = 0.0, pb = 0.0;
        for (int w = 0; w < 8; ++w) {
            pa += (double)s0[w];
            pb += (double)s1[w];
        }
        partials[0] = pa;
        partials[1] = pb;
    }
}

// Update rule of the current pass: the plain symmetric Sinkhorn step, or (from
// ctl->plain_passes on, accelerated scheme) the over-relaxed step with momentum.
struct PassRule {
    bool accel;
    float half_relax, momentum;
};

__device__ __forceinline__ PassRule pass_rule(const BalanceCtl* ctl) {
    PassRule r;
    const float relax = ctl->relax, mom = ctl->momentum;
    r.accel = relax > 0.f && ctl->pass >= ctl->plain_passes;  // a zeroed block is the plain scheme
    r.half_relax = 0.5f * relax;
    r.momentum = mom;
    return r;
}

// One thread's share of a balancing pass's epilogue (Eq. S2 iterated) on the
// kXH x kXW tile at (y0, x0): pixels (y0 + ry, x0 + cx) and (y0 + ry + 8, x0 + cx).
// t = K1 d (K1(s, s) = 1), the next scaling, and the running maxima e = max |d t - 1|
// and m = max d t.  The plain step is d <- sqrt(d / t).  The accelerated step
// works on u = log d: u <- u - relax (u + log t) / 2 + momentum (u - u_prev), i.e.
// d <- d (d t)^(-relax/2) (d / d_prev)^momentum, with both logarithms formed from
// quantities near one (log1p of d t - 1 and of (d - d_prev) / d_prev) and the
// factor applied as d + d expm1(.), so that the step keeps the relative precision
// of d near convergence.  d_prev is read from d_out before it is overwritten (the
// two scaling buffers alternate, so d_out holds the scaling of two passes back).
template <int SL = 0>
__device__ __forceinline__ void balance_pixels(const Cover& cv, int H, int W, const float* __restrict__ d_in,
                                               float* __restrict__ d_out, float* __restrict__ t_out, int y0, int x0,
                                               int cx, int ry, const PassRule& rule, float& e, float& m) {
    const TileCover tc = tile_cover(cv, y0, x0);
    const int pj = x0 + cx;
    const int lj = pj - (x0 / kTmaTW) * kTmaTW;
    // both rows' loads before the first store
    float dv[2], gv[2], dp[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int py = ry + 8 * r;
        const bool ok = y0 + py < H && pj < W;
        const size_t s = (size_t)(y0 + py) * W + pj;
        dv[r] = ok ? d_in[s] : 0.f;
        dp[r] = (ok && rule.accel) ? d_out[s] : 1.f;
        gv[r] = ok ? tile_gather_comp<SL>(tc, py, lj) : 0.f;
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int pi = y0 + ry + 8 * r;
        if (pi >= H || pj >= W) continue;
        const size_t s = (size_t)pi * W + pj;
        const float ds = dv[r];
        const float tt = ds + gv[r];  // (K1 d)_s with K1(s, s) = 1
        if (rule.accel) {
            const float lf = fmaf(-rule.half_relax, log1pf(fmaf(ds, tt, -1.f)),
                                  rule.momentum * log1pf((ds - dp[r]) / dp[r]));
            d_out[s] = fmaf(ds, expm1f(lf), ds);
        } else {
            d_out[s] = sqrtf(ds / tt);
        }
        t_out[s] = tt;
        e = fmaxf(e, fabsf(fmaf(ds, tt, -1.f)));  // |d_s t_s - 1| with a single rounding
        m = fmaxf(m, ds * tt);
    }
}

}  // namespace dsg
