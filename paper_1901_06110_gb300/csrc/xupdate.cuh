// Device helpers of the linearized x-update (Algorithm 1, first two steps) shared
// by the stand-alone x-update kernels and the kernel that fuses the combine of a
// W application with the next x-update.
#pragma once

#include "common.cuh"
#include "internal.h"

namespace dsg {

__device__ __forceinline__ float project(float x, int constraint) {
    if (constraint == 2) return fminf(fmaxf(x, 0.f), 1.f);
    if (constraint == 1) return fmaxf(x, 0.f);
    return x;
}

// h'(max(x, eps)) of the single-photon likelihood (Eq. obj), 1 - e^{-z} = -expm1(-z)
__device__ __forceinline__ float spi_hprime(float xv, int k1, int K, float eta, float eps) {
    const float t = fmaxf(xv, eps);
    const float zz = eta * t / (float)K;
    const float em = -expm1f(-zz);
    const float e = expf(-zz);
    return (eta / (float)K) * ((float)(K - k1) - (float)k1 * e / em);
}

// Super-resolution gradient on a kXH x kXW tile of high-resolution pixels.  The
// tile stages the x values it depends on (the adjoint needs r = A x - y on the
// low-resolution pixels within blur_r of the tile, and each of those needs x
// within blur_r of its even pixel), forms r on that low-resolution window with
// separable sums, then the vertical half of A^T r; sr_tile_grad finishes A^T r at
// one pixel.
constexpr int kXH = 16, kXW = 32;
constexpr int kMaxBlurR = 8;
constexpr int kLH = (kXH - 1 + 2 * kMaxBlurR) / 2 + 2 + 1;  // low-res rows, worst case
constexpr int kLW = (kXW - 1 + 2 * kMaxBlurR) / 2 + 2 + 1;  // low-res cols, worst case
constexpr int kSH = 2 * (kLH - 1) + 2 * kMaxBlurR + 1;      // staged x rows
constexpr int kSW = 2 * (kLW - 1) + 2 * kMaxBlurR + 1;      // staged x cols

__device__ __forceinline__ int floor_div2(int a) { return a >> 1; }  // arithmetic shift: floor(a / 2)

struct SrTile {
    float X[kSH * kSW];
    float Hs[kSH * kLW];
    float Rl[kLH * kLW];
    float V[kXH * kLW];
    int rows[kSH], cols[kSW];
    int lrows[kLH], lcols[kLW];  // wrapped low-resolution indices of the window
    float tp[2 * kMaxBlurR + 1];
    int qy_lo, qx_lo, G, y0, LH, LW, SH, SW;
};

// The tile's work is split so that every global load is issued before the first
// shared-memory phase: sr_tile_index (index tables; synchronises), sr_tile_load
// (global loads into registers, no synchronisation: a caller can issue its own
// loads alongside) and sr_tile_compute (smem phases; synchronises).  All threads
// of a (32, 8) block must call the three in order.  Loops run over 2-D thread
// coordinates, so no index is divided at run time.
constexpr int kXRows = (kSH + 7) / 8;   // staged x rows per thread
constexpr int kXCols = (kSW + 31) / 32;  // staged x columns per thread
constexpr int kYRows = (kLH + 7) / 8;    // low-resolution rows per thread
struct SrTileRegs {
    float x[kXRows][kXCols];
    float y[kYRows];
};

__device__ __forceinline__ void sr_tile_index(SrTile& T, int H, int W, const BlurTaps& taps, int y0, int x0) {
    const int R = taps.r;
    const int G = R > 0 ? R : 1;  // staging margin (covers the tile's own pixels when R = 0)
    const int h = H / 2, w = W / 2;
    const int qy_lo = floor_div2(y0 - G), qy_hi = floor_div2(y0 + kXH - 1 + G);
    const int qx_lo = floor_div2(x0 - G), qx_hi = floor_div2(x0 + kXW - 1 + G);
    const int LH = qy_hi - qy_lo + 1, LW = qx_hi - qx_lo + 1;
    const int SH = 2 * (LH - 1) + 2 * G + 1, SW = 2 * (LW - 1) + 2 * G + 1;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    if (tid == 0) {
        T.qy_lo = qy_lo;
        T.qx_lo = qx_lo;
        T.G = G;
        T.y0 = y0;
        T.LH = LH;
        T.LW = LW;
        T.SH = SH;
        T.SW = SW;
    }
    for (int a = tid; a < SH; a += 256) T.rows[a] = wrap_index(2 * qy_lo - G + a, H);
    for (int b = tid; b < SW; b += 256) T.cols[b] = wrap_index(2 * qx_lo - G + b, W);
    for (int l = tid; l < LH; l += 256) T.lrows[l] = wrap_index(qy_lo + l, h);
    for (int c = tid; c < LW; c += 256) T.lcols[c] = wrap_index(qx_lo + c, w);
    if (tid < 2 * R + 1) T.tp[tid] = taps.t[tid];
    __syncthreads();
}

__device__ __forceinline__ void sr_tile_load(const SrTile& T, const float* __restrict__ x_in,
                                             const float* __restrict__ y, int W, SrTileRegs& rg) {
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int w = W / 2;
#pragma unroll
    for (int ia = 0; ia < kXRows; ++ia) {
        const int a = ty + 8 * ia;
#pragma unroll
        for (int ib = 0; ib < kXCols; ++ib) {
            const int b = tx + 32 * ib;
            rg.x[ia][ib] = (a < T.SH && b < T.SW) ? __ldg(x_in + (size_t)T.rows[a] * W + T.cols[b]) : 0.f;
        }
    }
    // the low-resolution column of this lane (one per lane: LW <= 32 for blur radii up to 8)
#pragma unroll
    for (int il = 0; il < kYRows; ++il) {
        const int l = ty + 8 * il;
        rg.y[il] = (l < T.LH && tx < T.LW) ? __ldg(y + (size_t)T.lrows[l] * w + T.lcols[tx]) : 0.f;
    }
}

__device__ __forceinline__ void sr_tile_compute(SrTile& T, const SrTileRegs& rg, int R) {
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int G = T.G, SH = T.SH, SW = T.SW, LH = T.LH, LW = T.LW, qy_lo = T.qy_lo, y0 = T.y0;
#pragma unroll
    for (int ia = 0; ia < kXRows; ++ia) {
        const int a = ty + 8 * ia;
#pragma unroll
        for (int ib = 0; ib < kXCols; ++ib) {
            const int b = tx + 32 * ib;
            if (a < SH && b < SW) T.X[a * kSW + b] = rg.x[ia][ib];
        }
    }
    __syncthreads();
    // horizontal blur sums at the even columns 2 qx: staged column 2c + G - b
    for (int a = ty; a < SH; a += 8) {
        for (int c = tx; c < LW; c += 32) {
            const float* xr = T.X + a * kSW + 2 * c + G;
            float acc = 0.f;
            for (int b = -R; b <= R; ++b) acc = fmaf(T.tp[b + R], xr[-b], acc);
            T.Hs[a * kLW + c] = acc;
        }
    }
    __syncthreads();
    // r = A x - y on the low-resolution window
#pragma unroll
    for (int il = 0; il < kYRows; ++il) {
        const int l = ty + 8 * il;
        if (l < LH && tx < LW) {
            const float* hc = T.Hs + (2 * l + G) * kLW + tx;
            float acc = 0.f;
            for (int a = -R; a <= R; ++a) acc = fmaf(T.tp[a + R], hc[-a * kLW], acc);
            T.Rl[l * kLW + tx] = acc - rg.y[il];
        }
    }
    __syncthreads();
    // vertical adjoint sums: V(p_y, c) = sum_{a : p_y + a even} t(a) r((p_y + a) / 2, c)
    for (int py = ty; py < kXH; py += 8) {
        const int p = y0 + py;
        const int a0 = -R + ((p - R) & 1);
        for (int c = tx; c < LW; c += 32) {
            float acc = 0.f;
            for (int a = a0; a <= R; a += 2)
                acc = fmaf(T.tp[a + R], T.Rl[(((p + a) >> 1) - qy_lo) * kLW + c], acc);
            T.V[py * kLW + c] = acc;
        }
    }
    __syncthreads();
}

// (A^T (A x - y)) at tile row py, image column pj
__device__ __forceinline__ float sr_tile_grad(const SrTile& T, int R, int py, int pj) {
    float g = 0.f;
    for (int b = -R + ((pj - R) & 1); b <= R; b += 2)
        g = fmaf(T.tp[b + R], T.V[py * kLW + ((pj + b) >> 1) - T.qx_lo], g);
    return g;
}

// staged x at image pixel (pi, pj) of the tile
__device__ __forceinline__ float sr_tile_x(const SrTile& T, int pi, int pj) {
    return T.X[(pi - (2 * T.qy_lo - T.G)) * kSW + (pj - (2 * T.qx_lo - T.G))];
}

// Linearized x-update (Algorithm 1, first two steps) for super-resolution on the
// kXH x kXW tile at (y0, x0): x_out = Pi_C(mu (alpha x_in + rho (v - u) - A^T(A x_in - y))),
// z = x_out + u.  All threads of a (32, 8) block must call it.
__device__ __forceinline__ void sr_xupdate_body(SrTile& tile, const float* __restrict__ x_in,
                                                float* __restrict__ x_out, const float* __restrict__ y, int H,
                                                int W, const BlurTaps& taps, const float* __restrict__ v,
                                                const float* __restrict__ u, float* __restrict__ z, float mu,
                                                float alpha, float rho, int constraint, int y0, int x0) {
    sr_tile_index(tile, H, W, taps, y0, x0);
    SrTileRegs rg;
    sr_tile_load(tile, x_in, y, W, rg);
    // prefetch the per-pixel inputs while the tile loads are in flight
    const int pj = x0 + threadIdx.x;
    float vv[2], uu[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int pi = y0 + threadIdx.y + 8 * r;
        const bool ok = pi < H && pj < W;
        const size_t q = (size_t)pi * W + pj;
        vv[r] = ok ? v[q] : 0.f;
        uu[r] = ok ? u[q] : 0.f;
    }
    sr_tile_compute(tile, rg, taps.r);
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int py = threadIdx.y + 8 * r;
        const int pi = y0 + py;
        if (pi >= H || pj >= W) continue;
        const float g = sr_tile_grad(tile, taps.r, py, pj);
        const size_t q = (size_t)pi * W + pj;
        const float xv = sr_tile_x(tile, pi, pj);
        const float xn = project(mu * (alpha * xv + rho * (vv[r] - uu[r]) - g), constraint);
        x_out[q] = xn;
        z[q] = xn + uu[r];
    }
}

}  // namespace dsg
