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

__device__ __forceinline__ int floor_div2(int a) { return a >= 0 ? a / 2 : -((1 - a) / 2); }

struct SrTile {
    float X[kSH * kSW];
    float Hs[kSH * kLW];
    float Rl[kLH * kLW];
    float V[kXH * kLW];
    int rows[kSH], cols[kSW];
    float tp[2 * kMaxBlurR + 1];
    int qy_lo, qx_lo, G, y0;
};

// All threads of a 256-thread block must call this (it synchronises).
__device__ __forceinline__ void sr_tile_prepare(SrTile& T, const float* __restrict__ x_in,
                                                const float* __restrict__ y, int H, int W,
                                                const BlurTaps& taps, int y0, int x0) {
    const int R = taps.r;
    const int G = R > 0 ? R : 1;  // staging margin (covers the tile's own pixels when R = 0)
    const int h = H / 2, w = W / 2;
    const int qy_lo = floor_div2(y0 - G), qy_hi = floor_div2(y0 + kXH - 1 + G);
    const int qx_lo = floor_div2(x0 - G), qx_hi = floor_div2(x0 + kXW - 1 + G);
    const int LH = qy_hi - qy_lo + 1, LW = qx_hi - qx_lo + 1;
    const int SH = 2 * (LH - 1) + 2 * G + 1, SW = 2 * (LW - 1) + 2 * G + 1;
    const int tid = threadIdx.x;
    if (tid == 0) {
        T.qy_lo = qy_lo;
        T.qx_lo = qx_lo;
        T.G = G;
        T.y0 = y0;
    }
    for (int a = tid; a < SH; a += 256) T.rows[a] = wrap_index(2 * qy_lo - G + a, H);
    for (int b = tid; b < SW; b += 256) T.cols[b] = wrap_index(2 * qx_lo - G + b, W);
    if (tid < 2 * R + 1) T.tp[tid] = taps.t[tid];
    __syncthreads();
    for (int idx = tid; idx < SH * SW; idx += 256) {
        const int a = idx / SW, b = idx - a * SW;
        T.X[a * kSW + b] = x_in[(size_t)T.rows[a] * W + T.cols[b]];
    }
    __syncthreads();
    // horizontal blur sums at the even columns 2 qx: staged column 2c + G - b
    for (int idx = tid; idx < SH * LW; idx += 256) {
        const int a = idx / LW, c = idx - a * LW;
        const float* xr = T.X + a * kSW + 2 * c + G;
        float acc = 0.f;
        for (int b = -R; b <= R; ++b) acc = fmaf(T.tp[b + R], xr[-b], acc);
        T.Hs[a * kLW + c] = acc;
    }
    __syncthreads();
    // r = A x - y on the low-resolution window
    for (int idx = tid; idx < LH * LW; idx += 256) {
        const int l = idx / LW, c = idx - l * LW;
        const float* hc = T.Hs + (2 * l + G) * kLW + c;
        float acc = 0.f;
        for (int a = -R; a <= R; ++a) acc = fmaf(T.tp[a + R], hc[-a * kLW], acc);
        const int qy = wrap_index(qy_lo + l, h), qx = wrap_index(qx_lo + c, w);
        T.Rl[l * kLW + c] = acc - y[(size_t)qy * w + qx];
    }
    __syncthreads();
    // vertical adjoint sums: V(p_y, c) = sum_{a : p_y + a even} t(a) r((p_y + a) / 2, c)
    for (int idx = tid; idx < kXH * LW; idx += 256) {
        const int py = idx / LW, c = idx - py * LW;
        const int p = y0 + py;
        float acc = 0.f;
        for (int a = -R + ((p - R) & 1); a <= R; a += 2)
            acc = fmaf(T.tp[a + R], T.Rl[(floor_div2(p + a) - qy_lo) * kLW + c], acc);
        T.V[py * kLW + c] = acc;
    }
    __syncthreads();
}

// (A^T (A x - y)) at tile row py, image column pj
__device__ __forceinline__ float sr_tile_grad(const SrTile& T, int R, int py, int pj) {
    float g = 0.f;
    for (int b = -R + ((pj - R) & 1); b <= R; b += 2)
        g = fmaf(T.tp[b + R], T.V[py * kLW + floor_div2(pj + b) - T.qx_lo], g);
    return g;
}

// staged x at image pixel (pi, pj) of the tile
__device__ __forceinline__ float sr_tile_x(const SrTile& T, int pi, int pj) {
    return T.X[(pi - (2 * T.qy_lo - T.G)) * kSW + (pj - (2 * T.qx_lo - T.G))];
}

}  // namespace dsg
