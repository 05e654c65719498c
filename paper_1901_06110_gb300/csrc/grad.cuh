// Gradient of the super-resolution data term f(x) = 1/2 ||y - A x||^2 (Sec. 2 and
// Eq. dataterm, with the sign of the gradient read as A^T(A x - y)):
//   g = A^T (A x - y),  A = keep the even-index pixels of a periodic, separable
//   (2R + 1) x (2R + 1) blur.
// sr_grad_tile computes a 32 x 32 tile of g with one (256-thread) block.  The x
// values within reach of the tile are staged in shared memory once; then four
// separable passes follow: the blur along rows at the even columns, the blur along
// columns at the even rows minus y (the residual A x - y on the low-resolution
// window), the column half of A^T and its row half.  The blur radius is a template
// parameter, so every tap loop is unrolled and the taps are read from the
// kernel parameters.
#pragma once

#include "common.cuh"
#include "internal.h"

namespace dsg {

constexpr int kGT = 32;  // output tile side

// (A x)(q) = sum_a t(a) sum_b t(b) x(2q - (a, b)), periodic: the low-resolution pixel q
// = (qi, qj) of the blurred, decimated image.  Both tap loops unroll (R is a template
// parameter), so a row's loads are issued together.
template <int R>
__device__ __forceinline__ float sr_forward_at(const float* __restrict__ x, int H, int W, const BlurTaps& taps,
                                               int qi, int qj) {
    int cols[2 * R + 1];
#pragma unroll
    for (int b = -R; b <= R; ++b) cols[b + R] = wrap_index(2 * qj - b, W);
    float acc = 0.f;
#pragma unroll
    for (int a = -R; a <= R; ++a) {
        const float* row = x + (size_t)wrap_index(2 * qi - a, H) * W;
        float ra = 0.f;
#pragma unroll
        for (int b = -R; b <= R; ++b) ra = fmaf(taps.t[b + R], __ldg(row + cols[b + R]), ra);
        acc = fmaf(taps.t[a + R], ra, acc);
    }
    return acc;
}

template <int R>
struct GradDims {
    static constexpr int G = R > 0 ? R : 1;              // staging margin
    static constexpr int L = (kGT - 1 + 2 * G) / 2 + 2;  // low-resolution rows (cols) of the window, upper bound
    static constexpr int S = 2 * (L - 1) + 2 * G + 1;    // staged x rows (cols)
};

template <int R>
struct GradSmem {
    float X[GradDims<R>::S][GradDims<R>::S];
    float Hs[GradDims<R>::S][GradDims<R>::L];
    float Rl[GradDims<R>::L][GradDims<R>::L];
    float V[kGT][GradDims<R>::L];
    int rows[GradDims<R>::S], cols[GradDims<R>::S], lrows[GradDims<R>::L], lcols[GradDims<R>::L];
};

// g on the 32 x 32 tile at (y0, x0), handed to epi(s, i, j, g(i, j), g(i, j + 1)) for each
// even column j of the tile inside the image; all 256 threads of the block call it.
// Each thread receives two such pixel pairs (s = 0, 1), and pre(s, i, j) is called for
// them before the stencil passes, so that the caller's loads for the epilogue are in
// flight while g is formed.
template <int R, typename Pre, typename Epi>
__device__ __forceinline__ void sr_grad_tile_apply2(GradSmem<R>& sm, const float* __restrict__ x,
                                                    const float* __restrict__ y, int H, int W, const BlurTaps& taps,
                                                    int y0, int x0, Pre&& pre, Epi&& epi) {
    using Dm = GradDims<R>;
    constexpr int G = Dm::G, L = Dm::L, S = Dm::S;
    auto& X = sm.X;
    auto& Hs = sm.Hs;
    auto& Rl = sm.Rl;
    auto& V = sm.V;
    int* rows = sm.rows;
    int* cols = sm.cols;
    int* lrows = sm.lrows;
    int* lcols = sm.lcols;
    const int tid = threadIdx.y * 32 + threadIdx.x, lane = tid & 31, warp = tid >> 5;  // blocks of 256 or (32, 8)
    const int h = H >> 1, w = W >> 1;
    // the thread's epilogue pixels: rows 2 warp + lane / 16 (+ 16), column x0 + 2 (lane % 16)
    const int k = lane & 15;
    const int py0 = 2 * warp + (lane >> 4);
#pragma unroll
    for (int sl = 0; sl < 2; ++sl) {
        const int pi = y0 + py0 + 16 * sl, pj = x0 + 2 * k;
        if (pi < H && pj < W) pre(sl, pi, pj);
    }
    // low-resolution window: rows qy_lo .. qy_lo + L - 1 (and columns likewise); the
    // staged x rows start at high-resolution row 2 qy_lo - G
    const int qy_lo = (y0 - G) >> 1, qx_lo = (x0 - G) >> 1;
    for (int a = tid; a < S; a += 256) {
        rows[a] = wrap_index(2 * qy_lo - G + a, H);
        cols[a] = wrap_index(2 * qx_lo - G + a, W);
    }
    for (int l = tid; l < L; l += 256) {
        lrows[l] = wrap_index(qy_lo + l, h);
        lcols[l] = wrap_index(qx_lo + l, w);
    }
    __syncthreads();
    // every load of this thread is issued before the first store to shared memory
    constexpr int kLoads = (S * S + 255) / 256;
    float xv[kLoads];
#pragma unroll
    for (int k = 0; k < kLoads; ++k) {
        const int i = tid + 256 * k;
        if (i < S * S) {
            const int a = i / S, b = i - a * S;
            xv[k] = __ldg(x + (size_t)rows[a] * W + cols[b]);
        }
    }
#pragma unroll
    for (int k = 0; k < kLoads; ++k) {
        const int i = tid + 256 * k;
        if (i < S * S) {
            const int a = i / S, b = i - a * S;
            X[a][b] = xv[k];
        }
    }
    __syncthreads();
    // row blur at the even columns: Hs[a][c] = sum_b t_b x(staged row a, 2 (qx_lo + c) - b)
    for (int i = tid; i < S * L; i += 256) {
        const int a = i / L, c = i - a * L;
        float acc = 0.f;
#pragma unroll
        for (int b = -R; b <= R; ++b) acc = fmaf(taps.t[b + R], X[a][2 * c + G - b], acc);
        Hs[a][c] = acc;
    }
    __syncthreads();
    // column blur at the even rows minus the observation: r = A x - y (y null: r = A x)
    for (int i = tid; i < L * L; i += 256) {
        const int l = i / L, c = i - l * L;
        const float yv = y ? __ldg(y + (size_t)lrows[l] * w + lcols[c]) : 0.f;
        float acc = 0.f;
#pragma unroll
        for (int a = -R; a <= R; ++a) acc = fmaf(taps.t[a + R], Hs[2 * l + G - a][c], acc);
        Rl[l][c] = acc - yv;
    }
    __syncthreads();
    // column half of A^T: V(p, c) = sum_{a : p + a even} t_a r((p + a) / 2, c).  Rows
    // 2 pr (even p: even a) and 2 pr + 1 (odd p: odd a) are done together, so each
    // tap set is fixed at compile time; y0 is even.
    for (int pr = warp; pr < kGT / 2; pr += 8) {
        const int base = (y0 >> 1) + pr - qy_lo;  // window row of (y0 + 2 pr) / 2
        for (int c = lane; c < L; c += 32) {
            float e = 0.f, o = 0.f;
#pragma unroll
            for (int a = -R; a <= R; ++a) {
                if ((a & 1) == 0)
                    e = fmaf(taps.t[a + R], Rl[base + (a >> 1)][c], e);
                else
                    o = fmaf(taps.t[a + R], Rl[base + ((a + 1) >> 1)][c], o);
            }
            V[2 * pr][c] = e;
            V[2 * pr + 1][c] = o;
        }
    }
    __syncthreads();
    // row half of A^T at columns 2k (even b) and 2k + 1 (odd b)
    const int cbase = (x0 >> 1) + k - qx_lo;  // window column of (x0 + 2 k) / 2
    static_assert(kGT == 32, "two epilogue pixel pairs per thread");
#pragma unroll
    for (int sl = 0; sl < 2; ++sl) {
        const int py = py0 + 16 * sl;
        float e = 0.f, o = 0.f;
#pragma unroll
        for (int b = -R; b <= R; ++b) {
            if ((b & 1) == 0)
                e = fmaf(taps.t[b + R], V[py][cbase + (b >> 1)], e);
            else
                o = fmaf(taps.t[b + R], V[py][cbase + ((b + 1) >> 1)], o);
        }
        const int pi = y0 + py, pj = x0 + 2 * k;
        if (pi < H && pj < W) epi(sl, pi, pj, e, o);
    }
}

// The same without the prefetch: epi(i, j, g(i, j), g(i, j + 1)).
template <int R, typename Epi>
__device__ __forceinline__ void sr_grad_tile_apply(GradSmem<R>& sm, const float* __restrict__ x,
                                                   const float* __restrict__ y, int H, int W, const BlurTaps& taps,
                                                   int y0, int x0, Epi&& epi) {
    sr_grad_tile_apply2<R>(
        sm, x, y, H, W, taps, y0, x0, [](int, int, int) {},
        [&](int, int pi, int pj, float e, float o) { epi(pi, pj, e, o); });
}

// g stored on the 32 x 32 tile at (y0, x0)
template <int R>
__device__ __forceinline__ void sr_grad_tile(GradSmem<R>& sm, const float* __restrict__ x, const float* __restrict__ y,
                                             int H, int W, const BlurTaps& taps, float* __restrict__ g, int y0,
                                             int x0) {
    sr_grad_tile_apply<R>(sm, x, y, H, W, taps, y0, x0, [=](int pi, int pj, float e, float o) {
        *reinterpret_cast<float2*>(g + (size_t)pi * W + pj) = make_float2(e, o);
    });
}

}  // namespace dsg
