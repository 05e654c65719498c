// Gradient of the super-resolution data term f(x) = 1/2 ||y - A x||^2 (Sec. 2 and
// Eq. dataterm, with the sign of the gradient read as A^T(A x - y)):
//   g = A^T (A x - y),  A = keep the even-index pixels of a periodic, separable
//   (2R + 1) x (2R + 1) blur.
// One block computes a 32 x 32 tile of g.  The x values within reach of the tile
// are staged in shared memory once; then four separable passes follow: the blur
// along rows at the even columns, the blur along columns at the even rows minus y
// (the residual A x - y on the low-resolution window), the column half of A^T and
// its row half.  The blur radius is a template parameter, so every tap loop is
// unrolled and the taps are read from the kernel parameters.
#include "common.cuh"
#include "internal.h"
#include "xupdate.cuh"

namespace dsg {

namespace {

constexpr int kGT = 32;  // output tile side

template <int R>
struct GradDims {
    static constexpr int G = R > 0 ? R : 1;              // staging margin
    static constexpr int L = (kGT - 1 + 2 * G) / 2 + 2;  // low-resolution rows (cols) of the window, upper bound
    static constexpr int S = 2 * (L - 1) + 2 * G + 1;    // staged x rows (cols)
};

template <int R>
__global__ void __launch_bounds__(256)
sr_grad_kernel(const float* __restrict__ x, const float* __restrict__ y, int H, int W, BlurTaps taps,
               float* __restrict__ g) {
    using Dm = GradDims<R>;
    constexpr int G = Dm::G, L = Dm::L, S = Dm::S;
    __shared__ float X[S][S];
    __shared__ float Hs[S][L];
    __shared__ float Rl[L][L];
    __shared__ float V[kGT][L];
    __shared__ int rows[S], cols[S], lrows[L], lcols[L];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int y0 = blockIdx.y * kGT, x0 = blockIdx.x * kGT;
    const int h = H >> 1, w = W >> 1;
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
    // column blur at the even rows minus the observation: r = A x - y
    for (int i = tid; i < L * L; i += 256) {
        const int l = i / L, c = i - l * L;
        const float yv = __ldg(y + (size_t)lrows[l] * w + lcols[c]);
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
    const int k = lane & 15;
    const int cbase = (x0 >> 1) + k - qx_lo;  // window column of (x0 + 2 k) / 2
    for (int py = 2 * warp + (lane >> 4); py < kGT; py += 16) {
        float e = 0.f, o = 0.f;
#pragma unroll
        for (int b = -R; b <= R; ++b) {
            if ((b & 1) == 0)
                e = fmaf(taps.t[b + R], V[py][cbase + (b >> 1)], e);
            else
                o = fmaf(taps.t[b + R], V[py][cbase + ((b + 1) >> 1)], o);
        }
        const int pi = y0 + py, pj = x0 + 2 * k;
        if (pi < H && pj < W) *reinterpret_cast<float2*>(g + (size_t)pi * W + pj) = make_float2(e, o);
    }
}

// x <- Pi_C(mu (alpha x + rho (v - u) - g)) and z = x + u at each pixel (Algorithm 1,
// first two steps, with the gradient given)
__global__ void __launch_bounds__(256)
xupdate_point_kernel(float* __restrict__ x, const float* __restrict__ g, const float* __restrict__ v,
                     const float* __restrict__ u, float* __restrict__ z, int n, float mu, float alpha, float rho,
                     int constraint) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const float up = u[p];
    const float xn = project(mu * (alpha * x[p] + rho * (v[p] - up) - g[p]), constraint);
    x[p] = xn;
    z[p] = xn + up;
}

template <int R>
cudaError_t grad_launch(const float* x, const float* y, int H, int W, const BlurTaps& taps, float* g,
                        cudaStream_t st) {
    const dim3 grid((W + kGT - 1) / kGT, (H + kGT - 1) / kGT);
    sr_grad_kernel<R><<<grid, 256, 0, st>>>(x, y, H, W, taps, g);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sr_grad(const float* x, const float* y, int H, int W, BlurTaps taps, float* g,
                           cudaStream_t st) {
    if ((H & 1) || (W & 1)) return cudaErrorInvalidValue;
    switch (taps.r) {
        case 0: return grad_launch<0>(x, y, H, W, taps, g, st);
        case 1: return grad_launch<1>(x, y, H, W, taps, g, st);
        case 2: return grad_launch<2>(x, y, H, W, taps, g, st);
        case 3: return grad_launch<3>(x, y, H, W, taps, g, st);
        case 4: return grad_launch<4>(x, y, H, W, taps, g, st);
        case 5: return grad_launch<5>(x, y, H, W, taps, g, st);
        case 6: return grad_launch<6>(x, y, H, W, taps, g, st);
        case 7: return grad_launch<7>(x, y, H, W, taps, g, st);
        case 8: return grad_launch<8>(x, y, H, W, taps, g, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_xupdate_point(float* x, const float* g, const float* v, const float* u, float* z, int n, float mu,
                                 float alpha, float rho, int constraint, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    xupdate_point_kernel<<<(n + 255) / 256, 256, 0, st>>>(x, g, v, u, z, n, mu, alpha, rho, constraint);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace dsg
