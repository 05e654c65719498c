// Forward models, measurements, guides and the fused linearized x-update of
// Algorithm 1 (Sec. 2 and Sec. 4).
//
// Super-resolution (Sec. 4.1): A = periodic blur by a normalised Gaussian h,
// then keep pixels (2i, 2j).  The 2D Gaussian is separable, h(a, b) = t(a) t(b)
// with t the normalised 1D Gaussian, so the blur is evaluated as two nested 1D
// sums.  A^T r = adjoint blur of r zero-filled at (2i, 2j): only the taps with
// p + a even contribute.
//
// Single-photon imaging (Sec. 4.2): grad f(x)_i = h'(max(x_i, eps)) with
// h'(t) = (eta/K) (K0 - K1 e^{-z} / (1 - e^{-z})), z = eta t / K; 1 - e^{-z} is
// evaluated as -expm1(-z).
#include <type_traits>
#include <math.h>

#include "common.cuh"
#include "grad.cuh"
#include "internal.h"
#include "xupdate.cuh"

namespace dsg {

BlurTaps make_blur_taps(float sigma, int r) {
    BlurTaps t{};
    t.r = r;
    double s = 0.0, v[17];
    for (int a = -r; a <= r; ++a) {
        v[a + r] = exp(-(double)a * a / (2.0 * (double)sigma * sigma));
        s += v[a + r];
    }
    for (int a = -r; a <= r; ++a) t.t[a + r] = (float)(v[a + r] / s);
    return t;
}

namespace {

constexpr int kBX = 32, kBY = 8;

dim3 grid2(int H, int W) { return dim3((W + kBX - 1) / kBX, (H + kBY - 1) / kBY); }

// out(q) = (A x)(q) + c aux(q), periodic
template <int R>
__global__ void sr_forward_kernel(const float* __restrict__ x, int H, int W, BlurTaps taps,
                                  const float* __restrict__ aux, float c, float* __restrict__ out) {
    const int h = H / 2, w = W / 2;
    const int qj = blockIdx.x * kBX + threadIdx.x;
    const int qi = blockIdx.y * kBY + threadIdx.y;
    if (qi >= h || qj >= w) return;
    const float acc = sr_forward_at<R>(x, H, W, taps, qi, qj);
    const size_t q = (size_t)qi * w + qj;
    out[q] = aux ? fmaf(c, aux[q], acc) : acc;
}

// (A^T r)(p) = sum_a t(a) sum_b t(b) u(p + (a, b)), u = r zero-filled at even pixels:
// the taps a (b) with p + a (p + b) even, in increasing order
template <int R>
__device__ __forceinline__ float sr_adjoint_at(const float* __restrict__ rlo, int H, int W,
                                              const BlurTaps& taps, int pi, int pj) {
    const int w = W / 2;
    const int pa = (pi - R) & 1, pb = (pj - R) & 1;  // parity of the first tap used
    int cols[R + 1];
#pragma unroll
    for (int k = 0; k <= R; ++k) {
        const int b = -R + pb + 2 * k;
        cols[k] = b <= R ? wrap_index(pj + b, W) >> 1 : 0;
    }
    float acc = 0.f;
#pragma unroll
    for (int k = 0; k <= R; ++k) {
        const int a = -R + pa + 2 * k;
        if (a > R) break;
        const float* row = rlo + (size_t)(wrap_index(pi + a, H) >> 1) * w;
        float ra = 0.f;
#pragma unroll
        for (int kb = 0; kb <= R; ++kb) {
            const int b = -R + pb + 2 * kb;
            if (b > R) break;
            ra = fmaf(taps.t[b + R], __ldg(row + cols[kb]), ra);
        }
        acc = fmaf(taps.t[a + R], ra, acc);
    }
    return acc;
}

template <int R>
__global__ void sr_adjoint_kernel(const float* __restrict__ rlo, int H, int W, BlurTaps taps,
                                  float* __restrict__ out) {
    const int pj = blockIdx.x * kBX + threadIdx.x;
    const int pi = blockIdx.y * kBY + threadIdx.y;
    if (pi >= H || pj >= W) return;
    out[(size_t)pi * W + pj] = sr_adjoint_at<R>(rlo, H, W, taps, pi, pj);
}

template <int R>
__global__ void sr_xupdate_kernel(const float* __restrict__ rlo, int H, int W, BlurTaps taps,
                                  float* __restrict__ x, const float* __restrict__ v,
                                  const float* __restrict__ u, float* __restrict__ z, float mu,
                                  float alpha, float rho, int constraint) {
    const int pj = blockIdx.x * kBX + threadIdx.x;
    const int pi = blockIdx.y * kBY + threadIdx.y;
    if (pi >= H || pj >= W) return;
    const size_t p = (size_t)pi * W + pj;
    const float g = sr_adjoint_at<R>(rlo, H, W, taps, pi, pj);
    const float up = u[p];
    const float xb = mu * (alpha * x[p] + rho * (v[p] - up) - g);
    const float xn = project(xb, constraint);
    x[p] = xn;
    z[p] = xn + up;
}

__global__ void __launch_bounds__(256, 4)
sr_xupdate_fused_kernel(const float* __restrict__ x_in, float* __restrict__ x_out, const float* __restrict__ y,
                        int H, int W, BlurTaps taps, const float* __restrict__ v, const float* __restrict__ u,
                        float* __restrict__ z, float mu, float alpha, float rho, int constraint) {
    __shared__ SrTile tile;
    sr_xupdate_body(tile, x_in, x_out, y, H, W, taps, v, u, z, mu, alpha, rho, constraint, blockIdx.y * kXH,
                    blockIdx.x * kXW);
}

__global__ void spi_grad_kernel(const float* __restrict__ x, const uint8_t* __restrict__ counts, int n,
                                int K, float eta, float eps, float* __restrict__ grad) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    grad[p] = spi_hprime(x[p], counts[p], K, eta, eps);
}

__global__ void spi_xupdate_kernel(const uint8_t* __restrict__ counts, int n, int K, float eta,
                                   float eps, float* __restrict__ x, const float* __restrict__ v,
                                   const float* __restrict__ u, float* __restrict__ z, float mu,
                                   float alpha, float rho, int constraint) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const float xv = x[p];
    const float g = spi_hprime(xv, counts[p], K, eta, eps);
    const float up = u[p];
    const float xn = project(mu * (alpha * xv + rho * (v[p] - up) - g), constraint);
    x[p] = xn;
    z[p] = xn + up;
}

// Keys cubic (a = -0.5) 2x upsampling with periodic wrap: even outputs copy the
// sample; odd outputs sit half-way and take weights (-1, 9, 9, -1) / 16.
__device__ __forceinline__ void keys_taps(int p, int n, int idx[4], float wt[4], int& cnt) {
    const int j = p >> 1;
    if ((p & 1) == 0) {
        idx[0] = j;
        wt[0] = 1.f;
        cnt = 1;
    } else {
        idx[0] = wrap_index(j - 1, n); wt[0] = -0.0625f;
        idx[1] = j;                    wt[1] = 0.5625f;
        idx[2] = wrap_index(j + 1, n); wt[2] = 0.5625f;
        idx[3] = wrap_index(j + 2, n); wt[3] = -0.0625f;
        cnt = 4;
    }
}

__global__ void sr_guide_kernel(const float* __restrict__ y, int h, int w, float* __restrict__ g) {
    const int pj = blockIdx.x * kBX + threadIdx.x;
    const int pi = blockIdx.y * kBY + threadIdx.y;
    if (pi >= 2 * h || pj >= 2 * w) return;
    int ii[4], jj[4], ni, nj;
    float wi[4], wj[4];
    keys_taps(pi, h, ii, wi, ni);
    keys_taps(pj, w, jj, wj, nj);
    float acc = 0.f;
    for (int a = 0; a < ni; ++a) {
        float ra = 0.f;
        for (int b = 0; b < nj; ++b) ra = fmaf(wj[b], y[(size_t)ii[a] * w + jj[b]], ra);
        acc = fmaf(wi[a], ra, acc);
    }
    g[(size_t)pi * (2 * w) + pj] = acc;
}

__global__ void spi_observe_kernel(const float* __restrict__ x, const float* __restrict__ arrivals,
                                   int H, int W, int ks, float eta, uint8_t* __restrict__ bits) {
    const int Ws = W * ks, Hs = H * ks;
    const int b = blockIdx.x * kBX + threadIdx.x;
    const int a = blockIdx.y * kBY + threadIdx.y;
    if (a >= Hs || b >= Ws) return;
    const float lam = __fdiv_rn(__fmul_rn(eta, x[(size_t)(a / ks) * W + b / ks]), (float)(ks * ks));
    const size_t q = (size_t)a * Ws + b;
    bits[q] = arrivals[q] < lam ? 1 : 0;
}

__global__ void spi_counts_kernel(const uint8_t* __restrict__ bits, int H, int W, int ks,
                                  uint8_t* __restrict__ counts) {
    const int j = blockIdx.x * kBX + threadIdx.x;
    const int i = blockIdx.y * kBY + threadIdx.y;
    if (i >= H || j >= W) return;
    const size_t Ws = (size_t)W * ks;
    int n = 0;
    for (int a = 0; a < ks; ++a) {
        const uint8_t* row = bits + (size_t)(i * ks + a) * Ws + (size_t)j * ks;
        for (int b = 0; b < ks; ++b) n += row[b];
    }
    counts[(size_t)i * W + j] = (uint8_t)n;
}

__device__ __forceinline__ float spi_mle(int k1, int K, float eta) {
    if (k1 >= K) return 1.f;
    const float m = -((float)K / eta) * log1pf(-(float)k1 / (float)K);
    return fminf(fmaxf(m, 0.f), 1.f);
}

__global__ void spi_guide_kernel(const uint8_t* __restrict__ counts, int H, int W, int K, float eta,
                                 float* __restrict__ g) {
    const int j = blockIdx.x * kBX + threadIdx.x;
    const int i = blockIdx.y * kBY + threadIdx.y;
    if (i >= H || j >= W) return;
    float acc = 0.f;
    for (int a = -1; a <= 1; ++a) {
        const int ii = sym_index(i + a, H);
        for (int b = -1; b <= 1; ++b) acc += spi_mle(counts[(size_t)ii * W + sym_index(j + b, W)], K, eta);
    }
    g[(size_t)i * W + j] = acc / 9.f;
}

__global__ void init_kernel(const float* __restrict__ guide, int n, float* __restrict__ x,
                            float* __restrict__ v, float* __restrict__ u) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const float g = fminf(fmaxf(guide[p], 0.f), 1.f);
    x[p] = g;
    v[p] = g;
    u[p] = 0.f;
}

}  // namespace

// the blur radii 0..8 as template arguments
template <typename F>
cudaError_t by_blur_r(int r, F&& f) {
    switch (r) {
        case 0: return f(std::integral_constant<int, 0>{});
        case 1: return f(std::integral_constant<int, 1>{});
        case 2: return f(std::integral_constant<int, 2>{});
        case 3: return f(std::integral_constant<int, 3>{});
        case 4: return f(std::integral_constant<int, 4>{});
        case 5: return f(std::integral_constant<int, 5>{});
        case 6: return f(std::integral_constant<int, 6>{});
        case 7: return f(std::integral_constant<int, 7>{});
        case 8: return f(std::integral_constant<int, 8>{});
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_sr_forward(const float* x, int H, int W, BlurTaps taps, const float* aux, float c,
                              float* out, cudaStream_t st) {
    return by_blur_r(taps.r, [&](auto rr) {
        sr_forward_kernel<decltype(rr)::value><<<grid2(H / 2, W / 2), dim3(kBX, kBY), 0, st>>>(x, H, W, taps, aux, c,
                                                                                              out);
        count_launches(1);
        return cudaGetLastError();
    });
}

cudaError_t launch_sr_adjoint(const float* r, int H, int W, BlurTaps taps, float* out, cudaStream_t st) {
    return by_blur_r(taps.r, [&](auto rr) {
        sr_adjoint_kernel<decltype(rr)::value><<<grid2(H, W), dim3(kBX, kBY), 0, st>>>(r, H, W, taps, out);
        count_launches(1);
        return cudaGetLastError();
    });
}

cudaError_t launch_sr_xupdate(const float* r, int H, int W, BlurTaps taps, float* x, const float* v,
                              const float* u, float* z, float mu, float alpha, float rho,
                              int constraint, cudaStream_t st) {
    return by_blur_r(taps.r, [&](auto rr) {
        sr_xupdate_kernel<decltype(rr)::value><<<grid2(H, W), dim3(kBX, kBY), 0, st>>>(r, H, W, taps, x, v, u, z, mu,
                                                                                      alpha, rho, constraint);
        count_launches(1);
        return cudaGetLastError();
    });
}

cudaError_t launch_sr_xupdate_fused(const float* x_in, float* x_out, const float* y, int H, int W,
                                    BlurTaps taps, const float* v, const float* u, float* z, float mu,
                                    float alpha, float rho, int constraint, cudaStream_t st) {
    if (taps.r > kMaxBlurR) return cudaErrorInvalidValue;
    dim3 grid((W + kXW - 1) / kXW, (H + kXH - 1) / kXH);
    sr_xupdate_fused_kernel<<<grid, dim3(32, 8), 0, st>>>(x_in, x_out, y, H, W, taps, v, u, z, mu, alpha, rho,
                                                          constraint);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_spi_grad(const float* x, const uint8_t* counts, int n, int K, float eta, float eps,
                            float* grad, cudaStream_t st) {
    spi_grad_kernel<<<(n + 255) / 256, 256, 0, st>>>(x, counts, n, K, eta, eps, grad);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_spi_xupdate(const uint8_t* counts, int n, int K, float eta, float eps, float* x,
                               const float* v, const float* u, float* z, float mu, float alpha,
                               float rho, int constraint, cudaStream_t st) {
    spi_xupdate_kernel<<<(n + 255) / 256, 256, 0, st>>>(counts, n, K, eta, eps, x, v, u, z, mu, alpha,
                                                         rho, constraint);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_sr_guide(const float* y, int h, int w, float* guide, cudaStream_t st) {
    sr_guide_kernel<<<grid2(2 * h, 2 * w), dim3(kBX, kBY), 0, st>>>(y, h, w, guide);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_spi_observe(const float* x, const float* arrivals, int H, int W, int k_side,
                               float eta, uint8_t* bits, cudaStream_t st) {
    spi_observe_kernel<<<grid2(H * k_side, W * k_side), dim3(kBX, kBY), 0, st>>>(x, arrivals, H, W,
                                                                                k_side, eta, bits);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_spi_counts(const uint8_t* bits, int H, int W, int k_side, uint8_t* counts,
                              cudaStream_t st) {
    spi_counts_kernel<<<grid2(H, W), dim3(kBX, kBY), 0, st>>>(bits, H, W, k_side, counts);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_spi_guide(const uint8_t* counts, int H, int W, int K, float eta, float* guide,
                             cudaStream_t st) {
    spi_guide_kernel<<<grid2(H, W), dim3(kBX, kBY), 0, st>>>(counts, H, W, K, eta, guide);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_init(const float* guide, int n, float* x, float* v, float* u, cudaStream_t st) {
    init_kernel<<<(n + 255) / 256, 256, 0, st>>>(guide, n, x, v, u);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace dsg
