// Kernels of the super-resolution gradient (see grad.cuh) and the per-pixel
// x-update that consumes it.
#include "common.cuh"
#include "grad.cuh"
#include "internal.h"
#include "xupdate.cuh"

namespace dsg {

namespace {

template <int R>
__global__ void __launch_bounds__(256)
sr_grad_kernel(const float* __restrict__ x, const float* __restrict__ y, int H, int W, BlurTaps taps,
               float* __restrict__ g) {
    __shared__ GradSmem<R> sm;
    sr_grad_tile<R>(sm, x, y, H, W, taps, g, blockIdx.y * kGT, blockIdx.x * kGT);
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
