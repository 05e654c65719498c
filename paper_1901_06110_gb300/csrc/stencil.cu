// Stencil passes over the half-window weight planes: the balancing pass (second
// aggregation of Algorithm 2, iterated as symmetric Sinkhorn-Knopp) and the
// application of W (third aggregation of Algorithm 2), optionally fused with the
// dual update and residual reductions of Algorithm 1.
//
// A plane k holds K1(s, s + o_k) at s.  A pixel s gathers the forward neighbour
// s + o from plane k at s and the backward neighbour s - o from the same plane at
// s - o (symmetry K1(s, s - o) = K1(s - o, s)), so W is stored once and read
// without atomics.  Sums run over the offset rows o_y = 0..N_s; each row is
// accumulated in FP32 and the rows are added with an error-free transformation,
// in the same order for every pixel.
#include "common.cuh"
#include "internal.h"

namespace dsg {

namespace {

constexpr int kBX = 32;
constexpr int kBY = 8;
constexpr int kThreads = kBX * kBY;

// sum_{r != s} K1(s, r) a(r) b(r) with b = 1 when B is null (planes of row pitch Wp)
template <typename WT, bool kHasB>
__device__ __forceinline__ float stencil_gather(const WT* __restrict__ P, size_t plane, int H, int W,
                                                int rs, int i, int j, const float* __restrict__ A,
                                                const float* __restrict__ B, float b_s) {
    const int Wp = plane_pitch(W);
    CompSum total;
    for (int oy = 0; oy <= rs; ++oy) {
        const int ox0 = oy == 0 ? 1 : -rs;
        const WT* Pk = P + (size_t)row_first_k(oy, rs) * plane;
        float row = 0.f;
        const int fi = i + oy, bi = i - oy;
        for (int ox = ox0; ox <= rs; ++ox, Pk += plane) {
            const int fj = j + ox, bj = j - ox;
            if (fi < H && fj >= 0 && fj < W) {
                const size_t r = (size_t)fi * W + fj;
                const float w = to_f32(Pk[(size_t)i * Wp + j]);
                const float a = __ldg(A + r);
                row = fmaf(w, kHasB ? a * (__ldg(B + r) - b_s) : a, row);
            }
            if (bi >= 0 && bj >= 0 && bj < W) {
                const size_t r = (size_t)bi * W + bj;
                const float w = to_f32(Pk[(size_t)bi * Wp + bj]);
                const float a = __ldg(A + r);
                row = fmaf(w, kHasB ? a * (__ldg(B + r) - b_s) : a, row);
            }
        }
        total.add(row);
    }
    return total.value();
}

template <typename WT>
__global__ void __launch_bounds__(kThreads)
sinkhorn_pass_kernel(const WT* __restrict__ P, int H, int W, int rs, const float* __restrict__ d_in,
                     float* __restrict__ d_out, PassStat* __restrict__ stats,
                     BalanceCtl* __restrict__ ctl, int pass) {
    if (*(volatile int*)&ctl->done) return;
    const int j = blockIdx.x * kBX + threadIdx.x;
    const int i = blockIdx.y * kBY + threadIdx.y;
    double eps = 0.0, rsum = 0.0;
    if (i < H && j < W) {
        const size_t s = (size_t)i * W + j;
        const size_t plane = (size_t)H * plane_pitch(W);
        const float ds = d_in[s];
        // t = K1 d: the diagonal term (K1(s, s) = 1) plus the off-diagonal gather
        const float off = stencil_gather<WT, false>(P, plane, H, W, rs, i, j, d_in, nullptr, 0.f);
        const float t = ds + off;
        d_out[s] = sqrtf(ds / t);
        const double prod = (double)ds * (double)t;
        eps = fabs(prod - 1.0);
        rsum = prod;
    }
    __shared__ double s_eps[kThreads / 32], s_m[kThreads / 32];
    const int lane = (threadIdx.y * kBX + threadIdx.x) & 31;
    const int warp = (threadIdx.y * kBX + threadIdx.x) >> 5;
    eps = warp_max(eps);
    rsum = warp_max(rsum);
    if (lane == 0) { s_eps[warp] = eps; s_m[warp] = rsum; }
    __syncthreads();
    if (warp == 0) {
        eps = lane < kThreads / 32 ? s_eps[lane] : 0.0;
        rsum = lane < kThreads / 32 ? s_m[lane] : 0.0;
        eps = warp_max(eps);
        rsum = warp_max(rsum);
        if (lane == 0) {
            PassStat* ps = stats + pass;
            atomic_max_nonneg(&ps->eps_bits, eps);
            atomic_max_nonneg(&ps->m_bits, rsum);
            __threadfence();
            const unsigned nblocks = gridDim.x * gridDim.y;
            const unsigned ticket = atomicAdd(&ps->arrive, 1u);
            if (ticket == nblocks - 1) {
                // last block of this pass: decide whether to stop
                __threadfence();
                const double e = __longlong_as_double(
                    (long long)atomicAdd(&ps->eps_bits, 0ull));
                int done = 0, status = 0;
                if (e <= ctl->tol) {
                    done = 1;
                } else if (pass >= ctl->maxit) {
                    done = 1;
                    status = 6;
                } else if (e < 0.99 * ctl->best) {
                    ctl->best = e;
                    ctl->since_best = 0;
                } else if (++ctl->since_best >= 3) {
                    done = 1;
                    status = 7;
                }
                if (done) {
                    ctl->final_pass = pass;
                    ctl->status = status;
                    __threadfence();
                    *(volatile int*)&ctl->done = 1;
                }
            }
        }
    }
}

template <typename WT>
__global__ void __launch_bounds__(kThreads)
apply_kernel(const WT* __restrict__ P, int H, int W, int rs, const float* __restrict__ d, float inv_m,
             const float* __restrict__ z, float* __restrict__ y) {
    const int j = blockIdx.x * kBX + threadIdx.x;
    const int i = blockIdx.y * kBY + threadIdx.y;
    if (i >= H || j >= W) return;
    const size_t s = (size_t)i * W + j;
    const size_t plane = (size_t)H * plane_pitch(W);
    const float zs = z[s];
    // y_s = z_s + (d_s / m) sum_{r != s} K1(s, r) d_r (z_r - z_s): W z with the
    // diagonal closed so that the row sums are one (Eq. S3)
    const float acc = stencil_gather<WT, true>(P, plane, H, W, rs, i, j, d, z, zs);
    y[s] = fmaf(d[s] * inv_m, acc, zs);
}

template <typename WT>
__global__ void __launch_bounds__(kThreads)
apply_dual_kernel(const WT* __restrict__ P, int H, int W, int rs, const float* __restrict__ d,
                  float inv_m, const float* __restrict__ z, float* __restrict__ v,
                  float* __restrict__ u, SolveRed red, int iter) {
    const int j = blockIdx.x * kBX + threadIdx.x;
    const int i = blockIdx.y * kBY + threadIdx.y;
    double sp = 0.0, sd = 0.0;
    if (i < H && j < W) {
        const size_t s = (size_t)i * W + j;
        const size_t plane = (size_t)H * plane_pitch(W);
        const float zs = z[s];
        const float acc = stencil_gather<WT, true>(P, plane, H, W, rs, i, j, d, z, zs);
        const float vn = fmaf(d[s] * inv_m, acc, zs);
        const float vo = v[s];
        const float uo = u[s];
        const float un = zs - vn;  // u + x - v with z = x + u
        v[s] = vn;
        u[s] = un;
        const double dp = (double)un - (double)uo;  // x - v
        const double dd = (double)vn - (double)vo;  // v - v_prev
        sp = dp * dp;
        sd = dd * dd;
    }
    __shared__ double s_p[kThreads / 32], s_d[kThreads / 32];
    const int t = threadIdx.y * kBX + threadIdx.x;
    const int lane = t & 31, warp = t >> 5;
    sp = warp_sum(sp);
    sd = warp_sum(sd);
    if (lane == 0) { s_p[warp] = sp; s_d[warp] = sd; }
    __syncthreads();
    __shared__ bool is_last;
    if (t == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) { a += s_p[w]; b += s_d[w]; }
        const unsigned bid = blockIdx.y * gridDim.x + blockIdx.x;
        red.partials[2 * bid] = a;
        red.partials[2 * bid + 1] = b;
        __threadfence();
        const unsigned nblocks = gridDim.x * gridDim.y;
        is_last = atomicAdd(red.arrive + iter, 1u) == nblocks - 1;
    }
    __syncthreads();
    if (is_last) {
        // fixed-order reduction of the per-block partials
        __threadfence();
        const unsigned nblocks = gridDim.x * gridDim.y;
        double a = 0.0, b = 0.0;
        for (unsigned q = t; q < nblocks; q += kThreads) {
            a += ((volatile double*)red.partials)[2 * q];
            b += ((volatile double*)red.partials)[2 * q + 1];
        }
        __shared__ double r_a[kThreads], r_b[kThreads];
        r_a[t] = a;
        r_b[t] = b;
        __syncthreads();
        for (int w = kThreads / 2; w > 0; w >>= 1) {
            if (t < w) { r_a[t] += r_a[t + w]; r_b[t] += r_b[t + w]; }
            __syncthreads();
        }
        if (t == 0) {
            red.hist[2 * iter] = r_a[0];
            red.hist[2 * iter + 1] = r_b[0];
        }
    }
}

__global__ void fill_kernel(float* p, float value, size_t n) {
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n;
         q += (size_t)gridDim.x * blockDim.x)
        p[q] = value;
}

dim3 pixel_grid(int H, int W) { return dim3((W + kBX - 1) / kBX, (H + kBY - 1) / kBY); }

template <typename WT>
cudaError_t sinkhorn_t(const void* planes, int H, int W, int rs, const float* d_in, float* d_out,
                       PassStat* stats, BalanceCtl* ctl, int pass, cudaStream_t st) {
    sinkhorn_pass_kernel<WT><<<pixel_grid(H, W), dim3(kBX, kBY), 0, st>>>(
        (const WT*)planes, H, W, rs, d_in, d_out, stats, ctl, pass);
    count_launches(1);
    return cudaGetLastError();
}

template <typename WT>
cudaError_t apply_t(const void* planes, int H, int W, int rs, const float* d, float inv_m,
                    const float* z, float* y, cudaStream_t st) {
    apply_kernel<WT><<<pixel_grid(H, W), dim3(kBX, kBY), 0, st>>>((const WT*)planes, H, W, rs, d,
                                                                  inv_m, z, y);
    count_launches(1);
    return cudaGetLastError();
}

template <typename WT>
cudaError_t apply_dual_t(const void* planes, int H, int W, int rs, const float* d, float inv_m,
                         const float* z, float* v, float* u, SolveRed red, int iter,
                         cudaStream_t st) {
    apply_dual_kernel<WT><<<pixel_grid(H, W), dim3(kBX, kBY), 0, st>>>(
        (const WT*)planes, H, W, rs, d, inv_m, z, v, u, red, iter);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace

int apply_grid_blocks(int H, int W) {
    const dim3 g = pixel_grid(H, W);
    return (int)(g.x * g.y);
}

cudaError_t launch_fill(float* p, float value, size_t n, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    fill_kernel<<<blocks, 256, 0, st>>>(p, value, n);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_sinkhorn_pass(int dtype, const void* planes, int H, int W, int search_r,
                                 const float* d_in, float* d_out, PassStat* stats, BalanceCtl* ctl,
                                 int pass, cudaStream_t st) {
    switch (dtype) {
        case 0: return sinkhorn_t<float>(planes, H, W, search_r, d_in, d_out, stats, ctl, pass, st);
        case 1: return sinkhorn_t<__half>(planes, H, W, search_r, d_in, d_out, stats, ctl, pass, st);
        default:
            return sinkhorn_t<__nv_bfloat16>(planes, H, W, search_r, d_in, d_out, stats, ctl, pass, st);
    }
}

cudaError_t launch_apply(int dtype, const void* planes, int H, int W, int search_r, const float* d,
                         float inv_m, const float* z, float* y, cudaStream_t st) {
    switch (dtype) {
        case 0: return apply_t<float>(planes, H, W, search_r, d, inv_m, z, y, st);
        case 1: return apply_t<__half>(planes, H, W, search_r, d, inv_m, z, y, st);
        default: return apply_t<__nv_bfloat16>(planes, H, W, search_r, d, inv_m, z, y, st);
    }
}

cudaError_t launch_apply_dual(int dtype, const void* planes, int H, int W, int search_r,
                              const float* d, float inv_m, const float* z, float* v, float* u,
                              SolveRed red, int iter, cudaStream_t st) {
    switch (dtype) {
        case 0: return apply_dual_t<float>(planes, H, W, search_r, d, inv_m, z, v, u, red, iter, st);
        case 1: return apply_dual_t<__half>(planes, H, W, search_r, d, inv_m, z, v, u, red, iter, st);
        default:
            return apply_dual_t<__nv_bfloat16>(planes, H, W, search_r, d, inv_m, z, v, u, red, iter, st);
    }
}

}  // namespace dsg
