// Super-resolution operator with either boundary, and the conjugate-gradient steps
// of standard PnP-ADMM (the standard-vs-linearized comparison of Sec. 4.1).
//
//   (A x)(q) = sum_a t(a) sum_b t(b) x(e(2q - (a, b))),  e = periodic wrap or
//              half-sample symmetric reflection of the index into the image,
//   (A^T r)(p) = sum of t(a) t(b) r(q) over every (q, a, b) that A sends to p.
// The adjoint gathers per pixel: the positions of the extended grid that map to
// pixel i are i - H, i, i + H (periodic) or i, -1 - i, 2H - 1 - i (symmetric), of
// which those within the blur radius of the image take part; with H, W >= 2R no
// two of them coincide, so no term is counted twice and no atomics are needed.
//
// Conjugate gradients for (A^T A + rho I) x = b keep their scalars in device
// memory (each dot product: fixed-order double block sums, then one reducing
// block), so the steps run back to back without host round trips.
#include <type_traits>

#include "common.cuh"
#include "internal.h"
#include "xupdate.cuh"

namespace dsg {

namespace {

template <int BC>  // 0 periodic, 1 symmetric
__device__ __forceinline__ int ext_index(int k, int n) {
    return BC == 1 ? sym_index(k, n) : wrap_index(k, n);
}

// the (at most 3) extended positions e in [-R, n - 1 + R] that map to index i
template <int BC>
__device__ __forceinline__ int ext_candidates(int i, int n, int R, int (&e)[3]) {
    int c[3];
    if (BC == 1) {
        c[0] = i;
        c[1] = -1 - i;
        c[2] = 2 * n - 1 - i;
    } else {
        c[0] = i;
        c[1] = i - n;
        c[2] = i + n;
    }
    int m = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k)
        if (c[k] >= -R && c[k] <= n - 1 + R) e[m++] = c[k];
    return m;
}

constexpr int kBX = 32, kBY = 8;

// The blur radius R is a template parameter: the tap loops unroll, and a row's loads
// are issued ahead of the FMA chain that consumes them.
template <int BC, int R>
__global__ void __launch_bounds__(256)
sr_forward_bc_kernel(const float* __restrict__ x, int H, int W, BlurTaps taps, const float* __restrict__ aux, float c,
                     float* __restrict__ out) {
    const int h = H / 2, w = W / 2;
    const int qj = blockIdx.x * kBX + threadIdx.x;
    const int qi = blockIdx.y * kBY + threadIdx.y;
    if (qi >= h || qj >= w) return;
    int cols[2 * R + 1];
#pragma unroll
    for (int b = -R; b <= R; ++b) cols[b + R] = ext_index<BC>(2 * qj - b, W);
    float acc = 0.f;
#pragma unroll
    for (int a = -R; a <= R; ++a) {
        const float* row = x + (size_t)ext_index<BC>(2 * qi - a, H) * W;
        float ra = 0.f;
#pragma unroll
        for (int b = -R; b <= R; ++b) ra = fmaf(taps.t[b + R], __ldg(row + cols[b + R]), ra);
        acc = fmaf(taps.t[a + R], ra, acc);
    }
    const size_t q = (size_t)qi * w + qj;
    out[q] = aux ? fmaf(c, aux[q], acc) : acc;
}

// out = A^T rlo + rho * pin (pin may be null); with part, the block's sum of pin * out
template <int BC, int R>
__global__ void __launch_bounds__(256)
sr_adjoint_bc_kernel(const float* __restrict__ rlo, int H, int W, BlurTaps taps, float rho,
                     const float* __restrict__ pin, float* __restrict__ out, double* __restrict__ part) {
    const int h = H / 2, w = W / 2;
    const int pj = blockIdx.x * kBX + threadIdx.x;
    const int pi = blockIdx.y * kBY + threadIdx.y;
    double prod = 0.0;
    if (pi < H && pj < W) {
        int ei[3], ej[3];
        const int mi = ext_candidates<BC>(pi, H, R, ei);
        const int mj = ext_candidates<BC>(pj, W, R, ej);
        float acc = 0.f;
        for (int ci = 0; ci < mi; ++ci) {
            const int e = ei[ci];
            // the taps a with (e + a) even, in increasing order
#pragma unroll
            for (int k = 0; k <= R; ++k) {
                const int a = -R + ((e - R) & 1) + 2 * k;
                if (a > R) break;
                const int qi = (e + a) >> 1;
                if (qi < 0 || qi >= h) continue;
                const float* row = rlo + (size_t)qi * w;
                float ra = 0.f;
                for (int cj = 0; cj < mj; ++cj) {
                    const int f = ej[cj];
#pragma unroll
                    for (int kb = 0; kb <= R; ++kb) {
                        const int b = -R + ((f - R) & 1) + 2 * kb;
                        if (b > R) break;
                        const int qj = (f + b) >> 1;
                        if (qj < 0 || qj >= w) continue;
                        ra = fmaf(taps.t[b + R], __ldg(row + qj), ra);
                    }
                }
                acc = fmaf(taps.t[a + R], ra, acc);
            }
        }
        const size_t p = (size_t)pi * W + pj;
        if (pin) acc = fmaf(rho, pin[p], acc);
        out[p] = acc;
        if (part) prod = (double)pin[p] * (double)acc;
    }
    if (!part) return;
    prod = warp_sum(prod);
    __shared__ double s[8];
    const int t = threadIdx.y * kBX + threadIdx.x;
    if ((t & 31) == 0) s[t >> 5] = prod;
    __syncthreads();
    if (t == 0) {
        double b = 0.0;
        for (int k = 0; k < 8; ++k) b += s[k];
        part[blockIdx.y * gridDim.x + blockIdx.x] = b;
    }
}

constexpr int kVB = 256;  // threads of the 1-D vector kernels

__device__ __forceinline__ void block_partial(double v, double* part) {
    v = warp_sum(v);
    __shared__ double s[kVB / 32];
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int k = 0; k < kVB / 32; ++k) b += s[k];
        part[blockIdx.x] = b;
    }
}

// r = aty + rho (v - u) - mx, p = r; block sums of r * r
__global__ void __launch_bounds__(kVB)
cg_init_kernel(const float* __restrict__ aty, const float* __restrict__ v, const float* __restrict__ u, float rho,
               const float* __restrict__ mx, float* __restrict__ r, float* __restrict__ p, int n,
               double* __restrict__ part) {
    const int i = blockIdx.x * kVB + threadIdx.x;
    double rr = 0.0;
    if (i < n) {
        const float ri = fmaf(rho, v[i] - u[i], aty[i]) - mx[i];
        r[i] = ri;
        p[i] = ri;
        rr = (double)ri * (double)ri;
    }
    block_partial(rr, part);
}

// alpha = rs / pq (st); x += alpha p; r -= alpha q; block sums of r * r
__global__ void __launch_bounds__(kVB)
cg_step_kernel(float* __restrict__ x, float* __restrict__ r, const float* __restrict__ p, const float* __restrict__ q,
               const CgScalars* __restrict__ st, int n, double* __restrict__ part) {
    const int i = blockIdx.x * kVB + threadIdx.x;
    const float alpha = (float)st->alpha;
    double rr = 0.0;
    if (i < n) {
        x[i] = fmaf(alpha, p[i], x[i]);
        const float ri = fmaf(-alpha, q[i], r[i]);
        r[i] = ri;
        rr = (double)ri * (double)ri;
    }
    block_partial(rr, part);
}

// p = r + beta p
__global__ void __launch_bounds__(kVB)
cg_dir_kernel(const float* __restrict__ r, float* __restrict__ p, const CgScalars* __restrict__ st, int n) {
    const int i = blockIdx.x * kVB + threadIdx.x;
    if (i < n) p[i] = fmaf((float)st->beta, p[i], r[i]);
}

// fixed-order sum of the block partials, then: mode 0 rs = sum; mode 1 pq = sum and
// alpha = rs / pq; mode 2 beta = sum / rs and rs = sum
__global__ void __launch_bounds__(1024)
cg_reduce_kernel(const double* __restrict__ part, int nb, CgScalars* __restrict__ st, int mode) {
    double a = 0.0;
    for (int k = threadIdx.x; k < nb; k += 1024) a += part[k];
    __shared__ double s[1024];
    s[threadIdx.x] = a;
    __syncthreads();
    for (int w = 512; w > 0; w >>= 1) {
        if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    const double sum = s[0];
    if (mode == 0) {
        st->rs = sum;
    } else if (mode == 1) {
        st->pq = sum;
        st->alpha = sum > 0.0 ? st->rs / sum : 0.0;
    } else {
        st->beta = st->rs > 0.0 ? sum / st->rs : 0.0;
        st->rs = sum;
    }
}

// x <- Pi_C(x), z = x + u
__global__ void __launch_bounds__(kVB)
project_z_kernel(float* __restrict__ x, const float* __restrict__ u, float* __restrict__ z, int n, int constraint) {
    const int i = blockIdx.x * kVB + threadIdx.x;
    if (i >= n) return;
    const float xn = project(x[i], constraint);
    x[i] = xn;
    z[i] = xn + u[i];
}

dim3 grid_hi(int H, int W) { return dim3((W + kBX - 1) / kBX, (H + kBY - 1) / kBY); }
dim3 grid_lo(int H, int W) { return dim3((W / 2 + kBX - 1) / kBX, (H / 2 + kBY - 1) / kBY); }
int vblocks(int n) { return (n + kVB - 1) / kVB; }

}  // namespace

bool sr_bc_supported(int H, int W, int blur_r) { return H >= 2 * blur_r && W >= 2 * blur_r && H >= 2 && W >= 2; }

int sr_adjoint_bc_blocks(int H, int W) {
    const dim3 g = grid_hi(H, W);
    return (int)(g.x * g.y);
}

int cg_vector_blocks(int n) { return vblocks(n); }

// the boundary (0 periodic, 1 symmetric) and the blur radius 0..8 as template arguments
template <typename F>
cudaError_t by_bc_r(int bc, int r, F&& f) {
    auto with_r = [&](auto b) -> cudaError_t {
        switch (r) {
            case 0: return f(b, std::integral_constant<int, 0>{});
            case 1: return f(b, std::integral_constant<int, 1>{});
            case 2: return f(b, std::integral_constant<int, 2>{});
            case 3: return f(b, std::integral_constant<int, 3>{});
            case 4: return f(b, std::integral_constant<int, 4>{});
            case 5: return f(b, std::integral_constant<int, 5>{});
            case 6: return f(b, std::integral_constant<int, 6>{});
            case 7: return f(b, std::integral_constant<int, 7>{});
            case 8: return f(b, std::integral_constant<int, 8>{});
            default: return cudaErrorInvalidValue;
        }
    };
    return bc == 1 ? with_r(std::integral_constant<int, 1>{}) : with_r(std::integral_constant<int, 0>{});
}

cudaError_t launch_sr_forward_bc(int bc, const float* x, int H, int W, BlurTaps taps, const float* aux, float c,
                                 float* out, cudaStream_t st) {
    return by_bc_r(bc, taps.r, [&](auto b, auto r) {
        sr_forward_bc_kernel<decltype(b)::value, decltype(r)::value>
            <<<grid_lo(H, W), dim3(kBX, kBY), 0, st>>>(x, H, W, taps, aux, c, out);
        count_launches(1);
        return cudaGetLastError();
    });
}

cudaError_t launch_sr_adjoint_bc(int bc, const float* rlo, int H, int W, BlurTaps taps, float rho, const float* pin,
                                 float* out, double* part, cudaStream_t st) {
    return by_bc_r(bc, taps.r, [&](auto b, auto r) {
        sr_adjoint_bc_kernel<decltype(b)::value, decltype(r)::value>
            <<<grid_hi(H, W), dim3(kBX, kBY), 0, st>>>(rlo, H, W, taps, rho, pin, out, part);
        count_launches(1);
        return cudaGetLastError();
    });
}

cudaError_t launch_cg_init(const float* aty, const float* v, const float* u, float rho, const float* mx, float* r,
                           float* p, int n, double* part, cudaStream_t st) {
    cg_init_kernel<<<vblocks(n), kVB, 0, st>>>(aty, v, u, rho, mx, r, p, n, part);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_cg_step(float* x, float* r, const float* p, const float* q, const CgScalars* s, int n,
                           double* part, cudaStream_t st) {
    cg_step_kernel<<<vblocks(n), kVB, 0, st>>>(x, r, p, q, s, n, part);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_cg_dir(const float* r, float* p, const CgScalars* s, int n, cudaStream_t st) {
    cg_dir_kernel<<<vblocks(n), kVB, 0, st>>>(r, p, s, n);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_cg_reduce(const double* part, int nb, CgScalars* s, int mode, cudaStream_t st) {
    cg_reduce_kernel<<<1, 1024, 0, st>>>(part, nb, s, mode);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_project_z(float* x, const float* u, float* z, int n, int constraint, cudaStream_t st) {
    project_z_kernel<<<vblocks(n), kVB, 0, st>>>(x, u, z, n, constraint);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace dsg
