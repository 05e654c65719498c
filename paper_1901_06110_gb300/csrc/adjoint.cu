// Differentiable form of linearized PnP-ADMM with DSG-NLM: an unrolled forward
// solve that records checkpoints, and its hand-written adjoint.
//
// Forward (fixed discrete choices, so the output is piecewise smooth in the inputs):
//   K1 from the guide with bandwidth h (Eq. NLM, S1), stored as half-window planes;
//   T balancing passes d^{p+1} = sqrt(d^p / t^p), t^p = K1 d^p, from d^0 = 1 (Eq. S2);
//   m = max_s d_s t_s with t = K1 d (first maximiser s*), W from Eq. S3;
//   N iterations of Algorithm 1 from x = v = clip(guide), u = 0, recording (x, v, u)
//   and the gradient grad f(x_k) each x-update used.
//
// Backward, for the cotangent of x_N:
//   iteration k (reverse): a = vh - uh, zh = W a + uh (W is symmetric; zh is not stored),
//     g = Pi_C'(xbar_k) (xh + zh),  xh <- mu (alpha g - A^T A g),  vh <- mu rho g,
//     uh <- zh - mu rho g,  yh += mu A g (summed as A applied to sum mu g),
//     rhoh += sum g mu ((v_k - u_k) - xbar_k);
//   W depends on the pair weights w_sr = d_s d_r K1_sr / m (the diagonal closes the
//   rows), and dL/dw_sr = G_sr = sum_k (a_k(s) - a_k(r)) (z_k(r) - z_k(s)), z_k = x_{k+1} + u_k,
//   computed once per half-window pair into planes (pair pass G);
//   then through m, the T balancing passes, K1 = Lambda exp(-D c), c = 1 / (2 N_p^2 h^2)
//   (pair pass B), the patch distances D = box-sum of (g(p) - g(p + o))^2 and the
//   reflection of the guide.
// Every reduction has a fixed order, so results are bitwise repeatable.
//
// The images of a call advance in lockstep: every step of the forward and of the
// backward is one launch over all images (the image is blockIdx.z, or its high part),
// reading each image's buffers and scalars from a per-image view in device memory, and
// every phase-1 stencil pass is one launch of the batched weight stream over the tiles
// of all images.  The arithmetic of each image is that of the image alone; only the
// number of launches and how they fill the GPU change with the batch.  The steps that
// need neighbouring pixels but not the weights (grad f(x_{k+1}) in the forward,
// A^T A g in the backward) run on a side stream beside the weight stream they do not
// depend on; the per-pixel updates move into the steps around them.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "../../include/dsgnlm.h"
#include "combine.cuh"
#include "common.cuh"
#include "epilogue.cuh"
#include "grad.cuh"
#include "handle.h"
#include "internal.h"
#include "launch.h"
#include "tma.cuh"
#include "xupdate.cuh"

namespace dsg {

namespace {

constexpr int kAdjTH = 16, kAdjTW = 32;  // pair-pass tiles, block (32, 8), 2 rows per thread
constexpr int kMaxHalfOffsets = 2 * 12 * 13;  // n_h at the largest search radius (12)
constexpr int kPairSplit = 2;  // pair passes G and B: the half offsets in this many chunks (grid z)

// Everything the kernels of one image read: sizes, scalars and device buffers of its
// tape and handle, and the caller's inputs and outputs of the current call.
struct TapeView {
    int H, W, rp, rs, T, N, constraint;
    float mu, alpha, rho, c, hfac;
    BlurTaps taps;
    Cover cv;             // the handle's phase-1 partial regions
    const void* planes;   // K1 as half-window planes (the handle's weight type)
    const float* y;       // observation [H/2][W/2] (caller's)
    const float* guide;   // guide [H][W] (caller's)
    float *X, *V, *U;     // recorded iterates, N + 1 slots each
    float* Gr;            // recorded gradients, N slots
    float *Dh, *Th;       // recorded scalings d^0..d^T and row sums t^0..t^T
    float* scratch;       // the scaling after pass T (not recorded)
    float* z;             // the handle's z = x + u of the iteration
    double* cpart;        // the handle's per-block residual sums of the dual step (unused sums)
    float* m;             // m and 1/m
    unsigned long long* mkey;
    int* sstar;           // first maximiser of d t
    float *xh, *vh, *uh, *g, *gs, *dh, *dh0, *base, *thp, *Dhat, *Gp, *AZ;
    float* AZ4;           // (a_2u, a_2u+1, z_2u, z_2u+1) per pixel, u < ceil(N / 2) (pair pass G)
    float* gpart;         // partials of the patch-distance adjoint (the G or the D-hat memory)
    long long gp_cap, dh0_cap, gpart_cap;  // floats allocated at Gp, dh0, gpart (the checked build's bounds)
    alignas(64) unsigned char bd_kmap[128];  // tensor maps of the weight and G planes for the fused
    alignas(64) unsigned char bd_gmap[128];  // pass B (boxes of the D-hat window)
    alignas(64) unsigned char gt_kmap[128];  // tensor map of the weight planes for pass G (kQH x 32 tiles)
    alignas(64) unsigned char gt_amap[128];  // tensor map of the interleaved (a, z) copy (pass G windows)
    double *mh, *rho_part, *h_part, *m_part;  // mh: cotangents of m, rho, h
    float* x_out;         // x_N (caller's)
    const float* x_bar;   // its cotangent (caller's)
    float* y_bar;         // dL/dy (caller's)
    float* guide_bar;     // dL/dguide (caller's)
};

__device__ __forceinline__ float proj_deriv(float xb, int constraint) {
    if (constraint == 2) return (xb > 0.f && xb < 1.f) ? 1.f : 0.f;
    if (constraint == 1) return xb > 0.f ? 1.f : 0.f;
    return 1.f;
}

// ------------------------------------------------------------------------ forward

// d^0 = 1 and the maximiser key cleared, per image
__global__ void __launch_bounds__(256) adj_prep_kernel(const TapeView* __restrict__ tv) {
    griddep_enter();
    const TapeView& v = tv[blockIdx.z];
    const int n = v.H * v.W;
    for (int q = blockIdx.x * 256 + threadIdx.x; q < n; q += gridDim.x * 256) v.Dh[q] = 1.f;
    if (blockIdx.x == 0 && threadIdx.x == 0) *v.mkey = 0ull;
}

// Epilogue of balancing pass p (Eq. S2): t^p = K1 d^p from the phase-1 partial sums,
// d^{p+1} = sqrt(d^p / t^p) (the plain step), both recorded
__global__ void __launch_bounds__(256) adj_balance_kernel(const TapeView* __restrict__ tv, int p) {
    griddep_enter();
    const TapeView& v = tv[blockIdx.z];
    const size_t n = (size_t)v.H * v.W;
    float* d_out = p < v.T ? v.Dh + (size_t)(p + 1) * n : v.scratch;
    const PassRule plain{false, 0.f, 0.f};
    float e = 0.f, mx = 0.f;  // the residual maxima are not needed here
    balance_pixels<0>(v.cv, v.H, v.W, v.Dh + (size_t)p * n, d_out, v.Th + (size_t)p * n, blockIdx.y * kXH,
                      blockIdx.x * kXW, threadIdx.x, threadIdx.y, plain, e, mx);
}

// m = max_s d_s t_s and its first maximiser.  Each candidate becomes one 64-bit key:
// the bits of d_s t_s (positive floats order like their bit patterns) above the
// complement of s, so a larger key is a larger value or, for equal values, a smaller
// index.  Every warp folds its best key in with atomicMax, which does not depend on
// the order of arrival; the finish kernel unpacks the key.
__global__ void __launch_bounds__(256) adj_m_key_kernel(const TapeView* __restrict__ tv) {
    griddep_enter();
    const TapeView& v = tv[blockIdx.z];
    const int n = v.H * v.W;
    const float* d = v.Dh + (size_t)v.T * n;
    const float* t = v.Th + (size_t)v.T * n;
    unsigned long long best = 0ull;
    for (int q = blockIdx.x * 256 + threadIdx.x; q < n; q += gridDim.x * 256) {
        const unsigned long long k =
            ((unsigned long long)__float_as_uint(d[q] * t[q]) << 32) | (unsigned long long)(0xffffffffu - (unsigned)q);
        best = k > best ? k : best;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long other = __shfl_xor_sync(0xffffffffu, best, o);
        best = other > best ? other : best;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(v.mkey, best);
}

// one thread per image
__global__ void adj_m_finish_kernel(const TapeView* __restrict__ tv, int count) {
    griddep_enter();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const TapeView& v = tv[i];
    const unsigned long long k = *v.mkey;
    const float m = __uint_as_float((unsigned)(k >> 32));
    v.m[0] = m;
    v.m[1] = (float)(1.0 / (double)m);  // 1/m as the host would form it, read by the kernels that follow
    *v.sstar = (int)(0xffffffffu - (unsigned)(k & 0xffffffffull));
}

// x = v = clip(guide, 0, 1), u = 0 into slot 0
__global__ void __launch_bounds__(256) adj_init_kernel(const TapeView* __restrict__ tv) {
    griddep_enter();
    const TapeView& v = tv[blockIdx.z];
    const int n = v.H * v.W;
    const int q = blockIdx.x * 256 + threadIdx.x;
    if (q >= n) return;
    const float x0 = fminf(fmaxf(v.guide[q], 0.f), 1.f);
    v.X[q] = x0;
    v.V[q] = x0;
    v.U[q] = 0.f;
}

// x-update of recorded iteration k (Algorithm 1, first two steps) from the states of
// slot k into slot k + 1, on the 32 x 32 tile at (y0, x0):
//   g = A^T (A x_k - y) (recorded),  x_{k+1} = Pi_C(mu (alpha x_k + rho (v_k - u_k) - g)),
//   z = x_{k+1} + u_k,  and v_k, u_k copied into slot k + 1 for the dual step to update.
// x_k is read in halos and x_{k+1} written to another buffer, so tiles do not race.
template <int R>
__device__ __forceinline__ void fwd_xupdate_tile(GradSmem<R>& sm, const TapeView& v, int k, int y0, int x0) {
    const int H = v.H, W = v.W;
    const size_t n = (size_t)H * W;
    const float* xk = v.X + (size_t)k * n;
    const float* vk = v.V + (size_t)k * n;
    const float* uk = v.U + (size_t)k * n;
    float* grec = v.Gr + (size_t)k * n;
    float* x1 = v.X + (size_t)(k + 1) * n;
    float* v1 = v.V + (size_t)(k + 1) * n;
    float* u1 = v.U + (size_t)(k + 1) * n;
    float* z = v.z;
    const float mu = v.mu, alpha = v.alpha, rho = v.rho;
    const int constraint = v.constraint;
    float2 xp[2], vp2[2], up2[2];  // the epilogue pixels' x_k, v_k, u_k, loaded before the stencil
    sr_grad_tile_apply2<R>(
        sm, xk, v.y, H, W, v.taps, y0, x0,
        [&](int sl, int pi, int pj) {
            const size_t q = (size_t)pi * W + pj;  // even: a float2 per pair
            xp[sl] = *reinterpret_cast<const float2*>(xk + q);
            vp2[sl] = *reinterpret_cast<const float2*>(vk + q);
            up2[sl] = *reinterpret_cast<const float2*>(uk + q);
        },
        [&](int sl, int pi, int pj, float e, float o) {
            const size_t q = (size_t)pi * W + pj;
            const float g2[2] = {e, o}, x2[2] = {xp[sl].x, xp[sl].y}, v2[2] = {vp2[sl].x, vp2[sl].y},
                        u2[2] = {up2[sl].x, up2[sl].y};
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const float up = u2[c], vp = v2[c];
                const float xn = project(mu * (alpha * x2[c] + rho * (vp - up) - g2[c]), constraint);
                grec[q + c] = g2[c];
                x1[q + c] = xn;
                z[q + c] = xn + up;
                v1[q + c] = vp;
                u1[q + c] = up;
            }
        });
}

template <int R>
__global__ void __launch_bounds__(256, 4) adj_fwd_xupdate_kernel(const TapeView* __restrict__ tv, int k) {
    griddep_enter();
    __shared__ GradSmem<R> sm;
    fwd_xupdate_tile<R>(sm, tv[blockIdx.z], k, blockIdx.y * kGT, blockIdx.x * kGT);
}

// g_k = A^T (A x_k - y) recorded into its slot, on 32 x 32 tiles.  Only x_k is read, so it
// runs beside the weight stream of z_{k-1} = x_k + u_{k-1}.
template <int R>
__global__ void __launch_bounds__(256, 4) adj_fwd_grad_kernel(const TapeView* __restrict__ tv, int k) {
    griddep_enter();
    __shared__ GradSmem<R> sm;
    const TapeView& v = tv[blockIdx.z];
    const size_t n = (size_t)v.H * v.W;
    sr_grad_tile<R>(sm, v.X + (size_t)k * n, v.y, v.H, v.W, v.taps, v.Gr + (size_t)k * n, blockIdx.y * kGT,
                    blockIdx.x * kGT);
}

// The dual step of recorded iteration k and, with do_x, the x-step of iteration k + 1,
// per pixel on the kXH x kXW tile of the block (two pixels per thread, rows i and i + 8):
//   v_{k+1} = W z with z = x_{k+1} + u_k (the third aggregation of Algorithm 2 with the
//   closure of Eq. S3, from the phase-1 partial sums and 1/m on the device),
//   u_{k+1} = u_k + x_{k+1} - v_{k+1} = z - v_{k+1},
//   x_{k+2} = Pi_C(mu (alpha x_{k+1} + rho (v_{k+1} - u_{k+1}) - g_{k+1})),  z <- x_{k+2} + u_{k+1},
// g_{k+1} recorded beforehand by adj_fwd_grad_kernel.  z is read and written at the
// thread's own pixels only.
__global__ void __launch_bounds__(256) adj_fwd_dual_x_kernel(const TapeView* __restrict__ tv, int k, int do_x) {
    griddep_enter();
    const TapeView& v = tv[blockIdx.z];
    const int H = v.H, W = v.W;
    const size_t n = (size_t)H * W;
    const int y0 = blockIdx.y * kXH, x0 = blockIdx.x * kXW;
    const int j = x0 + threadIdx.x, lj = j - (x0 / kTmaTW) * kTmaTW;
    const float inv_m = __ldg(v.m + 1);
    const float* d = v.Dh + (size_t)v.T * n;
    const float* t = v.Th + (size_t)v.T * n;
    float* z = v.z;
    float* v1 = v.V + (size_t)(k + 1) * n;
    float* u1 = v.U + (size_t)(k + 1) * n;
    const float* x1 = do_x ? v.X + (size_t)(k + 1) * n : nullptr;
    const float* g1 = do_x ? v.Gr + (size_t)(k + 1) * n : nullptr;
    float* x2 = do_x ? v.X + (size_t)(k + 2) * n : nullptr;
    const float mu = v.mu, alpha = v.alpha, rho = v.rho;
    const TileCover tc = tile_cover(v.cv, y0, x0);
    float zs[2], ds[2], ts[2], xs[2], gs[2], A[2];
    bool ok[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const int i = y0 + threadIdx.y + 8 * c;
        ok[c] = i < H && j < W;
        const size_t q = ok[c] ? (size_t)i * W + j : 0;
        zs[c] = z[q];
        ds[c] = d[q];
        ts[c] = t[q];
        xs[c] = do_x ? x1[q] : 0.f;
        gs[c] = do_x ? g1[q] : 0.f;
    }
#pragma unroll
    for (int c = 0; c < 2; ++c) A[c] = ok[c] ? tile_gather(tc, threadIdx.y + 8 * c, lj) : 0.f;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        if (!ok[c]) continue;
        const size_t q = (size_t)(y0 + threadIdx.y + 8 * c) * W + j;
        const float dm = ds[c] * inv_m;
        const float cs = 1.f - dm * (ts[c] - ds[c]);
        const float vn = fmaf(dm, A[c], cs * zs[c]);
        const float un = zs[c] - vn;
        v1[q] = vn;
        u1[q] = un;
        if (do_x) {
            const float xn = project(mu * (alpha * xs[c] + rho * (vn - un) - gs[c]), v.constraint);
            x2[q] = xn;
            z[q] = xn + un;
        }
    }
}

// x_N to the caller's buffer
__global__ void __launch_bounds__(256) adj_xout_kernel(const TapeView* __restrict__ tv) {
    griddep_enter();
    const TapeView& v = tv[blockIdx.z];
    const size_t n = (size_t)v.H * v.W;
    const size_t q = (size_t)blockIdx.x * 256 + threadIdx.x;
    if (q < n) v.x_out[q] = v.X[(size_t)v.N * n + q];
}

// ----------------------------------------------------------------------- backward

// cotangents cleared, xh = x_bar, and the iteration N - 1 inputs of the reverse sweep:
// a_{N-1} = vh - uh = 0, z_{N-1} = x_N + u_{N-1} (a in its plane, a and z in the
// interleaved copy)
__global__ void __launch_bounds__(256) adj_bwd_prep_kernel(const TapeView* __restrict__ tv, int nrb) {
    griddep_enter();
    const TapeView& v = tv[blockIdx.z];
    const size_t n = (size_t)v.H * v.W;
    const size_t q = (size_t)blockIdx.x * 256 + threadIdx.x;
    if (q < (size_t)nrb) v.rho_part[q] = 0.0;
    if (q >= n) return;
    v.xh[q] = v.x_bar[q];
    v.gs[q] = 0.f;
    v.vh[q] = 0.f;
    v.uh[q] = 0.f;
    const int N = v.N;
    v.AZ[(size_t)(N - 1) * n + q] = 0.f;
    float* s4 = v.AZ4 + 4 * ((size_t)((N - 1) >> 1) * n + q);
    const int lane = (N - 1) & 1;
    s4[lane] = 0.f;
    s4[2 + lane] = v.X[(size_t)N * n + q] + v.U[(size_t)(N - 1) * n + q];
    if (lane == 0) {  // N odd: the pair's second iteration does not exist and adds zeros
        s4[1] = 0.f;
        s4[3] = 0.f;
    }
}

// W a finished from the phase-1 partial sums (W a = c_s a_s + (d_s / m) sum_r K1 d_r a_r,
// the closure of Eq. S3), then zh = W a + uh, g = Pi_C'(xbar_k)(xh + zh), the block's
// partial of sum g mu ((v - u) - xbar), and the per-pixel cotangent updates (vh, uh, gs
// and the earlier iteration's inputs a and z).  Blocks of 32 x 8 threads, 16 x 32 pixels.
// a_zero: a = 0 (no weight stream ran; W a = 0).
__global__ void __launch_bounds__(256) adj_wa_g_kernel(const TapeView* __restrict__ tv, int k, int a_zero) {
    griddep_enter();
    const TapeView& v = tv[blockIdx.z];
    const int H = v.H, W = v.W;
    const size_t n = (size_t)H * W;
    const int j = blockIdx.x * 32 + threadIdx.x;
    const float inv_m = __ldg(v.m + 1);
    const float mu = v.mu, alpha = v.alpha, rho = v.rho;
    const float* d = v.Dh + (size_t)v.T * n;
    const float* t_fin = v.Th + (size_t)v.T * n;
    const float *ak = v.AZ + (size_t)k * n, *vk = v.V + (size_t)k * n, *uk = v.U + (size_t)k * n;
    const float *xk = v.X + (size_t)k * n, *gk = v.Gr + (size_t)k * n;
    const bool more = k > 0;
    const float* uprev = more ? v.U + (size_t)(k - 1) * n : uk;
    float* a_next = more ? v.AZ + (size_t)(k - 1) * n : nullptr;
    float* s4 = more ? v.AZ4 + 4 * (size_t)((k - 1) >> 1) * n + ((k - 1) & 1) : nullptr;  // lane of iteration k - 1
    // the thread's two pixels, rows i and i + 8 of the block's 16 x 32 tile: every load of
    // both is issued before the first use
    float ds[2], ts[2], as[2], uhs[2], vs[2], us[2], xs[2], grs[2], xhs[2], gss[2], ups[2], A[2];
    bool ok[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const int i = blockIdx.y * 16 + threadIdx.y + 8 * c;
        ok[c] = i < H && j < W;
        const size_t q = ok[c] ? (size_t)i * W + j : 0;
        ds[c] = d[q];
        ts[c] = t_fin[q];
        as[c] = ak[q];
        uhs[c] = v.uh[q];
        vs[c] = vk[q];
        us[c] = uk[q];
        xs[c] = xk[q];
        grs[c] = gk[q];
        xhs[c] = v.xh[q];
        gss[c] = v.gs[q];
        ups[c] = uprev[q];
        A[c] = (a_zero || !ok[c]) ? 0.f : gather_partials(v.cv, i, j);
    }
    float r = 0.f;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        if (!ok[c]) continue;
        const size_t q = (size_t)(blockIdx.y * 16 + threadIdx.y + 8 * c) * W + j;
        const float dm = ds[c] * inv_m;
        const float cs = 1.f - dm * (ts[c] - ds[c]);
        const float wa = fmaf(dm, A[c], cs * as[c]);
        const float zz = wa + uhs[c];
        const float vu = vs[c] - us[c];
        const float xb = mu * (alpha * xs[c] + rho * vu - grs[c]);
        const float gg = proj_deriv(xb, v.constraint) * (xhs[c] + zz);
        v.g[q] = gg;
        r += gg * mu * (vu - xb);
        // the cotangent updates that need no neighbours: vh = mu rho g, uh = zh - mu rho g,
        // gs += mu g, and for k > 0 the earlier iteration's a = vh - uh and z = x_k + u_{k-1}
        const float vv = mu * rho * gg;
        const float uu = zz - vv;
        v.vh[q] = vv;
        v.uh[q] = uu;
        v.gs[q] = gss[c] + mu * gg;
        if (more) {
            const float an = vv - uu;
            a_next[q] = an;
            s4[4 * q] = an;
            s4[4 * q + 2] = xs[c] + ups[c];
        }
    }
    const int t = threadIdx.y * 32 + threadIdx.x;
    const double acc = block_sum_256(r, t);
    // a fixed slot per block, accumulated in a fixed order over the iterations
    if (t == 0) v.rho_part[blockIdx.y * gridDim.x + blockIdx.x] += acc;
}

// Reverse iteration k, after g: xh = mu (alpha g - A^T A g), the A^T A g on 32 x 32 tiles.
// It is the only step of the iteration that needs neighbouring pixels, so it runs beside
// the weight stream of the earlier iteration's a (which the W a finish forms per pixel).
// g is only read, so the halo reads do not race with the writes.
template <int R>
__global__ void __launch_bounds__(256, 4) adj_ata_update_kernel(const TapeView* __restrict__ tv, int k) {
    griddep_enter();
    __shared__ GradSmem<R> sm;
    const TapeView& v = tv[blockIdx.z];
    const int W = v.W;
    const float* g = v.g;
    float* xh = v.xh;
    const float mu = v.mu, alpha = v.alpha;
    float2 gp[2];  // the epilogue pixels' g, loaded before the stencil (pixel pairs: q even)
    sr_grad_tile_apply2<R>(
        sm, g, nullptr, v.H, W, v.taps, blockIdx.y * kGT, blockIdx.x * kGT,
        [&](int sl, int pi, int pj) { gp[sl] = *reinterpret_cast<const float2*>(g + (size_t)pi * W + pj); },
        [&](int sl, int pi, int pj, float e, float o) {
            const size_t q = (size_t)pi * W + pj;
            xh[q] = mu * (alpha * gp[sl].x - e);
            xh[q + 1] = mu * (alpha * gp[sl].y - o);
        });
    (void)k;
}

// fixed-order sum of one partial array of each image into one of its cotangents:
// which 0: m_part -> mh[0], 1: rho_part -> mh[1], 2: h_part -> mh[2]; one block per image
__global__ void __launch_bounds__(256) adj_sum_kernel(const TapeView* __restrict__ tv, int which, int count_m,
                                                      int count_rho) {
    griddep_enter();
    const TapeView& v = tv[blockIdx.x];
    const double* part = which == 1 ? v.rho_part : which == 2 ? v.h_part : v.m_part;
    const int count = which == 1 ? count_rho : count_m;
    double a = 0.0;
    for (int q = threadIdx.x; q < count; q += 256) a += part[q];
    __shared__ double s[256];
    s[threadIdx.x] = a;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) v.mh[which] = s[0];
}

// Through m = d_{s*} t_{s*}: dh_{s*} += mh (t_{s*} + d_{s*}); dh_j += mh d_{s*} K1(s*, j),
// j != s*; one block per image
template <typename WT>
__global__ void adj_mterms_kernel(const TapeView* __restrict__ tv) {
    griddep_enter();
    const TapeView& v = tv[blockIdx.x];
    const WT* __restrict__ P = static_cast<const WT*>(v.planes);
    const int H = v.H, W = v.W, rs = v.rs;
    const size_t n = (size_t)H * W;
    const float* d = v.Dh + (size_t)v.T * n;
    const float* t = v.Th + (size_t)v.T * n;
    float* dh = v.dh;
    const int ss = *v.sstar;
    const int si = ss / W, sj = ss - si * W;
    const float mh = (float)v.mh[0];
    const int Wp = plane_pitch(W);
    const size_t plane = (size_t)H * Wp;
    const int side = 2 * rs + 1;
    for (int q = threadIdx.x; q < side * side; q += blockDim.x) {
        const int oy = q / side - rs, ox = q % side - rs;
        const int ri = si + oy, rj = sj + ox;
        if (ri < 0 || ri >= H || rj < 0 || rj >= W) continue;
        if (oy == 0 && ox == 0) {
            dh[ss] += mh * (t[ss] + d[ss]);
            continue;
        }
        // K1(s*, r): plane of the half offset +-o at the lower-indexed end
        const bool fwd = oy > 0 || (oy == 0 && ox > 0);
        const int ay = fwd ? oy : -oy, ax = fwd ? ox : -ox;
        const int k = ay == 0 ? ax - 1 : rs + (ay - 1) * (2 * rs + 1) + ax + rs;
        const size_t at = (size_t)k * plane + (fwd ? (size_t)si * Wp + sj : (size_t)ri * Wp + rj);
        const float K = to_f32(P[at]);
        dh[(size_t)ri * W + rj] += mh * d[ss] * K;
    }
}

// Balancing pass T - 1 backwards: th = -0.5 dh' d'/t, base = 0.5 dh' d'/d (d' = d^T)
__global__ void __launch_bounds__(256) adj_sk_pre_kernel(const TapeView* __restrict__ tv) {
    griddep_enter();
    const TapeView& v = tv[blockIdx.z];
    const size_t n = (size_t)v.H * v.W;
    const size_t q = (size_t)blockIdx.x * 256 + threadIdx.x;
    if (q >= n) return;
    const int T = v.T;
    const float w = 0.5f * v.dh[q] * v.Dh[(size_t)T * n + q];
    v.thp[(size_t)(T - 1) * n + q] = -w / v.Th[(size_t)(T - 1) * n + q];
    v.base[q] = w / v.Dh[(size_t)(T - 1) * n + q];
}

// dh^p = base + K1 th^p = base + th^p + sum_{r != s} K1 th^p_r (phase-1 partial sums in
// cv), the cotangent of d^p, and from it pass p - 1's th^{p-1} = -0.5 dh^p d^p / t^{p-1}
// and base = 0.5 dh^p d^p / d^{p-1} (base rewritten in place)
__global__ void __launch_bounds__(256) adj_sk_finish_pre_kernel(const TapeView* __restrict__ tv, int p) {
    griddep_enter();
    const TapeView& v = tv[blockIdx.z];
    const int H = v.H, W = v.W;
    const size_t n = (size_t)H * W;
    const int j = blockIdx.x * 32 + threadIdx.x;
    const int i = blockIdx.y * 8 + threadIdx.y;
    if (i >= H || j >= W) return;
    const size_t s = (size_t)i * W + j;
    const float* th = v.thp + (size_t)p * n;
    const float dh = v.base[s] + th[s] + gather_partials(v.cv, i, j);
    const float w = 0.5f * dh * v.Dh[(size_t)p * n + s];
    v.thp[(size_t)(p - 1) * n + s] = -w / v.Th[(size_t)(p - 1) * n + s];
    v.base[s] = w / v.Dh[(size_t)(p - 1) * n + s];
}

// Stage `nf` fields (each n floats apart) over rows [r0, r0 + RH), cols [c0, c0 + RW), zero outside.
__device__ __forceinline__ void stage_fields(float* S, const float* __restrict__ F, int nf, size_t n, int H, int W,
                                             int r0, int c0, int RH, int RW) {
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const int cells = RH * RW;
    for (int f = 0; f < nf; ++f)
        for (int idx = tid; idx < cells; idx += 256) {
            const int a = idx / RW, b = idx - a * RW;
            const int i = r0 + a, j = c0 + b;
            S[f * cells + idx] = (i >= 0 && i < H && j >= 0 && j < W) ? F[f * n + (size_t)i * W + j] : 0.f;
        }
}

// Pair pass B: the cotangent of every stored weight K1(s, s + o),
//   Kh = G d_s d_r / m + sum_p (th^p_s d^p_r + th^p_r d^p_s) + [s or r = s*] mh d_s d_r,
// then Dh = -c K1 Kh (written as planes) and per-block partials of dL/dh = sum Kh K1 D 2c/h.
// G comes from the planes of pair pass G; fields staged over the tile and its forward
// halo: d^p (T + 1) and th^p (T).  Grid z = image * kPairSplit + chunk, the half
// offsets split as in pass G.
template <typename WT>
__global__ void __launch_bounds__(256, 3) adj_pairs_b_kernel(const TapeView* __restrict__ tv) {
    griddep_enter();
    extern __shared__ float S[];
    const int img = blockIdx.z / kPairSplit, zc = blockIdx.z - img * kPairSplit;
    const TapeView& v = tv[img];
    const WT* __restrict__ P = static_cast<const WT*>(v.planes);
    const int H = v.H, W = v.W, rs = v.rs, T = v.T;
    const float c = v.c, hfac = v.hfac;
    const float inv_m = __ldg(v.m + 1);
    const int y0 = blockIdx.y * kAdjTH, x0 = blockIdx.x * kAdjTW;
    const int RH = kAdjTH + rs, RW = kAdjTW + 2 * rs, cells = RH * RW;
    const size_t n = (size_t)H * W;
    stage_fields(S, v.Dh, T + 1, n, H, W, y0, x0 - rs, RH, RW);
    stage_fields(S + (T + 1) * cells, v.thp, T, n, H, W, y0, x0 - rs, RH, RW);
    __syncthreads();
    const float* Sdp = S;                  // d^0 .. d^T
    const float* Sth = S + (T + 1) * cells;  // th^0 .. th^{T-1}
    const float* Sd = Sdp + T * cells;     // d = d^T
    __shared__ float lglam[kMaxHalfOffsets];
    {
        const float inv_hat = 1.0f / (float)(rs + 1);
        for (int k = threadIdx.y * 32 + threadIdx.x; k < num_half_offsets(rs); k += 256) {
            int oy, ox;
            half_offset(k, rs, oy, ox);
            lglam[k] = logf((1.0f - fabsf((float)oy) * inv_hat) * (1.0f - fabsf((float)ox) * inv_hat));
        }
    }
    __syncthreads();
    const float inv_c = 1.0f / c;
    const int kz0 = num_half_offsets(rs) * zc / kPairSplit;
    const int kz1 = num_half_offsets(rs) * (zc + 1) / kPairSplit;
    const int ss = *v.sstar;
    const float mh = (float)v.mh[0];
    const int Wp = plane_pitch(W);
    const size_t plane = (size_t)H * Wp;
    const float* Gp = v.Gp;
    float* Dhat = v.Dhat;
    float hpart = 0.f;
    const int j = x0 + threadIdx.x;
    for (int py = threadIdx.y; py < kAdjTH; py += 8) {
        const int i = y0 + py;
        if (i >= H || j >= W) continue;
        const int cs = py * RW + threadIdx.x + rs;
        const int sidx = i * W + j;
        float hp = 0.f;  // this pixel's sum of Kh K1 D over its chunk (FP32)
        int oy, ox;
        half_offset(kz0, rs, oy, ox);
        // branch-free body (off-image pairs are masked), so the unrolled iterations issue
        // their loads together
#pragma unroll 2
        for (int k = kz0; k < kz1; ++k) {
            {
                const size_t at = (size_t)k * plane + (size_t)i * Wp + j;
                const int rj = j + ox;
                const bool in = i + oy < H && rj >= 0 && rj < W;
                const float K = in ? to_f32(P[at]) : 0.f;
                const float G = in ? Gp[at] : 0.f;
                const int cr = cs + oy * RW + ox;
                float Kh = G * Sd[cs] * Sd[cr] * inv_m;
                for (int p = 0; p < T; ++p)
                    Kh += Sth[p * cells + cs] * Sdp[p * cells + cr] + Sth[p * cells + cr] * Sdp[p * cells + cs];
                const int ridx = (i + oy) * W + rj;
                if (sidx == ss || ridx == ss) Kh = fmaf(mh, Sd[cs] * Sd[cr], Kh);
                Dhat[at] = in ? -c * K * Kh : 0.f;
                // D = -log(K1 / lam) / c, lam the hat weight of the offset
                hp = (in && K > 0.f) ? fmaf(Kh * K, (lglam[k] - logf(K)) * inv_c, hp) : hp;
            }
            if (++ox > rs) {
                ++oy;
                ox = -rs;
            }
        }
        hpart += hp;
    }
    const int t = threadIdx.y * 32 + threadIdx.x;
    const double acc = block_sum_256(hpart, t);
    if (t == 0) v.h_part[(zc * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = acc * (double)hfac;
}

// Patch-distance adjoint.  With g the reflected guide on the grid extended by the
// patch radius (p in [-rp, H + rp) x [-rp, W + rp)) and, per offset o,
//   E_o(q) = sum_{t in patch} Dh_o(q - t)               (box sum, Dh = 0 off the image)
//   F_o(q) = 2 E_o(q) (g(q) - g(q + o)),
// the cotangent of g(p) is ge(p) = sum_o F_o(p) - F_o(p - o): the first term from the
// patch at q = p, the second from the patch whose partner pixel is p.
//
// One kernel per tile Q of the extended grid (kQH x kQW) and chunk of the half
// offsets (grid z = image * chunks + chunk).  For each offset of the chunk in turn the
// block stages D-hat over Q and its patch halo, forms E_o on Q by row sums then column
// sums in shared memory, and adds F_o(q) to q's own sum (a register) and -F_o(q) to
// q + o in a shared accumulator over Q, rs rows below and rs columns either side.  No
// two q of one offset share q + o, and the offsets are separated by the barriers of the
// box sums, so every accumulator element is summed in offset order.  The block writes
// its accumulator window (own sums added) as one partial; the fold gathers ge(p) from
// the partials of every chunk and of the (up to six) tiles whose windows hold p, in a
// fixed order.  E is never stored; the partials reuse the memory of the G planes,
// which pair pass B has read.
constexpr int kQH = 16, kQW = 32;

__host__ __device__ __forceinline__ int bg_win_h(int rs) { return kQH + rs; }
__host__ __device__ __forceinline__ int bg_win_w(int rs) { return kQW + 2 * rs; }

__global__ void __launch_bounds__(256) adj_boxguide_kernel(const TapeView* __restrict__ tv, int chunks) {
    griddep_enter();
    extern __shared__ float S[];
    const int img = blockIdx.z / chunks, zc = blockIdx.z - img * chunks;
    const TapeView& v = tv[img];
    const int H = v.H, W = v.W, rp = v.rp, rs = v.rs;
    const int nh = num_half_offsets(rs);
    const int k0 = nh * zc / chunks, k1 = nh * (zc + 1) / chunks;
    const int q0y = blockIdx.y * kQH - rp, q0x = blockIdx.x * kQW - rp;  // image coords of Q's origin
    const int DH = kQH + 2 * rp, DW = kQW + 2 * rp;  // D-hat window: rows q0y - rp + [0, DH), cols q0x - rp + [0, DW)
    const int AH = bg_win_h(rs), AW = bg_win_w(rs);  // accumulator window: rows q0y + [0, AH), cols q0x - rs + [0, AW)
    float* Gs = S;             // [AH][AW] the reflected guide over the window
    float* Ac = Gs + AH * AW;  // [AH][AW]
    float* Ds = Ac + AH * AW;  // [DH][DW]
    float* Rs = Ds + DH * DW;  // [DH][kQW] row sums
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * 32 + tx;
    for (int idx = tid; idx < AH * AW; idx += 256) {
        const int a = idx / AW, b = idx - a * AW;
        Gs[idx] = v.guide[(size_t)sym_index(q0y + a, H) * W + sym_index(q0x - rs + b, W)];
        Ac[idx] = 0.f;
    }
    const int Wp = plane_pitch(W);
    const size_t plane = (size_t)H * Wp;
    const int w = 2 * rp;
    float own0 = 0.f, own1 = 0.f;  // q = (ty, tx) and (ty + 8, tx) of Q
    const int c0 = ty * AW + tx + rs, c1 = c0 + 8 * AW;  // their cells in the window
    int oy, ox;
    half_offset(k0, rs, oy, ox);
    for (int k = k0; k < k1; ++k) {
        const float* Dk = v.Dhat + (size_t)k * plane;
        for (int a = ty; a < DH; a += 8) {
            const int i = q0y - rp + a;
            const bool rin = i >= 0 && i < H;
            const float* row = Dk + (size_t)(rin ? i : 0) * Wp;
            for (int b = tx; b < DW; b += 32) {
                const int j = q0x - rp + b;
                Ds[a * DW + b] = (rin && j >= 0 && j < W) ? row[j] : 0.f;
            }
        }
        __syncthreads();  // Ds of this offset written; Ac of the previous offset updated
        for (int a = ty; a < DH; a += 8) {
            const float* r = Ds + a * DW + tx;
            float s = 0.f;
            for (int t = 0; t <= w; ++t) s += r[t];
            Rs[a * kQW + tx] = s;
        }
        __syncthreads();  // Rs written; Ds free for the next offset
        const int sh = oy * AW + ox;
        {
            const float* r = Rs + ty * kQW + tx;
            float e = 0.f;
            for (int t = 0; t <= w; ++t) e += r[t * kQW];
            const float F = 2.f * e * (Gs[c0] - Gs[c0 + sh]);
            own0 += F;
            Ac[c0 + sh] -= F;
        }
        {
            const float* r = Rs + (ty + 8) * kQW + tx;
            float e = 0.f;
            for (int t = 0; t <= w; ++t) e += r[t * kQW];
            const float F = 2.f * e * (Gs[c1] - Gs[c1 + sh]);
            own1 += F;
            Ac[c1 + sh] -= F;
        }
        if (++ox > rs) {
            ++oy;
            ox = -rs;
        }
    }
    __syncthreads();
    Ac[c0] += own0;
    Ac[c1] += own1;
    __syncthreads();
    const size_t obase = (((size_t)zc * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x) * (size_t)(AH * AW);
    if (DSG_IN_RANGE(obase + AH * AW - 1, v.gpart_cap, kChkAdjWindows))
        for (int idx = tid; idx < AH * AW; idx += 256) v.gpart[obase + idx] = Ac[idx];
}

// Pair pass B fused with the patch-distance adjoint.  Per tile Q of the extended grid
// (kQH x (32 - 2 rp), so that Q with its patch halo is 32 columns wide) and chunk of the
// half offsets (grid z = image * chunks + chunk), for each offset o of the chunk in turn:
//   1. D-hat(s, o) = -c K1 Kh at every s of Q and its patch halo (the pixels whose
//      D-hat enters the box sums over Q), Kh as in pair pass B, into shared memory;
//      pixels of Q itself also add Kh K1 D to the block's dL/dh partial, with
//      D = (log2 lam - log2 K1) ln 2 / c recovered from the stored weight;
//   2. row sums across the lanes of each warp (a warp holds one row of the 32-wide
//      window), then, after the offset's one barrier, column sums: E_o on Q;
//   3. the scatter of F_o(q) = 2 E_o(q) (g(q) - g(q + o)) as in the box-and-gather
//      kernel, into the same partial layout (windows of Q's width).
// D-hat is never stored.  The halo's D-hat is recomputed by the neighbouring tiles
// ((kQH + 2 rp) 32 / (kQH (32 - 2 rp)) of the pairs, 1.43 at rp = 2), which costs less
// than writing the planes and reading them back.  The row sums alternate between two
// buffers by offset parity, so one barrier per offset orders everything; shared-memory
// accesses are conflict-free.
// K1 and G of the window arrive by TMA, two offsets ahead, into a ring of two stages
// (one thread issues the copies once every thread has finished with the stage).  The
// tensors' rows are W wide and the planes are zero where s + o leaves the image (the
// weight build writes zeros there), so pairs off the image contribute exact zeros with
// no per-pair test.  The balancing fields are staged as pairs (d^p, d^{p+1}) and
// (th^p, th^{p+1}), so that the sum over the passes takes one packed FP32x2 FMA per
// pair of passes.  The patch radius RP is a template argument (1 to 3); RS > 0 and
// TT >= 0 fix the search radius and the number of balancing passes (field strides
// become constants and the fields at s stay in registers), RS = 0 and TT = -1 read
// them from the view.
template <int RP>
struct Bd {
    static constexpr int QW = 32 - 2 * RP;  // tile width
    static constexpr int DH = kQH + 2 * RP;  // D-hat window rows (32 columns)
    static constexpr int NC = (DH + 7) / 8;  // window rows per thread
};
// TMA box widths: the window's 32 columns from the 16-byte-aligned column at or left of
// its first column
__host__ __device__ constexpr int bd_box_w(int esz) { return esz == 4 ? 36 : 40; }
__host__ __device__ constexpr int bd_stage_bytes(int rows, int cols, int esz) {
    return (rows * cols * esz + 127) & ~127;
}

__host__ __device__ __forceinline__ int bd_qw(int rp) { return 32 - 2 * rp; }
__host__ __device__ __forceinline__ int bd_field_h(int rp, int rs) { return kQH + 2 * rp + rs; }
__host__ __device__ __forceinline__ int bd_field_w(int rs) { return 32 + 2 * rs; }
__host__ __device__ __forceinline__ int bd_win_w(int rp, int rs) { return bd_qw(rp) + 2 * rs; }

template <typename WT, int RP, int RS, int TT>
__global__ void __launch_bounds__(256, 3)
    adj_pairs_bd_kernel(const TapeView* __restrict__ tv, int chunks, unsigned* err, long long budget) {
    griddep_enter();
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int rp = RP, QW = Bd<RP>::QW, DH = Bd<RP>::DH, NC = Bd<RP>::NC;
    constexpr int KBW = bd_box_w((int)sizeof(WT)), GBW = bd_box_w(4);
    constexpr int KBYTES = DH * KBW * (int)sizeof(WT), GBYTES = DH * GBW * 4;
    constexpr int KST = bd_stage_bytes(DH, KBW, (int)sizeof(WT)), GST = bd_stage_bytes(DH, GBW, 4);
    constexpr int NP = TT >= 0 ? (TT + 1) / 2 : 1;  // field pairs held in registers per cell
    const int img = blockIdx.z / chunks, zc = blockIdx.z - img * chunks;
    const TapeView& v = tv[img];
    const int H = v.H, W = v.W;
    const int rs = RS > 0 ? RS : v.rs;
    const int T = TT >= 0 ? TT : v.T;
    const int P = (T + 1) / 2;
    const int nh = num_half_offsets(rs);
    const int k0 = nh * zc / chunks, k1 = nh * (zc + 1) / chunks;
    const int q0y = blockIdx.y * kQH - rp, q0x = blockIdx.x * QW - rp;  // image coords of Q's origin
    const int FH = bd_field_h(rp, rs), FW = bd_field_w(rs);  // field window, origin (q0y - rp, q0x - rp - rs)
    const int AH = bg_win_h(rs), AW = bd_win_w(rp, rs);      // accumulator window, origin (q0y, q0x - rs)
    const int fcells = FH * FW;
    const size_t n = (size_t)H * W;
    // stage st: K1 at smem + st KST, G at smem + 2 KST + st GST
    float* Rs = reinterpret_cast<float*>(smem + 2 * KST + 2 * GST);  // [2][DH][32] row sums (QW used), by offset parity
    float2* DP = reinterpret_cast<float2*>(Rs + 2 * DH * 32);        // [P][FH][FW] (d^2q, d^2q+1)
    float2* TP = DP + (size_t)P * fcells;                            // [P][FH][FW] (th^2q, th^2q+1)
    float* Dd = reinterpret_cast<float*>(TP + (size_t)P * fcells);   // [FH][FW] d = d^T
    float* Gs = Dd + fcells;                                         // [AH][AW] the reflected guide
    float* Ac = Gs + AH * AW;                                        // [AH][AW] the scatter accumulator
    __shared__ float lglam[kMaxHalfOffsets];
    __shared__ __align__(8) uint64_t bars[2];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * 32 + tx;
    const CUtensorMap* kmap = reinterpret_cast<const CUtensorMap*>(v.bd_kmap);
    const CUtensorMap* gmap = reinterpret_cast<const CUtensorMap*>(v.bd_gmap);
    const int xw = q0x - rp, yw = q0y - rp;  // the D-hat window's first column and row
    const int xk = xw & ~(16 / (int)sizeof(WT) - 1), xg = xw & ~3;
    const int xoK = xw - xk, xoG = xw - xg;
    uint64_t policy = 0;
    auto issue = [&](int k, int st) {
        mbar_arrive_expect_tx(&bars[st], (unsigned)(KBYTES + GBYTES));
        tma_load_3d(smem + st * KST, kmap, &bars[st], xk, yw, k, policy);
        tma_load_3d(smem + 2 * KST + st * GST, gmap, &bars[st], xg, yw, k, policy);
    };
    if (tid == 0) {
        tmap_acquire(kmap);
        tmap_acquire(gmap);
        policy = evict_first_policy();
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (k0 < k1) issue(k0, 0);
        if (k0 + 1 < k1) issue(k0 + 1, 1);
    }
    // stage the fields over the field window (zero off the image), the guide and a zero
    // accumulator over the accumulator window, and log2 of every offset's hat weight
#pragma unroll 2
    for (int idx = tid; idx < fcells; idx += 256) {
        const int a = idx / FW, b = idx - a * FW;
        const int i = q0y - rp + a, j = q0x - rp - rs + b;
        const bool in = i >= 0 && i < H && j >= 0 && j < W;
        const size_t q = in ? (size_t)i * W + j : 0;
        for (int u = 0; u < P; ++u) {
            const int p0 = 2 * u, p1 = p0 + 1;
            const bool in1 = in && p1 < T;
            DP[u * fcells + idx] = make_float2(in ? v.Dh[p0 * n + q] : 0.f, in1 ? v.Dh[p1 * n + q] : 0.f);
            TP[u * fcells + idx] = make_float2(in ? v.thp[p0 * n + q] : 0.f, in1 ? v.thp[p1 * n + q] : 0.f);
        }
        Dd[idx] = in ? v.Dh[T * n + q] : 0.f;
    }
    for (int idx = tid; idx < AH * AW; idx += 256) {
        const int a = idx / AW, b = idx - a * AW;
        Gs[idx] = v.guide[(size_t)sym_index(q0y + a, H) * W + sym_index(q0x - rs + b, W)];
        Ac[idx] = 0.f;
    }
    {
        const float inv_hat = 1.0f / (float)(rs + 1);
        for (int k = tid; k < nh; k += 256) {
            int oy, ox;
            half_offset(k, rs, oy, ox);
            lglam[k] = __log2f((1.0f - fabsf((float)oy) * inv_hat) * (1.0f - fabsf((float)ox) * inv_hat));
        }
    }
    __syncthreads();
    // the thread's D-hat cells (a, b) = (ty + 8 m, tx), m < NC: row a's field cell of s
    // and s's flat index (each m steps them by a constant), which cells are pixels of Q
    // (bit m), and (TT >= 0) the fields at s
    const int j = q0x - rp + tx;
    const int i0 = q0y - rp + ty;
    const int fs0 = ty * FW + tx + rs, sidx0 = i0 * W + j;
    unsigned ownb = 0u;
    float2 svD[NC][NP], svT[NC][NP];
    float svd[NC];
#pragma unroll
    for (int m = 0; m < NC; ++m) {
        const int a = ty + 8 * m;
        const int i = i0 + 8 * m;
        const bool in = a < DH && i >= 0 && i < H && j >= 0 && j < W;
        ownb |= (in && a >= rp && a < rp + kQH && tx >= rp && tx < rp + QW) ? 1u << m : 0u;
        const int cs = a < DH ? fs0 + 8 * m * FW : fs0;
        svd[m] = Dd[cs];
        if constexpr (TT >= 0) {
#pragma unroll
            for (int u = 0; u < NP; ++u) {
                svD[m][u] = DP[u * fcells + cs];
                svT[m][u] = TP[u * fcells + cs];
            }
        }
    }
    const float c = v.c, inv_m = __ldg(v.m + 1), mh = (float)v.mh[0];
    const float inv_c2 = 0.693147180559945f / c;  // ln 2 / c
    const int ss = *v.sstar;
    float hp = 0.f;  // the own pixels' sum of Kh K1 D over the chunk (FP32)
    float own0 = 0.f, own1 = 0.f;  // q = (ty, tx) and (ty + 8, tx) of Q
    const int c0 = ty * AW + tx + rs, c1 = c0 + 8 * AW;
    const bool qcol = tx < QW;
    bool gave_up = false;
    int oy, ox;
    half_offset(k0, rs, oy, ox);
    for (int k = k0; k < k1; ++k) {
        const int st = (k - k0) & 1;
        const unsigned par = (unsigned)((k - k0) >> 1) & 1u;
        // the stage's copies; after a wait that ran out (here or in another block) the
        // block stops waiting, and the error word makes the call fail
        if (!gave_up && !mbar_try_wait(&bars[st], par)) {
            if (*(volatile unsigned*)err != 0u || !mbar_wait_consumer(&bars[st], par, budget)) {
                gave_up = true;
                if (tid == 0) atomicOr(err, 1u);
            }
        }
        const WT* Kw = reinterpret_cast<const WT*>(smem + st * KST) + xoK + tx;
        const float* Gw = reinterpret_cast<const float*>(smem + 2 * KST + st * GST) + xoG + tx;
        const int fo = oy * FW + ox;
        const int oW = oy * W + ox;
        const float lk = lglam[k];
        // 1. D-hat of offset k at the thread's cells and its row sums over the patch width:
        // a warp holds one row of the 32-wide window, so the sums run across its lanes
        // (the lanes past Q's width form sums that are not used)
        float* Rk = Rs + (k & 1) * (DH * 32);
#pragma unroll
        for (int m = 0; m < NC; ++m) {
            const int a = ty + 8 * m;
            if (m < 2 || a < DH) {
                const float K = to_f32(Kw[a * KBW]);
                const float G = Gw[a * GBW];
                const int cs = fs0 + 8 * m * FW, cr = cs + fo;
                const float ds = svd[m], dr = Dd[cr];
                // the two halves of the balancing terms in independent chains
                float2 acc = make_float2(0.f, 0.f), acc2 = make_float2(0.f, 0.f);
                if constexpr (TT >= 0) {
#pragma unroll
                    for (int u = 0; u < NP; ++u) {
                        acc = __ffma2_rn(svT[m][u], DP[u * fcells + cr], acc);    // th^p_s d^p_r
                        acc2 = __ffma2_rn(TP[u * fcells + cr], svD[m][u], acc2);  // th^p_r d^p_s
                    }
                } else {
                    for (int u = 0; u < P; ++u) {
                        acc = __ffma2_rn(TP[u * fcells + cs], DP[u * fcells + cr], acc);
                        acc2 = __ffma2_rn(TP[u * fcells + cr], DP[u * fcells + cs], acc2);
                    }
                }
                float Kh = fmaf(G * ds, dr * inv_m, (acc.x + acc.y) + (acc2.x + acc2.y));
                const int si = sidx0 + 8 * m * W;
                if (si == ss || si + oW == ss) Kh = fmaf(mh, ds * dr, Kh);
                if ((ownb >> m) & 1u) hp = K > 0.f ? fmaf(Kh * K, (lk - __log2f(K)) * inv_c2, hp) : hp;
                const float val = -c * K * Kh;
                float rsum = val;
#pragma unroll
                for (int t = 1; t <= 2 * rp; ++t) rsum += __shfl_down_sync(0xffffffffu, val, t);
                Rk[a * 32 + tx] = rsum;
            }
        }
        // the row sums of this offset written, the stage read; the scatter of the offset
        // before (which read the other row-sum buffer) done
        __syncthreads();
        if (tid == 0 && k + 2 < k1) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(k + 2, st);
        }
        // 3. the scatter
        if (qcol) {
            const int sh = oy * AW + ox;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int cq = h == 0 ? c0 : c1;
                const float* r = Rk + (ty + 8 * h) * 32 + tx;
                float e = r[0];
#pragma unroll
                for (int t = 1; t <= 2 * rp; ++t) e += r[t * 32];
                const float F = 2.f * e * (Gs[cq] - Gs[cq + sh]);
                if (h == 0)
                    own0 += F;
                else
                    own1 += F;
                Ac[cq + sh] -= F;
            }
        }
        if (++ox > rs) {
            ++oy;
            ox = -rs;
        }
    }
    // the block's dL/dh partial (the barrier inside also ends every scatter)
    const double hacc = block_sum_256(hp, tid);
    if (tid == 0) v.h_part[(zc * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = hacc * (double)v.hfac;
    if (qcol) {
        Ac[c0] += own0;
        Ac[c1] += own1;
    }
    __syncthreads();
    const size_t obase = (((size_t)zc * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x) * (size_t)(AH * AW);
    if (DSG_IN_RANGE(obase + AH * AW - 1, v.gpart_cap, kChkAdjWindows))
        for (int idx = tid; idx < AH * AW; idx += 256) v.gpart[obase + idx] = Ac[idx];
}

// The window partials of the offset chunks added into chunk 0's (in chunk order), so
// that the gathers read one partial per window: which 0 the patch-distance adjoint's
// (gpart), 1 pair pass G's (dh0); `elems` values per chunk and image, grid z = image.
__global__ void __launch_bounds__(256) adj_chunk_sum_kernel(const TapeView* __restrict__ tv, int which, int elems,
                                                            int chunks) {
    griddep_enter();
    const TapeView& v = tv[blockIdx.z];
    float* part = which == 0 ? v.gpart : v.dh0;
    const int e = blockIdx.x * 256 + threadIdx.x;
    if (e >= elems) return;
    if (!DSG_IN_RANGE((size_t)(chunks - 1) * elems + e, which == 0 ? v.gpart_cap : v.dh0_cap, kChkAdjWindows)) return;
    float acc = part[e];
    for (int z = 1; z < chunks; ++z) acc += part[(size_t)z * elems + e];
    part[e] = acc;
}

// ge(p) of the extended-grid position p = (pi, pj) (image coords), tiles of width qw: the
// partials of every chunk and of the tiles whose accumulator windows hold p (rows ty0 - 1, ty0; columns
// tx0 - 1 .. tx0 + 1), chunk by chunk in that order.  The six candidates are tested once
// and their loads issued together (a candidate that does not hold p adds nothing).
__device__ __forceinline__ float gather_ge(const float* __restrict__ part, int pi, int pj, int rp, int rs, int tiles_y,
                                           int tiles_x, int chunks, int qw, long long cap) {
    const int AH = bg_win_h(rs), AW = qw + 2 * rs;
    const int ty0 = (pi + rp) / kQH, tx0 = (pj + rp) / qw;
    size_t off[6];
    bool ok[6];
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int w = 0; w < 3; ++w) {
            const int ty = ty0 - 1 + u, tx = tx0 - 1 + w;
            const int a = pi - (ty * kQH - rp), b = pj - (tx * qw - rp - rs);
            const bool in = ty >= 0 && ty < tiles_y && tx >= 0 && tx < tiles_x && a < AH && b >= 0 && b < AW;
            ok[u * 3 + w] = in;
            off[u * 3 + w] = in ? ((size_t)ty * tiles_x + tx) * (size_t)(AH * AW) + (size_t)a * AW + b : 0;
        }
    const size_t zstride = (size_t)tiles_y * tiles_x * (size_t)(AH * AW);
    float acc = 0.f;
    for (int z = 0; z < chunks; ++z) {
        const float* pz = part + (size_t)z * zstride;
        float v[6];
#pragma unroll
        for (int c = 0; c < 6; ++c)
            v[c] = (ok[c] && DSG_IN_RANGE((size_t)z * zstride + off[c], cap, kChkAdjWindows)) ? pz[off[c]] : 0.f;
#pragma unroll
        for (int c = 0; c < 6; ++c)
            if (ok[c]) acc += v[c];
    }
    return acc;
}

// gb(q) = (xh0 + vh0)(q) [0 < g(q) < 1] + sum of ge(p) over the extended p that reflect
// onto q (p = 2 n m + q or 2 n m - 1 - q per axis), in a fixed order: per axis the
// reflections -1 - q (q < rp), q, 2 n - 1 - q (q >= n - rp) while rp < n, the general
// enumeration otherwise
__global__ void __launch_bounds__(256) adj_fold_kernel(const TapeView* __restrict__ tv, int tiles_y, int tiles_x,
                                                       int chunks, int qw) {
    griddep_enter();
    const TapeView& v = tv[blockIdx.z];
    const int H = v.H, W = v.W, rp = v.rp, rs = v.rs;
    const int j = blockIdx.x * 32 + threadIdx.x;
    const int i = blockIdx.y * 8 + threadIdx.y;
    if (i >= H || j >= W) return;
    const size_t q = (size_t)i * W + j;
    const float g = v.guide[q];
    float acc = (g > 0.f && g < 1.f) ? v.xh[q] + v.vh[q] : 0.f;
    if (rp < H && rp < W) {
        int ri[3], rj[3], ni = 0, nj = 0;
        if (i < rp) ri[ni++] = -1 - i;
        ri[ni++] = i;
        if (i >= H - rp) ri[ni++] = 2 * H - 1 - i;
        if (j < rp) rj[nj++] = -1 - j;
        rj[nj++] = j;
        if (j >= W - rp) rj[nj++] = 2 * W - 1 - j;
        for (int a = 0; a < ni; ++a)
            for (int b = 0; b < nj; ++b)
                acc += gather_ge(v.gpart, ri[a], rj[b], rp, rs, tiles_y, tiles_x, chunks, qw, v.gpart_cap);
    } else {
        const int my = rp / (2 * H) + 1, mx = rp / (2 * W) + 1;
        for (int m = -my; m <= my; ++m)
            for (int cy = 0; cy < 2; ++cy) {
                const int pi = cy == 0 ? 2 * H * m - 1 - i : 2 * H * m + i;
                if (pi < -rp || pi >= H + rp) continue;
                for (int n = -mx; n <= mx; ++n)
                    for (int cx = 0; cx < 2; ++cx) {
                        const int pj = cx == 0 ? 2 * W * n - 1 - j : 2 * W * n + j;
                        if (pj < -rp || pj >= W + rp) continue;
                        acc += gather_ge(v.gpart, pi, pj, rp, rs, tiles_y, tiles_x, chunks, qw, v.gpart_cap);
                    }
            }
    }
    v.guide_bar[q] = acc;
}

// dL/dy = sum_k mu A g_k = A gs (A linear), every image (grid z)
template <int R>
__global__ void __launch_bounds__(256) adj_ybar_kernel(const TapeView* __restrict__ tv) {
    griddep_enter();
    const TapeView& v = tv[blockIdx.z];
    const int h = v.H / 2, w = v.W / 2;
    const int qj = blockIdx.x * 32 + threadIdx.x;
    const int qi = blockIdx.y * 8 + threadIdx.y;
    if (qi >= h || qj >= w) return;
    v.y_bar[(size_t)qi * w + qj] = sr_forward_at<R>(v.gs, v.H, v.W, v.taps, qi, qj);
}

// Pair pass G with the mirrored half of the scaling's cotangent.  Over the half-window
// pairs (s, r = s + o):
//   G_sr = sum_k (a_k(s) - a_k(r)) (z_k(r) - z_k(s)),
// stored as planes like K1 (values where s + o leaves the image are not used: K1 is
// zero there), per-block partials of -(1/m^2) sum G d_s d_r K1, and the window partials
// of dh0 = sum over the full window of G_sr d_r K1_sr: the forward term G d_r K1 of s
// and the mirrored term G d_s K1 of r (G and K1 are symmetric in (s, r)).
// Per tile of kQH x 32 pixels and chunk of the half offsets (grid z = image * chunks +
// chunk), one offset at a time: each thread forms G for its two pixels, adds the
// forward terms in registers and the mirrored terms into a shared accumulator over the
// tile, rs rows below and rs columns either side (no two pixels of one offset share
// r; the offsets are separated by a barrier), which the block writes as one window
// partial (its own pixels' forward sums added).  The weight tile of every offset
// arrives by TMA two offsets ahead.  Staged over the window: (a_2u, a_2u+1, z_2u,
// z_2u+1) as one float4 per pair of iterations (zeros past N; TMA copies of the
// interleaved copy the reverse sweep writes, zeros off the image) and d;
// the differences and products of the two iterations of a pair go through the packed
// FP32x2 units (a difference as an FMA with -1, which is exact).  With NPK > 0
// (= ceil(N / 2)) the values at s are held in registers; NPK = 0 reads them from
// shared memory.
template <typename WT, int NPK>
__global__ void __launch_bounds__(256, 2)
    adj_pairs_gt_kernel(const TapeView* __restrict__ tv, int chunks, unsigned* err, long long budget) {
    griddep_enter();
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int KBYTES = kQH * 32 * (int)sizeof(WT);
    constexpr int KST = bd_stage_bytes(kQH, 32, (int)sizeof(WT));
    constexpr int NR = NPK > 0 ? NPK : 1;
    const int img = blockIdx.z / chunks, zc = blockIdx.z - img * chunks;
    const TapeView& v = tv[img];
    const int H = v.H, W = v.W, rs = v.rs, N = v.N;
    const int np = NPK > 0 ? NPK : (N + 1) / 2;
    const int nh = num_half_offsets(rs);
    const int k0 = nh * zc / chunks, k1 = nh * (zc + 1) / chunks;
    const int y0 = blockIdx.y * kQH, x0 = blockIdx.x * 32;
    const int FH = kQH + rs, FW = 32 + 2 * rs, fcells = FH * FW;  // window: rows y0 + [0, FH), cols x0 - rs + [0, FW)
    const int AZST = bd_stage_bytes(FH, 4 * FW, 4);              // one iteration pair's window
    const size_t n = (size_t)H * W;
    unsigned char* az = smem + 2 * KST;  // [np] windows of float4 [FH][FW]
    float* Sd = reinterpret_cast<float*>(az + (size_t)np * AZST);
    float* Ac = Sd + fcells;
    auto AZ4 = [&](int u, int cell) -> const float4& {
        return reinterpret_cast<const float4*>(az + (size_t)u * AZST)[cell];
    };
    __shared__ __align__(8) uint64_t bars[3];  // the two weight stages, the (a, z) windows
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * 32 + tx;
    const CUtensorMap* kmap = reinterpret_cast<const CUtensorMap*>(v.gt_kmap);
    const CUtensorMap* amap = reinterpret_cast<const CUtensorMap*>(v.gt_amap);
    uint64_t policy = 0;
    auto issue = [&](int k, int st) {
        mbar_arrive_expect_tx(&bars[st], (unsigned)KBYTES);
        tma_load_3d(smem + st * KST, kmap, &bars[st], x0, y0, k, policy);
    };
    if (tid == 0) {
        tmap_acquire(kmap);
        tmap_acquire(amap);
        policy = evict_first_policy();
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_init(&bars[2], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        // the (a, z) windows: zeros off the image (the tensor's bounds), kept in L2
        mbar_arrive_expect_tx(&bars[2], (unsigned)(np * FH * 4 * FW * 4));
        for (int u = 0; u < np; ++u) tma_load_3d(az + (size_t)u * AZST, amap, &bars[2], 4 * (x0 - rs), y0, u, 0ull);
        if (k0 < k1) issue(k0, 0);
        if (k0 + 1 < k1) issue(k0 + 1, 1);
    }
    const float* d = v.Dh + (size_t)v.T * n;
    for (int idx = tid; idx < fcells; idx += 256) {
        const int a = idx / FW, b = idx - a * FW;
        const int i = y0 + a, j = x0 - rs + b;
        const bool in = i < H && j >= 0 && j < W;
        Sd[idx] = in ? d[(size_t)i * W + j] : 0.f;
        Ac[idx] = 0.f;
    }
    __syncthreads();
    bool gave_up = false;
    if (!mbar_try_wait(&bars[2], 0u) && !mbar_wait_consumer(&bars[2], 0u, budget)) {
        gave_up = true;
        if (tid == 0) atomicOr(err, 1u);
    }
    // the thread's pixels (ty + 8 m, tx), m = 0, 1, of the tile
    const int Wp = plane_pitch(W);
    const size_t plane = (size_t)H * Wp;
    const int j = x0 + tx;
    const int cs0 = ty * FW + tx + rs;
    float2 sa[2][NR], sz[2][NR];
    float ds[2], accd[2] = {0.f, 0.f};
    bool in[2];
#pragma unroll
    for (int m = 0; m < 2; ++m) {
        const int cs = cs0 + 8 * m * FW;
        in[m] = y0 + ty + 8 * m < H && j < W;
        ds[m] = Sd[cs];
        if constexpr (NPK > 0) {
#pragma unroll
            for (int u = 0; u < NPK; ++u) {
                const float4 t = AZ4(u, cs);
                sa[m][u] = make_float2(t.x, t.y);
                sz[m][u] = make_float2(t.z, t.w);
            }
        }
    }
    const float2 m1 = make_float2(-1.f, -1.f);
    float accm = 0.f;
    // the thread's first G element of plane 0 (row ty; row ty + 8 is 8 Wp further on), and
    // the allocation's bound, read once
    const size_t goff = (size_t)(y0 + ty) * Wp + j;
    float* const gbase = v.Gp + goff;
    const long long gcap = v.gp_cap;
    (void)gcap;
    int oy, ox;
    half_offset(k0, rs, oy, ox);
    for (int k = k0; k < k1; ++k) {
        const int st = (k - k0) & 1;
        const unsigned par = (unsigned)((k - k0) >> 1) & 1u;
        if (!gave_up && !mbar_try_wait(&bars[st], par)) {
            if (*(volatile unsigned*)err != 0u || !mbar_wait_consumer(&bars[st], par, budget)) {
                gave_up = true;
                if (tid == 0) atomicOr(err, 1u);
            }
        }
        const WT* Kt = reinterpret_cast<const WT*>(smem + st * KST);
        const int fo = oy * FW + ox;
        float* const Gk = gbase + (size_t)k * plane;
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            const int row = ty + 8 * m;
            const float K = to_f32(Kt[row * 32 + tx]);
            const int cs = cs0 + 8 * m * FW, cr = cs + fo;
            // the iteration pairs' products in two independent chains (even and odd pairs)
            float2 acc0 = make_float2(0.f, 0.f), acc1 = make_float2(0.f, 0.f);
            if constexpr (NPK > 0) {
#pragma unroll
                for (int u = 0; u < NPK; ++u) {
                    const float4 r4 = AZ4(u, cr);
                    const float2 da = __ffma2_rn(make_float2(r4.x, r4.y), m1, sa[m][u]);  // a(s) - a(r)
                    const float2 dz = __ffma2_rn(sz[m][u], m1, make_float2(r4.z, r4.w));  // z(r) - z(s)
                    if (u & 1)
                        acc1 = __ffma2_rn(da, dz, acc1);
                    else
                        acc0 = __ffma2_rn(da, dz, acc0);
                }
            } else {
                for (int u = 0; u < np; ++u) {
                    const float4 s4 = AZ4(u, cs), r4 = AZ4(u, cr);
                    const float2 da = __ffma2_rn(make_float2(r4.x, r4.y), m1, make_float2(s4.x, s4.y));
                    const float2 dz = __ffma2_rn(make_float2(s4.z, s4.w), m1, make_float2(r4.z, r4.w));
                    if (u & 1)
                        acc1 = __ffma2_rn(da, dz, acc1);
                    else
                        acc0 = __ffma2_rn(da, dz, acc0);
                }
            }
            const float G = (acc0.x + acc0.y) + (acc1.x + acc1.y);
            if (in[m] && DSG_IN_RANGE(goff + (size_t)k * plane + (size_t)(8 * m) * Wp, gcap, kChkAdjPlanes))
                Gk[(size_t)(8 * m) * Wp] = G;
            const float dr = Sd[cr];
            const float GK = G * K;
            accd[m] = fmaf(GK, dr, accd[m]);
            accm = fmaf(GK * ds[m], dr, accm);
            Ac[cr] = fmaf(GK, ds[m], Ac[cr]);
        }
        __syncthreads();  // the stage read; the mirrored terms of this offset added
        if (tid == 0 && k + 2 < k1) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(k + 2, st);
        }
        if (++ox > rs) {
            ++oy;
            ox = -rs;
        }
    }
    const float inv_m = __ldg(v.m + 1);
    const double macc = block_sum_256(-accm * inv_m * inv_m, tid);
    if (tid == 0) v.m_part[(zc * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = macc;
#pragma unroll
    for (int m = 0; m < 2; ++m) Ac[cs0 + 8 * m * FW] += accd[m];
    __syncthreads();
    const size_t obase = (((size_t)zc * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x) * (size_t)fcells;
    if (DSG_IN_RANGE(obase + fcells - 1, v.dh0_cap, kChkAdjWindows))
        for (int idx = tid; idx < fcells; idx += 256) v.dh0[obase + idx] = Ac[idx];
}

// dh(s) = (1/m) dh0(s), dh0 gathered from the window partials of pair pass G (every
// chunk, and every tile whose window holds s, in a fixed order)
__global__ void __launch_bounds__(256) adj_dh_kernel(const TapeView* __restrict__ tv, int tiles_y, int tiles_x,
                                                     int chunks) {
    griddep_enter();
    const TapeView& v = tv[blockIdx.z];
    const int H = v.H, W = v.W;
    const int j = blockIdx.x * 32 + threadIdx.x;
    const int i = blockIdx.y * 8 + threadIdx.y;
    if (i >= H || j >= W) return;
    const float inv_m = __ldg(v.m + 1);
    v.dh[(size_t)i * W + j] = gather_ge(v.dh0, i, j, 0, v.rs, tiles_y, tiles_x, chunks, 32, v.dh0_cap) * inv_m;
}

// the scalar cotangents of every image (m, rho, h) in one array, read back in one copy
__global__ void adj_gather_scalars_kernel(const TapeView* __restrict__ tv, int count, double* __restrict__ out) {
    griddep_enter();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    for (int w = 0; w < 3; ++w) out[3 * i + w] = tv[i].mh[w];
}

int nblk(size_t n) { return (int)((n + 255) / 256); }

// f(std::integral_constant<int, R>{}) for the blur radius R = taps.r (0..8)
template <typename F>
cudaError_t by_blur_radius(int r, F&& f) {
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

size_t pairs_g_smem(int N, int rs, int dtype) {
    const int esz = dtype == DSGNLM_F32 ? 4 : 2;
    const int FH = kQH + rs, FW = 32 + 2 * rs;
    return 2 * (size_t)bd_stage_bytes(kQH, 32, esz) + (size_t)((N + 1) / 2) * bd_stage_bytes(FH, 4 * FW, 4) +
           sizeof(float) * 2 * (size_t)FH * FW;
}
size_t pairs_b_smem(int T, int rs) {
    return sizeof(float) * (size_t)(2 * T + 1) * (kAdjTH + rs) * (kAdjTW + 2 * rs);
}
// the fused pass B with the patch-distance adjoint: fields, guide, accumulator, D-hat and
// row sums; used for patch radii 1 to 3 while two blocks fit on an SM, otherwise pass B
// writes the D-hat planes and the box-and-gather kernel reads them
size_t pairs_bd_smem(int T, int rp, int rs, int dtype) {
    const int esz = dtype == DSGNLM_F32 ? 4 : 2;
    const int DH = kQH + 2 * rp, P = (T + 1) / 2;
    const size_t fcells = (size_t)bd_field_h(rp, rs) * bd_field_w(rs);
    return 2 * (size_t)bd_stage_bytes(DH, bd_box_w(esz), esz) + 2 * (size_t)bd_stage_bytes(DH, bd_box_w(4), 4) +
           sizeof(float) * 2 * (size_t)DH * 32 + sizeof(float2) * 2 * (size_t)P * fcells + sizeof(float) * fcells +
           sizeof(float) * 2 * (size_t)bg_win_h(rs) * bd_win_w(rp, rs);
}
constexpr size_t kBdSmemMax = 110 * 1024;
bool use_pairs_bd(int T, int rp, int rs, int dtype) {
    return rp >= 1 && rp <= 3 && pairs_bd_smem(T, rp, rs, dtype) <= kBdSmemMax;
}

}  // namespace

DSG_CHECK_WORD_ACCESSOR(check_word_adjoint)

}  // namespace dsg

using namespace dsg;

struct lpnp_tape {
    dsgnlm_t den = nullptr;
    int H = 0, W = 0, rp = 0, rs = 0, T = 0, N = 0, constraint = 2;
    float h = 0.f, alpha = 1.f, rho = 1.f, mu = 0.5f, c = 0.f;
    BlurTaps taps{};
    const float* y = nullptr;      // caller's observation (kept valid until the backward)
    const float* guide = nullptr;  // caller's guide
    int blur_r = 0;
    float blur_sigma = 1.f;
    DevBuf Dh, Th, X, V, U, Gr, AZ, AZ4, xh, vh, uh, g, gs, dh, dh0, base, thp, Dhat, Gp, m, mkey, sstar, mh,
        rho_part, h_part, m_part, scratch;
    // tables of a call this tape leads (the first image of the batch): per-image views,
    // phase-1 instance tables and work items in one device buffer, uploaded from one
    // pinned buffer; the scalar cotangents of all images and their pinned copy
    DevBuf tables, scal;
    unsigned char* stage = nullptr;
    size_t stage_bytes = 0;
    double* hs = nullptr;  // pinned [count][3] + the handle's error word after it
    int hs_count = 0;
    cudaEvent_t staged = nullptr;  // the upload from `stage` has been read
    cudaEvent_t ev = nullptr;      // fork and join of the images' handle streams
    // tensor maps of the fused pass B (the handle's weight planes and this tape's G
    // planes), encoded again when the planes, sizes or type change
    alignas(64) unsigned char bd_kmap[128], bd_gmap[128];
    const void* bd_kbase = nullptr;
    const void* bd_gbase = nullptr;
    int bd_key[5] = {0, 0, 0, 0, 0};
    alignas(64) unsigned char gt_kmap[128];  // the weight planes for pair pass G
    const void* gt_kbase = nullptr;
    int gt_key[4] = {0, 0, 0, 0};
    alignas(64) unsigned char gt_amap[128];  // the interleaved (a, z) copy for pair pass G
    const void* gt_abase = nullptr;
    int gt_akey[4] = {0, 0, 0, 0};
    // the launch sequences of the forward (after the weight builds) and of the backward,
    // recorded as CUDA graphs by the call this tape leads, and the keys they were recorded for
    cudaGraphExec_t fwd_exec = nullptr, bwd_exec = nullptr;
    // the side stream of the steps that run beside the weight streams, the events that
    // fork and join it, and the stream the launch sequences are recorded on
    cudaStream_t side = nullptr, cap = nullptr;
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    std::vector<uint64_t> fwd_key, bwd_key;
    uint64_t fwd_launches = 0, bwd_launches = 0;
};

namespace {

dsgnlm_status tape_ck(cudaError_t e) {
    if (e == cudaSuccess) return DSGNLM_OK;
    record_cuda_error(e);
    return e == cudaErrorMemoryAllocation ? DSGNLM_ENOMEM : DSGNLM_ECUDA;
}

#define TAPE_CK(expr)                                   \
    do {                                                \
        dsgnlm_status s_ = tape_ck(expr);               \
        if (s_ != DSGNLM_OK) return s_;                 \
    } while (0)

#define PDL_CK(expr)                     \
    do {                                 \
        cudaError_t e_ = (expr);         \
        if (e_ != cudaSuccess) return e_; \
    } while (0)

// every launch of this file: programmatic stream serialization (launch.h); every kernel
// of this file waits for its predecessors (griddep_enter) before it touches memory
template <typename... KArgs, typename... Args>
cudaError_t pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args... args) {
    return launch_pdl(kern, grid, block, smem, st, args...);
}

cudaError_t ensure_event(cudaEvent_t& e) {
    return e ? cudaSuccess : cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
}

// Queue `seq` (a function of the stream that queues a fixed launch sequence and returns a
// status) on `st` through a CUDA graph: replayed when `key` equals the key the graph was
// recorded for, recorded anew otherwise.  The recording runs on `cap`, a stream of the
// tape's own (the caller's stream may be the legacy default stream, which cannot record);
// the graph is then launched on `st`.  The graph keeps the programmatic launch edges,
// and its replay takes one launch from the host and shorter gaps between the kernels.
// Every kernel parameter of the sequence must be a function of the key: the per-call
// pointers live in the tables in device memory, uploaded before the replay.  If the
// recording fails, the sequence is queued directly.
template <typename F>
dsgnlm_status run_recorded(cudaGraphExec_t& exec, std::vector<uint64_t>& rec_key, uint64_t& rec_launches,
                           const std::vector<uint64_t>& key, cudaStream_t st, cudaStream_t cap, F&& seq) {
    if (exec && rec_key == key) {
        TAPE_CK(cudaGraphLaunch(exec, st));
        count_launches(rec_launches);
        return DSGNLM_OK;
    }
    if (exec) {
        cudaGraphExecDestroy(exec);
        exec = nullptr;
    }
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return seq(st);
    }
    set_capture_counting(true);
    const dsgnlm_status s = seq(cap);
    set_capture_counting(false);
    const uint64_t n = recorded_launches();
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cap, &g);
    if (e == cudaSuccess && s == DSGNLM_OK) e = cudaGraphInstantiate(&exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess || s != DSGNLM_OK) {
        exec = nullptr;
        (void)cudaGetLastError();
        if (s != DSGNLM_OK) return s;
        return seq(st);
    }
    rec_key = key;
    rec_launches = n;
    TAPE_CK(cudaGraphLaunch(exec, st));
    count_launches(n);
    return DSGNLM_OK;
}

// The view of image i (the caller's pointers of the current call included).
TapeView make_view(const lpnp_tape* tp, const float* x_out, const float* x_bar, float* y_bar, float* guide_bar) {
    const dsgnlm* den = tp->den;
    TapeView v{};
    v.H = tp->H;
    v.W = tp->W;
    v.rp = tp->rp;
    v.rs = tp->rs;
    v.T = tp->T;
    v.N = tp->N;
    v.constraint = tp->constraint;
    v.mu = tp->mu;
    v.alpha = tp->alpha;
    v.rho = tp->rho;
    v.c = tp->c;
    v.hfac = 2.f * tp->c / tp->h;
    v.taps = tp->taps;
    v.cv = Cover{den->plan.partials, den->plan.tiles_x, den->plan.tiles_y, den->plan.splits.n, tp->rs,
                 den->plan.part_cap};
    v.planes = den->planes.p;
    v.y = tp->y;
    v.guide = tp->guide;
    v.X = tp->X.as<float>();
    v.V = tp->V.as<float>();
    v.U = tp->U.as<float>();
    v.Gr = tp->Gr.as<float>();
    v.Dh = tp->Dh.as<float>();
    v.Th = tp->Th.as<float>();
    v.scratch = tp->scratch.as<float>();
    v.z = den->z.as<float>();
    v.cpart = den->partials.as<double>();
    v.m = tp->m.as<float>();
    v.mkey = tp->mkey.as<unsigned long long>();
    v.sstar = tp->sstar.as<int>();
    v.xh = tp->xh.as<float>();
    v.vh = tp->vh.as<float>();
    v.uh = tp->uh.as<float>();
    v.g = tp->g.as<float>();
    v.gs = tp->gs.as<float>();
    v.dh = tp->dh.as<float>();
    v.dh0 = tp->dh0.as<float>();
    v.base = tp->base.as<float>();
    v.thp = tp->thp.as<float>();
    v.Dhat = tp->Dhat.as<float>();
    v.Gp = tp->Gp.as<float>();
    v.AZ = tp->AZ.as<float>();
    v.AZ4 = tp->AZ4.as<float>();
    v.mh = tp->mh.as<double>();
    v.rho_part = tp->rho_part.as<double>();
    v.h_part = tp->h_part.as<double>();
    v.m_part = tp->m_part.as<double>();
    v.x_out = const_cast<float*>(x_out);
    v.x_bar = x_bar;
    v.y_bar = y_bar;
    v.guide_bar = guide_bar;
    return v;
}

// The phase-1 instance of image i for one stencil pass over q = d (z null) or d z.
BatchInst p1_inst(const dsgnlm* den, const float* d, const float* z) {
    BatchInst b{};
    b.H = den->H;
    b.W = den->W;
    b.tiles_x = den->plan.tiles_x;
    b.tiles_y = den->plan.tiles_y;
    b.splits = den->plan.splits;
    b.d = d;
    b.z = z;
    b.part = den->plan.partials;
    b.part_cap = den->plan.part_cap;
    b.done = nullptr;
    return b;
}

constexpr size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// The tables of one call of a batch: views, phase-1 instance tables (`passes` passes,
// each `count` instances) and the phase-1 work items of all images, uploaded in one
// copy on `st`.  Pointers into the device buffer are returned.
struct Tables {
    const TapeView* views;
    const BatchInst* insts;
    const int4* work;
    int nwork;
    const BuildJob* jobs;  // the forward's weight builds (null for the backward)
};

dsgnlm_status upload_tables(lpnp_tape* lead, dsgnlm* const* dens, int count, const std::vector<TapeView>& views,
                            const std::vector<BatchInst>& insts, cudaStream_t st, Tables& out,
                            const std::vector<BuildJob>* jobs = nullptr) {
    std::vector<int4> work;
    for (int i = 0; i < count; ++i) {
        const TmaPlan& pl = dens[i]->plan;
        for (int sl = 0; sl < pl.splits.n; ++sl)
            for (int ty = 0; ty < pl.tiles_y; ++ty)
                for (int tx = 0; tx < pl.tiles_x; ++tx) work.push_back(make_int4(i, ty, tx, sl));
    }
    const size_t bv = align256(sizeof(TapeView) * views.size());
    const size_t bi = align256(sizeof(BatchInst) * insts.size());
    const size_t bw = align256(sizeof(int4) * work.size());
    const size_t bj = jobs ? align256(sizeof(BuildJob) * jobs->size()) : 0;
    const size_t total = bv + bi + bw + bj;
    TAPE_CK(lead->tables.ensure(total));
    TAPE_CK(ensure_event(lead->staged));
    // the previous upload from the staging buffer must have been read before it is rewritten
    TAPE_CK(cudaEventSynchronize(lead->staged));
    if (lead->stage_bytes < total) {
        if (lead->stage) cudaFreeHost(lead->stage);
        lead->stage = nullptr;
        lead->stage_bytes = 0;
        TAPE_CK(cudaMallocHost((void**)&lead->stage, total));
        lead->stage_bytes = total;
    }
    std::memcpy(lead->stage, views.data(), sizeof(TapeView) * views.size());
    std::memcpy(lead->stage + bv, insts.data(), sizeof(BatchInst) * insts.size());
    std::memcpy(lead->stage + bv + bi, work.data(), sizeof(int4) * work.size());
    if (jobs) std::memcpy(lead->stage + bv + bi + bw, jobs->data(), sizeof(BuildJob) * jobs->size());
    TAPE_CK(cudaMemcpyAsync(lead->tables.p, lead->stage, total, cudaMemcpyHostToDevice, st));
    TAPE_CK(cudaEventRecord(lead->staged, st));
    unsigned char* base = static_cast<unsigned char*>(lead->tables.p);
    out.views = reinterpret_cast<const TapeView*>(base);
    out.insts = reinterpret_cast<const BatchInst*>(base + bv);
    out.work = reinterpret_cast<const int4*>(base + bv + bi);
    out.nwork = (int)work.size();
    out.jobs = jobs ? reinterpret_cast<const BuildJob*>(base + bv + bi + bw) : nullptr;
    return DSGNLM_OK;
}

BatchMaps batch_maps(dsgnlm* const* dens, int count) {
    BatchMaps maps;
    for (int i = 0; i < count; ++i) std::memcpy(maps.m[i], dens[i]->plan.tmap, 128);
    return maps;
}

// The lead tape's side stream and the events that fork work onto it and join it back
// (created before any recording)
dsgnlm_status ensure_side(lpnp_tape* lead) {
    if (!lead->side) TAPE_CK(cudaStreamCreateWithFlags(&lead->side, cudaStreamNonBlocking));
    if (!lead->cap) TAPE_CK(cudaStreamCreateWithFlags(&lead->cap, cudaStreamNonBlocking));
    TAPE_CK(ensure_event(lead->fork_ev));
    TAPE_CK(ensure_event(lead->join_ev));
    return DSGNLM_OK;
}

// The other images' handle streams wait for the work queued on `st` (so that work the
// caller queues on them afterwards follows the batch).
dsgnlm_status join_streams(lpnp_tape* lead, dsgnlm* const* dens, int count, cudaStream_t st) {
    TAPE_CK(ensure_event(lead->ev));
    TAPE_CK(cudaEventRecord(lead->ev, st));
    for (int i = 1; i < count; ++i)
        if (dens[i]->stream != st) TAPE_CK(cudaStreamWaitEvent(dens[i]->stream, lead->ev, 0));
    return DSGNLM_OK;
}

// The recorded forward of `count` images in lockstep on the first handle's stream: the
// weights of every image (each on its handle's stream, joined into the first), the T
// balancing passes with every d^p and t^p kept, m with its first maximiser and 1/m on
// the device, and N iterations of Algorithm 1, every state recorded.  Nothing waits for
// the device.
dsgnlm_status lock_forward(lpnp_tape* const* tapes, dsgnlm* const* dens, int count, const float* const* y,
                           const float* const* guide, int H, int W, int patch_r, int search_r, float bandwidth,
                           int balance_passes, float alpha, float rho, int iters, float blur_sigma, int blur_r,
                           float* const* x_out) {
    if (H < 2 || W < 2 || (H & 1) || (W & 1) || iters < 1 || iters > 256 || balance_passes < 0 ||
        balance_passes > 64 || !(rho > 0.f) || !(alpha >= 0.f) || blur_r < 0 || blur_r > 8 || !(blur_sigma > 0.f))
        return DSGNLM_EINVAL;
    if (!tma_path_supports(search_r) || count > kMaxBatch) return DSGNLM_EINVAL;
    // shared memory of the pair passes of the backward (fields over a tile + halo)
    if (pairs_g_smem(iters, search_r, DSGNLM_F32) > 220 * 1024 || pairs_b_smem(balance_passes, search_r) > 220 * 1024)
        return DSGNLM_EINVAL;
    lpnp_tape* lead = tapes[0];
    cudaStream_t st = dens[0]->stream;
    const size_t n = (size_t)H * W;
    const int T = balance_passes, N = iters;
    // 1. every image's planes and phase-1 plan, the offset split of each sized for the
    // batch; the weights themselves are built by one batched launch in the recorded
    // sequence below.  Work queued on the other handles' streams comes first.
    for (int i = 0; i < count; ++i) {
        dens[i]->share = count;
        dsgnlm_status s = build_handle(dens[i], guide[i], H, W, patch_r, search_r, bandwidth, false);
        dens[i]->share = 1;
        if (s != DSGNLM_OK) return s;
        if (!dens[i]->fast || dens[i]->dtype != dens[0]->dtype) return DSGNLM_EINVAL;
        if (i > 0 && dens[i]->stream != st) {
            TAPE_CK(ensure_event(tapes[i]->ev));
            TAPE_CK(cudaEventRecord(tapes[i]->ev, dens[i]->stream));
            TAPE_CK(cudaStreamWaitEvent(st, tapes[i]->ev, 0));
        }
    }
    // 2. each tape's sizes, scalars and buffers
    const double np = 2.0 * patch_r + 1.0;
    for (int i = 0; i < count; ++i) {
        lpnp_tape* tp = tapes[i];
        dsgnlm* den = dens[i];
        tp->den = den;
        tp->H = H;
        tp->W = W;
        tp->rp = patch_r;
        tp->rs = search_r;
        tp->T = T;
        tp->N = N;
        tp->h = bandwidth;
        tp->alpha = alpha;
        tp->rho = rho;
        tp->mu = (float)(1.0 / ((double)alpha + (double)rho));
        tp->c = (float)(1.0 / (2.0 * np * np * (double)bandwidth * (double)bandwidth));
        tp->taps = make_blur_taps(blur_sigma, blur_r);
        tp->blur_sigma = blur_sigma;
        tp->blur_r = blur_r;
        tp->y = y[i];
        tp->guide = guide[i];
        TAPE_CK(tp->Dh.ensure(sizeof(float) * n * (T + 1)));
        TAPE_CK(tp->Th.ensure(sizeof(float) * n * (T + 1)));
        TAPE_CK(tp->X.ensure(sizeof(float) * n * (N + 1)));
        TAPE_CK(tp->V.ensure(sizeof(float) * n * (N + 1)));
        TAPE_CK(tp->U.ensure(sizeof(float) * n * (N + 1)));
        TAPE_CK(tp->Gr.ensure(sizeof(float) * n * N));
        TAPE_CK(tp->scratch.ensure(sizeof(float) * n));
        TAPE_CK(tp->m.ensure(2 * sizeof(float)));  // m and 1/m
        TAPE_CK(tp->sstar.ensure(sizeof(int)));
        TAPE_CK(tp->mkey.ensure(sizeof(unsigned long long)));
        TAPE_CK(den->partials.ensure(sizeof(double) * 2 * (size_t)combine_xupdate_blocks(H, W)));
        TAPE_CK(den->z.ensure(sizeof(float) * n));
    }
    // 3. the tables: views; phase-1 passes 0..T of the balance (q = d^p), then W z
    std::vector<TapeView> views(count);
    std::vector<BatchInst> insts((size_t)(T + 2) * count);
    for (int i = 0; i < count; ++i) {
        views[i] = make_view(tapes[i], x_out[i], nullptr, nullptr, nullptr);
        for (int p = 0; p <= T; ++p)
            insts[(size_t)p * count + i] = p1_inst(dens[i], tapes[i]->Dh.as<float>() + (size_t)p * n, nullptr);
        insts[(size_t)(T + 1) * count + i] =
            p1_inst(dens[i], tapes[i]->Dh.as<float>() + (size_t)T * n, dens[i]->z.as<float>());
    }
    std::vector<BuildJob> jobs(count);
    const float build_c2 = (float)((double)lead->c * 1.4426950408889634);  // c log2 e
    for (int i = 0; i < count; ++i)
        jobs[i] = BuildJob{guide[i], dens[i]->planes.p,
                           (long long)(dens[i]->planes.bytes / weight_elem_bytes(dens[i]->dtype)), build_c2};
    Tables tb{};
    dsgnlm_status s = upload_tables(lead, dens, count, views, insts, st, tb, &jobs);
    if (s != DSGNLM_OK) return s;
    s = ensure_side(lead);
    if (s != DSGNLM_OK) return s;
    const BatchMaps maps = batch_maps(dens, count);
    unsigned* err = dens[0]->err.as<unsigned>();
    const int dtype = dens[0]->dtype;
    const dim3 eg((W + kXW - 1) / kXW, (H + kXH - 1) / kXH, count);  // per-pixel epilogue blocks
    const dim3 ng(std::min(nblk(n), 1024), 1, count);
    // 4. the work, one launch per step over all images, recorded once per configuration
    // as a CUDA graph and replayed
    const dim3 gg((W + kGT - 1) / kGT, (H + kGT - 1) / kGT, count);
    const BlurTaps taps = make_blur_taps(blur_sigma, blur_r);
    auto seq = [&](cudaStream_t st) -> dsgnlm_status {
        // on the side stream, beside the weight build and the balance (which do not depend
        // on x): x = v = clip(guide), u = 0, and the x-step of iteration 0 with its
        // recorded gradient
        TAPE_CK(cudaEventRecord(lead->fork_ev, st));
        TAPE_CK(cudaStreamWaitEvent(lead->side, lead->fork_ev, 0));
        TAPE_CK(pdl(adj_init_kernel, dim3(nblk(n), 1, count), dim3(256), 0, lead->side, tb.views));
        TAPE_CK(by_blur_radius(taps.r, [&](auto rc) {
            return pdl(adj_fwd_xupdate_kernel<decltype(rc)::value>, gg, dim3(256), 0, lead->side, tb.views, 0);
        }));
        TAPE_CK(cudaEventRecord(lead->join_ev, lead->side));
        // the weights of every image (Eq. NLM, Eq. S1), one launch
        TAPE_CK(launch_build_batched(dtype, tb.jobs, count, H, W, patch_r, search_r, lead->c, st));
        TAPE_CK(pdl(adj_prep_kernel, dim3(ng), dim3(256), 0, st, tb.views));
        count_launches(3);
        TAPE_CK(cudaGetLastError());
        for (int p = 0; p <= T; ++p) {
            TAPE_CK(launch_tma_gather_batched(dtype, search_r, maps, tb.insts + (size_t)p * count, tb.work,
                                              tb.nwork, err, st));
            TAPE_CK(pdl(adj_balance_kernel, dim3(eg), dim3(32, 8), 0, st, tb.views, p));
            count_launches(1);
            TAPE_CK(cudaGetLastError());
        }
        TAPE_CK(pdl(adj_m_key_kernel, dim3(ng), dim3(256), 0, st, tb.views));
        TAPE_CK(pdl(adj_m_finish_kernel, dim3((count + 63) / 64), dim3(64), 0, st, tb.views, count));
        count_launches(2);
        TAPE_CK(cudaGetLastError());
        TAPE_CK(cudaStreamWaitEvent(st, lead->join_ev, 0));
        // iteration k: the weight stream of z_k and, beside it on the side stream, the
        // gradient of x_{k+1}; then the dual step of k with the x-step of k + 1
        for (int k = 0; k < N; ++k) {
            const int do_x = k + 1 < N;
            if (do_x) {
                TAPE_CK(cudaEventRecord(lead->fork_ev, st));
                TAPE_CK(cudaStreamWaitEvent(lead->side, lead->fork_ev, 0));
                TAPE_CK(by_blur_radius(taps.r, [&](auto rc) {
                    return pdl(adj_fwd_grad_kernel<decltype(rc)::value>, gg, dim3(256), 0, lead->side, tb.views,
                               k + 1);
                }));
                TAPE_CK(cudaEventRecord(lead->join_ev, lead->side));
                count_launches(1);
            }
            TAPE_CK(launch_tma_gather_batched(dtype, search_r, maps, tb.insts + (size_t)(T + 1) * count, tb.work,
                                              tb.nwork, err, st));
            if (do_x) TAPE_CK(cudaStreamWaitEvent(st, lead->join_ev, 0));
            TAPE_CK(pdl(adj_fwd_dual_x_kernel, eg, dim3(32, 8), 0, st, tb.views, k, do_x));
            count_launches(1);
        }
        TAPE_CK(pdl(adj_xout_kernel, dim3(nblk(n), 1, count), dim3(256), 0, st, tb.views));
        count_launches(1);
        TAPE_CK(cudaGetLastError());
        return DSGNLM_OK;
    };
    std::vector<uint64_t> key = {(uint64_t)count,  (uint64_t)H,      (uint64_t)W, (uint64_t)patch_r,
                                 (uint64_t)search_r, (uint64_t)T,    (uint64_t)N, (uint64_t)dtype,
                                 (uint64_t)taps.r,   (uint64_t)(uintptr_t)tb.views, (uint64_t)tb.nwork,
                                 (uint64_t)(uintptr_t)err};
    for (int i = 0; i < count; ++i) {
        key.push_back((uint64_t)(uintptr_t)dens[i]->planes.p);
        key.push_back((uint64_t)dens[i]->plan.splits.n);
    }
    s = run_recorded(lead->fwd_exec, lead->fwd_key, lead->fwd_launches, key, st, lead->cap, seq);
    if (s != DSGNLM_OK) return s;
    // 5. every handle holds its image's W; its m and 1/m stay on the device until a
    // host-side use of the handle reads them back
    for (int i = 0; i < count; ++i) {
        dsgnlm* den = dens[i];
        den->d_final = tapes[i]->Dh.as<float>() + (size_t)T * n;
        den->t_final = tapes[i]->Th.as<float>() + (size_t)T * n;
        den->iters = T;
        den->balanced = true;
        den->inv_m_dev = false;  // the balance control block does not hold this W's 1/m
        den->m_pending = tapes[i]->m.as<float>();
    }
    return join_streams(lead, dens, count, st);
}

// The reverse sweep of `count` recorded images in lockstep on the first tape's handle
// stream, then one read-back of every image's scalar cotangents and of the wait-error
// word.
dsgnlm_status lock_backward(lpnp_tape* const* tapes, int count, const float* const* x_bar, float* const* y_bar,
                            float* const* guide_bar, double* h_bar, double* rho_bar) {
    lpnp_tape* lead = tapes[0];
    if (count > kMaxBatch || !lead->den) return DSGNLM_EINVAL;
    const int H = lead->H, W = lead->W, N = lead->N, T = lead->T, rs = lead->rs, rp = lead->rp;
    std::vector<dsgnlm*> dens(count);
    for (int i = 0; i < count; ++i) {
        const lpnp_tape* tp = tapes[i];
        dsgnlm* den = tp->den;
        if (!den || !tp->X.p) return DSGNLM_EINVAL;  // no recording
        if (tp->H != H || tp->W != W || tp->N != N || tp->T != T || tp->rs != rs || tp->rp != rp ||
            tp->taps.r != lead->taps.r || den->dtype != lead->den->dtype)
            return DSGNLM_EINVAL;
        // the handle's planes must still hold this tape's K1
        if (den->H != H || den->W != W || den->rs != rs || den->nh != num_half_offsets(rs)) return DSGNLM_EINVAL;
        dens[i] = den;
    }
    cudaStream_t st = dens[0]->stream;
    const size_t n = (size_t)H * W;
    const int nh = num_half_offsets(rs);
    const dim3 pgrid2((W + 31) / 32, (H + 7) / 8, count);  // per-pixel passes in 32 x 8 blocks
    const dim3 wgrid((W + 31) / 32, (H + 15) / 16, count);  // the W a finish: 16 x 32 pixels per block
    const int nrb = (int)(wgrid.x * wgrid.y);                // its blocks' rho partials
    const int pgx = (W + kAdjTW - 1) / kAdjTW, pgy = (H + kAdjTH - 1) / kAdjTH;  // tiles of pair passes G and B
    const int npb = pgx * pgy * kPairSplit;  // pair-pass blocks (with the offset chunks)
    // patch-distance adjoint: tiles of the extended grid, the half offsets in kPairSplit
    // chunks (a number that does not depend on the batch, so that an image's sums have
    // the same order alone and in a batch)
    const bool fused = use_pairs_bd(T, rp, rs, lead->den->dtype);
    const int bg_qw = fused ? bd_qw(rp) : kQW;  // tile width (the fused pass: the window 32 wide)
    const int bg_ty = (H + 2 * rp + kQH - 1) / kQH, bg_tx = (W + 2 * rp + bg_qw - 1) / bg_qw;
    const int bg_chunks = std::min(kPairSplit, nh);
    const size_t bg_part = (size_t)bg_chunks * bg_ty * bg_tx * bg_win_h(rs) * (bg_qw + 2 * rs);
    const int nbd = bg_tx * bg_ty * bg_chunks;  // blocks of the fused pass (with the offset chunks)
    const int nhb = fused ? nbd : npb;         // blocks that write dL/dh partials
    for (int i = 0; i < count; ++i) {
        lpnp_tape* tp = tapes[i];
        DevBuf* nbufs[] = {&tp->xh, &tp->vh, &tp->uh, &tp->g, &tp->gs, &tp->dh, &tp->base};
        for (DevBuf* b : nbufs) TAPE_CK(b->ensure(sizeof(float) * n));
        TAPE_CK(tp->AZ.ensure(sizeof(float) * n * N));
        TAPE_CK(tp->AZ4.ensure(sizeof(float4) * n * ((N + 1) / 2)));
        TAPE_CK(tp->thp.ensure(sizeof(float) * n * (T > 0 ? T : 1)));
        // window partials of pair pass G (the forward and mirrored sums of dh0)
        TAPE_CK(tp->dh0.ensure(sizeof(float) * (size_t)kPairSplit * pgx * pgy * (kQH + rs) * (32 + 2 * rs)));
        // fused: the partials of the patch-distance adjoint in the D-hat memory (no D-hat
        // planes); otherwise the D-hat planes, and the partials in the G memory once pass
        // B has read G
        TAPE_CK(tp->Dhat.ensure(sizeof(float) * (fused ? bg_part : (size_t)nh * H * plane_pitch(W))));
        TAPE_CK(tp->Gp.ensure(sizeof(float) * std::max((size_t)nh * H * plane_pitch(W), fused ? 0 : bg_part)));
        TAPE_CK(tp->rho_part.ensure(sizeof(double) * nrb));
        TAPE_CK(tp->h_part.ensure(sizeof(double) * std::max(npb, nhb)));
        TAPE_CK(tp->m_part.ensure(sizeof(double) * npb));
        TAPE_CK(tp->mh.ensure(sizeof(double) * 3));
    }
    // tables: views; phase-1 passes W a_k (k = 0..N-1), then K1 th^p (p = 0..T-1)
    std::vector<TapeView> views(count);
    std::vector<BatchInst> insts((size_t)(N + T) * count);
    for (int i = 0; i < count; ++i) {
        lpnp_tape* tp = tapes[i];
        views[i] = make_view(tp, nullptr, x_bar[i], y_bar[i], guide_bar[i]);
        views[i].gpart = fused ? tp->Dhat.as<float>() : tp->Gp.as<float>();
        views[i].gp_cap = (long long)(tp->Gp.bytes / sizeof(float));
        views[i].dh0_cap = (long long)(tp->dh0.bytes / sizeof(float));
        views[i].gpart_cap = (long long)((fused ? tp->Dhat.bytes : tp->Gp.bytes) / sizeof(float));
        {
            const int dt = dens[i]->dtype;
            const int key[4] = {H, W, nh, dt};
            if (tp->gt_kbase != dens[i]->planes.p || std::memcmp(key, tp->gt_key, sizeof key) != 0) {
                TAPE_CK(encode_tile_map(tp->gt_kmap, dens[i]->planes.p, dt, H, W, nh, 32, kQH));
                tp->gt_kbase = dens[i]->planes.p;
                std::memcpy(tp->gt_key, key, sizeof key);
            }
            std::memcpy(views[i].gt_kmap, tp->gt_kmap, 128);
            // the (a, z) copy as FP32 rows of 4 W values, boxes of the pass's windows
            const int np = (N + 1) / 2;
            const int akey[4] = {H, W, np, rs};
            if (tp->gt_abase != tp->AZ4.p || std::memcmp(akey, tp->gt_akey, sizeof akey) != 0) {
                TAPE_CK(encode_tile_map(tp->gt_amap, tp->AZ4.p, DSGNLM_F32, H, 4 * W, np, 4 * (32 + 2 * rs), kQH + rs,
                                        4 * W));
                tp->gt_abase = tp->AZ4.p;
                std::memcpy(tp->gt_akey, akey, sizeof akey);
            }
            std::memcpy(views[i].gt_amap, tp->gt_amap, 128);
        }
        if (fused) {
            const int dt = dens[i]->dtype;
            const int key[5] = {H, W, nh, dt, rp};
            if (tp->bd_kbase != dens[i]->planes.p || tp->bd_gbase != tp->Gp.p ||
                std::memcmp(key, tp->bd_key, sizeof key) != 0) {
                const int esz = dt == DSGNLM_F32 ? 4 : 2;
                TAPE_CK(encode_tile_map(tp->bd_kmap, dens[i]->planes.p, dt, H, W, nh, bd_box_w(esz), kQH + 2 * rp));
                TAPE_CK(encode_tile_map(tp->bd_gmap, tp->Gp.p, DSGNLM_F32, H, W, nh, bd_box_w(4), kQH + 2 * rp));
                tp->bd_kbase = dens[i]->planes.p;
                tp->bd_gbase = tp->Gp.p;
                std::memcpy(tp->bd_key, key, sizeof key);
            }
            std::memcpy(views[i].bd_kmap, tp->bd_kmap, 128);
            std::memcpy(views[i].bd_gmap, tp->bd_gmap, 128);
        }
        const float* dT = tp->Dh.as<float>() + (size_t)T * n;
        for (int k = 0; k < N; ++k)
            insts[(size_t)k * count + i] = p1_inst(dens[i], dT, tp->AZ.as<float>() + (size_t)k * n);
        for (int p = 0; p < T; ++p)
            insts[(size_t)(N + p) * count + i] = p1_inst(dens[i], tp->thp.as<float>() + (size_t)p * n, nullptr);
    }
    Tables tb{};
    dsgnlm_status s = upload_tables(lead, dens.data(), count, views, insts, st, tb);
    if (s != DSGNLM_OK) return s;
    const BatchMaps maps = batch_maps(dens.data(), count);
    unsigned* err = dens[0]->err.as<unsigned>();
    const int dtype = dens[0]->dtype;
    const dim3 gg((W + kGT - 1) / kGT, (H + kGT - 1) / kGT, count);  // A^T A tiles
    const dim3 ng(nblk(n), 1, count);
    // the side stream and its events, and the scalar cotangents' device and pinned host
    // buffers (before any recording)
    {
        const dsgnlm_status ss = ensure_side(lead);
        if (ss != DSGNLM_OK) return ss;
    }
    TAPE_CK(lead->scal.ensure(sizeof(double) * 3 * (size_t)count));
    if (lead->hs_count < count) {
        if (lead->hs) cudaFreeHost(lead->hs);
        lead->hs = nullptr;
        lead->hs_count = 0;
        TAPE_CK(cudaMallocHost((void**)&lead->hs, sizeof(double) * (3 * (size_t)count + 1)));
        lead->hs_count = count;
    }
    unsigned* err_host = reinterpret_cast<unsigned*>(lead->hs + 3 * (size_t)count);
    // the reverse sweep, the pair passes, the balance and the guide, and the read-back of
    // every image's (m, rho, h) cotangents with the wait-error word: recorded once per
    // configuration as a CUDA graph and replayed
    auto seq = [&](cudaStream_t st) -> dsgnlm_status {
        TAPE_CK(pdl(adj_bwd_prep_kernel, dim3(ng), dim3(256), 0, st, tb.views, nrb));
        count_launches(1);
        TAPE_CK(cudaGetLastError());
        // iteration k: W a_k (W symmetric; no weight stream in the last iteration, where
        // a = vh - uh = 0) finished with g and the per-pixel cotangent updates, which also
        // form a_{k-1}; then the weight stream of a_{k-1} on this stream and, beside it on
        // the side stream, xh = mu (alpha g - A^T A g) (the only step with neighbours)
        auto ata = [&](cudaStream_t s2) {
            return by_blur_radius(lead->taps.r, [&](auto rc) {
                return pdl(adj_ata_update_kernel<decltype(rc)::value>, gg, dim3(256), 0, s2, tb.views, 0);
            });
        };
        for (int k = N - 1; k >= 0; --k) {
            const int a_zero = k == N - 1;
            TAPE_CK(pdl(adj_wa_g_kernel, wgrid, dim3(32, 8), 0, st, tb.views, k, a_zero));
            count_launches(2);
            if (k > 0) {
                TAPE_CK(cudaEventRecord(lead->fork_ev, st));
                TAPE_CK(cudaStreamWaitEvent(lead->side, lead->fork_ev, 0));
                TAPE_CK(ata(lead->side));
                TAPE_CK(cudaEventRecord(lead->join_ev, lead->side));
                TAPE_CK(launch_tma_gather_batched(dtype, rs, maps, tb.insts + (size_t)(k - 1) * count, tb.work,
                                                  tb.nwork, err, st));
                TAPE_CK(cudaStreamWaitEvent(st, lead->join_ev, 0));
            } else {
                TAPE_CK(ata(st));
            }
        }
        // pair pass G with the mirrored terms, the gather of dh, then the cotangent of m and
        // its terms
        auto pairs_gt = [&](auto wt) -> cudaError_t {
            using WT = decltype(wt);
            const size_t smem = pairs_g_smem(N, rs, dtype);
            const dim3 grid(pgx, pgy, kPairSplit * count);
            auto run = [&](auto kern) -> cudaError_t {
                cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                if (e != cudaSuccess) return e;
                return pdl(kern, grid, dim3(32, 8), smem, st, tb.views, kPairSplit, err, kDefaultWaitBudget);
            };
            cudaError_t e;
            switch ((N + 1) / 2) {
                case 1: e = run(adj_pairs_gt_kernel<WT, 1>); break;
                case 2: e = run(adj_pairs_gt_kernel<WT, 2>); break;
                case 3: e = run(adj_pairs_gt_kernel<WT, 3>); break;
                case 4: e = run(adj_pairs_gt_kernel<WT, 4>); break;
                case 5: e = run(adj_pairs_gt_kernel<WT, 5>); break;
                case 6: e = run(adj_pairs_gt_kernel<WT, 6>); break;
                case 7: e = run(adj_pairs_gt_kernel<WT, 7>); break;
                case 8: e = run(adj_pairs_gt_kernel<WT, 8>); break;
                default: e = run(adj_pairs_gt_kernel<WT, 0>); break;
            }
            count_launches(1);
            if (e != cudaSuccess) return e;
            {
                const int elems = pgx * pgy * (kQH + rs) * (32 + 2 * rs);
                PDL_CK(pdl(adj_chunk_sum_kernel, dim3((elems + 255) / 256, 1, count), dim3(256), 0, st,
                    tb.views, 1, elems,
                           kPairSplit));
            }
            PDL_CK(pdl(adj_dh_kernel, pgrid2, dim3(32, 8), 0, st, tb.views, pgy, pgx, 1));
            count_launches(1);
            PDL_CK(pdl(adj_sum_kernel, dim3(count), dim3(256), 0, st, tb.views, 0, npb, nrb));
            PDL_CK(pdl(adj_mterms_kernel<WT>, dim3(count), dim3(256), 0, st, tb.views));
            count_launches(3);
            return cudaGetLastError();
        };
        auto pairs_b = [&](auto wt) -> cudaError_t {
            using WT = decltype(wt);
            const size_t smem = pairs_b_smem(T, rs);
            cudaError_t e =
                cudaFuncSetAttribute(adj_pairs_b_kernel<WT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            PDL_CK(pdl(adj_pairs_b_kernel<WT>, dim3(pgx, pgy, kPairSplit * count), dim3(32, 8), smem, st, tb.views));
            count_launches(1);
            return cudaGetLastError();
        };
        switch (dtype) {
            case DSGNLM_F32: TAPE_CK(pairs_gt(float{})); break;
            case DSGNLM_F16: TAPE_CK(pairs_gt(__half{})); break;
            default: TAPE_CK(pairs_gt(__nv_bfloat16{})); break;
        }
        // balancing passes backwards: th^p from the cotangent of d^{p+1}, then K1 th^p; the
        // finish of pass p forms the cotangent of d^p and at once th^{p-1} of the next pass
        // (the cotangent of d^0 = 1 is not needed, so K1 th^0 is not streamed and pass 0 has
        // no finish)
        if (T > 0) {
            TAPE_CK(pdl(adj_sk_pre_kernel, dim3(ng), dim3(256), 0, st, tb.views));
            count_launches(1);
            TAPE_CK(cudaGetLastError());
        }
        for (int p = T - 1; p >= 1; --p) {
            TAPE_CK(launch_tma_gather_batched(dtype, rs, maps, tb.insts + (size_t)(N + p) * count, tb.work,
                                              tb.nwork, err, st));
            TAPE_CK(pdl(adj_sk_finish_pre_kernel, pgrid2, dim3(32, 8), 0, st, tb.views, p));
            count_launches(1);
            TAPE_CK(cudaGetLastError());
        }
        if (fused) {
            // pair pass B with the box sums and the scatter of the patch-distance adjoint
            auto bd = [&](auto wt) -> cudaError_t {
                using WT = decltype(wt);
                const size_t smem = pairs_bd_smem(T, rp, rs, dtype);
                auto run = [&](auto kern) -> cudaError_t {
                    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                    if (e != cudaSuccess) return e;
                    return pdl(kern, dim3(bg_tx, bg_ty, bg_chunks * count), dim3(32, 8), smem, st, tb.views,
                               bg_chunks, err, kDefaultWaitBudget);
                };
                if (rp == 2 && rs == 7 && T == 4) return run(adj_pairs_bd_kernel<WT, 2, 7, 4>);
                switch (rp) {
                    case 1: return run(adj_pairs_bd_kernel<WT, 1, 0, -1>);
                    case 2: return run(adj_pairs_bd_kernel<WT, 2, 0, -1>);
                    default: return run(adj_pairs_bd_kernel<WT, 3, 0, -1>);
                }
            };
            switch (dtype) {
                case DSGNLM_F32: TAPE_CK(bd(float{})); break;
                case DSGNLM_F16: TAPE_CK(bd(__half{})); break;
                default: TAPE_CK(bd(__nv_bfloat16{})); break;
            }
            count_launches(1);
            {
                const int elems = bg_tx * bg_ty * bg_win_h(rs) * (bg_qw + 2 * rs);
                TAPE_CK(pdl(adj_chunk_sum_kernel, dim3((elems + 255) / 256, 1, count), dim3(256), 0, st,
                    tb.views, 0, elems,
                            bg_chunks));
            }
            TAPE_CK(pdl(adj_fold_kernel, dim3(pgrid2), dim3(32, 8), 0, st, tb.views, bg_ty, bg_tx, 1, bg_qw));
            count_launches(2);
            TAPE_CK(cudaGetLastError());
        } else {
            // pair pass B: D-hat planes and dL/dh partials
            switch (dtype) {
                case DSGNLM_F32: TAPE_CK(pairs_b(float{})); break;
                case DSGNLM_F16: TAPE_CK(pairs_b(__half{})); break;
                default: TAPE_CK(pairs_b(__nv_bfloat16{})); break;
            }
            // patch distances back to the guide: box sums and the scatter of every offset per
            // tile of the extended grid, then the gather of the partials and the fold through
            // the reflection
            const size_t bsmem =
                sizeof(float) * (size_t)(2 * bg_win_h(rs) * bg_win_w(rs) + (kQH + 2 * rp) * (kQW + 2 * rp) +
                                         (kQH + 2 * rp) * kQW);
            TAPE_CK(cudaFuncSetAttribute(adj_boxguide_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bsmem));
            TAPE_CK(pdl(adj_boxguide_kernel, dim3(bg_tx, bg_ty, bg_chunks * count), dim3(32, 8), bsmem, st, tb.views,
                        bg_chunks));
            TAPE_CK(pdl(adj_fold_kernel, dim3(pgrid2), dim3(32, 8), 0, st, tb.views, bg_ty, bg_tx, bg_chunks, bg_qw));
            count_launches(2);
            TAPE_CK(cudaGetLastError());
        }
        // dL/dy = sum_k mu A g_k = A gs
        TAPE_CK(by_blur_radius(lead->taps.r, [&](auto rc) {
            return pdl(adj_ybar_kernel<decltype(rc)::value>, dim3((W / 2 + 31) / 32, (H / 2 + 7) / 8, count),
                       dim3(32, 8), 0, st, tb.views);
        }));
        count_launches(1);
        TAPE_CK(pdl(adj_sum_kernel, dim3(count), dim3(256), 0, st, tb.views, 1, npb, nrb));
        TAPE_CK(pdl(adj_sum_kernel, dim3(count), dim3(256), 0, st, tb.views, 2, nhb, nrb));
        count_launches(2);
        TAPE_CK(cudaGetLastError());
        // every image's (m, rho, h) cotangents and the wait-error word, read back once
        TAPE_CK(pdl(adj_gather_scalars_kernel, dim3((count + 63) / 64), dim3(64), 0, st, tb.views, count,
                    lead->scal.as<double>()));
        count_launches(1);
        TAPE_CK(cudaGetLastError());
        TAPE_CK(cudaMemcpyAsync(lead->hs, lead->scal.p, sizeof(double) * 3 * (size_t)count, cudaMemcpyDeviceToHost,
                                st));
        TAPE_CK(cudaMemcpyAsync(err_host, err, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
        return DSGNLM_OK;
    };
    std::vector<uint64_t> key = {(uint64_t)count,  (uint64_t)H,     (uint64_t)W,  (uint64_t)rp,
                                 (uint64_t)rs,     (uint64_t)T,     (uint64_t)N,  (uint64_t)dtype,
                                 (uint64_t)lead->taps.r, (uint64_t)(uintptr_t)tb.views, (uint64_t)tb.nwork,
                                 (uint64_t)(uintptr_t)err, (uint64_t)(uintptr_t)lead->scal.p,
                                 (uint64_t)(uintptr_t)lead->hs};
    for (int i = 0; i < count; ++i) {
        key.push_back((uint64_t)(uintptr_t)dens[i]->planes.p);
        key.push_back((uint64_t)dens[i]->plan.splits.n);
    }
    s = run_recorded(lead->bwd_exec, lead->bwd_key, lead->bwd_launches, key, st, lead->cap, seq);
    if (s != DSGNLM_OK) return s;
    s = join_streams(lead, dens.data(), count, st);
    if (s != DSGNLM_OK) return s;
    TAPE_CK(cudaStreamSynchronize(st));
    if (*err_host) {
        TAPE_CK(cudaMemsetAsync(err, 0, sizeof(unsigned), st));
        TAPE_CK(cudaStreamSynchronize(st));
        return DSGNLM_TIMEOUT;
    }
    for (int i = 0; i < count; ++i) {
        if (rho_bar) rho_bar[i] = lead->hs[3 * i + 1];
        if (h_bar) h_bar[i] = lead->hs[3 * i + 2];
    }
    return DSGNLM_OK;
}

}  // namespace

extern "C" {

dsgnlm_status lpnp_tape_create(lpnp_tape_t* out) {
    if (!out) return DSGNLM_EINVAL;
    *out = new (std::nothrow) lpnp_tape();
    return *out ? DSGNLM_OK : DSGNLM_ENOMEM;
}

void lpnp_tape_destroy(lpnp_tape_t t) {
    if (!t) return;
    if (t->den) cudaStreamSynchronize(t->den->stream);
    if (t->staged) cudaEventSynchronize(t->staged);
    DevBuf* bufs[] = {&t->Dh,  &t->Th,   &t->X,  &t->V,       &t->U,     &t->Gr,     &t->AZ, &t->AZ4, &t->xh,
                      &t->vh,  &t->uh,   &t->g,  &t->gs,      &t->dh,    &t->dh0,    &t->base,
                      &t->thp, &t->Dhat, &t->Gp, &t->m,     &t->mkey,   &t->sstar,  &t->mh,
                      &t->rho_part, &t->h_part, &t->m_part, &t->scratch, &t->tables, &t->scal};
    for (DevBuf* b : bufs) b->release();
    if (t->stage) cudaFreeHost(t->stage);
    if (t->hs) cudaFreeHost(t->hs);
    if (t->staged) cudaEventDestroy(t->staged);
    if (t->ev) cudaEventDestroy(t->ev);
    if (t->side) cudaStreamSynchronize(t->side);
    if (t->fork_ev) cudaEventDestroy(t->fork_ev);
    if (t->join_ev) cudaEventDestroy(t->join_ev);
    if (t->side) cudaStreamDestroy(t->side);
    if (t->cap) cudaStreamDestroy(t->cap);
    if (t->fwd_exec) cudaGraphExecDestroy(t->fwd_exec);
    if (t->bwd_exec) cudaGraphExecDestroy(t->bwd_exec);
    delete t;
}

dsgnlm_status lpnp_unrolled_forward(lpnp_tape_t tp, dsgnlm_t den, const float* y, const float* guide, int H, int W,
                                    int patch_r, int search_r, float bandwidth, int balance_passes, float alpha,
                                    float rho, int iters, float blur_sigma, int blur_r, float* x_out) {
    NvtxRange nvtx_range("lpnp_unrolled_forward");
    if (!tp || !den || !y || !guide || !x_out) return DSGNLM_EINVAL;
    dsgnlm_status s = lock_forward(&tp, &den, 1, &y, &guide, H, W, patch_r, search_r, bandwidth, balance_passes,
                                   alpha, rho, iters, blur_sigma, blur_r, &x_out);
    if (s != DSGNLM_OK) cudaStreamSynchronize(den->stream);  // nothing left running on the inputs
    return s;
}

dsgnlm_status lpnp_unrolled_forward_batched(lpnp_tape_t* tapes, dsgnlm_t* dens, int count, const float* const* y,
                                            const float* const* guide, int H, int W, int patch_r, int search_r,
                                            float bandwidth, int balance_passes, float alpha, float rho, int iters,
                                            float blur_sigma, int blur_r, float* const* x_out) {
    NvtxRange nvtx_range("lpnp_unrolled_forward_batched");
    if (!tapes || !dens || !y || !guide || !x_out || count < 1) return DSGNLM_EINVAL;
    for (int i = 0; i < count; ++i) {
        if (!tapes[i] || !dens[i] || !x_out[i] || !y[i] || !guide[i]) return DSGNLM_EINVAL;
        for (int j = 0; j < i; ++j)
            if (tapes[j] == tapes[i] || dens[j] == dens[i]) return DSGNLM_EINVAL;
    }
    dsgnlm_status s = lock_forward(tapes, dens, count, y, guide, H, W, patch_r, search_r, bandwidth, balance_passes,
                                   alpha, rho, iters, blur_sigma, blur_r, x_out);
    if (s != DSGNLM_OK)  // on a failure, nothing of the batch is left running on the caller's buffers
        for (int j = 0; j < count; ++j) cudaStreamSynchronize(dens[j]->stream);
    return s;
}

dsgnlm_status lpnp_backward(lpnp_tape_t tp, const float* x_bar, float* y_bar, float* guide_bar, double* h_bar,
                            double* rho_bar) {
    NvtxRange nvtx_range("lpnp_backward");
    if (!tp || !x_bar || !y_bar || !guide_bar) return DSGNLM_EINVAL;
    dsgnlm_status s = lock_backward(&tp, 1, &x_bar, &y_bar, &guide_bar, h_bar, rho_bar);
    if (s != DSGNLM_OK && tp->den) cudaStreamSynchronize(tp->den->stream);  // nothing left in flight
    return s;
}

dsgnlm_status lpnp_backward_batched(lpnp_tape_t* tapes, int count, const float* const* x_bar, float* const* y_bar,
                                    float* const* guide_bar, double* h_bar, double* rho_bar) {
    NvtxRange nvtx_range("lpnp_backward_batched");
    if (!tapes || !x_bar || !y_bar || !guide_bar || count < 1) return DSGNLM_EINVAL;
    for (int i = 0; i < count; ++i) {
        if (!tapes[i] || !x_bar[i] || !y_bar[i] || !guide_bar[i]) return DSGNLM_EINVAL;
        for (int j = 0; j < i; ++j)
            if (tapes[j] == tapes[i] || (tapes[i]->den && tapes[j]->den == tapes[i]->den)) return DSGNLM_EINVAL;
    }
    dsgnlm_status s = lock_backward(tapes, count, x_bar, y_bar, guide_bar, h_bar, rho_bar);
    if (s != DSGNLM_OK)
        for (int j = 0; j < count; ++j)  // nothing left in flight
            if (tapes[j]->den) cudaStreamSynchronize(tapes[j]->den->stream);
    return s;
}

}  // extern "C"
