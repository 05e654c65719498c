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
//   iteration k (reverse): a = vh - uh, zh = W a + uh (W is symmetric),
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
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "../../include/dsgnlm.h"
#include "combine.cuh"
#include "common.cuh"
#include "grad.cuh"
#include "handle.h"
#include "host_pool.h"
#include "internal.h"
#include "xupdate.cuh"

namespace dsg {

namespace {

constexpr int kAdjTH = 16, kAdjTW = 32;  // pair-pass tiles, block (32, 8), 2 rows per thread
constexpr int kMaxHalfOffsets = 2 * 12 * 13;  // n_h at the largest search radius (12)
constexpr int kPairSplit = 4;  // pair passes G and B: the half offsets in this many chunks (grid z)

__device__ __forceinline__ float proj_deriv(float xb, int constraint) {
    if (constraint == 2) return (xb > 0.f && xb < 1.f) ? 1.f : 0.f;
    if (constraint == 1) return xb > 0.f ? 1.f : 0.f;
    return 1.f;
}

// m = max_s d_s t_s and its first maximiser.  Each candidate becomes one 64-bit key:
// the bits of d_s t_s (positive floats order like their bit patterns) above the
// complement of s, so a larger key is a larger value or, for equal values, a smaller
// index.  Every warp folds its best key in with atomicMax, which does not depend on
// the order of arrival; the finish kernel unpacks the key.
__global__ void __launch_bounds__(256) adj_m_key_kernel(const float* __restrict__ d, const float* __restrict__ t,
                                                        int n, unsigned long long* __restrict__ key) {
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
    if ((threadIdx.x & 31) == 0) atomicMax(key, best);
}

__global__ void adj_m_finish_kernel(const unsigned long long* __restrict__ key, float* __restrict__ m_out,
                                    int* __restrict__ s_out) {
    const unsigned long long k = *key;
    const float m = __uint_as_float((unsigned)(k >> 32));
    m_out[0] = m;
    m_out[1] = (float)(1.0 / (double)m);  // 1/m as the host would form it, read by the kernels that follow
    *s_out = (int)(0xffffffffu - (unsigned)(k & 0xffffffffull));
}

// x-update of one recorded forward iteration (Algorithm 1, first two steps) from the
// states of slot k into slot k + 1, on 32 x 32 tiles:
//   g = A^T (A x_k - y) (recorded),  x_{k+1} = Pi_C(mu (alpha x_k + rho (v_k - u_k) - g)),
//   z = x_{k+1} + u_k,  and v_k, u_k copied into slot k + 1 for the dual step to update.
// x_k is read in halos and x_{k+1} written to another buffer, so tiles do not race.
template <int R>
__global__ void __launch_bounds__(256)
adj_fwd_xupdate_kernel(const float* __restrict__ xk, const float* __restrict__ vk, const float* __restrict__ uk,
                       const float* __restrict__ y, int H, int W, BlurTaps taps, float mu, float alpha, float rho,
                       int constraint, float* __restrict__ grec, float* __restrict__ x1, float* __restrict__ v1,
                       float* __restrict__ u1, float* __restrict__ z) {
    __shared__ GradSmem<R> sm;
    sr_grad_tile_apply<R>(sm, xk, y, H, W, taps, blockIdx.y * kGT, blockIdx.x * kGT,
                          [&](int pi, int pj, float e, float o) {
                              const size_t q = (size_t)pi * W + pj;
                              const float g2[2] = {e, o};
#pragma unroll
                              for (int c = 0; c < 2; ++c) {
                                  const float up = uk[q + c], vp = vk[q + c];
                                  const float xn = project(mu * (alpha * xk[q + c] + rho * (vp - up) - g2[c]), constraint);
                                  grec[q + c] = g2[c];
                                  x1[q + c] = xn;
                                  z[q + c] = xn + up;
                                  v1[q + c] = vp;
                                  u1[q + c] = up;
                              }
                          });
}

// Reverse iteration k, after g: ata = A^T A g on 32 x 32 tiles, then per pixel
//   xh = mu (alpha g - ata), vh = mu rho g, uh = zh - mu rho g, gs += mu g (the
//   observation's cotangent is A gs, A being linear), and when a_next is given the
//   inputs of the earlier iteration: a_{k-1} = vh - uh, z_{k-1} = x_k + u_{k-1}.
// g is only read, so the halo reads do not race with the writes.
template <int R>
__global__ void __launch_bounds__(256)
adj_ata_update_kernel(const float* __restrict__ g, int H, int W, BlurTaps taps, const float* __restrict__ zh,
                      float mu, float alpha, float rho, float* __restrict__ xh, float* __restrict__ vh,
                      float* __restrict__ uh, float* __restrict__ gs, const float* __restrict__ xk,
                      const float* __restrict__ uprev, float* __restrict__ a_next, float* __restrict__ z_next) {
    __shared__ GradSmem<R> sm;
    sr_grad_tile_apply<R>(sm, g, nullptr, H, W, taps, blockIdx.y * kGT, blockIdx.x * kGT,
                          [&](int pi, int pj, float e, float o) {
                              const size_t q = (size_t)pi * W + pj;
                              const float ata[2] = {e, o};
#pragma unroll
                              for (int c = 0; c < 2; ++c) {
                                  const float gg = g[q + c];
                                  const float vv = mu * rho * gg;
                                  const float uu = zh[q + c] - vv;
                                  xh[q + c] = mu * (alpha * gg - ata[c]);
                                  vh[q + c] = vv;
                                  uh[q + c] = uu;
                                  gs[q + c] += mu * gg;
                                  if (a_next) {
                                      a_next[q + c] = vv - uu;
                                      z_next[q + c] = xk[q + c] + uprev[q + c];
                                  }
                              }
                          });
}

// a_k = vh - uh, z_k = x_{k+1} + u_k
__global__ void adj_az_kernel(int n, const float* __restrict__ vh, const float* __restrict__ uh,
                              const float* __restrict__ x1, const float* __restrict__ u0, float* __restrict__ a,
                              float* __restrict__ z) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    a[q] = vh[q] - uh[q];
    z[q] = x1[q] + u0[q];
}

// W a finished from the phase-1 partial sums (W a = c_s a_s + (d_s / m) sum_r K1 d_r a_r,
// the closure of Eq. S3), then zh = W a + uh, g = Pi_C'(xbar_k)(xh + zh) and the block's
// partial of sum g mu ((v - u) - xbar).  Blocks of 32 x 8 pixels.
__global__ void __launch_bounds__(256)
adj_wa_g_kernel(Cover cv, int H, int W, const float* __restrict__ d, const float* __restrict__ t_fin,
                const float* __restrict__ inv_m_p, const float* __restrict__ a, const float* __restrict__ uh, const float* __restrict__ xh,
                const float* __restrict__ xk, const float* __restrict__ vk, const float* __restrict__ uk,
                const float* __restrict__ gradk, float mu, float alpha, float rho, int constraint,
                float* __restrict__ g, float* __restrict__ zh, double* __restrict__ rho_part) {
    const int j = blockIdx.x * 32 + threadIdx.x;
    const int i = blockIdx.y * 8 + threadIdx.y;
    const float inv_m = __ldg(inv_m_p);
    double r = 0.0;
    if (i < H && j < W) {
        const size_t q = (size_t)i * W + j;
        const float A = gather_partials(cv, i, j);
        const float ds = d[q];
        const float dm = ds * inv_m;
        const float cs = 1.f - dm * (t_fin[q] - ds);
        const float wa = fmaf(dm, A, cs * a[q]);
        const float zz = wa + uh[q];
        const float vu = vk[q] - uk[q];
        const float xb = mu * (alpha * xk[q] + rho * vu - gradk[q]);
        const float gg = proj_deriv(xb, constraint) * (xh[q] + zz);
        g[q] = gg;
        zh[q] = zz;
        r = (double)gg * (double)mu * ((double)vu - (double)xb);
    }
    r = warp_sum(r);
    __shared__ double sr[8];
    const int t = threadIdx.y * 32 + threadIdx.x;
    if ((t & 31) == 0) sr[t >> 5] = r;
    __syncthreads();
    if (t == 0) {
        double acc = 0.0;
        for (int w = 0; w < 8; ++w) acc += sr[w];
        rho_part[blockIdx.y * gridDim.x + blockIdx.x] += acc;  // fixed slot per block, fixed order over iterations
    }
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

// Pair pass G, over the half-window pairs (s, r = s + o): the pair term
//   G_sr = sum_k (a_k(s) - a_k(r)) (z_k(r) - z_k(s))
// stored as planes like K1 (0 where r is off the image), the forward half of
// dh0(s) = sum_o G_sr d_r K1_sr, and per-block partials of
// -(1/m^2) sum over half-window pairs of G d_s d_r K1.  G is symmetric in (s, r), so
// the other half of dh comes from these planes (pair pass T).  Grid z splits the half
// offsets into kPairSplit contiguous chunks; chunk z writes its own dh0 plane and
// partials.
// Staged over the tile and its forward halo: (a_k, z_k, a_{k+1}, z_{k+1}) as one float4
// per pair of iterations (zeros past N, which add exact zeros), then d.  With NP > 0
// (NP = ceil(N / 2)) the values at s are held in registers and the loop is unrolled;
// NP = 0 reads them from shared memory.  Both sum in the same order.
template <typename WT, int NP>
__global__ void __launch_bounds__(256, 2)
adj_pairs_g_kernel(const WT* __restrict__ P, int H, int W, int rs, int N, const float* __restrict__ AZ,
                   const float* __restrict__ d, const float* __restrict__ inv_m_p, float* __restrict__ Gp,
                   float* __restrict__ dh0, double* __restrict__ m_part) {
    extern __shared__ float4 S4[];
    const float inv_m = __ldg(inv_m_p);
    const int y0 = blockIdx.y * kAdjTH, x0 = blockIdx.x * kAdjTW;
    const int RH = kAdjTH + rs, RW = kAdjTW + 2 * rs, cells = RH * RW;
    const size_t n = (size_t)H * W;
    const int np = (N + 1) >> 1;
    float* Sd = reinterpret_cast<float*>(S4 + (size_t)np * cells);
    const int nh = num_half_offsets(rs);
    const int kz0 = nh * (int)blockIdx.z / kPairSplit, kz1 = nh * ((int)blockIdx.z + 1) / kPairSplit;
    {
        const int tid = threadIdx.y * 32 + threadIdx.x;
        for (int idx = tid; idx < cells; idx += 256) {
            const int ra = idx / RW, cb = idx - ra * RW;
            const int i = y0 + ra, j = x0 - rs + cb;
            const bool in = i < H && j >= 0 && j < W;
            const size_t q = in ? (size_t)i * W + j : 0;
            for (int kp = 0; kp < np; ++kp) {
                const int k0 = 2 * kp, k1 = k0 + 1;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (in) {
                    v.x = AZ[(size_t)k0 * n + q];
                    v.y = AZ[(size_t)(N + k0) * n + q];
                    if (k1 < N) {
                        v.z = AZ[(size_t)k1 * n + q];
                        v.w = AZ[(size_t)(N + k1) * n + q];
                    }
                }
                S4[(size_t)kp * cells + idx] = v;
            }
            Sd[idx] = in ? d[q] : 0.f;
        }
    }
    __syncthreads();
    const int Wp = plane_pitch(W);
    const size_t plane = (size_t)H * Wp;
    double mpart = 0.0;
    const int j = x0 + threadIdx.x;
    for (int py = threadIdx.y; py < kAdjTH; py += 8) {
        const int i = y0 + py;
        if (i >= H || j >= W) continue;
        const int cs = py * RW + threadIdx.x + rs;  // cell of s
        float4 sv[NP > 0 ? NP : 1];
        if constexpr (NP > 0) {
#pragma unroll
            for (int kp = 0; kp < NP; ++kp) sv[kp] = S4[kp * cells + cs];
        }
        const float ds = Sd[cs];
        float accd = 0.f, accm = 0.f;
        int oy, ox;
        half_offset(kz0, rs, oy, ox);
        // branch-free body (an off-image partner r reads staged zeros and adds an exact
        // zero), so the unrolled iterations issue their loads together
#pragma unroll 4
        for (int k = kz0; k < kz1; ++k) {
            {
                const size_t at = (size_t)k * plane + (size_t)i * Wp + j;
                const int rj = j + ox;
                const bool in = i + oy < H && rj >= 0 && rj < W;
                const float K = in ? to_f32(P[at]) : 0.f;
                const int cr = cs + oy * RW + ox;
                float G = 0.f;
                if constexpr (NP > 0) {
#pragma unroll
                    for (int kp = 0; kp < NP; ++kp) {
                        const float4 r = S4[kp * cells + cr];
                        G = fmaf(sv[kp].x - r.x, r.y - sv[kp].y, G);
                        G = fmaf(sv[kp].z - r.z, r.w - sv[kp].w, G);
                    }
                } else {
                    for (int kp = 0; kp < np; ++kp) {
                        const float4 a = S4[kp * cells + cs], r = S4[kp * cells + cr];
                        G = fmaf(a.x - r.x, r.y - a.y, G);
                        G = fmaf(a.z - r.z, r.w - a.w, G);
                    }
                }
                Gp[at] = in ? G : 0.f;
                const float dr = Sd[cr];
                accd = fmaf(G * dr, K, accd);
                accm = fmaf(G * ds * dr, K, accm);
            }
            if (++ox > rs) {
                ++oy;
                ox = -rs;
            }
        }
        dh0[blockIdx.z * n + (size_t)i * W + j] = accd;
        mpart -= (double)accm * (double)inv_m * (double)inv_m;
    }
    mpart = warp_sum(mpart);
    __shared__ double sm[8];
    const int t = threadIdx.y * 32 + threadIdx.x;
    if ((t & 31) == 0) sm[t >> 5] = mpart;
    __syncthreads();
    if (t == 0) {
        double acc = 0.0;
        for (int w = 0; w < 8; ++w) acc += sm[w];
        m_part[(blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = acc;
    }
}

// Pair pass T: dh(s) = (1/m) (dh0(s) + sum_o G_{s-o, s} d_{s-o} K1_{s-o, s}), dh0 the
// sum of pass G's chunk planes (in chunk order) and the backward half-window read from
// the planes at s - o
template <typename WT>
__global__ void __launch_bounds__(256)
adj_pairs_t_kernel(const WT* __restrict__ P, const float* __restrict__ Gp, int H, int W, int rs,
                   const float* __restrict__ d, const float* __restrict__ dh0, const float* __restrict__ inv_m_p,
                   float* __restrict__ dh) {
    const int j = blockIdx.x * 32 + threadIdx.x;
    const int i = blockIdx.y * 8 + threadIdx.y;
    if (i >= H || j >= W) return;
    const float inv_m = __ldg(inv_m_p);
    const int Wp = plane_pitch(W);
    const size_t plane = (size_t)H * Wp;
    const size_t n = (size_t)H * W;
    float acc = dh0[(size_t)i * W + j];
    for (int z = 1; z < kPairSplit; ++z) acc += dh0[z * n + (size_t)i * W + j];
    for (int oy = 0; oy <= rs && i - oy >= 0; ++oy) {
        const int ri = i - oy;
        const int ox0 = oy == 0 ? 1 : -rs;
        int k = oy == 0 ? 0 : rs + (oy - 1) * (2 * rs + 1);  // half offset of (oy, ox0)
        const size_t row = (size_t)ri * Wp;
        const float* drow = d + (size_t)ri * W;
        // predicated loads (no early exit), so the unrolled loads issue together
#pragma unroll 4
        for (int ox = ox0; ox <= rs; ++ox, ++k) {
            const int rj = j - ox;
            const bool in = rj >= 0 && rj < W;
            const size_t at = (size_t)k * plane + row + (in ? rj : 0);
            const float g = in ? Gp[at] : 0.f;
            const float w = in ? to_f32(P[at]) : 0.f;
            const float dv = in ? drow[rj] : 0.f;
            acc = fmaf(g * dv, w, acc);
        }
    }
    dh[(size_t)i * W + j] = acc * inv_m;
}

// fixed-order sum of `count` doubles into *out (one block)
__global__ void __launch_bounds__(256) adj_sum_kernel(const double* __restrict__ part, int count, double* __restrict__ out) {
    double a = 0.0;
    for (int q = threadIdx.x; q < count; q += 256) a += part[q];
    __shared__ double s[256];
    s[threadIdx.x] = a;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = s[0];
}

// Through m = d_{s*} t_{s*}: dh_{s*} += mh (t_{s*} + d_{s*}); dh_j += mh d_{s*} K1(s*, j), j != s*
template <typename WT>
__global__ void adj_mterms_kernel(const WT* __restrict__ P, int H, int W, int rs, const float* __restrict__ d,
                                  const float* __restrict__ t, const int* __restrict__ s_star,
                                  const double* __restrict__ mh_ptr, float* __restrict__ dh) {
    const int ss = *s_star;
    const int si = ss / W, sj = ss - si * W;
    const float mh = (float)*mh_ptr;
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
        const float K = to_f32(fwd ? P[(size_t)k * plane + (size_t)si * Wp + sj] : P[(size_t)k * plane + (size_t)ri * Wp + rj]);
        dh[(size_t)ri * W + rj] += mh * d[ss] * K;
    }
}

// Balancing pass p backwards: th = -0.5 dh' d'/t, base = 0.5 dh' d'/d (d' = d^{p+1})
__global__ void adj_sk_pre_kernel(int n, const float* __restrict__ dhn, const float* __restrict__ dn,
                                  const float* __restrict__ dp, const float* __restrict__ tp, float* __restrict__ th,
                                  float* __restrict__ base) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const float w = 0.5f * dhn[q] * dn[q];
    th[q] = -w / tp[q];
    base[q] = w / dp[q];
}

// dh^p = base + K1 th^p = base + th^p + sum_{r != s} K1 th^p_r (phase-1 partial sums in
// cv), the cotangent of d^p, and from it pass p - 1's th^{p-1} = -0.5 dh^p d^p / t^{p-1}
// and base = 0.5 dh^p d^p / d^{p-1} (base rewritten in place)
__global__ void __launch_bounds__(256)
adj_sk_finish_pre_kernel(Cover cv, int H, int W, const float* __restrict__ th, float* __restrict__ base,
                         const float* __restrict__ dp, const float* __restrict__ dq, const float* __restrict__ tq,
                         float* __restrict__ th_prev) {
    const int j = blockIdx.x * 32 + threadIdx.x;
    const int i = blockIdx.y * 8 + threadIdx.y;
    if (i >= H || j >= W) return;
    const size_t s = (size_t)i * W + j;
    const float dh = base[s] + th[s] + gather_partials(cv, i, j);
    const float w = 0.5f * dh * dp[s];
    th_prev[s] = -w / tq[s];
    base[s] = w / dq[s];
}

// Pair pass B: the cotangent of every stored weight K1(s, s + o),
//   Kh = G d_s d_r / m + sum_p (th^p_s d^p_r + th^p_r d^p_s) + [s or r = s*] mh d_s d_r,
// then Dh = -c K1 Kh (written as planes) and per-block partials of dL/dh = sum Kh K1 D 2c/h.
// G comes from the planes of pair pass G; fields staged over the tile and its forward
// halo: d^p (T + 1) and th^p (T).  Grid z splits the half offsets as in pass G.
template <typename WT>
__global__ void __launch_bounds__(256, 3)
adj_pairs_b_kernel(const WT* __restrict__ P, const float* __restrict__ Gp, int H, int W, int rs, int T,
                   const float* __restrict__ Dh, const float* __restrict__ Th, const float* __restrict__ inv_m_p,
                   float c, float hfac, const int* __restrict__ s_star, const double* __restrict__ mh_ptr,
                   float* __restrict__ Dhat, double* __restrict__ h_part) {
    extern __shared__ float S[];
    const float inv_m = __ldg(inv_m_p);
    const int y0 = blockIdx.y * kAdjTH, x0 = blockIdx.x * kAdjTW;
    const int RH = kAdjTH + rs, RW = kAdjTW + 2 * rs, cells = RH * RW;
    const size_t n = (size_t)H * W;
    stage_fields(S, Dh, T + 1, n, H, W, y0, x0 - rs, RH, RW);
    stage_fields(S + (T + 1) * cells, Th, T, n, H, W, y0, x0 - rs, RH, RW);
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
    const int kz0 = num_half_offsets(rs) * (int)blockIdx.z / kPairSplit;
    const int kz1 = num_half_offsets(rs) * ((int)blockIdx.z + 1) / kPairSplit;
    const int ss = *s_star;
    const float mh = (float)*mh_ptr;
    const int Wp = plane_pitch(W);
    const size_t plane = (size_t)H * Wp;
    double hpart = 0.0;
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
        hpart += (double)hp * (double)hfac;
    }
    hpart = warp_sum(hpart);
    __shared__ double sm[8];
    const int t = threadIdx.y * 32 + threadIdx.x;
    if ((t & 31) == 0) sm[t >> 5] = hpart;
    __syncthreads();
    if (t == 0) {
        double acc = 0.0;
        for (int w = 0; w < 8; ++w) acc += sm[w];
        h_part[(blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = acc;
    }
}

// Patch-distance adjoint.  With g the reflected guide on the grid extended by the
// patch radius (p in [-rp, H + rp) x [-rp, W + rp)) and, per offset o,
//   E_o(q) = sum_{t in patch} Dh_o(q - t)               (box sum, Dh = 0 off the image)
//   F_o(q) = 2 E_o(q) (g(q) - g(q + o)),
// the cotangent of g(p) is ge(p) = sum_o F_o(p) - F_o(p - o): the first term from the
// patch at q = p, the second from the patch whose partner pixel is p.  Two kernels:
// the box sums of every D-hat plane onto the extended grid, then one thread per p
// summing its offsets in a fixed order (no atomics, so the result does not depend on
// scheduling).
constexpr int kBT = 32;  // box-sum tile side (extended grid)

__global__ void __launch_bounds__(256)
adj_box_kernel(const float* __restrict__ Dhat, int H, int W, int rp, float* __restrict__ E) {
    extern __shared__ float S[];
    const int k = blockIdx.z;
    const int q0y = blockIdx.y * kBT - rp, q0x = blockIdx.x * kBT - rp;  // image coords of the tile origin
    const int DW = kBT + 2 * rp;  // Dh over rows [q0y - rp, q0y + kBT + rp), same columns
    float* Ds = S;                // [DW][DW]
    float* Rs = Ds + DW * DW;     // horizontal sums [DW][kBT]
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int Wp = plane_pitch(W);
    const float* Dk = Dhat + (size_t)k * H * Wp;
    for (int a = ty; a < DW; a += 8) {
        const int i = q0y - rp + a;
        const bool row_in = i >= 0 && i < H;
        for (int b = tx; b < DW; b += 32) {
            const int j = q0x - rp + b;
            Ds[a * DW + b] = (row_in && j >= 0 && j < W) ? Dk[(size_t)i * Wp + j] : 0.f;
        }
    }
    __syncthreads();
    for (int a = ty; a < DW; a += 8) {
        float s = 0.f;
        for (int t = 0; t <= 2 * rp; ++t) s += Ds[a * DW + tx + t];
        Rs[a * kBT + tx] = s;
    }
    __syncthreads();
    const int XW = W + 2 * rp, XH = H + 2 * rp;
    float* Ek = E + (size_t)k * XH * XW;
    const int qx = q0x + tx;
    for (int a = ty; a < kBT; a += 8) {
        const int qy = q0y + a;
        if (qy >= H + rp || qx >= W + rp) continue;
        float s = 0.f;
        for (int t = 0; t <= 2 * rp; ++t) s += Rs[(a + t) * kBT + tx];
        Ek[(size_t)(qy + rp) * XW + (qx + rp)] = s;
    }
}

__global__ void __launch_bounds__(256)
adj_guide_kernel(const float* __restrict__ E, const float* __restrict__ guide, int H, int W, int rp, int rs,
                 float* __restrict__ ge) {
    extern __shared__ float Gs[];  // g over rows [p0y - rs, p0y + 8 + rs), cols [p0x - rs, p0x + 32 + rs)
    const int p0y = blockIdx.y * 8 - rp, p0x = blockIdx.x * 32 - rp;
    const int GH = 8 + 2 * rs, GW = 32 + 2 * rs;
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int a = ty; a < GH; a += 8) {
        const size_t row = (size_t)sym_index(p0y - rs + a, H) * W;
        for (int b = tx; b < GW; b += 32) Gs[a * GW + b] = guide[row + sym_index(p0x - rs + b, W)];
    }
    __syncthreads();
    const int py = p0y + ty, px = p0x + tx;
    const int XW = W + 2 * rp, XH = H + 2 * rp;
    if (py >= H + rp || px >= W + rp) return;
    const size_t plane = (size_t)XH * XW;
    const int ca = ty + rs, cb = tx + rs;  // p in Gs
    const float gp = Gs[ca * GW + cb];
    const size_t at = (size_t)(py + rp) * XW + (px + rp);
    float acc = 0.f;
    int oy, ox;
    half_offset(0, rs, oy, ox);
    const int nh = num_half_offsets(rs);
#pragma unroll 4
    for (int k = 0; k < nh; ++k) {
        const float* Ek = E + (size_t)k * plane;
        // q = p - o must lie on the extended grid (E is 0 beyond it)
        const int qy = py - oy, qx = px - ox;
        const bool qin = qy >= -rp && qx >= -rp && qx < W + rp;
        const float ep = Ek[at];
        const float eq = qin ? Ek[at - (size_t)oy * XW - ox] : 0.f;
        const float fp = 2.f * ep * (gp - Gs[(ca + oy) * GW + cb + ox]);
        const float fq = 2.f * eq * (Gs[(ca - oy) * GW + cb - ox] - gp);
        acc += fp - fq;
        if (++ox > rs) {
            ++oy;
            ox = -rs;
        }
    }
    ge[at] = acc;
}

// gb(q) = (xh0 + vh0)(q) [0 < g(q) < 1] + sum of ge(p) over the extended p that reflect
// onto q (p = 2 n m + q or 2 n m - 1 - q per axis), in a fixed order
__global__ void adj_fold_kernel(const float* __restrict__ ge, const float* __restrict__ xh0,
                                const float* __restrict__ vh0, const float* __restrict__ guide, int H, int W, int rp,
                                float* __restrict__ gb) {
    const int j = blockIdx.x * 32 + threadIdx.x;
    const int i = blockIdx.y * 8 + threadIdx.y;
    if (i >= H || j >= W) return;
    const size_t q = (size_t)i * W + j;
    const float g = guide[q];
    float acc = (g > 0.f && g < 1.f) ? xh0[q] + vh0[q] : 0.f;
    const int XW = W + 2 * rp;
    const int my = rp / (2 * H) + 1, mx = rp / (2 * W) + 1;
    for (int m = -my; m <= my; ++m)
        for (int cy = 0; cy < 2; ++cy) {
            const int pi = cy == 0 ? 2 * H * m - 1 - i : 2 * H * m + i;
            if (pi < -rp || pi >= H + rp) continue;
            for (int n = -mx; n <= mx; ++n)
                for (int cx = 0; cx < 2; ++cx) {
                    const int pj = cx == 0 ? 2 * W * n - 1 - j : 2 * W * n + j;
                    if (pj < -rp || pj >= W + rp) continue;
                    acc += ge[(size_t)(pi + rp) * XW + (pj + rp)];
                }
        }
    gb[q] = acc;
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

}  // namespace

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
    DevBuf Dh, Th, X, V, U, Gr, AZ, xh, vh, uh, zh, g, gs, dh[1], dh0, base, thp, Dhat, Gp, ge, gb, ctl,
        part, m, mkey, sstar, mh, rho_part, h_part, m_part, scratch;
    // m and 1/m on the device (written by the forward, read by the kernels that follow)
    const float* inv_m_dev() const { return m.as<float>() + 1; }
    // pinned host words read back after the stream work: m, the scalar cotangents and
    // the handle's wait-error flag
    struct Host {
        double hs[3];
        unsigned err;
        float m;
    };
    Host* host = nullptr;
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

size_t pairs_g_smem(int N, int rs) {
    return (sizeof(float4) * (size_t)((N + 1) / 2) + sizeof(float)) * (kAdjTH + rs) * (kAdjTW + 2 * rs);
}
size_t pairs_b_smem(int T, int rs) {
    return sizeof(float) * (size_t)(2 * T + 1) * (kAdjTH + rs) * (kAdjTW + 2 * rs);
}

// pair passes G and T: the planes of G and dh = (1/m) sum_{r ~ s} G_sr d_r K1_sr into dh[0]
// (dh0 holds the forward half, one plane per offset chunk, in between)
template <typename WT>
cudaError_t pairs_gt(const lpnp_tape* tp, const void* planes, cudaStream_t st, double* m_part) {
    const int H = tp->H, W = tp->W, rs = tp->rs, N = tp->N;
    const size_t smem = pairs_g_smem(N, rs);
    const float* d = tp->Dh.as<float>() + (size_t)tp->T * H * W;
    dim3 grid((W + kAdjTW - 1) / kAdjTW, (H + kAdjTH - 1) / kAdjTH, kPairSplit);
    auto run = [&](auto kern) -> cudaError_t {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<grid, dim3(32, 8), smem, st>>>((const WT*)planes, H, W, rs, N, tp->AZ.as<float>(), d, tp->inv_m_dev(),
                                              tp->Gp.as<float>(), tp->dh0.as<float>(), m_part);
        return cudaGetLastError();
    };
    cudaError_t e;
    switch ((N + 1) / 2) {
        case 1: e = run(adj_pairs_g_kernel<WT, 1>); break;
        case 2: e = run(adj_pairs_g_kernel<WT, 2>); break;
        case 3: e = run(adj_pairs_g_kernel<WT, 3>); break;
        case 4: e = run(adj_pairs_g_kernel<WT, 4>); break;
        case 5: e = run(adj_pairs_g_kernel<WT, 5>); break;
        case 6: e = run(adj_pairs_g_kernel<WT, 6>); break;
        case 7: e = run(adj_pairs_g_kernel<WT, 7>); break;
        case 8: e = run(adj_pairs_g_kernel<WT, 8>); break;
        default: e = run(adj_pairs_g_kernel<WT, 0>); break;
    }
    count_launches(1);
    if (e != cudaSuccess) return e;
    adj_pairs_t_kernel<WT><<<dim3((W + 31) / 32, (H + 7) / 8), dim3(32, 8), 0, st>>>(
        (const WT*)planes, tp->Gp.as<float>(), H, W, rs, d, tp->dh0.as<float>(), tp->inv_m_dev(), tp->dh[0].as<float>());
    count_launches(1);
    return cudaGetLastError();
}

template <typename WT>
cudaError_t pairs_b(const lpnp_tape* tp, const void* planes, cudaStream_t st) {
    const int H = tp->H, W = tp->W, rs = tp->rs;
    const size_t smem = pairs_b_smem(tp->T, rs);
    cudaError_t e = cudaFuncSetAttribute(adj_pairs_b_kernel<WT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((W + kAdjTW - 1) / kAdjTW, (H + kAdjTH - 1) / kAdjTH, kPairSplit);
    adj_pairs_b_kernel<WT><<<grid, dim3(32, 8), smem, st>>>(
        (const WT*)planes, tp->Gp.as<float>(), H, W, rs, tp->T, tp->Dh.as<float>(), tp->thp.as<float>(), tp->inv_m_dev(),
        tp->c, 2.f * tp->c / tp->h, tp->sstar.as<int>(), tp->mh.as<double>(), tp->Dhat.as<float>(),
        tp->h_part.as<double>());
    count_launches(1);
    return cudaGetLastError();
}

template <typename WT>
cudaError_t mterms(const lpnp_tape* tp, const void* planes, cudaStream_t st) {
    const size_t n = (size_t)tp->H * tp->W;
    adj_mterms_kernel<WT><<<1, 256, 0, st>>>((const WT*)planes, tp->H, tp->W, tp->rs,
                                             tp->Dh.as<float>() + (size_t)tp->T * n, tp->Th.as<float>() + (size_t)tp->T * n,
                                             tp->sstar.as<int>(), tp->mh.as<double>(), tp->dh[0].as<float>());
    count_launches(1);
    return cudaGetLastError();
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
    DevBuf* bufs[] = {&t->Dh, &t->Th, &t->X, &t->V, &t->U, &t->Gr, &t->AZ, &t->xh, &t->vh, &t->uh, &t->zh, &t->g,
                      &t->gs, &t->dh[0], &t->dh0, &t->base, &t->thp, &t->Dhat,
                      &t->Gp, &t->ge, &t->gb, &t->ctl, &t->part, &t->m, &t->mkey, &t->sstar, &t->mh, &t->rho_part, &t->h_part,
                      &t->m_part, &t->scratch};
    for (DevBuf* b : bufs) b->release();
    if (t->host) cudaFreeHost(t->host);
    delete t;
}

}  // extern "C"

namespace {

// First half of the recording: K1 into the handle, the T balancing passes with every
// d^p and t^p kept, m = max_s d_s t_s with its first maximiser and 1/m on the device,
// and the read-back of m queued on the handle's stream.  Nothing here waits for the
// device.  `share` images run at once (the handle's offset split is sized for them).
dsgnlm_status forward_begin(lpnp_tape* tp, dsgnlm* den, const float* y, const float* guide, int H, int W,
                            int patch_r, int search_r, float bandwidth, int balance_passes, float alpha, float rho,
                            int iters, float blur_sigma, int blur_r, int share) {
    if (!tp || !den || !y || !guide) return DSGNLM_EINVAL;
    if (H < 2 || W < 2 || (H & 1) || (W & 1) || iters < 1 || iters > 256 || balance_passes < 0 ||
        balance_passes > 64 || !(rho > 0.f) || !(alpha >= 0.f) || blur_r < 0 || blur_r > 8 || !(blur_sigma > 0.f))
        return DSGNLM_EINVAL;
    if (!tma_path_supports(search_r)) return DSGNLM_EINVAL;
    // shared memory of the pair passes of the backward (fields over a tile + halo)
    if (pairs_g_smem(iters, search_r) > 220 * 1024 || pairs_b_smem(balance_passes, search_r) > 220 * 1024)
        return DSGNLM_EINVAL;
    if (!tp->host) TAPE_CK(cudaMallocHost((void**)&tp->host, sizeof(lpnp_tape::Host)));
    den->share = share;
    dsgnlm_status s = dsgnlm_build(den, guide, H, W, patch_r, search_r, bandwidth);
    den->share = 1;
    if (s != DSGNLM_OK) return s;
    if (!den->fast) return DSGNLM_EINVAL;
    cudaStream_t st = den->stream;
    const size_t n = (size_t)H * W;
    const int T = balance_passes, N = iters;
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
    const double np = 2.0 * patch_r + 1.0;
    tp->c = (float)(1.0 / (2.0 * np * np * (double)bandwidth * (double)bandwidth));
    tp->taps = make_blur_taps(blur_sigma, blur_r);
    tp->blur_sigma = blur_sigma;
    tp->blur_r = blur_r;
    tp->y = y;
    tp->guide = guide;
    TAPE_CK(tp->Dh.ensure(sizeof(float) * n * (T + 1)));
    TAPE_CK(tp->Th.ensure(sizeof(float) * n * (T + 1)));
    TAPE_CK(tp->X.ensure(sizeof(float) * n * (N + 1)));
    TAPE_CK(tp->V.ensure(sizeof(float) * n * (N + 1)));
    TAPE_CK(tp->U.ensure(sizeof(float) * n * (N + 1)));
    TAPE_CK(tp->Gr.ensure(sizeof(float) * n * N));
    TAPE_CK(tp->scratch.ensure(sizeof(float) * n));
    TAPE_CK(tp->ctl.ensure(sizeof(BalanceCtl)));
    TAPE_CK(tp->part.ensure(sizeof(float2) * (size_t)balance_combine_blocks(H, W)));
    TAPE_CK(tp->m.ensure(2 * sizeof(float)));  // m and 1/m
    TAPE_CK(tp->sstar.ensure(sizeof(int)));
    TAPE_CK(tp->mkey.ensure(sizeof(unsigned long long)));
    TAPE_CK(cudaMemsetAsync(tp->ctl.p, 0, sizeof(BalanceCtl), st));  // done = 0: passes always run
    TAPE_CK(launch_fill(tp->Dh.as<float>(), 1.0f, n, st));
    // T balancing passes with every d^p and t^p kept, then t^T = K1 d^T
    BalanceCtl* ctl = tp->ctl.as<BalanceCtl>();
    for (int p = 0; p <= T; ++p) {
        float* dp = tp->Dh.as<float>() + (size_t)p * n;
        float* dn = p < T ? tp->Dh.as<float>() + (size_t)(p + 1) * n : tp->scratch.as<float>();
        TAPE_CK(launch_tma_gather(den->dtype, den->plan, H, W, search_r, dp, nullptr, den->err.as<unsigned>(),
                                  &ctl->done, st, den->wait_budget));
        TAPE_CK(launch_balance_epilogue(den->plan, H, W, search_r, dp, dn, tp->Th.as<float>() + (size_t)p * n,
                                        tp->part.as<float2>(), ctl, 0, cudaGraphConditionalHandle{}, 0, st));
    }
    const float* dT = tp->Dh.as<float>() + (size_t)T * n;
    const float* tT = tp->Th.as<float>() + (size_t)T * n;
    TAPE_CK(cudaMemsetAsync(tp->mkey.p, 0, sizeof(unsigned long long), st));
    adj_m_key_kernel<<<(int)std::min<size_t>((n + 255) / 256, 1024), 256, 0, st>>>(
        dT, tT, (int)n, tp->mkey.as<unsigned long long>());
    adj_m_finish_kernel<<<1, 1, 0, st>>>(tp->mkey.as<unsigned long long>(), tp->m.as<float>(), tp->sstar.as<int>());
    count_launches(2);
    TAPE_CK(cudaGetLastError());
    return DSGNLM_OK;
}

// Second half: fixes W on the handle and runs Algorithm 1 one iteration at a time,
// every state recorded (the same kernels and order of arithmetic as a one-iteration
// lpnp_solve, with the x-update writing into the next slot).  1/m is read on the
// device, so nothing here waits for the device either.  x_out receives x_N.
dsgnlm_status forward_finish(lpnp_tape* tp, float* x_out) {
    dsgnlm* den = tp->den;
    cudaStream_t st = den->stream;
    const size_t n = (size_t)tp->H * tp->W;
    const int T = tp->T, N = tp->N;
    // the handle now holds this W; its m and 1/m stay on the device until a host-side
    // use of the handle reads them back
    den->d_final = tp->Dh.as<float>() + (size_t)T * n;
    den->t_final = tp->Th.as<float>() + (size_t)T * n;
    den->iters = T;
    den->balanced = true;
    den->inv_m_dev = false;  // the balance control block does not hold this W's 1/m
    den->m_pending = tp->m.as<float>();
    TAPE_CK(launch_init(tp->guide, (int)n, tp->X.as<float>(), tp->V.as<float>(), tp->U.as<float>(), st));
    // Algorithm 1, one iteration at a time from slot k into slot k + 1: the x-update
    // (recording grad f(x_k)), then W z and the dual step in place on slot k + 1
    const int H = tp->H, W = tp->W;
    const int nblocks = combine_xupdate_blocks(H, W);
    TAPE_CK(den->partials.ensure(sizeof(double) * 2 * (size_t)nblocks));
    TAPE_CK(den->z.ensure(sizeof(float) * n));
    EpilogueArgs ea{};
    ea.H = H;
    ea.W = W;
    ea.d = den->d_final;
    ea.t = den->t_final;
    ea.inv_m = 1.f;
    ea.inv_m_dev = tp->inv_m_dev();
    ea.z = den->z.as<float>();
    ea.taps = tp->taps;
    ea.mu = tp->mu;
    ea.alpha = tp->alpha;
    ea.rho = tp->rho;
    ea.constraint = tp->constraint;
    ea.do_x = 0;
    ea.partials = den->partials.as<double>();
    const dim3 ggrid((W + kGT - 1) / kGT, (H + kGT - 1) / kGT);
    for (int k = 0; k < N; ++k) {
        const float* xk = tp->X.as<float>() + (size_t)k * n;
        const float* vk = tp->V.as<float>() + (size_t)k * n;
        const float* uk = tp->U.as<float>() + (size_t)k * n;
        float* v1 = tp->V.as<float>() + (size_t)(k + 1) * n;
        float* u1 = tp->U.as<float>() + (size_t)(k + 1) * n;
        TAPE_CK(by_blur_radius(tp->taps.r, [&](auto rc) {
            adj_fwd_xupdate_kernel<decltype(rc)::value><<<ggrid, 256, 0, st>>>(
                xk, vk, uk, tp->y, H, W, tp->taps, tp->mu, tp->alpha, tp->rho, tp->constraint,
                tp->Gr.as<float>() + (size_t)k * n, tp->X.as<float>() + (size_t)(k + 1) * n, v1, u1, ea.z);
            return cudaGetLastError();
        }));
        count_launches(1);
        TAPE_CK(launch_tma_gather(den->dtype, den->plan, H, W, tp->rs, den->d_final, ea.z, den->err.as<unsigned>(),
                                  nullptr, st, den->wait_budget));
        ea.v = v1;
        ea.u = u1;
        TAPE_CK(launch_combine_update(0, den->plan, tp->rs, ea, st));
    }
    TAPE_CK(cudaMemcpyAsync(x_out, tp->X.as<float>() + (size_t)N * n, sizeof(float) * n, cudaMemcpyDeviceToDevice, st));
    return DSGNLM_OK;
}

// The reverse sweep, queued on the handle's stream up to the read-back of the scalar
// cotangents and of the wait-error flag into the tape's pinned words.
dsgnlm_status backward_begin(lpnp_tape* tp, const float* x_bar, float* y_bar, float* guide_bar) {
    if (!tp || !tp->den || !tp->host || !x_bar || !y_bar || !guide_bar) return DSGNLM_EINVAL;
    dsgnlm* den = tp->den;
    cudaStream_t st = den->stream;
    const int H = tp->H, W = tp->W, N = tp->N, T = tp->T, rs = tp->rs, rp = tp->rp;
    const size_t n = (size_t)H * W;
    const int nh = num_half_offsets(rs);
    // the handle's planes must still hold this tape's K1
    if (den->H != H || den->W != W || den->rs != rs || den->nh != nh) return DSGNLM_EINVAL;
    DevBuf* nbufs[] = {&tp->xh, &tp->vh, &tp->uh, &tp->zh, &tp->g,
                       &tp->gs, &tp->dh[0], &tp->base, &tp->gb};
    for (DevBuf* b : nbufs) TAPE_CK(b->ensure(sizeof(float) * n));
    TAPE_CK(tp->AZ.ensure(sizeof(float) * n * 2 * N));
    TAPE_CK(tp->thp.ensure(sizeof(float) * n * (T > 0 ? T : 1)));
    TAPE_CK(tp->dh0.ensure(sizeof(float) * n * kPairSplit));
    TAPE_CK(tp->Dhat.ensure(sizeof(float) * (size_t)nh * H * plane_pitch(W)));
    // the G planes, later the box sums E on the extended grid (pass B has then read G)
    TAPE_CK(tp->Gp.ensure(sizeof(float) * (size_t)nh *
                          std::max((size_t)H * plane_pitch(W), (size_t)(H + 2 * rp) * (W + 2 * rp))));
    const size_t ne = (size_t)(H + 2 * rp) * (W + 2 * rp);
    TAPE_CK(tp->ge.ensure(sizeof(float) * ne));
    const int nb = nblk(n);
    const dim3 pgrid((W + kAdjTW - 1) / kAdjTW, (H + kAdjTH - 1) / kAdjTH);
    const int npb = (int)(pgrid.x * pgrid.y) * kPairSplit;  // pair-pass blocks (with the offset chunks)
    const dim3 pgrid2((W + 31) / 32, (H + 7) / 8);           // per-pixel passes in 32 x 8 blocks
    const dim3 ggrid((W + kGT - 1) / kGT, (H + kGT - 1) / kGT);  // A^T A tiles
    const int nrb = (int)(pgrid2.x * pgrid2.y);
    const Cover cover{den->plan.partials, den->plan.tiles_x, den->plan.tiles_y, den->plan.splits.n, rs};
    TAPE_CK(tp->rho_part.ensure(sizeof(double) * nrb));
    TAPE_CK(tp->h_part.ensure(sizeof(double) * npb));
    TAPE_CK(tp->m_part.ensure(sizeof(double) * npb));
    TAPE_CK(tp->mh.ensure(sizeof(double) * 3));
    TAPE_CK(cudaMemsetAsync(tp->rho_part.p, 0, sizeof(double) * nrb, st));
    TAPE_CK(cudaMemsetAsync(tp->gs.p, 0, sizeof(float) * n, st));
    TAPE_CK(cudaMemsetAsync(tp->vh.p, 0, sizeof(float) * n, st));
    TAPE_CK(cudaMemsetAsync(tp->uh.p, 0, sizeof(float) * n, st));
    TAPE_CK(cudaMemcpyAsync(tp->xh.p, x_bar, sizeof(float) * n, cudaMemcpyDeviceToDevice, st));
    const float mu = tp->mu, alpha = tp->alpha, rho = tp->rho;
    const float* dT = tp->Dh.as<float>() + (size_t)T * n;
    const float* tT = tp->Th.as<float>() + (size_t)T * n;
    float* A = tp->AZ.as<float>();
    float* Z = A + (size_t)N * n;
    // a_{N-1} = vh - uh = 0 and z_{N-1} = x_N + u_{N-1}; every earlier pair is written by
    // the update of the iteration after it
    adj_az_kernel<<<nb, 256, 0, st>>>((int)n, tp->vh.as<float>(), tp->uh.as<float>(),
                                      tp->X.as<float>() + (size_t)N * n, tp->U.as<float>() + (size_t)(N - 1) * n,
                                      A + (size_t)(N - 1) * n, Z + (size_t)(N - 1) * n);
    count_launches(1);
    TAPE_CK(cudaGetLastError());
    for (int k = N - 1; k >= 0; --k) {
        const float* xk = tp->X.as<float>() + (size_t)k * n;
        const float* vk = tp->V.as<float>() + (size_t)k * n;
        const float* uk = tp->U.as<float>() + (size_t)k * n;
        float* ak = A + (size_t)k * n;
        // W a (W symmetric), finished with g and zh; xbar_k from the recorded grad f(x_k)
        TAPE_CK(launch_tma_gather(den->dtype, den->plan, H, W, rs, dT, ak, den->err.as<unsigned>(), nullptr, st, den->wait_budget));
        adj_wa_g_kernel<<<pgrid2, dim3(32, 8), 0, st>>>(cover, H, W, dT, tT, tp->inv_m_dev(), ak, tp->uh.as<float>(),
                                                        tp->xh.as<float>(), xk, vk, uk,
                                                        tp->Gr.as<float>() + (size_t)k * n, mu, alpha, rho,
                                                        tp->constraint, tp->g.as<float>(), tp->zh.as<float>(),
                                                        tp->rho_part.as<double>());
        count_launches(1);
        TAPE_CK(cudaGetLastError());
        // A^T A g and the updates of the cotangents, with the next (earlier) iteration's inputs
        const bool more = k > 0;
        TAPE_CK(by_blur_radius(tp->taps.r, [&](auto rc) {
            adj_ata_update_kernel<decltype(rc)::value><<<ggrid, 256, 0, st>>>(
                tp->g.as<float>(), H, W, tp->taps, tp->zh.as<float>(), mu, alpha, rho, tp->xh.as<float>(),
                tp->vh.as<float>(), tp->uh.as<float>(), tp->gs.as<float>(), xk, more ? uk - n : nullptr,
                more ? ak - n : nullptr, more ? Z + (size_t)(k - 1) * n : nullptr);
            return cudaGetLastError();
        }));
        count_launches(1);
    }
    // pair passes G and T: the G planes, dh, partials of mh
    double* m_part = tp->m_part.as<double>();
    double* mh = tp->mh.as<double>();
    switch (den->dtype) {
        case DSGNLM_F32: TAPE_CK(pairs_gt<float>(tp, den->planes.p, st, m_part)); break;
        case DSGNLM_F16: TAPE_CK(pairs_gt<__half>(tp, den->planes.p, st, m_part)); break;
        default: TAPE_CK(pairs_gt<__nv_bfloat16>(tp, den->planes.p, st, m_part)); break;
    }
    adj_sum_kernel<<<1, 256, 0, st>>>(m_part, npb, mh);
    count_launches(1);
    TAPE_CK(cudaGetLastError());
    switch (den->dtype) {
        case DSGNLM_F32: TAPE_CK(mterms<float>(tp, den->planes.p, st)); break;
        case DSGNLM_F16: TAPE_CK(mterms<__half>(tp, den->planes.p, st)); break;
        default: TAPE_CK(mterms<__nv_bfloat16>(tp, den->planes.p, st)); break;
    }
    // balancing passes backwards: th^p from the cotangent of d^{p+1}, then K1 th^p; the
    // finish of pass p forms the cotangent of d^p and at once th^{p-1} of the next pass
    // (the cotangent of d^0 = 1 is not needed, so pass 0 has no finish)
    if (T > 0) {
        adj_sk_pre_kernel<<<nb, 256, 0, st>>>((int)n, tp->dh[0].as<float>(), tp->Dh.as<float>() + (size_t)T * n,
                                              tp->Dh.as<float>() + (size_t)(T - 1) * n,
                                              tp->Th.as<float>() + (size_t)(T - 1) * n,
                                              tp->thp.as<float>() + (size_t)(T - 1) * n, tp->base.as<float>());
        count_launches(1);
        TAPE_CK(cudaGetLastError());
    }
    for (int p = T - 1; p >= 0; --p) {
        float* th = tp->thp.as<float>() + (size_t)p * n;
        TAPE_CK(launch_tma_gather(den->dtype, den->plan, H, W, rs, th, nullptr, den->err.as<unsigned>(), nullptr, st, den->wait_budget));
        if (p == 0) break;
        adj_sk_finish_pre_kernel<<<pgrid2, dim3(32, 8), 0, st>>>(
            cover, H, W, th, tp->base.as<float>(), tp->Dh.as<float>() + (size_t)p * n,
            tp->Dh.as<float>() + (size_t)(p - 1) * n, tp->Th.as<float>() + (size_t)(p - 1) * n, th - n);
        count_launches(1);
        TAPE_CK(cudaGetLastError());
    }
    // pair pass B: D-hat planes and dL/dh partials
    switch (den->dtype) {
        case DSGNLM_F32: TAPE_CK(pairs_b<float>(tp, den->planes.p, st)); break;
        case DSGNLM_F16: TAPE_CK(pairs_b<__half>(tp, den->planes.p, st)); break;
        default: TAPE_CK(pairs_b<__nv_bfloat16>(tp, den->planes.p, st)); break;
    }
    // patch distances back to the guide: box sums of the D-hat planes onto the extended
    // grid (reusing the G planes' memory, which pass B has finished with), then the
    // gather of every extended position
    {
        float* E = tp->Gp.as<float>();
        const int DW = kBT + 2 * rp;
        const size_t bsmem = sizeof(float) * (size_t)(DW * DW + DW * kBT);
        TAPE_CK(cudaFuncSetAttribute(adj_box_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bsmem));
        adj_box_kernel<<<dim3((W + 2 * rp + kBT - 1) / kBT, (H + 2 * rp + kBT - 1) / kBT, nh), 256, bsmem, st>>>(
            tp->Dhat.as<float>(), H, W, rp, E);
        const size_t gsmem = sizeof(float) * (size_t)(8 + 2 * rs) * (32 + 2 * rs);
        adj_guide_kernel<<<dim3((W + 2 * rp + 31) / 32, (H + 2 * rp + 7) / 8), dim3(32, 8), gsmem, st>>>(
            E, tp->guide, H, W, rp, rs, tp->ge.as<float>());
        count_launches(2);
        TAPE_CK(cudaGetLastError());
    }
    adj_fold_kernel<<<dim3((W + 31) / 32, (H + 7) / 8), dim3(32, 8), 0, st>>>(
        tp->ge.as<float>(), tp->xh.as<float>(), tp->vh.as<float>(), tp->guide, H, W, rp, guide_bar);
    count_launches(1);
    TAPE_CK(cudaGetLastError());
    // dL/dy = sum_k mu A g_k = A gs
    TAPE_CK(launch_sr_forward(tp->gs.as<float>(), H, W, tp->taps, nullptr, 0.f, y_bar, st));
    adj_sum_kernel<<<1, 256, 0, st>>>(tp->rho_part.as<double>(), nrb, mh + 1);
    adj_sum_kernel<<<1, 256, 0, st>>>(tp->h_part.as<double>(), npb, mh + 2);
    count_launches(2);
    TAPE_CK(cudaGetLastError());
    TAPE_CK(cudaMemcpyAsync(tp->host->hs, mh, sizeof tp->host->hs, cudaMemcpyDeviceToHost, st));
    TAPE_CK(cudaMemcpyAsync(&tp->host->err, den->err.p, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    return DSGNLM_OK;
}

dsgnlm_status backward_finish(lpnp_tape* tp, double* h_bar, double* rho_bar) {
    TAPE_CK(cudaStreamSynchronize(tp->den->stream));
    if (tp->host->err) {
        TAPE_CK(cudaMemsetAsync(tp->den->err.p, 0, sizeof(unsigned), tp->den->stream));
        return DSGNLM_TIMEOUT;
    }
    if (rho_bar) *rho_bar = tp->host->hs[1];
    if (h_bar) *h_bar = tp->host->hs[2];
    return DSGNLM_OK;
}

}  // namespace

extern "C" {

dsgnlm_status lpnp_unrolled_forward(lpnp_tape_t tp, dsgnlm_t den, const float* y, const float* guide, int H, int W,
                                    int patch_r, int search_r, float bandwidth, int balance_passes, float alpha,
                                    float rho, int iters, float blur_sigma, int blur_r, float* x_out) {
    NvtxRange nvtx_range("lpnp_unrolled_forward");
    if (!x_out || !y || !guide) return DSGNLM_EINVAL;
    dsgnlm_status s = forward_begin(tp, den, y, guide, H, W, patch_r, search_r, bandwidth, balance_passes, alpha, rho,
                                    iters, blur_sigma, blur_r, 1);
    if (s == DSGNLM_OK) s = forward_finish(tp, x_out);
    if (s != DSGNLM_OK && den) cudaStreamSynchronize(den->stream);  // nothing left running on the inputs
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
    // each image's weights, balance and iterations, queued from the host pool's threads
    // on its handle's stream; nothing waits for the device (1/m is read there)
    std::vector<dsgnlm_status> st(count, DSGNLM_OK);
    HostPool::run(count, [&](int i) {
        st[i] = forward_begin(tapes[i], dens[i], y[i], guide[i], H, W, patch_r, search_r, bandwidth, balance_passes,
                              alpha, rho, iters, blur_sigma, blur_r, count);
        if (st[i] == DSGNLM_OK) st[i] = forward_finish(tapes[i], x_out[i]);
    });
    for (int i = 0; i < count; ++i)
        if (st[i] != DSGNLM_OK) {
            // on a failure, nothing of the batch is left running on the caller's buffers
            for (int j = 0; j < count; ++j) cudaStreamSynchronize(dens[j]->stream);
            return st[i];
        }
    return DSGNLM_OK;
}

dsgnlm_status lpnp_backward(lpnp_tape_t tp, const float* x_bar, float* y_bar, float* guide_bar, double* h_bar,
                            double* rho_bar) {
    NvtxRange nvtx_range("lpnp_backward");
    if (!x_bar || !y_bar || !guide_bar) return DSGNLM_EINVAL;
    dsgnlm_status s = backward_begin(tp, x_bar, y_bar, guide_bar);
    if (s != DSGNLM_OK) {
        if (tp && tp->den) cudaStreamSynchronize(tp->den->stream);  // nothing left in flight
        return s;
    }
    return backward_finish(tp, h_bar, rho_bar);
}

dsgnlm_status lpnp_backward_batched(lpnp_tape_t* tapes, int count, const float* const* x_bar, float* const* y_bar,
                                    float* const* guide_bar, double* h_bar, double* rho_bar) {
    NvtxRange nvtx_range("lpnp_backward_batched");
    if (!tapes || !x_bar || !y_bar || !guide_bar || count < 1) return DSGNLM_EINVAL;
    for (int i = 0; i < count; ++i) {
        if (!tapes[i]) return DSGNLM_EINVAL;
        for (int j = 0; j < i; ++j)
            if (tapes[j] == tapes[i]) return DSGNLM_EINVAL;
    }
    std::vector<dsgnlm_status> st(count, DSGNLM_OK);
    HostPool::run(count, [&](int i) { st[i] = backward_begin(tapes[i], x_bar[i], y_bar[i], guide_bar[i]); });
    for (int i = 0; i < count; ++i)
        if (st[i] != DSGNLM_OK) {
            for (int j = 0; j < count; ++j)  // nothing left in flight
                if (tapes[j]->den) cudaStreamSynchronize(tapes[j]->den->stream);
            return st[i];
        }
    dsgnlm_status first = DSGNLM_OK;
    for (int i = 0; i < count; ++i) {
        dsgnlm_status r = backward_finish(tapes[i], h_bar ? h_bar + i : nullptr, rho_bar ? rho_bar + i : nullptr);
        if (first == DSGNLM_OK) first = r;
    }
    return first;
}

}  // extern "C"
