// Weight build: fast patch distances and the hat-windowed NLM kernel (Eq. NLM,
// Eq. S1; the first aggregation of Algorithm 2 and the fast patch distances of
// Sec. 3), stored as half-window planes.
//
// One CTA owns a 32 x 32 spatial tile and a chunk of consecutive half-window
// offsets.  It stages the guide tile with the halo every offset of the chunk
// needs (patch radius on all sides plus the search radius downwards and
// sideways; half-window offsets never point upwards) in shared memory once, then
// for each offset o:
//   E(p) = (g(p) - g(p + o))^2                 over the tile + patch halo
//   R(p) = sum_{|t_x| <= r_p} E(p + (0, t_x))   horizontal patch sums
//   D(s) = sum_{|t_y| <= r_p} R(s + (t_y, 0))   vertical patch sums
//   K1(s, s + o) = Lambda(o / (N_s + 1)) exp(-D(s) / (2 N_p^2 h^2)),  0 if s + o is
//   outside the image,
// and writes the plane row-contiguously.  The sums are direct (2 r_p + 1 terms
// each), so every D(s) is computed in the same order wherever the tile
// boundaries fall; the cost per offset is O(r_p), against O(r_p^2) for the
// direct patch sum.
#include "common.cuh"
#include "internal.h"

namespace dsg {

namespace {

constexpr int kTW = 32;   // tile columns (= threadIdx.x)
constexpr int kTH = 32;   // tile rows
constexpr int kBY = 8;    // threadIdx.y
constexpr int kThreads = kTW * kBY;
constexpr int kChunk = 22;  // offsets per CTA

// RP >= 0: patch radius known at compile time; RP < 0: runtime radius rp_rt.
template <typename WT, int RP>
__global__ void __launch_bounds__(kThreads)
build_kernel(const float* __restrict__ guide, int H, int W, int rp_rt, int rs, float c,
             WT* __restrict__ planes) {
    extern __shared__ float smem[];
    const int rp = RP >= 0 ? RP : rp_rt;
    const int nh = num_half_offsets(rs);
    const int y0 = blockIdx.y * kTH;
    const int x0 = blockIdx.x * kTW;
    const int k_begin = blockIdx.z * kChunk;
    const int k_end = min(nh, k_begin + kChunk);

    // staged guide: rows y0 - rp .. y0 + TH + rp + rs - 1,
    //               cols x0 - rp - rs .. x0 + TW + rp + rs - 1
    const int GH = kTH + 2 * rp + rs;
    const int GW = kTW + 2 * rp + 2 * rs;
    const int EH = kTH + 2 * rp;
    const int EW = kTW + 2 * rp;
    float* G = smem;
    float* E = G + GH * GW;
    float* R = E + EH * EW;
    int* rows = reinterpret_cast<int*>(R + EH * kTW);
    int* cols = rows + GH;

    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * kTW + tx;
    for (int a = tid; a < GH; a += kThreads) rows[a] = sym_index(y0 - rp + a, H);
    for (int b = tid; b < GW; b += kThreads) cols[b] = sym_index(x0 - rp - rs + b, W);
    __syncthreads();
    for (int a = ty; a < GH; a += kBY) {
        const float* grow = guide + (size_t)rows[a] * W;
        for (int b = tx; b < GW; b += kTW) G[a * GW + b] = grow[cols[b]];
    }
    __syncthreads();

    const int Wp = plane_pitch(W);
    const size_t plane = (size_t)H * Wp;
    const float inv_hat = 1.0f / (float)(rs + 1);
    for (int k = k_begin; k < k_end; ++k) {
        int oy, ox;
        half_offset(k, rs, oy, ox);
        // E(p) = (g(p) - g(p + o))^2 over the tile + patch halo
        for (int ey = ty; ey < EH; ey += kBY) {
            const float* ga = G + ey * GW + rs;
            const float* gb = G + (ey + oy) * GW + rs + ox;
            for (int ex = tx; ex < EW; ex += kTW) {
                const float df = ga[ex] - gb[ex];
                E[ey * EW + ex] = df * df;
            }
        }
        __syncthreads();
        // R(p) = sum over the 2 rp + 1 columns of the patch row
        for (int ry = ty; ry < EH; ry += kBY) {
            const float* e = E + ry * EW + tx;
            float acc = 0.f;
#pragma unroll
            for (int t = 0; t <= 2 * (RP >= 0 ? RP : 0); ++t) acc += e[t];
            if (RP < 0)
                for (int t = 1; t <= 2 * rp; ++t) acc += e[t];
            R[ry * kTW + tx] = acc;
        }
        __syncthreads();
        const float hat = (1.0f - fabsf((float)oy) * inv_hat) * (1.0f - fabsf((float)ox) * inv_hat);
        WT* out = planes + (size_t)k * plane;
        const int j = x0 + tx;
        const bool col_ok = j < W && j + ox >= 0 && j + ox < W;
        for (int py = ty; py < kTH; py += kBY) {
            const int i = y0 + py;
            if (i >= H || j >= W) continue;
            const float* r = R + py * kTW + tx;
            float D = 0.f;
#pragma unroll
            for (int t = 0; t <= 2 * (RP >= 0 ? RP : 0); ++t) D += r[t * kTW];
            if (RP < 0)
                for (int t = 1; t <= 2 * rp; ++t) D += r[t * kTW];
            const bool inside = col_ok && (i + oy < H);
            const float w = inside ? hat * __expf(-D * c) : 0.f;
            out[(size_t)i * Wp + j] = from_f32<WT>(w);
        }
        // E is rewritten next while R is still being read: they are distinct
        // buffers, and R is rewritten only after the next barrier.
    }
}

template <typename WT, int RP>
cudaError_t launch_build_rp(const float* guide, int H, int W, int rp, int rs, float c, WT* planes,
                            cudaStream_t st) {
    const int nh = num_half_offsets(rs);
    if (nh == 0) return cudaSuccess;
    const int GH = kTH + 2 * rp + rs, GW = kTW + 2 * rp + 2 * rs;
    const int EH = kTH + 2 * rp, EW = kTW + 2 * rp;
    const size_t smem = sizeof(float) * (size_t)(GH * GW + EH * EW + EH * kTW) + sizeof(int) * (GH + GW);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(build_kernel<WT, RP>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((W + kTW - 1) / kTW, (H + kTH - 1) / kTH, (nh + kChunk - 1) / kChunk);
    build_kernel<WT, RP><<<grid, dim3(kTW, kBY), smem, st>>>(guide, H, W, rp, rs, c, planes);
    count_launches(1);
    return cudaGetLastError();
}

template <typename WT>
cudaError_t launch_build_t(const float* guide, int H, int W, int rp, int rs, float c, WT* planes,
                           cudaStream_t st) {
    switch (rp) {
        case 1: return launch_build_rp<WT, 1>(guide, H, W, rp, rs, c, planes, st);
        case 2: return launch_build_rp<WT, 2>(guide, H, W, rp, rs, c, planes, st);
        case 3: return launch_build_rp<WT, 3>(guide, H, W, rp, rs, c, planes, st);
        case 4: return launch_build_rp<WT, 4>(guide, H, W, rp, rs, c, planes, st);
        case 5: return launch_build_rp<WT, 5>(guide, H, W, rp, rs, c, planes, st);
        default: return launch_build_rp<WT, -1>(guide, H, W, rp, rs, c, planes, st);
    }
}

}  // namespace

cudaError_t launch_build(int dtype, const float* guide, int H, int W, int patch_r, int search_r,
                         float c, void* planes, cudaStream_t st) {
    switch (dtype) {
        case 0: return launch_build_t(guide, H, W, patch_r, search_r, c, (float*)planes, st);
        case 1: return launch_build_t(guide, H, W, patch_r, search_r, c, (__half*)planes, st);
        default: return launch_build_t(guide, H, W, patch_r, search_r, c, (__nv_bfloat16*)planes, st);
    }
}

}  // namespace dsg
