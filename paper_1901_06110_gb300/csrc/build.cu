// Weight build: fast patch distances and the hat-windowed NLM kernel (Eq. NLM,
// Eq. S1; the first aggregation of Algorithm 2 and the fast patch distances of
// Sec. 3), stored as half-window planes.
//
// One CTA owns a 32 x 64 spatial tile and a chunk of consecutive half-window
// offsets.  It stages the guide tile with the halo every offset of the chunk
// needs (patch radius on all sides plus the search radius downwards and
// sideways; half-window offsets never point upwards) in shared memory once, then
// for each offset o:
//   V(p) = sum_{|t_y| <= r_p} (g(p + (t_y, 0)) - g(p + (t_y, 0) + o))^2
//          vertical patch sums, as a sliding window down a column over 8
//          consecutive outputs (one direct sum, then one add and one subtract
//          per output), one thread per column, and
//   D(s) = sum_{|t_x| <= r_p} V(s + (0, t_x))   horizontal patch sums,
//   K1(s, s + o) = Lambda(o / (N_s + 1)) exp(-D(s) / (2 N_p^2 h^2)),  0 if s + o is
//   outside the image,
// and writes the plane row-contiguously.  Segments sit at fixed positions of the
// image grid (tiles are aligned to 8), so results do not depend on scheduling.
#include "common.cuh"
#include "internal.h"

namespace dsg {

namespace {

constexpr int kTW = 64;    // tile columns
constexpr int kTH = 32;    // tile rows
constexpr int kThreads = 256;
constexpr int kSeg = 8;    // outputs per sliding-window segment
constexpr int kChunk = 22; // offsets per CTA
constexpr int kMaxRp = 10; // DSGNLM_MAX_PATCH_R

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
    const int EW = kTW + 2 * rp;
    float* G = smem;
    float* V = G + GH * GW;  // vertical patch sums, [kTH][EW]
    int* rows = reinterpret_cast<int*>(V + kTH * EW);
    int* cols = rows + GH;

    const int tid = threadIdx.x;
    for (int a = tid; a < GH; a += kThreads) rows[a] = sym_index(y0 - rp + a, H);
    for (int b = tid; b < GW; b += kThreads) cols[b] = sym_index(x0 - rp - rs + b, W);
    __syncthreads();
    {
        const int tx = tid & 63, ty = tid >> 6;
        for (int a = ty; a < GH; a += 4) {
            const float* grow = guide + (size_t)rows[a] * W;
            for (int b = tx; b < GW; b += 64) G[a * GW + b] = grow[cols[b]];
        }
    }
    __syncthreads();

    const int Wp = plane_pitch(W);
    const size_t plane = (size_t)H * Wp;
    const float inv_hat = 1.0f / (float)(rs + 1);
    const int n_vtask = EW * (kTH / kSeg);
    const int hx = tid & 63, hy = tid >> 6;  // horizontal phase: column, 8-row segment
    for (int k = k_begin; k < k_end; ++k) {
        int oy, ox;
        half_offset(k, rs, oy, ox);
        // V(i, c) = sum_{t_y} (g(i + t_y, c) - g(i + t_y + o_y, c + o_x))^2: one column and
        // 8 consecutive output rows per task, as a sliding window down the column
        for (int task = tid; task < n_vtask; task += kThreads) {
            const int seg = task / EW;
            const int cc = task - seg * EW;
            const int r0 = seg * kSeg;  // first output row; staged row r0 + t is image row y0 - rp + r0 + t
            const float* ga = G + r0 * GW + cc + rs;
            const float* gb = G + (r0 + oy) * GW + cc + rs + ox;
            float e[kSeg + 2 * kMaxRp];
            const int ne = kSeg + 2 * rp;
#pragma unroll
            for (int t = 0; t < kSeg + 2 * (RP >= 0 ? RP : kMaxRp); ++t) {
                if (RP < 0 && t >= ne) break;
                const float df = ga[t * GW] - gb[t * GW];
                e[t] = df * df;
            }
            float acc = 0.f;
#pragma unroll
            for (int t = 0; t <= 2 * (RP >= 0 ? RP : kMaxRp); ++t) {
                if (RP < 0 && t > 2 * rp) break;
                acc += e[t];
            }
            V[r0 * EW + cc] = acc;
#pragma unroll
            for (int q = 1; q < kSeg; ++q) {
                acc += e[q + 2 * rp] - e[q - 1];
                V[(r0 + q) * EW + cc] = acc;
            }
        }
        __syncthreads();
        // D(i, j) = sum_{t_x} V(i, j + t_x), then the weight
        const float hat = (1.0f - fabsf((float)oy) * inv_hat) * (1.0f - fabsf((float)ox) * inv_hat);
        WT* out = planes + (size_t)k * plane;
        const int j = x0 + hx;
        const bool col_ok = j < W && j + ox >= 0 && j + ox < W;
#pragma unroll
        for (int q = 0; q < kSeg; ++q) {
            const int r = hy * kSeg + q;
            const float* vr = V + r * EW + hx;
            float D = 0.f;
#pragma unroll
            for (int t = 0; t <= 2 * (RP >= 0 ? RP : kMaxRp); ++t) {
                if (RP < 0 && t > 2 * rp) break;
                D += vr[t];
            }
            const int i = y0 + r;
            if (i < H && j < W) {
                const bool inside = col_ok && (i + oy < H);
                const float w = inside ? hat * __expf(-D * c) : 0.f;
                out[(size_t)i * Wp + j] = from_f32<WT>(w);
            }
        }
        __syncthreads();  // V is rewritten by the next offset
    }
}

template <typename WT, int RP>
cudaError_t launch_build_rp(const float* guide, int H, int W, int rp, int rs, float c, WT* planes,
                            cudaStream_t st) {
    const int nh = num_half_offsets(rs);
    if (nh == 0) return cudaSuccess;
    const int GH = kTH + 2 * rp + rs, GW = kTW + 2 * rp + 2 * rs;
    const int EW = kTW + 2 * rp;
    const size_t smem = sizeof(float) * (size_t)(GH * GW + kTH * EW) + sizeof(int) * (GH + GW);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(build_kernel<WT, RP>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((W + kTW - 1) / kTW, (H + kTH - 1) / kTH, (nh + kChunk - 1) / kChunk);
    build_kernel<WT, RP><<<grid, kThreads, smem, st>>>(guide, H, W, rp, rs, c, planes);
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
