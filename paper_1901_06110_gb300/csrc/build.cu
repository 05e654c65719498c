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
//          vertical patch sums, as a sliding window down a column over 16
//          consecutive outputs (one direct sum, then one add and one subtract
//          per output), one thread per column and segment, and
//   D(s) = sum_{|t_x| <= r_p} V(s + (0, t_x))   horizontal patch sums, as a
//          sliding window along a row over 4 consecutive outputs per thread
//          (16-byte shared-memory loads, one 4-wide store per row),
//   K1(s, s + o) = Lambda(o / (N_s + 1)) exp(-D(s) / (2 N_p^2 h^2)),  0 if s + o is
//   outside the image,
// and writes the plane row-contiguously.  V is double-buffered: the vertical sums
// of offset k + 1 are formed in the same interval as the horizontal sums of
// offset k, so each offset costs one barrier.  Segments sit at fixed positions of
// the image grid (tiles are aligned to 16), so results do not depend on scheduling.
// A CTA takes a chunk of consecutive offsets, sized at launch so that the grid
// fills whole waves of resident CTAs; tiles whose pixels and offset partners all lie
// inside the image skip the per-pixel bounds test.
#include <mutex>
#include <utility>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace dsg {

namespace {

constexpr int kTW = 64;    // tile columns
constexpr int kTH = 32;    // tile rows
constexpr int kThreads = 256;
constexpr int kSeg = 16;   // outputs per vertical sliding-window segment
constexpr int kHW = 4;     // outputs per horizontal sliding window (one thread, one row)
constexpr int kMaxRp = 14; // DSGNLM_MAX_PATCH_R

// row length of the vertical sums: the tile plus the patch radius on both sides,
// rounded up so that every window start is 16-byte aligned and a window's last
// 16-byte load stays inside the row
__host__ __device__ constexpr int v_pitch(int rp) { return ((kTW + 2 * rp + 3) / 4) * 4 + 4; }
// The vertical sums of rows 16..31 start 16 floats further on, and the staged guide has an
// odd row pitch: a warp's vertical tasks alternate between the two row segments (lanes
// 2c and 2c + 1 take column c), and the two segments' accesses then fall in different
// banks (16 rows apart is 16 banks apart).
__host__ __device__ constexpr int v_row(int r, int vp) { return r * vp + (r >= kSeg ? 16 : 0); }
__host__ __device__ constexpr int v_floats(int rp) { return kTH * v_pitch(rp) + 16; }
__host__ __device__ constexpr int g_pitch(int rp, int rs) { return (kTW + 2 * rp + 2 * rs) | 1; }

template <typename WT>
__device__ __forceinline__ void store4(WT* p, const float (&w)[kHW]);
template <>
__device__ __forceinline__ void store4<float>(float* p, const float (&w)[kHW]) {
    *reinterpret_cast<float4*>(p) = make_float4(w[0], w[1], w[2], w[3]);
}
template <>
__device__ __forceinline__ void store4<__half>(__half* p, const float (&w)[kHW]) {
    __half2 a = __floats2half2_rn(w[0], w[1]), b = __floats2half2_rn(w[2], w[3]);
    uint2 u;
    u.x = *reinterpret_cast<unsigned*>(&a);
    u.y = *reinterpret_cast<unsigned*>(&b);
    *reinterpret_cast<uint2*>(p) = u;
}
template <>
__device__ __forceinline__ void store4<__nv_bfloat16>(__nv_bfloat16* p, const float (&w)[kHW]) {
    __nv_bfloat162 a = __floats2bfloat162_rn(w[0], w[1]), b = __floats2bfloat162_rn(w[2], w[3]);
    uint2 u;
    u.x = *reinterpret_cast<unsigned*>(&a);
    u.y = *reinterpret_cast<unsigned*>(&b);
    *reinterpret_cast<uint2*>(p) = u;
}

// 2^x by the hardware's approximate base-2 exponential (relative error about 2^-22)
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// RP >= 0: patch radius known at compile time; RP < 0: runtime radius rp_rt.  RS >= 0:
// search radius known at compile time (the staged guide's row stride and every
// shared-memory address offset of the vertical sums are then constants); RS < 0:
// runtime radius rs_rt.
template <typename WT, int RP, int RS>
__global__ void __launch_bounds__(kThreads, RP < 0 ? 1 : (RP <= 5 ? 4 : 3))
build_kernel(const float* __restrict__ guide, int H, int W, int rp_rt, int rs_rt, float c2, int chunk,
             WT* __restrict__ planes, long long cap, const BuildJob* __restrict__ jobs, int zchunks) {
    extern __shared__ __align__(16) float smem[];
    const int rp = RP >= 0 ? RP : rp_rt;
    const int rs = RS >= 0 ? RS : rs_rt;
    const int nh = num_half_offsets(rs);
    const int y0 = blockIdx.y * kTH;
    const int x0 = blockIdx.x * kTW;
    int kz = blockIdx.z;
    if (jobs) {  // batched: grid z = image x offset chunk
        const int img = blockIdx.z / zchunks;
        kz = blockIdx.z - img * zchunks;
        guide = jobs[img].guide;
        planes = static_cast<WT*>(jobs[img].planes);
        cap = jobs[img].cap;
        c2 = jobs[img].c2;
    }
    const int k_begin = kz * chunk;
    const int k_end = min(nh, k_begin + chunk);

    // staged guide: rows y0 - rp .. y0 + TH + rp + rs - 1,
    //               cols x0 - rp - rs .. x0 + TW + rp + rs - 1
    const int GH = kTH + 2 * rp + rs;
    const int GW = g_pitch(rp, rs);
    const int EW = kTW + 2 * rp;  // vertical sums per row: tile columns -rp .. TW + rp - 1
    const int VP = v_pitch(rp);
    float* V0 = smem;  // two buffers of vertical sums, [kTH][VP] each (rows 16.. staggered by 16)
    float* V1 = V0 + v_floats(rp);
    float* G = V1 + v_floats(rp);
    int* rows = reinterpret_cast<int*>(G + GH * GW);
    int* cols = rows + GH;

    const int tid = threadIdx.x;
    for (int a = tid; a < GH; a += kThreads) rows[a] = sym_index(y0 - rp + a, H);
    for (int b = tid; b < GW; b += kThreads) cols[b] = sym_index(x0 - rp - rs + b, W);
    for (int i = tid; i < 2 * v_floats(rp); i += kThreads) V0[i] = 0.f;  // the row tails are read, never used
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
    // the weight Lambda(o) exp(-D c) as one base-2 exponential: 2^(log2 Lambda(o) - D c
    // log2 e), with c2 = c log2 e from the host and log2 Lambda(o) once per offset
    const int n_vtask = EW * (kTH / kSeg);
    // V(i, cc) = sum_{t_y} (g(i + t_y, cc - rp) - g(i + t_y + o_y, cc - rp + o_x))^2 for the
    // tile's rows: one column and 8 consecutive output rows per task, as a sliding
    // window down the column (staged row r0 + t is image row y0 - rp + r0 + t)
    // every thread has at most one vertical task (2 (kTW + 2 r_p) <= kThreads), the same
    // for every offset: with the patch radius known at compile time, its own guide
    // column g(i + t_y, cc - rp) is read once into registers and kept for all offsets
    constexpr int kNG = RP >= 0 ? kSeg + 2 * RP : 1;
    float gown[kNG];
    if constexpr (RP >= 0) {
        if (tid < n_vtask) {
            const int seg = tid & 1, cc = tid >> 1;
            const float* ga = G + seg * kSeg * GW + cc + rs;
#pragma unroll
            for (int t = 0; t < kNG; ++t) gown[t] = ga[t * GW];
        }
    }
    auto vertical = [&](int oy, int ox, float* V) {
        for (int task = tid; task < n_vtask; task += kThreads) {
            const int seg = task & 1;  // lanes alternate between the two segments
            const int cc = task >> 1;
            const int r0 = seg * kSeg;
            const float* ga = G + r0 * GW + cc + rs;
            const float* gb = G + (r0 + oy) * GW + cc + rs + ox;
            float e[kSeg + 2 * kMaxRp];
            const int ne = kSeg + 2 * rp;
#pragma unroll
            for (int t = 0; t < kSeg + 2 * (RP >= 0 ? RP : kMaxRp); ++t) {
                if (RP < 0 && t >= ne) break;
                float a;
                if constexpr (RP >= 0)
                    a = gown[t];
                else
                    a = ga[t * GW];
                const float df = a - gb[t * GW];
                e[t] = df * df;
            }
            float acc = 0.f;
#pragma unroll
            for (int t = 0; t <= 2 * (RP >= 0 ? RP : kMaxRp); ++t) {
                if (RP < 0 && t > 2 * rp) break;
                acc += e[t];
            }
            float* Vs = V + v_row(r0, VP) + cc;
            Vs[0] = acc;
#pragma unroll
            for (int q = 1; q < kSeg; ++q) {
                acc += e[q + 2 * rp] - e[q - 1];
                Vs[q * VP] = acc;
            }
        }
    };
    // horizontal phase: thread = 4 consecutive columns (group hg) of rows hr and hr + 16
    const int hg = tid & 15, hr = tid >> 4;
    const int j0 = x0 + kHW * hg;
    constexpr int kNV = (kHW + 2 * (RP >= 0 ? RP : kMaxRp) + 3) / 4;  // 16-byte loads per window
    const int nv = (kHW + 2 * rp + 3) / 4;

    // the tile and every offset's partner pixel lie inside the image (half-window
    // offsets point down or sideways): no output needs the bounds test
    const bool interior = y0 + kTH + rs <= H && x0 >= rs && x0 + kTW + rs <= W;
    // offsets k and k + 1, advanced in half-window order (o_y = 0, o_x = 1..rs, then
    // o_y = 1.., o_x = -rs..rs)
    int oy, ox, oy1, ox1;
    half_offset(k_begin, rs, oy, ox);
    auto next_offset = [&](int& y, int& x) {
        if (++x > rs) {
            ++y;
            x = -rs;
        }
    };
    oy1 = oy;
    ox1 = ox;
    next_offset(oy1, ox1);
    if (k_begin < k_end) vertical(oy, ox, V0);
    __syncthreads();
    for (int k = k_begin; k < k_end; ++k) {
        float* Vc = ((k - k_begin) & 1) ? V1 : V0;
        float* Vn = ((k - k_begin) & 1) ? V0 : V1;
        if (k + 1 < k_end) vertical(oy1, ox1, Vn);  // in the same interval as the sums below
        // D(i, j) = sum_{t_x} V(i, j + t_x), then the weight
        const float lhat = __log2f((1.0f - fabsf((float)oy) * inv_hat) * (1.0f - fabsf((float)ox) * inv_hat));
        // columns whose partner j + o_x lies inside the image, and the rows whose partner does
        const int jlo = ox < 0 ? -ox : 0, jhi = ox > 0 ? W - ox : W;
        const int ihi = H - oy;
        WT* out = planes + (size_t)k * plane;
#pragma unroll
        for (int rr = 0; rr < kTH / 16; ++rr) {
            const int r = hr + 16 * rr;
            const int i = y0 + r;
            const float4* vr = reinterpret_cast<const float4*>(Vc + v_row(r, VP) + kHW * hg);
            float v[4 * kNV];
#pragma unroll
            for (int q = 0; q < kNV; ++q) {
                if (RP < 0 && q >= nv) break;
                const float4 f = vr[q];
                v[4 * q] = f.x;
                v[4 * q + 1] = f.y;
                v[4 * q + 2] = f.z;
                v[4 * q + 3] = f.w;
            }
            float D = 0.f;
#pragma unroll
            for (int t = 0; t <= 2 * (RP >= 0 ? RP : kMaxRp); ++t) {
                if (RP < 0 && t > 2 * rp) break;
                D += v[t];
            }
            float w[kHW];
            if (interior || (i < ihi && j0 >= jlo && j0 + kHW <= jhi)) {
#pragma unroll
                for (int jj = 0; jj < kHW; ++jj) {
                    if (jj > 0) D += v[jj + 2 * rp] - v[jj - 1];
                    w[jj] = ex2_approx(fmaf(D, -c2, lhat));
                }
                if (DSG_IN_RANGE((size_t)k * plane + (size_t)i * Wp + j0 + kHW - 1, cap, kChkPlanes))
                    store4<WT>(out + (size_t)i * Wp + j0, w);
            } else {
#pragma unroll
                for (int jj = 0; jj < kHW; ++jj) {
                    if (jj > 0) D += v[jj + 2 * rp] - v[jj - 1];
                    const int j = j0 + jj;
                    const bool inside = i < H && j < W && j + ox >= 0 && j + ox < W && i + oy < H;
                    w[jj] = inside ? ex2_approx(fmaf(D, -c2, lhat)) : 0.f;
                }
                // planes have a pitch of a multiple of 8: the 4 outputs are all inside the
                // row's pitch or all outside it
                if (i < H && j0 < Wp &&
                    DSG_IN_RANGE((size_t)k * plane + (size_t)i * Wp + j0 + kHW - 1, cap, kChkPlanes))
                    store4<WT>(out + (size_t)i * Wp + j0, w);
            }
        }
        oy = oy1;
        ox = ox1;
        next_offset(oy1, ox1);
        __syncthreads();  // Vc is rewritten two offsets on; Vn is complete
    }
}

// Resident CTAs on the device of one build instantiation at its shared-memory size
// (queried once per size; the size's attribute is set before)
template <typename WT, int RP, int RS>
int build_ctas_per_sm(size_t smem) {
    static std::mutex mu;
    static std::vector<std::pair<size_t, int>> known;
    std::lock_guard<std::mutex> lock(mu);
    for (const auto& kv : known)
        if (kv.first == smem) return kv.second;
    int per_sm = 0, dev = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, build_kernel<WT, RP, RS>, kThreads, smem) !=
            cudaSuccess ||
        cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess)
        return 0;
    const int slots = per_sm * sms;
    known.emplace_back(smem, slots);
    return slots;
}

// count == 0: one image (guide, planes, cap); count > 0: `count` images from `jobs`
template <typename WT, int RP, int RS>
cudaError_t launch_build_rp(const float* guide, int H, int W, int rp, int rs, float c, WT* planes, long long cap,
                            const BuildJob* jobs, int count, cudaStream_t st) {
    const int nh = num_half_offsets(rs);
    if (nh == 0) return cudaSuccess;
    const int GH = kTH + 2 * rp + rs, GW = kTW + 2 * rp + 2 * rs;
    const int GWp = g_pitch(rp, rs);
    const size_t smem = sizeof(float) * (size_t)(GH * GWp + 2 * v_floats(rp)) + sizeof(int) * (GH + GWp);
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(build_kernel<WT, RP, RS>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int slots_i = build_ctas_per_sm<WT, RP, RS>(smem);
    if (slots_i <= 0) {
        const cudaError_t e = cudaGetLastError();
        return e != cudaSuccess ? e : cudaErrorInvalidConfiguration;
    }
    // offsets per CTA: the chunk that makes the fewest waves of resident CTAs take the
    // least time (each CTA also stages its guide tile, worth about two offsets)
    const long long slots = slots_i;
    const int images = count > 0 ? count : 1;
    const long long tiles = (long long)((W + kTW - 1) / kTW) * ((H + kTH - 1) / kTH) * images;
    int chunk = nh;
    long long best = -1;
    for (int ch = 1; ch <= nh; ++ch) {
        const long long ctas = tiles * ((nh + ch - 1) / ch);
        const long long cost = ((ctas + slots - 1) / slots) * (ch + 2);
        if (best < 0 || cost < best) {
            best = cost;
            chunk = ch;
        }
    }
    const int zchunks = (nh + chunk - 1) / chunk;
    dim3 grid((W + kTW - 1) / kTW, (H + kTH - 1) / kTH, zchunks * images);
    const float c2 = (float)((double)c * 1.4426950408889634);  // c log2 e: the exponent in base 2
    build_kernel<WT, RP, RS><<<grid, kThreads, smem, st>>>(guide, H, W, rp, rs, c2, chunk, planes, cap,
                                                           count > 0 ? jobs : nullptr, zchunks);
    count_launches(1);
    return cudaGetLastError();
}

// Search radii with their own instantiations: the windows of the workloads (11x11,
// 15x15, 21x21) for the patch sizes they use, and the 21x21 window for every patch size
// of Table 1; other radii take the runtime-radius form.
template <typename WT, int RP>
cudaError_t launch_build_rs(const float* guide, int H, int W, int rp, int rs, float c, WT* planes, long long cap,
                            const BuildJob* jobs, int count, cudaStream_t st) {
    if constexpr (RP == 2) {
        if (rs == 5) return launch_build_rp<WT, RP, 5>(guide, H, W, rp, rs, c, planes, cap, jobs, count, st);
        if (rs == 7) return launch_build_rp<WT, RP, 7>(guide, H, W, rp, rs, c, planes, cap, jobs, count, st);
    }
    if constexpr (RP == 3 || RP == 5 || RP == 8 || RP == 11 || RP == 14) {
        if (rs == 10) return launch_build_rp<WT, RP, 10>(guide, H, W, rp, rs, c, planes, cap, jobs, count, st);
    }
    return launch_build_rp<WT, RP, -1>(guide, H, W, rp, rs, c, planes, cap, jobs, count, st);
}

template <typename WT>
cudaError_t launch_build_t(const float* guide, int H, int W, int rp, int rs, float c, WT* planes, long long cap,
                           const BuildJob* jobs, int count, cudaStream_t st) {
    switch (rp) {
        case 1: return launch_build_rs<WT, 1>(guide, H, W, rp, rs, c, planes, cap, jobs, count, st);
        case 2: return launch_build_rs<WT, 2>(guide, H, W, rp, rs, c, planes, cap, jobs, count, st);
        case 3: return launch_build_rs<WT, 3>(guide, H, W, rp, rs, c, planes, cap, jobs, count, st);
        case 4: return launch_build_rs<WT, 4>(guide, H, W, rp, rs, c, planes, cap, jobs, count, st);
        case 5: return launch_build_rs<WT, 5>(guide, H, W, rp, rs, c, planes, cap, jobs, count, st);
        // 17 x 17, 23 x 23 and 29 x 29 patches
        case 8: return launch_build_rs<WT, 8>(guide, H, W, rp, rs, c, planes, cap, jobs, count, st);
        case 11: return launch_build_rs<WT, 11>(guide, H, W, rp, rs, c, planes, cap, jobs, count, st);
        case 14: return launch_build_rs<WT, 14>(guide, H, W, rp, rs, c, planes, cap, jobs, count, st);
        default: return launch_build_rp<WT, -1, -1>(guide, H, W, rp, rs, c, planes, cap, jobs, count, st);
    }
}

}  // namespace

DSG_CHECK_WORD_ACCESSOR(check_word_build)

cudaError_t launch_build(int dtype, const float* guide, int H, int W, int patch_r, int search_r,
                         float c, void* planes, long long cap, cudaStream_t st) {
    switch (dtype) {
        case 0: return launch_build_t(guide, H, W, patch_r, search_r, c, (float*)planes, cap, nullptr, 0, st);
        case 1: return launch_build_t(guide, H, W, patch_r, search_r, c, (__half*)planes, cap, nullptr, 0, st);
        default:
            return launch_build_t(guide, H, W, patch_r, search_r, c, (__nv_bfloat16*)planes, cap, nullptr, 0, st);
    }
}

cudaError_t launch_build_batched(int dtype, const BuildJob* jobs, int count, int H, int W, int patch_r,
                                 int search_r, float c, cudaStream_t st) {
    if (!jobs || count < 1) return cudaErrorInvalidValue;
    switch (dtype) {
        case 0: return launch_build_t<float>(nullptr, H, W, patch_r, search_r, c, nullptr, 0, jobs, count, st);
        case 1: return launch_build_t<__half>(nullptr, H, W, patch_r, search_r, c, nullptr, 0, jobs, count, st);
        default:
            return launch_build_t<__nv_bfloat16>(nullptr, H, W, patch_r, search_r, c, nullptr, 0, jobs, count, st);
    }
}

}  // namespace dsg
