// C ABI implementation: handle management, argument checks, the balancing control
// loop and the Algorithm 1 iteration loop.  Only host code lives here; every step
// of the method runs in the kernels of build.cu, stencil.cu and lpnp.cu.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "../../include/dsgnlm.h"
#include "common.cuh"
#include "handle.h"
#include "internal.h"

namespace dsg {
static std::atomic<uint64_t> g_launches{0};
static thread_local bool g_capturing = false;  // launches recorded into a graph are counted at replay
static thread_local uint64_t g_recorded = 0;   // launches recorded since set_capture_counting(true)
void count_launches(uint64_t n) {
    if (!g_capturing)
        g_launches.fetch_add(n, std::memory_order_relaxed);
    else
        g_recorded += n;
}
void set_capture_counting(bool recording) {
    g_capturing = recording;
    if (recording) g_recorded = 0;
}
uint64_t recorded_launches() { return g_recorded; }
// Tensor map of planes [nh][H][pitch] of the storage type `dtype`, pitch in elements
// (plane_pitch(W) when 0); the tensor's rows are W wide, so boxes read zeros past
// column W - 1 (and past row H - 1, and before row or column 0).
cudaError_t encode_tile_map(void* out, const void* base, int dtype, int H, int W, int nh, int box_w, int box_h,
                            int pitch) {
    // looked up once (a thread-safe static initialisation)
    static const PFN_cuTensorMapEncodeTiled_v12000 encode = [] {
        cudaDriverEntryPointQueryResult q;
        void* fn = nullptr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                         cudaEnableDefault, &q);
        return (e == cudaSuccess && q == cudaDriverEntryPointSuccess) ? (PFN_cuTensorMapEncodeTiled_v12000)fn
                                                                      : nullptr;
    }();
    if (!encode) return cudaErrorNotSupported;
    const size_t esz = dtype == DSGNLM_F32 ? 4 : 2;
    const CUtensorMapDataType dt = dtype == DSGNLM_F32   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : dtype == DSGNLM_F16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                         : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    const cuuint64_t dims[3] = {(cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)nh};
    const cuuint64_t pe = pitch > 0 ? (cuuint64_t)pitch : (cuuint64_t)plane_pitch(W);
    const cuuint64_t strides[2] = {pe * esz, pe * H * esz};
    const cuuint32_t box[3] = {(cuuint32_t)box_w, (cuuint32_t)box_h, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = encode((CUtensorMap*)out, dt, 3, const_cast<void*>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}
}  // namespace dsg

using namespace dsg;

namespace {

thread_local int g_last_cuda = 0;

}  // namespace

void dsg::record_cuda_error(cudaError_t e) { g_last_cuda = (int)e; }

namespace dsg {

DSG_CHECK_WORD_ACCESSOR(check_word_api)

namespace {
__global__ void check_selftest_kernel(long long index, long long bound) {
    (void)DSG_IN_RANGE(index, bound, kChkSelfTest);
}
}  // namespace

cudaError_t launch_check_selftest(long long index, long long bound) {
    check_selftest_kernel<<<1, 1>>>(index, bound);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace dsg

namespace {

dsgnlm_status fail_cuda(cudaError_t e) {
    g_last_cuda = (int)e;
    return e == cudaErrorMemoryAllocation ? DSGNLM_ENOMEM : DSGNLM_ECUDA;
}

#define DSG_CK(expr)                                  \
    do {                                              \
        cudaError_t e_ = (expr);                      \
        if (e_ != cudaSuccess) return fail_cuda(e_);  \
    } while (0)

// Tensor map of the weight planes [n_h][H][pitch] for the TMA stencil path.
cudaError_t encode_planes_map(void* out, void* planes, int dtype, int H, int W, int nh) {
    return encode_tile_map(out, planes, dtype, H, W, nh, tma_tile_w(), tma_tile_h());
}

// Split the column offsets -rs..rs into `n` contiguous slices of about equal
// offset counts (a column offset o_x carries rs offsets for o_x <= 0 and rs + 1
// for o_x > 0).
TmaSplits make_splits(int rs, int n) {
    TmaSplits t{};
    const int groups = 2 * rs + 1;
    n = n < 1 ? 1 : (n > groups ? groups : n);
    if (n > kMaxSlices) n = kMaxSlices;
    const int total = num_half_offsets(rs);
    int ox = -rs, cum = 0;
    for (int sl = 0; sl < n; ++sl) {
        t.ox_lo[sl] = ox;
        const int target = (int)(((long long)total * (sl + 1) + n - 1) / n);
        // leave at least one column offset for each remaining slice
        const int last_allowed = rs - (n - 1 - sl);
        while (true) {
            cum += ox > 0 ? rs + 1 : rs;
            if (ox >= last_allowed || cum >= target) break;
            ++ox;
        }
        t.ox_hi[sl] = ox;
        ++ox;
    }
    t.ox_hi[n - 1] = rs;
    t.n = n;
    return t;
}

}  // namespace

extern "C" {

dsgnlm_status dsgnlm_create(dsgnlm_t* out, void* stream, int weight_dtype) {
    if (!out) return DSGNLM_EINVAL;
    *out = nullptr;
    if (weight_dtype != DSGNLM_F32 && weight_dtype != DSGNLM_F16 && weight_dtype != DSGNLM_BF16)
        return DSGNLM_EINVAL;
    dsgnlm* h = new (std::nothrow) dsgnlm();
    if (!h) return DSGNLM_ENOMEM;
    h->stream = (cudaStream_t)stream;
    h->dtype = weight_dtype;
    *out = h;
    return DSGNLM_OK;
}

void dsgnlm_destroy(dsgnlm_t h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    h->release_all();
    delete h;
}

dsgnlm_status dsgnlm_set_stream(dsgnlm_t h, void* stream) {
    if (!h) return DSGNLM_EINVAL;
    h->stream = (cudaStream_t)stream;
    return DSGNLM_OK;
}

int dsgnlm_num_offsets(dsgnlm_t h) { return (h && h->built) ? h->nh : 0; }

dsgnlm_status dsgnlm_build(dsgnlm_t h, const float* guide, int H, int W, int patch_r,
                           int search_r, float bandwidth) {
    NvtxRange nvtx_range("dsgnlm_build");
    return build_handle(h, guide, H, W, patch_r, search_r, bandwidth, true);
}

}  // extern "C"

namespace dsg {

dsgnlm_status build_handle(dsgnlm* h, const float* guide, int H, int W, int patch_r, int search_r, float bandwidth,
                           bool launch) {
    if (!h || !guide || !aligned16(guide)) return DSGNLM_EINVAL;
    if (H < 1 || W < 1 || (size_t)H * (size_t)W > (size_t)1 << 31) return DSGNLM_EINVAL;
    if (patch_r < 0 || patch_r > DSGNLM_MAX_PATCH_R) return DSGNLM_EINVAL;
    if (search_r < 0 || search_r > DSGNLM_MAX_SEARCH_R) return DSGNLM_EINVAL;
    if (!(bandwidth > 0.f) || !std::isfinite(bandwidth)) return DSGNLM_EINVAL;
    const int nh = num_half_offsets(search_r);
    const int Wp = plane_pitch(W);
    const size_t bytes = (size_t)nh * (size_t)H * (size_t)Wp * weight_elem_bytes(h->dtype);
    h->built = false;
    h->balanced = false;
    h->inv_m_dev = false;
    h->fast = false;
    DSG_CK(h->planes.ensure(bytes));
    const double np = 2.0 * patch_r + 1.0;
    const float c = (float)(1.0 / (2.0 * np * np * (double)bandwidth * (double)bandwidth));
    if (launch)
        DSG_CK(h->timed(DSGNLM_PROF_BUILD, [&] {
            return launch_build(h->dtype, guide, H, W, patch_r, search_r, c, h->planes.p,
                                (long long)(h->planes.bytes / weight_elem_bytes(h->dtype)), h->stream);
        }));
    h->H = H;
    h->W = W;
    h->Wp = Wp;
    h->rp = patch_r;
    h->rs = search_r;
    h->nh = nh;
    h->bw = bandwidth;
    if (tma_path_supports(search_r)) {
        if (!h->num_sms) {
            int dev = 0;
            DSG_CK(cudaGetDevice(&dev));
            DSG_CK(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev));
        }
        TmaPlan& pl = h->plan;
        DSG_CK(encode_planes_map(pl.tmap, h->planes.p, h->dtype, H, W, nh));
        pl.tiles_x = (W + tma_tile_w() - 1) / tma_tile_w();
        pl.tiles_y = (H + tma_tile_h() - 1) / tma_tile_h();
        const int tiles = pl.tiles_x * pl.tiles_y;
        // about one CTA per resident slot (two per SM for FP32 weights, three for
        // 16-bit weights): split the offsets when tiles are scarce, counting the tiles
        // of the images that run beside this one
        int slices = (tma_ctas_per_sm(h->dtype) * h->num_sms) / (tiles * (h->share > 1 ? h->share : 1));
        pl.splits = make_splits(search_r, slices < 1 ? 1 : slices);
        DSG_CK(h->tma_part.ensure(sizeof(float) * tma_region_floats(search_r) * (size_t)tiles * pl.splits.n));
        pl.partials = h->tma_part.as<float>();
        pl.part_cap = (long long)(h->tma_part.bytes / sizeof(float));
        DSG_CK(h->err.ensure(sizeof(unsigned)));
        DSG_CK(cudaMemsetAsync(h->err.p, 0, sizeof(unsigned), h->stream));
        h->fast = true;
    }
    h->built = true;
    h->m_pending = nullptr;
    return DSGNLM_OK;
}

}  // namespace dsg

namespace {

// m and 1/m of a W whose balance ran elsewhere (m_pending): read back once, when a
// call first needs them on the host.
dsgnlm_status settle_m(dsgnlm* h) {
    if (!h->m_pending) return DSGNLM_OK;
    float mm[2] = {1.f, 1.f};
    DSG_CK(cudaStreamSynchronize(h->stream));
    DSG_CK(cudaMemcpy(mm, h->m_pending, sizeof mm, cudaMemcpyDeviceToHost));
    h->m = mm[0];
    h->inv_m = mm[1];
    h->m_pending = nullptr;
    return DSGNLM_OK;
}

// A phase-1 wait gave up during the call: clear the error word (so that the next
// call starts clean) and report it.
dsgnlm_status wait_timeout(dsgnlm* h, cudaStream_t st) {
    const cudaError_t e = cudaMemsetAsync(h->err.p, 0, sizeof(unsigned), st);
    if (e == cudaSuccess) cudaStreamSynchronize(st);
    return DSGNLM_TIMEOUT;
}

// Passes of the accelerated balance: two plain symmetric Sinkhorn steps, then
// Polyak's heavy-ball step on u = log d with the parameters that are optimal for a
// linear error map whose matrix (I + S) / 2 has its spectrum in [1/2, 1]; S, the
// balanced kernel, is symmetric, doubly stochastic and positive semidefinite (the
// Gaussian kernel of patch distances times the separable hat, a Schur product of
// positive semidefinite matrices), so its spectrum lies in [0, 1].  With
// q = sqrt(1/2): relax = 4 / (1 + q)^2, momentum = ((1 - q) / (1 + q))^2, a
// contraction of (1 - q) / (1 + q) = 0.17 per pass near the fixed point against
// 1/2 for the plain step.  The fixed point, d (K1 d) = 1, is that of the plain step.
void set_pass_rule(BalanceCtl& c, int scheme) {
    if (scheme != DSGNLM_BALANCE_ACCELERATED) return;  // zeros: the plain step in every pass
    const double q = std::sqrt(0.5);
    c.relax = (float)(4.0 / ((1.0 + q) * (1.0 + q)));
    c.momentum = (float)(((1.0 - q) / (1.0 + q)) * ((1.0 - q) / (1.0 + q)));
    c.plain_passes = 2;
}

// One balancing pass of the TMA path: phase-1 gather of K1 d, then the epilogue
// (next d, t, residual maxima and, in its last block, the decision).  `parity`
// selects the d and t buffers.
cudaError_t balance_pass(dsgnlm* h, int parity, cudaStream_t st, cudaGraphConditionalHandle cond, int use_cond) {
    BalanceCtl* ctl = h->ctl.as<BalanceCtl>();
    float* d_in = h->dbuf[parity].as<float>();
    float* d_out = h->dbuf[parity ^ 1].as<float>();
    cudaError_t e = launch_tma_gather(h->dtype, h->plan, h->H, h->W, h->rs, d_in, nullptr, h->err.as<unsigned>(),
                                      &ctl->done, st, h->wait_budget);
    if (e != cudaSuccess) return e;
    return launch_balance_epilogue(h->plan, h->H, h->W, h->rs, d_in, d_out, h->tbuf[parity].as<float>(),
                                   h->bal_part.as<float2>(), ctl, 1, cond, use_cond, st);
}

// Everything a recorded balance graph depends on.
void balance_key(const dsgnlm* h, unsigned char out[256]) {
    std::memset(out, 0, 256);
    const void* ptrs[9] = {h->planes.p, h->dbuf[0].p, h->dbuf[1].p, h->tbuf[0].p, h->tbuf[1].p,
                           h->bal_part.p, h->ctl.p, h->err.p, h->plan.partials};
    const int ints[5] = {h->H, h->W, h->rs, h->dtype, h->plan.splits.n};
    std::memcpy(out, ptrs, sizeof ptrs);
    std::memcpy(out + sizeof ptrs, ints, sizeof ints);
    std::memcpy(out + 128, h->plan.tmap, 128);
}

// Record the passes once as a graph: a WHILE node whose body holds two passes
// (even and odd buffers); the decision kernel clears the condition when the
// balance stops, and kernels after the stop return at once.
cudaError_t ensure_balance_graph(dsgnlm* h) {
    unsigned char key[256];
    balance_key(h, key);
    if (h->bal_exec && std::memcmp(key, h->bal_key, 256) == 0) return cudaSuccess;
    h->release_graphs();
    cudaError_t e = cudaSuccess;
    if (!h->cap_stream) {
        e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return e;
    }
    cudaGraph_t g = nullptr;
    e = cudaGraphCreate(&g, 0);
    if (e != cudaSuccess) return e;
    cudaGraphConditionalHandle cond;
    e = cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = cond;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    if (e == cudaSuccess) e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
    if (e == cudaSuccess) {
        cudaGraph_t body = np.conditional.phGraph_out[0];
        e = cudaStreamBeginCaptureToGraph(h->cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
        if (e == cudaSuccess) {
            g_capturing = true;
            cudaError_t e1 = balance_pass(h, 0, h->cap_stream, cond, 1);
            if (e1 == cudaSuccess) e1 = balance_pass(h, 1, h->cap_stream, cond, 1);
            g_capturing = false;
            cudaGraph_t captured = body;
            e = cudaStreamEndCapture(h->cap_stream, &captured);
            if (e == cudaSuccess) e = e1;
        }
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&h->bal_exec, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        h->bal_exec = nullptr;
        (void)cudaGetLastError();
        return e;
    }
    h->bal_graph = g;
    std::memcpy(h->bal_key, key, 256);
    return cudaSuccess;
}

}  // namespace

extern "C" {

dsgnlm_status dsgnlm_balance(dsgnlm_t h, double tol, int maxit, int* iters_out, double* resid_out) {
    NvtxRange nvtx_range("dsgnlm_balance");
    if (!h) return DSGNLM_EINVAL;
    if (!h->built) return DSGNLM_NOT_BUILT;
    if (!(tol >= 0.0) || maxit < 0 || maxit > 1000000) return DSGNLM_EINVAL;
    const size_t n = (size_t)h->H * h->W;
    h->balanced = false;
    h->inv_m_dev = false;
    DSG_CK(h->dbuf[0].ensure(n * sizeof(float)));
    DSG_CK(h->dbuf[1].ensure(n * sizeof(float)));
    if (h->fast) {
        DSG_CK(h->tbuf[0].ensure(n * sizeof(float)));
        DSG_CK(h->tbuf[1].ensure(n * sizeof(float)));
        DSG_CK(h->bal_part.ensure(sizeof(float2) * (size_t)balance_combine_blocks(h->H, h->W)));
    } else {
        DSG_CK(h->stats.ensure(sizeof(PassStat) * (size_t)(maxit + 1)));
        DSG_CK(cudaMemsetAsync(h->stats.p, 0, sizeof(PassStat) * (size_t)(maxit + 1), h->stream));
    }
    DSG_CK(h->ctl.ensure(sizeof(BalanceCtl)));
    DSG_CK(h->stage(sizeof(BalanceCtl) + sizeof(PassStat)));
    BalanceCtl c0{};
    c0.done = 0;
    c0.final_pass = -1;
    c0.status = 0;
    c0.since_best = 0;
    c0.best = INFINITY;
    c0.tol = tol;
    c0.maxit = maxit;
    c0.pass = 0;
    if (h->fast) set_pass_rule(c0, h->balance_scheme);
    std::memcpy(h->host_stage, &c0, sizeof c0);
    DSG_CK(cudaMemcpyAsync(h->ctl.p, h->host_stage, sizeof c0, cudaMemcpyHostToDevice, h->stream));
    DSG_CK(launch_fill(h->dbuf[0].as<float>(), 1.0f, n, h->stream));

    BalanceCtl c{};
    bool ran = false;
    if (h->fast && !h->bal_graph_failed) {
        if (ensure_balance_graph(h) == cudaSuccess) {
            DSG_CK(h->timed(DSGNLM_PROF_BALANCE, [&] { return cudaGraphLaunch(h->bal_exec, h->stream); }));
            DSG_CK(cudaMemcpyAsync(h->host_stage, h->ctl.p, sizeof c, cudaMemcpyDeviceToHost, h->stream));
            DSG_CK(cudaStreamSynchronize(h->stream));
            std::memcpy(&c, h->host_stage, sizeof c);
            // each WHILE iteration runs two passes of two kernels
            if (c.done) count_launches(4 * (uint64_t)((c.final_pass + 2) / 2));
            ran = true;
        } else {
            h->bal_graph_failed = true;  // conditional graphs unavailable: launch passes from the host
        }
    }
    if (!ran) {
        // Passes are launched in groups; a pass launched after the deciding one
        // returns at once (the done flag is checked on entry), so the group size
        // only trades wasted launches against host round trips.
        const int group = 4;
        for (int pass = 0; pass <= maxit; ++pass) {
            DSG_CK(h->timed(DSGNLM_PROF_BALANCE, [&] {
                if (h->fast) return balance_pass(h, pass & 1, h->stream, 0, 0);
                return launch_sinkhorn_pass(h->dtype, h->planes.p, h->H, h->W, h->rs, h->dbuf[pass & 1].as<float>(),
                                            h->dbuf[(pass + 1) & 1].as<float>(), h->stats.as<PassStat>(),
                                            h->ctl.as<BalanceCtl>(), pass, h->stream);
            }));
            if ((pass + 1) % group == 0 || pass == maxit) {
                DSG_CK(cudaMemcpyAsync(h->host_stage, h->ctl.p, sizeof c, cudaMemcpyDeviceToHost, h->stream));
                DSG_CK(cudaStreamSynchronize(h->stream));
                std::memcpy(&c, h->host_stage, sizeof c);
                if (c.done) break;
            }
        }
    }
    if (!c.done || c.final_pass < 0) return DSGNLM_ECUDA;  // cannot happen: pass maxit decides
    double eps = c.eps, m = c.m;
    if (h->fast) {
        unsigned errv = 0;
        DSG_CK(cudaMemcpy(&errv, h->err.p, sizeof errv, cudaMemcpyDeviceToHost));
        if (errv) return wait_timeout(h, h->stream);
        h->t_final = h->tbuf[c.final_pass & 1].as<float>();
    } else {
        PassStat ps{};
        DSG_CK(cudaMemcpyAsync(h->host_stage, h->stats.as<PassStat>() + c.final_pass, sizeof ps,
                               cudaMemcpyDeviceToHost, h->stream));
        DSG_CK(cudaStreamSynchronize(h->stream));
        std::memcpy(&ps, h->host_stage, sizeof ps);
        std::memcpy(&eps, &ps.eps_bits, sizeof eps);
        std::memcpy(&m, &ps.m_bits, sizeof m);
    }
    h->d_final = h->dbuf[c.final_pass & 1].as<float>();
    h->m = m;
    h->inv_m = (float)(1.0 / m);
    h->m_pending = nullptr;
    h->inv_m_dev = h->fast;  // the TMA path's control block holds the same 1/m
    h->iters = c.final_pass;
    h->resid = eps;
    h->balanced = true;
    if (iters_out) *iters_out = c.final_pass;
    if (resid_out) *resid_out = eps;
    if (c.status == 6) return DSGNLM_NOT_CONVERGED;
    if (c.status == 7) return DSGNLM_STALLED;
    return DSGNLM_OK;
}

dsgnlm_status dsgnlm_balance_batched(dsgnlm_t* hs, int count, double tol, int maxit, int slices, int* iters_out,
                                     double* resid_out, int* status_out) {
    NvtxRange nvtx_range("dsgnlm_balance_batched");
    if (!hs || count < 1 || count > kMaxBatch || slices < 0) return DSGNLM_EINVAL;
    if (!(tol >= 0.0) || maxit < 0 || maxit > 1000000) return DSGNLM_EINVAL;
    for (int i = 0; i < count; ++i) {
        dsgnlm* h = hs[i];
        if (!h) return DSGNLM_EINVAL;
        if (!h->built) return DSGNLM_NOT_BUILT;
        if (!h->fast || h->dtype != hs[0]->dtype || h->rs != hs[0]->rs) return DSGNLM_EINVAL;
        for (int j = 0; j < i; ++j)
            if (hs[j] == h) return DSGNLM_EINVAL;
    }
    dsgnlm* lead = hs[0];
    cudaStream_t st = lead->stream;
    for (int i = 1; i < count; ++i)  // work queued on other streams (their builds) comes first
        if (hs[i]->stream != st) DSG_CK(cudaStreamSynchronize(hs[i]->stream));
    std::vector<BatchInst> inst(2 * (size_t)count);
    std::vector<BatchBal> bal(count);
    std::vector<int4> work1, work2;
    BatchMaps maps;
    DSG_CK(lead->stage(sizeof(BalanceCtl) * (size_t)count));
    BalanceCtl* c0 = static_cast<BalanceCtl*>(lead->host_stage);
    for (int i = 0; i < count; ++i) {
        dsgnlm* h = hs[i];
        const int H = h->H, W = h->W;
        const size_t n = (size_t)H * W;
        const int nbx = (W + 31) / 32, nby = (H + 15) / 16;  // the 16 x 32 epilogue blocks
        if (nbx * nby != balance_combine_blocks(H, W)) return DSGNLM_EINVAL;
        h->balanced = false;
        h->inv_m_dev = false;
        DSG_CK(h->dbuf[0].ensure(n * sizeof(float)));
        DSG_CK(h->dbuf[1].ensure(n * sizeof(float)));
        DSG_CK(h->tbuf[0].ensure(n * sizeof(float)));
        DSG_CK(h->tbuf[1].ensure(n * sizeof(float)));
        DSG_CK(h->bal_part.ensure(sizeof(float2) * (size_t)balance_combine_blocks(H, W)));
        DSG_CK(h->ctl.ensure(sizeof(BalanceCtl)));
        BalanceCtl& c = c0[i];
        c = BalanceCtl{};
        c.final_pass = -1;
        c.best = INFINITY;
        c.tol = tol;
        c.maxit = maxit;
        set_pass_rule(c, h->balance_scheme);
        DSG_CK(cudaMemcpyAsync(h->ctl.p, &c, sizeof c, cudaMemcpyHostToDevice, st));
        DSG_CK(launch_fill(h->dbuf[0].as<float>(), 1.0f, n, st));
        std::memcpy(maps.m[i], h->plan.tmap, 128);
        const TmaSplits splits = slices > 0 ? make_splits(h->rs, slices) : h->plan.splits;
        const size_t tiles = (size_t)h->plan.tiles_x * h->plan.tiles_y;
        DSG_CK(h->tma_part.ensure(sizeof(float) * tma_region_floats(h->rs) * tiles * splits.n));
        h->plan.partials = h->tma_part.as<float>();  // the buffer may have grown
        h->plan.part_cap = (long long)(h->tma_part.bytes / sizeof(float));
        for (int par = 0; par < 2; ++par) {
            BatchInst& bi = inst[(size_t)par * count + i];
            bi = BatchInst{};
            bi.H = H;
            bi.W = W;
            bi.tiles_x = h->plan.tiles_x;
            bi.tiles_y = h->plan.tiles_y;
            bi.splits = splits;
            bi.d = h->dbuf[par].as<float>();
            bi.z = nullptr;
            bi.part = h->plan.partials;
            bi.part_cap = h->plan.part_cap;
            bi.done = &h->ctl.as<BalanceCtl>()->done;
        }
        BatchBal& b = bal[i];
        b.cv = Cover{h->plan.partials, h->plan.tiles_x, h->plan.tiles_y, splits.n, h->rs, h->plan.part_cap};
        b.H = H;
        b.W = W;
        b.nbx = nbx;
        b.nblocks = nbx * nby;
        for (int par = 0; par < 2; ++par) {
            b.d[par] = h->dbuf[par].as<float>();
            b.t[par] = h->tbuf[par].as<float>();
        }
        b.part = h->bal_part.as<float2>();
        b.ctl = h->ctl.as<BalanceCtl>();
        for (int sl = 0; sl < splits.n; ++sl)
            for (int ty = 0; ty < h->plan.tiles_y; ++ty)
                for (int tx = 0; tx < h->plan.tiles_x; ++tx) work1.push_back(make_int4(i, ty, tx, sl));
        for (int by = 0; by < nby; ++by)
            for (int bx = 0; bx < nbx; ++bx) work2.push_back(make_int4(i, by, bx, 0));
    }
    DSG_CK(lead->bb_inst.ensure(sizeof(BatchInst) * inst.size()));
    DSG_CK(lead->bb_bal.ensure(sizeof(BatchBal) * bal.size()));
    DSG_CK(lead->bb_work1.ensure(sizeof(int4) * work1.size()));
    DSG_CK(lead->bb_work2.ensure(sizeof(int4) * work2.size()));
    DSG_CK(lead->bb_flag.ensure(sizeof(unsigned)));
    DSG_CK(cudaMemcpyAsync(lead->bb_inst.p, inst.data(), sizeof(BatchInst) * inst.size(), cudaMemcpyHostToDevice, st));
    DSG_CK(cudaMemcpyAsync(lead->bb_bal.p, bal.data(), sizeof(BatchBal) * bal.size(), cudaMemcpyHostToDevice, st));
    DSG_CK(cudaMemcpyAsync(lead->bb_work1.p, work1.data(), sizeof(int4) * work1.size(), cudaMemcpyHostToDevice, st));
    DSG_CK(cudaMemcpyAsync(lead->bb_work2.p, work2.data(), sizeof(int4) * work2.size(), cudaMemcpyHostToDevice, st));
    DSG_CK(cudaMemsetAsync(lead->bb_flag.p, 0, sizeof(unsigned), st));
    DSG_CK(cudaMemsetAsync(lead->err.p, 0, sizeof(unsigned), st));
    // Passes in groups of four between host checks of the stopped count; an image's
    // items return at once after the pass that stops it.
    const BatchInst* dinst = lead->bb_inst.as<BatchInst>();
    const int n1 = (int)work1.size(), n2 = (int)work2.size();
    unsigned* stopped = lead->bb_flag.as<unsigned>();
    for (int pass = 0; pass <= maxit; ++pass) {
        const int par = pass & 1;
        DSG_CK(lead->timed(DSGNLM_PROF_BALANCE, [&] {
            cudaError_t e = launch_tma_gather_batched(lead->dtype, lead->rs, maps, dinst + (size_t)par * count,
                                                      lead->bb_work1.as<int4>(), n1, lead->err.as<unsigned>(), st);
            if (e != cudaSuccess) return e;
            return launch_batched_balance_epilogue(lead->bb_bal.as<BatchBal>(), lead->bb_work2.as<int4>(), n2, par,
                                                   stopped, st);
        }));
        if ((pass + 1) % 4 == 0 || pass == maxit) {
            unsigned done = 0;
            DSG_CK(cudaMemcpyAsync(lead->host_stage, stopped, sizeof done, cudaMemcpyDeviceToHost, st));
            DSG_CK(cudaStreamSynchronize(st));
            std::memcpy(&done, lead->host_stage, sizeof done);
            if (done >= (unsigned)count) break;
        }
    }
    for (int i = 0; i < count; ++i)
        DSG_CK(cudaMemcpyAsync(c0 + i, hs[i]->ctl.p, sizeof(BalanceCtl), cudaMemcpyDeviceToHost, st));
    unsigned errv = 0;
    DSG_CK(cudaMemcpyAsync(&errv, lead->err.p, sizeof errv, cudaMemcpyDeviceToHost, st));
    DSG_CK(cudaStreamSynchronize(st));
    if (errv) return wait_timeout(lead, st);
    for (int i = 0; i < count; ++i) {
        const BalanceCtl& c = c0[i];
        if (!c.done || c.final_pass < 0) return DSGNLM_ECUDA;  // cannot happen: pass maxit decides
        dsgnlm* h = hs[i];
        h->t_final = h->tbuf[c.final_pass & 1].as<float>();
        h->d_final = h->dbuf[c.final_pass & 1].as<float>();
        h->m = c.m;
        h->inv_m = (float)(1.0 / c.m);
        h->m_pending = nullptr;
        h->inv_m_dev = true;
        h->iters = c.final_pass;
        h->resid = c.eps;
        h->balanced = true;
        if (iters_out) iters_out[i] = c.final_pass;
        if (resid_out) resid_out[i] = c.eps;
        if (status_out)
            status_out[i] = c.status == 6 ? DSGNLM_NOT_CONVERGED : c.status == 7 ? DSGNLM_STALLED : DSGNLM_OK;
    }
    return DSGNLM_OK;
}

dsgnlm_status dsgnlm_apply(dsgnlm_t h, const float* x, float* y) {
    if (!h || !x || !y || x == y || !aligned16(x) || !aligned16(y)) return DSGNLM_EINVAL;
    if (!h->built) return DSGNLM_NOT_BUILT;
    if (!h->balanced) return DSGNLM_NOT_BALANCED;
    {
        const dsgnlm_status ms = settle_m(h);
        if (ms != DSGNLM_OK) return ms;
    }
    DSG_CK(h->timed(DSGNLM_PROF_APPLY, [&] {
        if (h->fast) {
            cudaError_t e = launch_tma_gather(h->dtype, h->plan, h->H, h->W, h->rs, h->d_final, x,
                                              h->err.as<unsigned>(), nullptr, h->stream, h->wait_budget);
            if (e != cudaSuccess) return e;
            return launch_tma_apply_finish(h->plan, h->H, h->W, h->rs, h->d_final, h->t_final, h->inv_m, x,
                                           y, h->stream);
        }
        return launch_apply(h->dtype, h->planes.p, h->H, h->W, h->rs, h->d_final, h->inv_m, x, y,
                            h->stream);
    }));
    return DSGNLM_OK;
}

dsgnlm_status dsgnlm_set_wait_budget(dsgnlm_t h, long long cycles) {
    if (!h || cycles > dsg::kDefaultWaitBudget) return DSGNLM_EINVAL;
    const long long b = cycles < 0 ? dsg::kDefaultWaitBudget : cycles;
    if (b != h->wait_budget) {
        // recorded graphs carry the budget in their kernel parameters
        DSG_CK(cudaStreamSynchronize(h->stream));
        h->release_graphs();
        h->wait_budget = b;
    }
    return DSGNLM_OK;
}

dsgnlm_status dsgnlm_set_balance_scheme(dsgnlm_t h, int scheme) {
    if (!h || (scheme != DSGNLM_BALANCE_SINKHORN && scheme != DSGNLM_BALANCE_ACCELERATED)) return DSGNLM_EINVAL;
    h->balance_scheme = scheme;
    return DSGNLM_OK;
}

dsgnlm_status dsgnlm_sync(dsgnlm_t h) {
    if (!h) return DSGNLM_EINVAL;
    DSG_CK(cudaStreamSynchronize(h->stream));
    if (!h->err.p) return DSGNLM_OK;
    unsigned errv = 0;
    DSG_CK(cudaMemcpy(&errv, h->err.p, sizeof errv, cudaMemcpyDeviceToHost));
    if (errv) return wait_timeout(h, h->stream);
    return DSGNLM_OK;
}

dsgnlm_status dsgnlm_copy_weights(dsgnlm_t h, void* dst) {
    if (!h || !dst) return DSGNLM_EINVAL;
    if (!h->built) return DSGNLM_NOT_BUILT;
    const size_t esz = weight_elem_bytes(h->dtype);
    if (h->nh)
        DSG_CK(cudaMemcpy2DAsync(dst, (size_t)h->W * esz, h->planes.p, (size_t)h->Wp * esz, (size_t)h->W * esz,
                                 (size_t)h->nh * h->H, cudaMemcpyDeviceToDevice, h->stream));
    return DSGNLM_OK;
}

dsgnlm_status dsgnlm_copy_scaling(dsgnlm_t h, float* d_dst, double* m_host) {
    if (!h) return DSGNLM_EINVAL;
    if (!h->built) return DSGNLM_NOT_BUILT;
    if (!h->balanced) return DSGNLM_NOT_BALANCED;
    {
        const dsgnlm_status ms = settle_m(h);
        if (ms != DSGNLM_OK) return ms;
    }
    if (d_dst)
        DSG_CK(cudaMemcpyAsync(d_dst, h->d_final, sizeof(float) * (size_t)h->H * h->W,
                               cudaMemcpyDeviceToDevice, h->stream));
    DSG_CK(cudaStreamSynchronize(h->stream));
    if (m_host) *m_host = h->m;
    return DSGNLM_OK;
}

dsgnlm_status lpnp_sr_observe(const float* x, const float* noise, int H, int W, float blur_sigma,
                              int blur_r, float* y, void* stream) {
    if (!x || !y || H < 2 || W < 2 || (H & 1) || (W & 1)) return DSGNLM_EINVAL;
    if (blur_r < 0 || blur_r > 8 || !(blur_sigma > 0.f)) return DSGNLM_EINVAL;
    DSG_CK(launch_sr_forward(x, H, W, make_blur_taps(blur_sigma, blur_r), noise, 1.0f, y,
                             (cudaStream_t)stream));
    return DSGNLM_OK;
}

dsgnlm_status lpnp_sr_observe_bc(const float* x, const float* noise, int H, int W, float blur_sigma, int blur_r,
                                 int boundary, float* y, void* stream) {
    if (boundary == LPNP_BC_PERIODIC) return lpnp_sr_observe(x, noise, H, W, blur_sigma, blur_r, y, stream);
    if (boundary != LPNP_BC_SYMMETRIC) return DSGNLM_EINVAL;
    if (!x || !y || H < 2 || W < 2 || (H & 1) || (W & 1)) return DSGNLM_EINVAL;
    if (blur_r < 0 || blur_r > 8 || !(blur_sigma > 0.f) || !sr_bc_supported(H, W, blur_r)) return DSGNLM_EINVAL;
    DSG_CK(launch_sr_forward_bc(1, x, H, W, make_blur_taps(blur_sigma, blur_r), noise, 1.0f, y,
                                (cudaStream_t)stream));
    return DSGNLM_OK;
}

dsgnlm_status lpnp_sr_guide(const float* y, int h, int w, float* guide, void* stream) {
    if (!y || !guide || h < 1 || w < 1) return DSGNLM_EINVAL;
    DSG_CK(launch_sr_guide(y, h, w, guide, (cudaStream_t)stream));
    return DSGNLM_OK;
}

dsgnlm_status lpnp_spi_observe(const float* x, const float* arrivals, int H, int W, int k_side,
                               float eta, uint8_t* bits, void* stream) {
    if (!x || !arrivals || !bits || H < 1 || W < 1 || k_side < 1 || k_side > 15 || !(eta > 0.f))
        return DSGNLM_EINVAL;
    DSG_CK(launch_spi_observe(x, arrivals, H, W, k_side, eta, bits, (cudaStream_t)stream));
    return DSGNLM_OK;
}

dsgnlm_status lpnp_spi_counts(const uint8_t* bits, int H, int W, int k_side, uint8_t* counts,
                              void* stream) {
    if (!bits || !counts || H < 1 || W < 1 || k_side < 1 || k_side > 15) return DSGNLM_EINVAL;
    DSG_CK(launch_spi_counts(bits, H, W, k_side, counts, (cudaStream_t)stream));
    return DSGNLM_OK;
}

dsgnlm_status lpnp_spi_guide(const uint8_t* counts, int H, int W, int K, float eta, float* guide,
                             void* stream) {
    if (!counts || !guide || H < 1 || W < 1 || K < 1 || K > 255 || !(eta > 0.f)) return DSGNLM_EINVAL;
    DSG_CK(launch_spi_guide(counts, H, W, K, eta, guide, (cudaStream_t)stream));
    return DSGNLM_OK;
}

dsgnlm_status lpnp_init(const float* guide, int n, float* x, float* v, float* u, void* stream) {
    if (!guide || !x || !v || !u || n < 1) return DSGNLM_EINVAL;
    DSG_CK(launch_init(guide, n, x, v, u, (cudaStream_t)stream));
    return DSGNLM_OK;
}

}  // extern "C"

namespace {

// Checks the data-term fields; with `for_solve` also the iterate buffers and, with
// `need_w`, the denoiser state.
dsgnlm_status check_problem(const lpnp_problem* p, bool for_solve, bool need_w = true) {
    if (!p || !p->den || p->H < 1 || p->W < 1) return DSGNLM_EINVAL;
    if (for_solve) {
        if (!p->x || !p->v || !p->u) return DSGNLM_EINVAL;
        if (!aligned16(p->x) || !aligned16(p->v) || !aligned16(p->u)) return DSGNLM_EINVAL;
        if (p->x == p->v || p->x == p->u || p->v == p->u) return DSGNLM_EINVAL;
        if (p->constraint < LPNP_C_NONE || p->constraint > LPNP_C_BOX01) return DSGNLM_EINVAL;
        if (!(p->alpha >= 0.f) || !std::isfinite(p->alpha)) return DSGNLM_EINVAL;
        if (need_w) {
            if (!p->den->built) return DSGNLM_NOT_BUILT;
            if (!p->den->balanced) return DSGNLM_NOT_BALANCED;
            if (p->H != p->den->H || p->W != p->den->W) return DSGNLM_EINVAL;
        }
    }
    if (p->kind == LPNP_SR2) {
        if (!p->y || (p->H & 1) || (p->W & 1)) return DSGNLM_EINVAL;
        if (p->blur_r < 0 || p->blur_r > 8 || !(p->blur_sigma > 0.f)) return DSGNLM_EINVAL;
        if (p->blur_boundary != LPNP_BC_PERIODIC && p->blur_boundary != LPNP_BC_SYMMETRIC) return DSGNLM_EINVAL;
        if (p->blur_boundary == LPNP_BC_SYMMETRIC && !sr_bc_supported(p->H, p->W, p->blur_r))
            return DSGNLM_EINVAL;
    } else if (p->kind == LPNP_SPI) {
        if (!p->counts || p->K < 1 || p->K > 255 || !(p->eta > 0.f) || !(p->spi_eps > 0.f))
            return DSGNLM_EINVAL;
    } else {
        return DSGNLM_EINVAL;
    }
    // a W balanced by the unrolled forward: its m and 1/m are needed on the host
    if (for_solve && need_w) return settle_m(p->den);
    return DSGNLM_OK;
}

}  // namespace

extern "C" {

dsgnlm_status lpnp_gradient(const lpnp_problem* p, const float* x, float* grad) {
    dsgnlm_status s = check_problem(p, false);
    if (s != DSGNLM_OK) return s;
    if (!x || !grad) return DSGNLM_EINVAL;
    dsgnlm* h = p->den;
    if (p->kind == LPNP_SR2) {
        DSG_CK(h->rlo.ensure(sizeof(float) * (size_t)(p->H / 2) * (p->W / 2)));
        const BlurTaps taps = make_blur_taps(p->blur_sigma, p->blur_r);
        if (p->blur_boundary == LPNP_BC_SYMMETRIC) {
            DSG_CK(launch_sr_forward_bc(1, x, p->H, p->W, taps, p->y, -1.0f, h->rlo.as<float>(), h->stream));
            DSG_CK(launch_sr_adjoint_bc(1, h->rlo.as<float>(), p->H, p->W, taps, 0.f, nullptr, grad, nullptr,
                                        h->stream));
        } else {
            DSG_CK(launch_sr_forward(x, p->H, p->W, taps, p->y, -1.0f, h->rlo.as<float>(), h->stream));
            DSG_CK(launch_sr_adjoint(h->rlo.as<float>(), p->H, p->W, taps, grad, h->stream));
        }
    } else {
        DSG_CK(launch_spi_grad(x, p->counts, p->H * p->W, p->K, p->eta, p->spi_eps, grad, h->stream));
    }
    return DSGNLM_OK;
}

}  // extern "C"

namespace {

// W rebuilt from the denoiser input (Sec. 4, A-DSG-NLM and the adapt-then-freeze
// schedule): in iterations k < iters the weights are built from z = x + u and
// balanced before W z is formed.
struct Adapt {
    int iters, patch_r, search_r;
    float bandwidth;
    double tol;
    int maxit;
};

// Build from the handle's z and balance; NOT_CONVERGED and STALLED still leave W
// exactly doubly stochastic and are accepted.
dsgnlm_status adapt_w(dsgnlm* h, const Adapt& ad, int H, int W) {
    dsgnlm_status s = dsgnlm_build(h, h->z.as<float>(), H, W, ad.patch_r, ad.search_r, ad.bandwidth);
    if (s != DSGNLM_OK) return s;
    s = dsgnlm_balance(h, ad.tol, ad.maxit, nullptr, nullptr);
    return (s == DSGNLM_NOT_CONVERGED || s == DSGNLM_STALLED) ? DSGNLM_OK : s;
}

template <typename T>
void key_put(std::vector<unsigned char>& k, const T& v) {
    const unsigned char* b = reinterpret_cast<const unsigned char*>(&v);
    k.insert(k.end(), b, b + sizeof(T));
}

dsgnlm_status solve_impl(const lpnp_problem* p, float rho, int iters, const Adapt* ad) {
    dsgnlm_status s = check_problem(p, true, ad == nullptr);
    if (s != DSGNLM_OK) return s;
    if (!(rho > 0.f) || !std::isfinite(rho) || iters < 0) return DSGNLM_EINVAL;
    if (iters == 0) return DSGNLM_OK;
    dsgnlm* h = p->den;
    const int H = p->H, W = p->W;
    const size_t n = (size_t)H * W;
    const bool fast = ad ? true : h->fast;  // the adaptive form runs on the TMA path only
    const int nblocks = fast ? combine_xupdate_blocks(H, W) : apply_grid_blocks(H, W);
    DSG_CK(h->z.ensure(n * sizeof(float)));
    DSG_CK(h->partials.ensure(sizeof(double) * 2 * (size_t)nblocks * (fast ? (size_t)iters : 1)));
    DSG_CK(h->arrive.ensure(sizeof(unsigned) * (size_t)iters));
    DSG_CK(h->hist.ensure(sizeof(double) * 2 * (size_t)iters));
    DSG_CK(cudaMemsetAsync(h->arrive.p, 0, sizeof(unsigned) * (size_t)iters, h->stream));
    SolveRed red{h->partials.as<double>(), h->arrive.as<unsigned>(), h->hist.as<double>()};
    const float mu = (float)(1.0 / ((double)p->alpha + (double)rho));
    const BlurTaps taps = make_blur_taps(p->blur_sigma > 0.f ? p->blur_sigma : 1.f,
                                         p->kind == LPNP_SR2 ? p->blur_r : 0);
    // Generic path: the super-resolution update reads x in halos, so x alternates
    // between the caller's buffer (A) and the handle's copy (B), the update of
    // iteration k writing B for even k and A for odd k.  TMA path: the gradient is
    // formed first, so every update works on A in place.
    float* xA = p->x;
    float* xB = p->kind == LPNP_SR2 ? h->x2.as<float>() : p->x;
    const bool sr = p->kind == LPNP_SR2;
    const bool sym = sr && p->blur_boundary == LPNP_BC_SYMMETRIC;
    if (sym && !fast) return DSGNLM_EINVAL;  // the symmetric blur runs on the stencil path only
    // the solve's view of the data term's input: the caller's buffer, or the handle's
    // copy of it when the solve runs as a recorded graph
    const float* yv = p->y;
    const uint8_t* cv = p->counts;
    // A^T (A x - y) of the current x: one tiled kernel (periodic) or the residual on the
    // low-resolution grid and its adjoint (symmetric)
    auto sr_gradient = [&](const float* xs, float* g, cudaStream_t s) -> cudaError_t {
        if (!sym) return launch_sr_grad(xs, yv, H, W, taps, g, s);
        cudaError_t e = launch_sr_forward_bc(1, xs, H, W, taps, yv, -1.0f, h->rlo.as<float>(), s);
        if (e != cudaSuccess) return e;
        return launch_sr_adjoint_bc(1, h->rlo.as<float>(), H, W, taps, 0.f, nullptr, g, nullptr, s);
    };
    if (fast) {
        // Iteration k: phase-1 gather of W z, then one per-pixel pass that finishes v
        // and u of iteration k and performs the x-update of iteration k + 1.  For SR
        // that update needs A^T(A x - y) at the current x, which depends on x alone:
        // it is computed on the side stream while phase 1 streams the weights.
        if (sr) {
            DSG_CK(h->gbuf.ensure(n * sizeof(float)));
            if (sym) DSG_CK(h->rlo.ensure(sizeof(float) * n / 4));
            if (iters > 1) DSG_CK(h->ensure_side());
        }
        // the per-iteration residual partials are reduced only when the history is read
        const int want_hist = p->resid_hist ? 1 : 0;
        const bool use_graph = !ad && !h->prof && iters > 1;
        if (use_graph) {
            const size_t obytes = sr ? sizeof(float) * (n / 4) : n;
            DSG_CK(h->obs.ensure(obytes));
            DSG_CK(cudaMemcpyAsync(h->obs.p, sr ? (const void*)p->y : (const void*)p->counts, obytes,
                                   cudaMemcpyDeviceToDevice, h->stream));
            if (sr)
                yv = h->obs.as<float>();
            else
                cv = h->obs.as<uint8_t>();
        }
        EpilogueArgs ea{};
        ea.H = H;
        ea.W = W;
        ea.d = h->d_final;
        ea.t = h->t_final;
        ea.inv_m = h->inv_m;
        ea.inv_m_dev = h->inv_m_dev ? &h->ctl.as<BalanceCtl>()->inv_m : nullptr;
        ea.z = h->z.as<float>();
        ea.v = p->v;
        ea.u = p->u;
        ea.y = yv;
        ea.g = h->gbuf.as<float>();
        ea.taps = taps;
        ea.counts = cv;
        ea.K = p->K;
        ea.eta = p->eta;
        ea.eps = p->spi_eps;
        ea.mu = mu;
        ea.alpha = p->alpha;
        ea.rho = rho;
        ea.constraint = p->constraint;
        ea.x_in = xA;
        ea.x_out = xA;
        const int kind = sr ? 0 : 1;
        // the x-update of iteration 0 (its gradient at the initial x, for SR)
        auto first_update = [&](cudaStream_t st) -> cudaError_t {
            if (!sr)
                return launch_spi_xupdate(cv, (int)n, p->K, p->eta, p->spi_eps, p->x, p->v, p->u,
                                          h->z.as<float>(), mu, p->alpha, rho, p->constraint, st);
            cudaError_t e = sr_gradient(xA, h->gbuf.as<float>(), st);
            if (e != cudaSuccess) return e;
            return launch_xupdate_point(xA, h->gbuf.as<float>(), p->v, p->u, h->z.as<float>(), (int)n, mu, p->alpha,
                                        rho, p->constraint, st);
        };
        // phase 1 of iteration it, the next gradient beside it, then the epilogue
        auto iteration = [&](int it, cudaStream_t st) -> cudaError_t {
            const bool do_x = it < iters - 1;
            cudaError_t e = cudaSuccess;
            if (sr && do_x) e = cudaEventRecord(h->ev_fork, st);
            if (e == cudaSuccess)
                e = h->timed(DSGNLM_PROF_APPLY, [&] {
                    return launch_tma_gather(h->dtype, h->plan, H, W, h->rs, h->d_final, h->z.as<float>(),
                                             h->err.as<unsigned>(), nullptr, st, h->wait_budget);
                });
            if (sr && do_x) {
                if (e == cudaSuccess) e = cudaStreamWaitEvent(h->side, h->ev_fork, 0);
                if (e == cudaSuccess) e = sr_gradient(xA, h->gbuf.as<float>(), h->side);
                if (e == cudaSuccess) e = cudaEventRecord(h->ev_join, h->side);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(st, h->ev_join, 0);
            }
            ea.do_x = do_x;
            ea.partials = h->partials.as<double>() + 2 * (size_t)nblocks * it;
            if (e == cudaSuccess)
                e = h->timed(DSGNLM_PROF_XUPDATE, [&] { return launch_combine_update(kind, h->plan, h->rs, ea, st); });
            return e;
        };
        bool ran = false;
        if (use_graph) {
            // The sequence is recorded once as a CUDA graph and replayed while everything
            // its kernel parameters bake in is unchanged: one launch per solve instead of
            // one per kernel, so the host's launch rate does not gap the GPU.  A single
            // iteration (a few kernels, often on fresh buffers) is launched directly.
            std::vector<unsigned char> key;
            // with 1/m read on the device, a new image of the same size (another m)
            // replays the same graph
            const int ints[14] = {H, W, iters, kind, (int)sym, h->dtype, h->rs, nblocks, p->constraint, p->K,
                                  h->plan.tiles_x, h->plan.tiles_y, want_hist, (int)h->inv_m_dev};
            const float fls[6] = {mu, p->alpha, rho, h->inv_m_dev ? 0.f : h->inv_m, p->eta, p->spi_eps};
            const void* ptrs[19] = {xA, p->v, p->u, yv, cv, h->z.p, h->gbuf.p, h->rlo.p, h->d_final,
                                    h->t_final, h->partials.p, h->hist.p, h->arrive.p, h->err.p, h->plan.partials,
                                    h->side, h->ev_fork, h->ev_join, h->ctl.p};
            key_put(key, ints);
            key_put(key, fls);
            key_put(key, ptrs);
            key_put(key, taps);
            key_put(key, h->plan.splits);
            key.insert(key.end(), h->plan.tmap, h->plan.tmap + 128);
            cudaError_t e = cudaSuccess;
            int slot = -1;
            for (int i = 0; i < dsgnlm::kSolveGraphs; ++i)
                if (h->s_exec[i] && h->s_key[i] == key) slot = i;
            if (slot < 0) {
                // record into the entry not used last
                slot = (h->s_last + 1) % dsgnlm::kSolveGraphs;
                if (h->s_exec[slot]) cudaGraphExecDestroy(h->s_exec[slot]);
                if (h->s_graph[slot]) cudaGraphDestroy(h->s_graph[slot]);
                h->s_exec[slot] = nullptr;
                h->s_graph[slot] = nullptr;
                h->s_key[slot].clear();
                if (!h->cap_stream) e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
                if (e == cudaSuccess) e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeRelaxed);
                if (e == cudaSuccess) {
                    g_capturing = true;
                    cudaError_t e1 = first_update(h->cap_stream);
                    for (int it = 0; it < iters && e1 == cudaSuccess; ++it) e1 = iteration(it, h->cap_stream);
                    if (e1 == cudaSuccess && want_hist)
                        e1 = launch_reduce_residuals(red, iters, nblocks, h->cap_stream);
                    g_capturing = false;
                    cudaGraph_t g = nullptr;
                    e = cudaStreamEndCapture(h->cap_stream, &g);
                    if (e == cudaSuccess) e = e1;
                    if (e == cudaSuccess) e = cudaGraphInstantiate(&h->s_exec[slot], g, 0);
                    if (e == cudaSuccess) {
                        h->s_graph[slot] = g;
                        h->s_key[slot] = key;
                    } else {
                        if (g) cudaGraphDestroy(g);
                        h->s_exec[slot] = nullptr;
                        (void)cudaGetLastError();
                    }
                }
            }
            if (h->s_exec[slot]) {
                h->s_last = slot;
                DSG_CK(cudaGraphLaunch(h->s_exec[slot], h->stream));
                const uint64_t grad = sr ? (sym ? 2 : 1) : 0;
                count_launches((sr ? grad + 1 : 1) + 2 * (uint64_t)iters + grad * (uint64_t)(iters - 1) + want_hist);
                ran = true;
            }
        }
        if (!ran) {  // launched directly: profiling, adaptive W, or no graph
            DSG_CK(h->timed(DSGNLM_PROF_XUPDATE, [&] { return first_update(h->stream); }));
            for (int it = 0; it < iters; ++it) {
                if (ad && it < ad->iters) {
                    s = adapt_w(h, *ad, H, W);
                    if (s != DSGNLM_OK) return s;
                    ea.d = h->d_final;
                    ea.t = h->t_final;
                    ea.inv_m = h->inv_m;
                }
                DSG_CK(iteration(it, h->stream));
            }
            if (want_hist) DSG_CK(launch_reduce_residuals(red, iters, nblocks, h->stream));
        }
    } else {
        if (sr) DSG_CK(h->x2.ensure(n * sizeof(float)));
        xB = sr ? h->x2.as<float>() : p->x;
        for (int it = 0; it < iters; ++it) {
            DSG_CK(h->timed(DSGNLM_PROF_XUPDATE, [&] {
                if (p->kind == LPNP_SR2) {
                    float* xa = (it & 1) ? xB : xA;
                    float* xb = (it & 1) ? xA : xB;
                    return launch_sr_xupdate_fused(xa, xb, p->y, H, W, taps, p->v, p->u, h->z.as<float>(), mu,
                                                   p->alpha, rho, p->constraint, h->stream);
                }
                return launch_spi_xupdate(p->counts, (int)n, p->K, p->eta, p->spi_eps, p->x, p->v, p->u,
                                          h->z.as<float>(), mu, p->alpha, rho, p->constraint, h->stream);
            }));
            DSG_CK(h->timed(DSGNLM_PROF_APPLY, [&] {
                return launch_apply_dual(h->dtype, h->planes.p, H, W, h->rs, h->d_final, h->inv_m,
                                         h->z.as<float>(), p->v, p->u, red, it, h->stream);
            }));
        }
    }
    if (!fast && sr && (iters & 1))
        DSG_CK(cudaMemcpyAsync(p->x, h->x2.p, n * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
    if (p->resid_hist) {
        DSG_CK(h->stage(sizeof(double) * 2 * (size_t)iters));
        DSG_CK(cudaMemcpyAsync(h->host_stage, h->hist.p, sizeof(double) * 2 * (size_t)iters,
                               cudaMemcpyDeviceToHost, h->stream));
        DSG_CK(cudaStreamSynchronize(h->stream));
        if (fast) {
            unsigned errv = 0;
            DSG_CK(cudaMemcpy(&errv, h->err.p, sizeof errv, cudaMemcpyDeviceToHost));
            if (errv) return wait_timeout(h, h->stream);
        }
        const double* hs = (const double*)h->host_stage;
        for (int it = 0; it < iters; ++it) {
            p->resid_hist[2 * it] = std::sqrt(hs[2 * it] / (double)n);
            p->resid_hist[2 * it + 1] = (double)rho * std::sqrt(hs[2 * it + 1] / (double)n);
        }
    }
    return DSGNLM_OK;
}

}  // namespace

extern "C" {

dsgnlm_status lpnp_solve(const lpnp_problem* p, float rho, int iters) {
    NvtxRange nvtx_range("lpnp_solve");
    return solve_impl(p, rho, iters, nullptr);
}

dsgnlm_status lpnp_solve_standard(const lpnp_problem* p, float rho, int iters, int cg_iters) {
    NvtxRange nvtx_range("lpnp_solve_standard");
    dsgnlm_status s = check_problem(p, true);
    if (s != DSGNLM_OK) return s;
    if (p->kind != LPNP_SR2 || cg_iters < 1 || !(rho > 0.f) || !std::isfinite(rho) || iters < 0) return DSGNLM_EINVAL;
    dsgnlm* h = p->den;
    if (!h->fast) return DSGNLM_EINVAL;
    if (iters == 0) return DSGNLM_OK;
    const int H = p->H, W = p->W, n = H * W;
    const int bc = p->blur_boundary;
    const BlurTaps taps = make_blur_taps(p->blur_sigma, p->blur_r);
    if (!sr_bc_supported(H, W, taps.r)) return DSGNLM_EINVAL;
    cudaStream_t st = h->stream;
    const int nblocks = combine_xupdate_blocks(H, W);
    const int nb_hi = sr_adjoint_bc_blocks(H, W), nb_v = cg_vector_blocks(n);
    DSG_CK(h->z.ensure(sizeof(float) * n));
    DSG_CK(h->rlo.ensure(sizeof(float) * n / 4));
    DSG_CK(h->cg_r.ensure(sizeof(float) * n));
    DSG_CK(h->cg_p.ensure(sizeof(float) * n));
    DSG_CK(h->cg_q.ensure(sizeof(float) * n));
    DSG_CK(h->cg_aty.ensure(sizeof(float) * n));
    DSG_CK(h->cg_part.ensure(sizeof(double) * (size_t)std::max(nb_hi, nb_v)));
    DSG_CK(h->cg_scal.ensure(sizeof(CgScalars)));
    DSG_CK(h->partials.ensure(sizeof(double) * 2 * (size_t)nblocks * iters));
    DSG_CK(h->hist.ensure(sizeof(double) * 2 * (size_t)iters));
    DSG_CK(h->arrive.ensure(sizeof(unsigned) * (size_t)iters));
    SolveRed red{h->partials.as<double>(), h->arrive.as<unsigned>(), h->hist.as<double>()};
    float* x = p->x;
    float* r = h->cg_r.as<float>();
    float* pv = h->cg_p.as<float>();
    float* q = h->cg_q.as<float>();
    float* lo = h->rlo.as<float>();
    float* aty = h->cg_aty.as<float>();
    double* part = h->cg_part.as<double>();
    CgScalars* sc = h->cg_scal.as<CgScalars>();
    // A^T y once
    DSG_CK(launch_sr_adjoint_bc(bc, p->y, H, W, taps, 0.f, nullptr, aty, nullptr, st));
    EpilogueArgs ea{};
    ea.H = H;
    ea.W = W;
    ea.d = h->d_final;
    ea.t = h->t_final;
    ea.inv_m = h->inv_m;
    ea.z = h->z.as<float>();
    ea.v = p->v;
    ea.u = p->u;
    ea.x_in = x;
    ea.x_out = x;
    ea.y = p->y;
    ea.taps = taps;
    ea.do_x = 0;  // the x-update is the CG solve of the next iteration
    for (int it = 0; it < iters; ++it) {
        DSG_CK(h->timed(DSGNLM_PROF_XUPDATE, [&]() -> cudaError_t {
            // (A^T A + rho I) x = A^T y + rho (v - u) by CG from the current x
            cudaError_t e = launch_sr_forward_bc(bc, x, H, W, taps, nullptr, 0.f, lo, st);
            if (e == cudaSuccess) e = launch_sr_adjoint_bc(bc, lo, H, W, taps, rho, x, q, nullptr, st);
            if (e == cudaSuccess) e = launch_cg_init(aty, p->v, p->u, rho, q, r, pv, n, part, st);
            if (e == cudaSuccess) e = launch_cg_reduce(part, nb_v, sc, 0, st);
            for (int k = 0; k < cg_iters && e == cudaSuccess; ++k) {
                e = launch_sr_forward_bc(bc, pv, H, W, taps, nullptr, 0.f, lo, st);
                if (e == cudaSuccess) e = launch_sr_adjoint_bc(bc, lo, H, W, taps, rho, pv, q, part, st);
                if (e == cudaSuccess) e = launch_cg_reduce(part, nb_hi, sc, 1, st);
                if (e == cudaSuccess) e = launch_cg_step(x, r, pv, q, sc, n, part, st);
                if (e == cudaSuccess) e = launch_cg_reduce(part, nb_v, sc, 2, st);
                if (e == cudaSuccess && k + 1 < cg_iters) e = launch_cg_dir(r, pv, sc, n, st);
            }
            if (e == cudaSuccess) e = launch_project_z(x, p->u, h->z.as<float>(), n, p->constraint, st);
            return e;
        }));
        DSG_CK(h->timed(DSGNLM_PROF_APPLY, [&] {
            return launch_tma_gather(h->dtype, h->plan, H, W, h->rs, h->d_final, h->z.as<float>(),
                                     h->err.as<unsigned>(), nullptr, st, h->wait_budget);
        }));
        ea.partials = h->partials.as<double>() + 2 * (size_t)nblocks * it;
        DSG_CK(h->timed(DSGNLM_PROF_XUPDATE, [&] { return launch_combine_update(0, h->plan, h->rs, ea, st); }));
    }
    DSG_CK(launch_reduce_residuals(red, iters, nblocks, st));
    if (p->resid_hist) {
        DSG_CK(h->stage(sizeof(double) * 2 * (size_t)iters));
        DSG_CK(cudaMemcpyAsync(h->host_stage, h->hist.p, sizeof(double) * 2 * (size_t)iters, cudaMemcpyDeviceToHost,
                               st));
        DSG_CK(cudaStreamSynchronize(st));
        unsigned errv = 0;
        DSG_CK(cudaMemcpy(&errv, h->err.p, sizeof errv, cudaMemcpyDeviceToHost));
        if (errv) return wait_timeout(h, st);
        const double* hs = (const double*)h->host_stage;
        for (int it = 0; it < iters; ++it) {
            p->resid_hist[2 * it] = std::sqrt(hs[2 * it] / (double)n);
            p->resid_hist[2 * it + 1] = (double)rho * std::sqrt(hs[2 * it + 1] / (double)n);
        }
    }
    return DSGNLM_OK;
}

dsgnlm_status lpnp_solve_adaptive(const lpnp_problem* p, float rho, int iters, int adapt_iters, int patch_r,
                                  int search_r, float bandwidth, double tol, int maxit) {
    NvtxRange nvtx_range("lpnp_solve_adaptive");
    if (adapt_iters < 1 || !tma_path_supports(search_r)) return DSGNLM_EINVAL;
    if (patch_r < 0 || patch_r > DSGNLM_MAX_PATCH_R || !(bandwidth > 0.f) || !std::isfinite(bandwidth))
        return DSGNLM_EINVAL;
    if (!(tol >= 0.0) || maxit < 1) return DSGNLM_EINVAL;
    const Adapt ad{adapt_iters, patch_r, search_r, bandwidth, tol, maxit};
    return solve_impl(p, rho, iters, &ad);
}

}  // extern "C"

namespace {


// Batched Algorithm 1.  `slices` > 0 splits the offsets of every image into that many
// slices (the batch fills the GPU by itself, so fewer slices than a lone image
// needs cut the partial-region traffic); 0 keeps each handle's own plan.  With
// `use_graph` the step sequence is recorded once into a CUDA graph on the lead
// handle and replayed while the batch is unchanged.
dsgnlm_status batched_impl(const lpnp_problem* probs, int count, float rho, int iters, int slices,
                           bool use_graph) {
    if (!probs || count < 1 || count > kMaxBatch || slices < 0) return DSGNLM_EINVAL;
    if (!(rho > 0.f) || !std::isfinite(rho) || iters < 0) return DSGNLM_EINVAL;
    for (int i = 0; i < count; ++i) {
        dsgnlm_status s = check_problem(&probs[i], true);
        if (s != DSGNLM_OK) return s;
        const dsgnlm* h = probs[i].den;
        if (!h->fast || probs[i].kind != probs[0].kind || h->dtype != probs[0].den->dtype || h->rs != probs[0].den->rs)
            return DSGNLM_EINVAL;
        if (probs[i].kind == LPNP_SR2 && probs[i].blur_boundary != LPNP_BC_PERIODIC)
            return DSGNLM_EINVAL;  // the batched gradient is the periodic tile kernel
        for (int j = 0; j < i; ++j)
            if (probs[j].den == h) return DSGNLM_EINVAL;  // each image needs its own handle
    }
    if (iters == 0) return DSGNLM_OK;
    dsgnlm* lead = probs[0].den;
    cudaStream_t st = lead->stream;
    const int kind = probs[0].kind == LPNP_SR2 ? 0 : 1;
    std::vector<BatchInst> inst(count);
    std::vector<BatchEpi> epi(count);
    std::vector<int4> work1, work2, work3;
    BatchMaps maps;
    for (int i = 0; i < count; ++i) {
        const lpnp_problem* p = &probs[i];
        dsgnlm* h = p->den;
        const int H = p->H, W = p->W;
        const size_t n = (size_t)H * W;
        const int gx = (W + 31) / 32, gy = (H + 15) / 16;
        const int nb = gx * gy;
        if (nb != combine_xupdate_blocks(H, W)) return DSGNLM_EINVAL;
        DSG_CK(h->z.ensure(n * sizeof(float)));
        if (p->kind == LPNP_SR2) {
            if (p->blur_r != probs[0].blur_r) return DSGNLM_EINVAL;  // one gradient kernel per batch
            DSG_CK(h->gbuf.ensure(n * sizeof(float)));
        }
        DSG_CK(h->partials.ensure(sizeof(double) * 2 * (size_t)nb * iters));
        const TmaSplits splits = slices > 0 ? make_splits(h->rs, slices) : h->plan.splits;
        const size_t tiles = (size_t)h->plan.tiles_x * h->plan.tiles_y;
        DSG_CK(h->tma_part.ensure(sizeof(float) * tma_region_floats(h->rs) * tiles * splits.n));
        h->plan.partials = h->tma_part.as<float>();  // the buffer may have grown
        h->plan.part_cap = (long long)(h->tma_part.bytes / sizeof(float));
        std::memcpy(maps.m[i], h->plan.tmap, 128);
        BatchInst& bi = inst[i];
        bi.H = H;
        bi.W = W;
        bi.tiles_x = h->plan.tiles_x;
        bi.tiles_y = h->plan.tiles_y;
        bi.splits = splits;
        bi.d = h->d_final;
        bi.z = h->z.as<float>();
        bi.part = h->plan.partials;
        bi.part_cap = h->plan.part_cap;
        for (int sl = 0; sl < bi.splits.n; ++sl)
            for (int ty = 0; ty < bi.tiles_y; ++ty)
                for (int tx = 0; tx < bi.tiles_x; ++tx) work1.push_back(make_int4(i, ty, tx, sl));
        BatchEpi& be = epi[i];
        EpilogueArgs& ea = be.a;
        ea = EpilogueArgs{};
        ea.H = H;
        ea.W = W;
        ea.d = h->d_final;
        ea.t = h->t_final;
        ea.inv_m = h->inv_m;
        ea.z = h->z.as<float>();
        ea.v = p->v;
        ea.u = p->u;
        ea.x_in = p->x;
        ea.x_out = p->x;
        ea.y = p->y;
        ea.g = p->kind == LPNP_SR2 ? h->gbuf.as<float>() : nullptr;
        ea.taps = make_blur_taps(p->blur_sigma > 0.f ? p->blur_sigma : 1.f, p->kind == LPNP_SR2 ? p->blur_r : 0);
        ea.counts = p->counts;
        ea.K = p->K;
        ea.eta = p->eta;
        ea.eps = p->spi_eps;
        ea.mu = (float)(1.0 / ((double)p->alpha + (double)rho));
        ea.alpha = p->alpha;
        ea.rho = rho;
        ea.constraint = p->constraint;
        ea.do_x = 1;
        be.cv = Cover{h->plan.partials, h->plan.tiles_x, h->plan.tiles_y, splits.n, h->rs, h->plan.part_cap};
        be.gx = gx;
        be.nblocks = nb;
        be.partials = h->partials.as<double>();
        for (int by = 0; by < gy; ++by)
            for (int bx = 0; bx < gx; ++bx) work2.push_back(make_int4(i, by, bx, 0));
        if (p->kind == LPNP_SR2)
            for (int by = 0; by < (H + 31) / 32; ++by)
                for (int bx = 0; bx < (W + 31) / 32; ++bx) work3.push_back(make_int4(i, by, bx, 0));
    }
    bool want_hist = false;
    for (int i = 0; i < count; ++i) want_hist |= probs[i].resid_hist != nullptr;
    DSG_CK(lead->b_inst.ensure(sizeof(BatchInst) * count));
    DSG_CK(lead->b_epi.ensure(sizeof(BatchEpi) * count));
    DSG_CK(lead->b_work1.ensure(sizeof(int4) * work1.size()));
    DSG_CK(lead->b_work2.ensure(sizeof(int4) * work2.size()));
    DSG_CK(lead->b_work3.ensure(sizeof(int4) * (work3.size() + 1)));
    if (want_hist) DSG_CK(lead->b_hist.ensure(sizeof(double) * 2 * (size_t)count * iters));
    // the tables carry the scalings and 1/m of the current balance: uploaded on every
    // call, read by the kernels (and a recorded graph) at run time
    DSG_CK(cudaMemcpyAsync(lead->b_inst.p, inst.data(), sizeof(BatchInst) * count, cudaMemcpyHostToDevice, st));
    DSG_CK(cudaMemcpyAsync(lead->b_epi.p, epi.data(), sizeof(BatchEpi) * count, cudaMemcpyHostToDevice, st));
    DSG_CK(cudaMemcpyAsync(lead->b_work1.p, work1.data(), sizeof(int4) * work1.size(), cudaMemcpyHostToDevice, st));
    DSG_CK(cudaMemcpyAsync(lead->b_work2.p, work2.data(), sizeof(int4) * work2.size(), cudaMemcpyHostToDevice, st));
    if (!work3.empty())
        DSG_CK(cudaMemcpyAsync(lead->b_work3.p, work3.data(), sizeof(int4) * work3.size(), cudaMemcpyHostToDevice, st));
    // every image must be ready on the lead stream: the other handles' work is ordered
    // before this call by the caller (same stream), as for lpnp_solve
    const BatchInst* dinst = lead->b_inst.as<BatchInst>();
    const BatchEpi* depi = lead->b_epi.as<BatchEpi>();
    const int4* w1 = lead->b_work1.as<int4>();
    const int4* w2 = lead->b_work2.as<int4>();
    const int4* w3 = lead->b_work3.as<int4>();
    const int n1 = (int)work1.size(), n2 = (int)work2.size(), n3 = (int)work3.size();
    const bool sr = kind == 0;
    const int blur_r = probs[0].blur_r;
    if (sr && iters > 1) DSG_CK(lead->ensure_side());
    // As the single-image solve: the SR gradient of the current x depends on x alone
    // and runs on the side stream while phase 1 streams the weights.
    auto steps = [&](cudaStream_t s) -> cudaError_t {
        cudaError_t e = lead->timed(DSGNLM_PROF_XUPDATE, [&] {
            if (sr) {
                const cudaError_t eg = launch_batched_grad(blur_r, depi, w3, n3, s);
                if (eg != cudaSuccess) return eg;
            }
            return launch_batched_xupdate0(kind, depi, w2, n2, s);
        });
        for (int it = 0; it < iters && e == cudaSuccess; ++it) {
            const bool do_x = it < iters - 1;
            if (sr && do_x) e = cudaEventRecord(lead->ev_fork, s);
            if (e == cudaSuccess)
                e = lead->timed(DSGNLM_PROF_APPLY, [&] {
                    return launch_tma_gather_batched(lead->dtype, lead->rs, maps, dinst, w1, n1,
                                                     lead->err.as<unsigned>(), s);
                });
            if (e == cudaSuccess && sr && do_x) {
                e = cudaStreamWaitEvent(lead->side, lead->ev_fork, 0);
                if (e == cudaSuccess) e = launch_batched_grad(blur_r, depi, w3, n3, lead->side);
                if (e == cudaSuccess) e = cudaEventRecord(lead->ev_join, lead->side);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(s, lead->ev_join, 0);
            }
            if (e == cudaSuccess)
                e = lead->timed(DSGNLM_PROF_XUPDATE,
                                [&] { return launch_batched_combine(kind, depi, w2, n2, it, !do_x, s); });
        }
        if (e == cudaSuccess && want_hist) e = launch_batched_reduce(depi, count, lead->b_hist.as<double>(), iters, s);
        return e;
    };
    bool ran = false;
    if (use_graph && !lead->prof) {
        // everything a recorded sequence bakes into its kernel parameters
        std::vector<unsigned char> key;
        const int ints[11] = {count, iters, kind, lead->dtype, lead->rs, n1, n2, n3, blur_r, (int)want_hist, slices};
        const void* ptrs[10] = {lead->b_inst.p, lead->b_epi.p, lead->b_work1.p, lead->b_work2.p, lead->b_work3.p,
                                lead->b_hist.p, lead->err.p, lead->side, lead->ev_fork, lead->ev_join};
        key_put(key, ints);
        key_put(key, ptrs);
        key.insert(key.end(), &maps.m[0][0], &maps.m[0][0] + 128 * (size_t)count);
        cudaError_t e = cudaSuccess;
        if (!lead->b_exec || key != lead->b_key) {
            if (lead->b_exec) cudaGraphExecDestroy(lead->b_exec);
            if (lead->b_graph) cudaGraphDestroy(lead->b_graph);
            lead->b_exec = nullptr;
            lead->b_graph = nullptr;
            lead->b_key.clear();
            if (!lead->cap_stream) e = cudaStreamCreateWithFlags(&lead->cap_stream, cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaStreamBeginCapture(lead->cap_stream, cudaStreamCaptureModeRelaxed);
            if (e == cudaSuccess) {
                g_capturing = true;
                const cudaError_t e1 = steps(lead->cap_stream);
                g_capturing = false;
                cudaGraph_t g = nullptr;
                e = cudaStreamEndCapture(lead->cap_stream, &g);
                if (e == cudaSuccess) e = e1;
                if (e == cudaSuccess) e = cudaGraphInstantiate(&lead->b_exec, g, 0);
                if (e == cudaSuccess) {
                    lead->b_graph = g;
                    lead->b_key = key;
                } else {
                    if (g) cudaGraphDestroy(g);
                    lead->b_exec = nullptr;
                    (void)cudaGetLastError();
                }
            }
        }
        if (lead->b_exec) {
            DSG_CK(cudaGraphLaunch(lead->b_exec, st));
            count_launches(1 + (sr ? 1 : 0) + (sr ? 3 : 2) * (uint64_t)iters - (sr ? 1 : 0) + (want_hist ? 1 : 0));
            ran = true;
        }
    }
    if (!ran) DSG_CK(steps(st));  // no graph: launch the steps directly
    if (want_hist) {
        std::vector<double> hs(2 * (size_t)count * iters);
        DSG_CK(cudaMemcpyAsync(hs.data(), lead->b_hist.p, sizeof(double) * hs.size(), cudaMemcpyDeviceToHost, st));
        DSG_CK(cudaStreamSynchronize(st));
        unsigned errv = 0;
        DSG_CK(cudaMemcpy(&errv, lead->err.p, sizeof errv, cudaMemcpyDeviceToHost));
        if (errv) return wait_timeout(lead, st);
        for (int i = 0; i < count; ++i) {
            if (!probs[i].resid_hist) continue;
            const double n = (double)probs[i].H * probs[i].W;
            for (int it = 0; it < iters; ++it) {
                probs[i].resid_hist[2 * it] = std::sqrt(hs[2 * ((size_t)i * iters + it)] / n);
                probs[i].resid_hist[2 * it + 1] = (double)rho * std::sqrt(hs[2 * ((size_t)i * iters + it) + 1] / n);
            }
        }
    }
    return DSGNLM_OK;
}

}  // namespace

extern "C" {

dsgnlm_status lpnp_solve_batched(const lpnp_problem* probs, int count, float rho, int iters) {
    NvtxRange nvtx_range("lpnp_solve_batched");
    return batched_impl(probs, count, rho, iters, 0, true);
}

dsgnlm_status lpnp_solve_batched_sched(const lpnp_problem* probs, int count, float rho, int iters, int slices) {
    NvtxRange nvtx_range("lpnp_solve_batched_sched");
    return batched_impl(probs, count, rho, iters, slices, true);
}

dsgnlm_status lpnp_tune_batched(const lpnp_problem* probs, int count, float rho, const int* candidates, int ncand,
                                int trial_iters, int* best_slices, float* ms_per_iter) {
    if (!probs || count < 1 || count > kMaxBatch || !candidates || ncand < 1 || trial_iters < 1 || !best_slices)
        return DSGNLM_EINVAL;
    for (int c = 0; c < ncand; ++c)
        if (candidates[c] < 0) return DSGNLM_EINVAL;
    for (int i = 0; i < count; ++i) {
        const dsgnlm_status s = check_problem(&probs[i], true);
        if (s != DSGNLM_OK) return s;
    }
    cudaStream_t st = probs[0].den->stream;
    // trial solves run on copies of the iterates; the weights are only read
    struct Scratch {
        std::vector<DevBuf> b;
        ~Scratch() {
            for (DevBuf& x : b) x.release();
        }
    } scratch;
    scratch.b.resize(3 * (size_t)count);
    std::vector<DevBuf>& bufs = scratch.b;
    std::vector<lpnp_problem> trial(probs, probs + count);
    for (int i = 0; i < count; ++i) {
        const size_t bytes = sizeof(float) * (size_t)probs[i].H * probs[i].W;
        float* src[3] = {probs[i].x, probs[i].v, probs[i].u};
        for (int k = 0; k < 3; ++k) {
            DevBuf& b = bufs[3 * (size_t)i + k];
            DSG_CK(b.ensure(bytes));
            DSG_CK(cudaMemcpyAsync(b.p, src[k], bytes, cudaMemcpyDeviceToDevice, st));
        }
        trial[i].x = bufs[3 * (size_t)i].as<float>();
        trial[i].v = bufs[3 * (size_t)i + 1].as<float>();
        trial[i].u = bufs[3 * (size_t)i + 2].as<float>();
        trial[i].resid_hist = nullptr;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    DSG_CK(cudaEventCreate(&e0));
    cudaError_t ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail_cuda(ce);
    }
    dsgnlm_status s = DSGNLM_OK;
    float best = INFINITY;
    for (int c = 0; c < ncand && s == DSGNLM_OK; ++c) {
        s = batched_impl(trial.data(), count, rho, 1, candidates[c], false);  // warm-up
        if (s != DSGNLM_OK) break;
        ce = cudaEventRecord(e0, st);
        if (ce == cudaSuccess) s = batched_impl(trial.data(), count, rho, trial_iters, candidates[c], false);
        if (ce == cudaSuccess && s == DSGNLM_OK) ce = cudaEventRecord(e1, st);
        if (ce == cudaSuccess && s == DSGNLM_OK) ce = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (ce == cudaSuccess && s == DSGNLM_OK) ce = cudaEventElapsedTime(&ms, e0, e1);
        if (ce != cudaSuccess) s = fail_cuda(ce);
        if (s != DSGNLM_OK) break;
        ms /= (float)trial_iters;
        if (ms_per_iter) ms_per_iter[c] = ms;
        if (ms < best) {
            best = ms;
            *best_slices = candidates[c];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s == DSGNLM_OK) DSG_CK(cudaStreamSynchronize(st));  // the copies are freed on return
    return s;
}
dsgnlm_status dsgnlm_profile_enable(dsgnlm_t h, int enable) {
    if (!h) return DSGNLM_EINVAL;
    h->prof = enable != 0;
    for (ProfPool& p : h->pools) p.used = 0;
    return DSGNLM_OK;
}

dsgnlm_status dsgnlm_profile_read(dsgnlm_t h, int kind, double* total_ms, int* launches) {
    if (!h || kind < 0 || kind >= kProfKinds) return DSGNLM_EINVAL;
    DSG_CK(cudaStreamSynchronize(h->stream));
    ProfPool& P = h->pools[kind];
    double acc = 0.0;
    for (int q = 0; q < P.used; ++q) {
        float ms = 0.f;
        DSG_CK(cudaEventElapsedTime(&ms, P.ev[2 * q], P.ev[2 * q + 1]));
        acc += ms;
    }
    if (total_ms) *total_ms = acc;
    if (launches) *launches = P.used;
    return DSGNLM_OK;
}

uint64_t dsgnlm_launch_count(void) { return g_launches.load(); }

int dsgnlm_is_checked(void) {
#ifdef DSGNLM_CHECKED
    return 1;
#else
    return 0;
#endif
}

dsgnlm_status dsgnlm_check_word(unsigned* word, int clear) {
    if (!word) return DSGNLM_EINVAL;
    DSG_CK(cudaDeviceSynchronize());
    const bool c = clear != 0;
    *word = check_word_adjoint(c) | check_word_api(c) | check_word_batched(c) | check_word_build(c) |
            check_word_epilogue(c) | check_word_stencil_tma(c);
    return DSGNLM_OK;
}

dsgnlm_status dsgnlm_check_selftest(long long index, long long bound) {
    DSG_CK(launch_check_selftest(index, bound));
    DSG_CK(cudaDeviceSynchronize());
    return DSGNLM_OK;
}

int dsgnlm_last_cuda_error(void) { return g_last_cuda; }

const char* dsgnlm_strerror(dsgnlm_status s) {
    switch (s) {
        case DSGNLM_OK: return "ok";
        case DSGNLM_EINVAL: return "invalid argument";
        case DSGNLM_ENOMEM: return "device allocation failed";
        case DSGNLM_ECUDA: return "CUDA error";
        case DSGNLM_NOT_BUILT: return "denoiser not built";
        case DSGNLM_NOT_BALANCED: return "denoiser not balanced";
        case DSGNLM_NOT_CONVERGED: return "balancing reached maxit above tol";
        case DSGNLM_STALLED: return "balancing residual stalled above tol";
        case DSGNLM_TIMEOUT: return "bounded device wait timed out";
    }
    return "unknown status";
}

}  // extern "C"
