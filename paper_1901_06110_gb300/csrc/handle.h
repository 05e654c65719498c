// The dsgnlm_t handle: weight planes, balancing state, solve workspace and the
// bookkeeping shared by the C ABI implementation files.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/dsgnlm.h"
#include "internal.h"

namespace dsg {

inline bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    cudaError_t ensure(size_t n) {
        if (n <= bytes && p) return cudaSuccess;
        release();
        if (n == 0) return cudaSuccess;
        cudaError_t e = cudaMalloc(&p, n);
        if (e != cudaSuccess) {
            p = nullptr;
            (void)cudaGetLastError();
            return e;
        }
        bytes = n;
        return cudaSuccess;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    template <typename T> T* as() const { return (T*)p; }
};

inline size_t weight_elem_bytes(int dtype) { return dtype == DSGNLM_F32 ? 4 : 2; }

// CUDA event pairs recorded around the launches of one kernel kind while
// profiling is enabled.
struct ProfPool {
    std::vector<cudaEvent_t> ev;
    int used = 0;  // pairs recorded since the last reset
    static constexpr int kMaxPairs = 1 << 16;
    void release() {
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
        ev.clear();
        used = 0;
    }
};

constexpr int kProfKinds = 4;

}  // namespace dsg

struct dsgnlm {
    using DevBuf = dsg::DevBuf;
    using ProfPool = dsg::ProfPool;
    using TmaPlan = dsg::TmaPlan;
    cudaStream_t stream = nullptr;
    int dtype = DSGNLM_F32;
    int H = 0, W = 0, Wp = 0, rp = 0, rs = 0, nh = 0;
    int num_sms = 0;
    // images whose launches share the GPU with this handle's while it is built; the
    // build splits the offsets over fewer slices when the others fill the SMs
    int share = 1;
    // TMA stencil path
    bool fast = false;
    TmaPlan plan{};
    DevBuf tma_part, tbuf[2], err, bal_part;
    // cycles a phase-1 consumer waits for a plane before giving up (dsgnlm_set_wait_budget)
    long long wait_budget = dsg::kDefaultWaitBudget;
    // device (m, 1/m) of a W balanced outside this handle's own balance (the unrolled
    // forward of the differentiable form), read back to m and inv_m on the first call
    // that needs them on the host; null when m and inv_m are current
    const float* m_pending = nullptr;
    // update rule of dsgnlm_balance / dsgnlm_balance_batched (dsgnlm_set_balance_scheme)
    int balance_scheme = DSGNLM_BALANCE_SINKHORN;
    float* t_final = nullptr;
    // balancing passes as a CUDA graph with a device-driven WHILE node
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t bal_graph = nullptr;
    cudaGraphExec_t bal_exec = nullptr;
    unsigned char bal_key[256] = {};
    bool bal_graph_failed = false;
    float bw = 0.f;
    bool built = false, balanced = false;
    DevBuf planes, dbuf[2], stats, ctl;
    float* d_final = nullptr;
    double m = 1.0;
    float inv_m = 1.f;
    int iters = 0;
    double resid = 0.0;
    // Algorithm 1 workspace
    DevBuf z, x2, rlo, partials, arrive, hist, gbuf;
    // the observation (SR) or the counts (SPI) copied in before a recorded solve, so the
    // solve graph does not depend on the caller's buffer
    DevBuf obs;
    // conjugate-gradient workspace of the standard ADMM x-update
    DevBuf cg_r, cg_p, cg_q, cg_aty, cg_part, cg_scal;
    // side stream of the solve: the SR gradient of an iteration runs there while the
    // main stream streams the weights (fork and join events)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // batched Algorithm 1 workspace (used when this handle leads a batch), and the
    // batch's step sequence as a CUDA graph with the values it was recorded for
    DevBuf b_inst, b_epi, b_work1, b_work2, b_work3, b_hist;
    // batched balance tables (used when this handle leads a batched balance)
    DevBuf bb_inst, bb_bal, bb_work1, bb_work2, bb_flag;
    cudaGraph_t b_graph = nullptr;
    cudaGraphExec_t b_exec = nullptr;
    std::vector<unsigned char> b_key;
    // the single-image solve's sequence as CUDA graphs, with the values each was
    // recorded for: two entries, since the balanced scaling alternates between two
    // buffers with the parity of the pass count; s_last is the most recent entry
    static constexpr int kSolveGraphs = 2;
    cudaGraph_t s_graph[kSolveGraphs] = {};
    cudaGraphExec_t s_exec[kSolveGraphs] = {};
    std::vector<unsigned char> s_key[kSolveGraphs];
    int s_last = 0;
    // the balance control block holds 1/m of the current W (set by the balances of
    // this handle, cleared when W comes from elsewhere)
    bool inv_m_dev = false;
    // optional per-kernel timing
    bool prof = false;
    ProfPool pools[dsg::kProfKinds];
    // pinned host staging for small device->host reads
    void* host_stage = nullptr;
    size_t host_stage_bytes = 0;

    cudaError_t stage(size_t n) {
        if (n <= host_stage_bytes) return cudaSuccess;
        if (host_stage) cudaFreeHost(host_stage);
        host_stage = nullptr;
        host_stage_bytes = 0;
        cudaError_t e = cudaMallocHost(&host_stage, n);
        if (e != cudaSuccess) {
            host_stage = nullptr;
            return e;
        }
        host_stage_bytes = n;
        return cudaSuccess;
    }
    cudaError_t ensure_side() {
        cudaError_t e = cudaSuccess;
        if (!side) e = cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking);
        if (e == cudaSuccess && !ev_fork) e = cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming);
        if (e == cudaSuccess && !ev_join) e = cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming);
        return e;
    }
    void release_graphs() {
        if (bal_exec) cudaGraphExecDestroy(bal_exec);
        if (bal_graph) cudaGraphDestroy(bal_graph);
        bal_exec = nullptr;
        bal_graph = nullptr;
        if (b_exec) cudaGraphExecDestroy(b_exec);
        if (b_graph) cudaGraphDestroy(b_graph);
        b_exec = nullptr;
        b_graph = nullptr;
        b_key.clear();
        for (int i = 0; i < kSolveGraphs; ++i) {
            if (s_exec[i]) cudaGraphExecDestroy(s_exec[i]);
            if (s_graph[i]) cudaGraphDestroy(s_graph[i]);
            s_exec[i] = nullptr;
            s_graph[i] = nullptr;
            s_key[i].clear();
        }
    }
    void release_all() {
        release_graphs();
        if (cap_stream) cudaStreamDestroy(cap_stream);
        cap_stream = nullptr;
        if (side) cudaStreamDestroy(side);
        side = nullptr;
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_join) cudaEventDestroy(ev_join);
        ev_fork = ev_join = nullptr;
        gbuf.release();
        obs.release();
        cg_r.release();
        cg_p.release();
        cg_q.release();
        cg_aty.release();
        cg_part.release();
        cg_scal.release();
        bal_part.release();
        tma_part.release();
        tbuf[0].release();
        tbuf[1].release();
        err.release();
        planes.release();
        dbuf[0].release();
        dbuf[1].release();
        stats.release();
        ctl.release();
        z.release();
        x2.release();
        b_inst.release();
        b_epi.release();
        b_work1.release();
        b_work2.release();
        b_work3.release();
        b_hist.release();
        bb_inst.release();
        bb_bal.release();
        bb_work1.release();
        bb_work2.release();
        bb_flag.release();
        rlo.release();
        partials.release();
        arrive.release();
        hist.release();
        if (host_stage) cudaFreeHost(host_stage);
        host_stage = nullptr;
        host_stage_bytes = 0;
        for (ProfPool& p : pools) p.release();
    }

    // Launch through `f`, bracketed by timing events when profiling is on.
    template <typename F>
    cudaError_t timed(int kind, F&& f) {
        if (!prof) return f();
        ProfPool& P = pools[kind];
        if (P.used >= ProfPool::kMaxPairs) return f();
        while ((int)P.ev.size() < 2 * (P.used + 1)) {
            cudaEvent_t e;
            cudaError_t err = cudaEventCreate(&e);
            if (err != cudaSuccess) return err;
            P.ev.push_back(e);
        }
        cudaError_t err = cudaEventRecord(P.ev[2 * P.used], stream);
        if (err != cudaSuccess) return err;
        err = f();
        if (err != cudaSuccess) return err;
        err = cudaEventRecord(P.ev[2 * P.used + 1], stream);
        if (err != cudaSuccess) return err;
        ++P.used;
        return cudaSuccess;
    }
};


namespace dsg {
// dsgnlm_build's work: validation, the planes and, with `launch`, the weight build on the
// handle's stream; then the phase-1 plan and the tensor map of the planes.  launch =
// false leaves the weights to a batched build that the caller queues.
dsgnlm_status build_handle(dsgnlm* h, const float* guide, int H, int W, int patch_r, int search_r, float bandwidth,
                           bool launch);
}  // namespace dsg
