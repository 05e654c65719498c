// Host-side launchers of the kernels, shared by the C ABI implementation.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

namespace dsg {

void count_launches(uint64_t n);

// A named NVTX range over one call of the C ABI, for timeline tools that record NVTX
// (build, balance, solve, the differentiable form); a push and a pop that cost next
// to nothing when no tool is attached.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
// while set (on this thread), count_launches adds nothing: the kernels being recorded
// into a graph are counted each time the graph is launched
void set_capture_counting(bool recording);
uint64_t recorded_launches();  // launches counted while recording, since set_capture_counting(true)
// the checked build's per-translation-unit index-check words (0 in the normal build)
unsigned check_word_adjoint(bool clear);
unsigned check_word_api(bool clear);
unsigned check_word_batched(bool clear);
unsigned check_word_build(bool clear);
unsigned check_word_epilogue(bool clear);
unsigned check_word_stencil_tma(bool clear);
cudaError_t launch_check_selftest(long long index, long long bound);
// makes `e` the value dsgnlm_last_cuda_error() returns in this thread
void record_cuda_error(cudaError_t e);

// balancing state in device memory, one slot per pass
struct PassStat {
    unsigned long long eps_bits;  // max_s |d_s t_s - 1| (FP64 bits)
    unsigned long long m_bits;    // max_s d_s t_s (FP64 bits)
    unsigned int arrive;          // blocks finished
    unsigned int pad;
};

struct BalanceCtl {
    int done;        // set by the deciding pass
    int final_pass;  // pass whose scaling is the result (= number of updates)
    int status;      // 0 ok, 6 not converged, 7 stalled
    int since_best;  // passes since the residual last improved by 1%
    double best;     // smallest residual seen
    double tol;
    int maxit;
    int pass;        // current pass (TMA path: advanced on the device)
    double eps;      // TMA path: residual of the last decided pass
    double m;        // TMA path: max row sum of the last decided pass
    float inv_m;     // TMA path: (float)(1 / m), written with m on the device
    unsigned arrive;  // TMA path: blocks of the current pass's epilogue that have finished
    // update rule of the passes from `plain_passes` on (accelerated scheme): on
    // u = log d, u <- u - relax (u + log t) / 2 + momentum (u - u_prev); relax = 0
    // (a zeroed block) keeps the plain step d <- sqrt(d / t) in every pass
    float relax;
    float momentum;
    int plain_passes;
};

// Solve-loop reduction state: per-block partial sums of every iteration (reduced
// after the loop by launch_reduce_residuals), one arrival counter per iteration
// (generic path) and one two-value history slot per iteration.
struct SolveRed {
    double* partials;        // [iters][nblocks][2] (TMA path) or [nblocks][2] (generic path)
    unsigned int* arrive;    // [iters]
    double* hist;            // [2 * iters]: sum (x-v)^2 and sum (v-v_prev)^2
};

// Weight planes are stored [n_h][H][pitch] with the row pitch a multiple of 8
// elements (16-byte aligned rows, as TMA requires); dtype 0 = FP32, 1 = FP16, 2 = BF16.
__host__ __device__ inline int plane_pitch(int W) { return (W + 7) & ~7; }

// One image of a batched build: its guide, its planes and the elements allocated there,
// and the exponent's scale c log2 e (c = 1 / (2 N_p^2 h^2)).
struct BuildJob {
    const float* guide;
    void* planes;
    long long cap;
    float c2;
};
// The weights of `count` images of one size in one launch (grid z = image x offset
// chunk); `jobs` is a device array, read by the kernel, so the launch can be recorded
// once and replayed for other images.
cudaError_t launch_build_batched(int dtype, const BuildJob* jobs, int count, int H, int W, int patch_r,
                                 int search_r, float c, cudaStream_t st);
cudaError_t launch_build(int dtype, const float* guide, int H, int W, int patch_r, int search_r,
                         float inv_two_np2_h2, void* planes, long long cap, cudaStream_t st);  // cap: weights allocated

// TMA stencil path (search radii with a compiled kernel)
constexpr int kMaxSlices = 25;
struct TmaSplits {
    int ox_lo[kMaxSlices];
    int ox_hi[kMaxSlices];
    int n;
};
struct Cover {  // where a pixel's phase-1 partial sums live
    const float* part;
    int tiles_x, tiles_y, slices, rs;
    long long cap;  // floats allocated at part (the checked build's bound)
};
struct TmaPlan {
    alignas(64) unsigned char tmap[128];  // CUtensorMap of the planes
    int tiles_x, tiles_y;
    TmaSplits splits;
    float* partials;  // [slices][tiles_y][tiles_x][region]
    long long part_cap;  // floats allocated at partials
};
// Batched phase 1: every instance's tensor map travels in the kernel parameters.
constexpr int kMaxBatch = 96;
// Cycles (about 2 s at 2 GHz) before a bounded device wait gives up.
constexpr long long kDefaultWaitBudget = 4000000000LL;
struct BatchMaps {
    alignas(64) unsigned char m[kMaxBatch][128];
};
struct BatchInst {  // per-instance data of a batched launch (device memory)
    int H, W, tiles_x, tiles_y;
    TmaSplits splits;
    const float* d;   // scaling
    const float* z;   // second factor of q (null: q = d)
    float* part;      // partial regions of this instance
    const int* done;  // null, or a flag that, when set, makes the instance's items return
    long long part_cap;  // floats allocated at part (the checked build's bound)
};
cudaError_t launch_tma_gather_batched(int dtype, int rs, const BatchMaps& maps, const BatchInst* insts,
                                      const int4* work, int nwork, unsigned* err, cudaStream_t st);
bool tma_path_supports(int rs);
// tensor map of planes [nh][H][pitch] of type dtype (DSGNLM_F32/F16/BF16), pitch in
// elements (plane_pitch(W) when 0), with boxes of box_w x box_h x 1; reads past the
// image (W x H) return zeros
cudaError_t encode_tile_map(void* out, const void* base, int dtype, int H, int W, int nh, int box_w, int box_h,
                            int pitch = 0);
int tma_tile_w();
int tma_ctas_per_sm(int dtype);  // resident phase-1 CTAs per SM for the weight type
int tma_tile_h();
size_t tma_region_floats(int rs);
int tma_p2_blocks(int H, int W);
// phase 1: partial sums of K1 q over every tile and offset slice, q = d (z null) or d z
// wait_budget: cycles a consumer waits for a plane before the CTA gives up and sets
// *err (kDefaultWaitBudget, about 2 s; 0 gives up at the first wait); pdl: launched with
// programmatic stream serialization (the kernel waits for its predecessor)
cudaError_t launch_tma_gather(int dtype, const TmaPlan& plan, int H, int W, int rs, const float* d,
                              const float* z, unsigned* err, const int* skip, cudaStream_t st,
                              long long wait_budget = kDefaultWaitBudget, bool pdl = false);
// phase 2 epilogues
cudaError_t launch_tma_apply_finish(const TmaPlan& plan, int H, int W, int rs, const float* d,
                                    const float* t, float inv_m, const float* z, float* y,
                                    cudaStream_t st);
cudaError_t launch_reduce_residuals(SolveRed red, int iters, int nblocks, cudaStream_t st);

cudaError_t launch_fill(float* p, float value, size_t n, cudaStream_t st);

cudaError_t launch_sinkhorn_pass(int dtype, const void* planes, int H, int W, int search_r,
                                 const float* d_in, float* d_out, PassStat* stats,
                                 BalanceCtl* ctl, int pass, cudaStream_t st);

cudaError_t launch_apply(int dtype, const void* planes, int H, int W, int search_r,
                         const float* d, float inv_m, const float* z, float* y, cudaStream_t st);

// v <- W z, u <- z - v (= u + x - v), residual partial sums into red at slot `iter`
cudaError_t launch_apply_dual(int dtype, const void* planes, int H, int W, int search_r,
                              const float* d, float inv_m, const float* z, float* v, float* u,
                              SolveRed red, int iter, cudaStream_t st);
int apply_grid_blocks(int H, int W);

struct BlurTaps {
    float t[17];  // normalised 1D Gaussian taps t[a + r], a = -r..r
    int r;
};
BlurTaps make_blur_taps(float sigma, int r);

// out(q) = (A x)(q) + c * aux(q) on the [H/2][W/2] grid (aux may be null)
cudaError_t launch_sr_forward(const float* x, int H, int W, BlurTaps taps, const float* aux,
                              float c, float* out, cudaStream_t st);
// grad = A^T r at [H][W] (r on [H/2][W/2])
cudaError_t launch_sr_adjoint(const float* r, int H, int W, BlurTaps taps, float* out,
                              cudaStream_t st);
// x <- Pi_C(mu (alpha x + rho (v - u) - A^T r)), z <- x + u
cudaError_t launch_sr_xupdate(const float* r, int H, int W, BlurTaps taps, float* x,
                              const float* v, const float* u, float* z, float mu, float alpha,
                              float rho, int constraint, cudaStream_t st);
// fused: r = A x_in - y, x_out <- Pi_C(mu (alpha x_in + rho (v - u) - A^T r)), z <- x_out + u
cudaError_t launch_sr_xupdate_fused(const float* x_in, float* x_out, const float* y, int H, int W,
                                    BlurTaps taps, const float* v, const float* u, float* z, float mu,
                                    float alpha, float rho, int constraint, cudaStream_t st);
// grad f for SPI
cudaError_t launch_spi_grad(const float* x, const uint8_t* counts, int n, int K, float eta,
                            float eps, float* grad, cudaStream_t st);
// SR operator with either boundary (bc 0 periodic, 1 symmetric; sym.cu):
// out = A x + c aux (low-resolution), out = A^T rlo + rho pin (pin may be null) with
// optional block sums of pin * out in part; valid when sr_bc_supported(H, W, r).
bool sr_bc_supported(int H, int W, int blur_r);
int sr_adjoint_bc_blocks(int H, int W);
cudaError_t launch_sr_forward_bc(int bc, const float* x, int H, int W, BlurTaps taps, const float* aux, float c,
                                 float* out, cudaStream_t st);
cudaError_t launch_sr_adjoint_bc(int bc, const float* rlo, int H, int W, BlurTaps taps, float rho, const float* pin,
                                 float* out, double* part, cudaStream_t st);
// conjugate-gradient steps with device-resident scalars
struct CgScalars {
    double rs, pq, alpha, beta;
};
int cg_vector_blocks(int n);
cudaError_t launch_cg_init(const float* aty, const float* v, const float* u, float rho, const float* mx, float* r,
                           float* p, int n, double* part, cudaStream_t st);
cudaError_t launch_cg_step(float* x, float* r, const float* p, const float* q, const CgScalars* s, int n,
                           double* part, cudaStream_t st);
cudaError_t launch_cg_dir(const float* r, float* p, const CgScalars* s, int n, cudaStream_t st);
cudaError_t launch_cg_reduce(const double* part, int nb, CgScalars* s, int mode, cudaStream_t st);
cudaError_t launch_project_z(float* x, const float* u, float* z, int n, int constraint, cudaStream_t st);
// g = A^T (A x - y) in one launch (H, W even, taps.r <= 8); y null: g = A^T A x
cudaError_t launch_sr_grad(const float* x, const float* y, int H, int W, BlurTaps taps, float* g,
                           cudaStream_t st);
// x <- Pi_C(mu (alpha x + rho (v - u) - g)), z = x + u, per pixel (x in place)
cudaError_t launch_xupdate_point(float* x, const float* g, const float* v, const float* u, float* z, int n, float mu,
                                 float alpha, float rho, int constraint, cudaStream_t st);
cudaError_t launch_spi_xupdate(const uint8_t* counts, int n, int K, float eta, float eps, float* x,
                               const float* v, const float* u, float* z, float mu, float alpha,
                               float rho, int constraint, cudaStream_t st);

cudaError_t launch_sr_guide(const float* y, int h, int w, float* guide, cudaStream_t st);
cudaError_t launch_spi_observe(const float* x, const float* arrivals, int H, int W, int k_side,
                               float eta, uint8_t* bits, cudaStream_t st);
cudaError_t launch_spi_counts(const uint8_t* bits, int H, int W, int k_side, uint8_t* counts,
                              cudaStream_t st);
cudaError_t launch_spi_guide(const uint8_t* counts, int H, int W, int K, float eta, float* guide,
                             cudaStream_t st);
cudaError_t launch_init(const float* guide, int n, float* x, float* v, float* u, cudaStream_t st);

// Epilogues (epilogue.cu)
int balance_combine_blocks(int H, int W);  // blocks (and residual pairs) of one balance epilogue
// One balancing pass's epilogue (t, next d, residual pairs); with `decide` the
// last block applies the stopping rule and, with use_cond, sets the graph's WHILE
// condition.
cudaError_t launch_balance_epilogue(const TmaPlan& plan, int H, int W, int rs, const float* d_in, float* d_out,
                                    float* t_out, float2* part, BalanceCtl* ctl, int decide,
                                    cudaGraphConditionalHandle cond, int use_cond, cudaStream_t st);

struct EpilogueArgs {
    int H, W;
    const float* d;
    const float* t;
    float inv_m;
    const float* inv_m_dev;  // when set, 1/m is read here instead (written by the balance)
    float* z;          // in: x + u of this iteration; out: x + u of the next one
    float* v;
    float* u;
    const float* x_in;   // x of the next update (SR, fused form: read in halos)
    float* x_out;        // its result (SR, fused form: another buffer; otherwise may equal x_in)
    const float* y;      // SR observation
    float* g;            // SR, per-pixel form: A^T (A x_in - y), computed beforehand
    BlurTaps taps;
    const uint8_t* counts;  // SPI
    int K;
    float eta, eps;
    float mu, alpha, rho;
    int constraint;
    int do_x;            // 0 on the last iteration
    double* partials;    // this iteration's per-block residual sums [nblocks][2]
};
int combine_xupdate_blocks(int H, int W);  // epilogue tiles (kXH x kXW) of an image
// Finish v, u of one iteration and perform the next x-update, per pixel (SR takes
// the gradient from args.g); one residual pair per epilogue tile.
cudaError_t launch_combine_update(int kind, const TmaPlan& plan, int rs, const EpilogueArgs& args,
                                  cudaStream_t st, bool pdl = false);

// Batched Algorithm 1 (batched.cu).  x is updated in place (a.x_in == a.x_out); SR
// reads the gradient of the current x from a.g.
struct BatchEpi {
    EpilogueArgs a;
    Cover cv;
    int gx;            // epilogue tiles per row
    int nblocks;       // epilogue tiles of the image
    double* partials;  // [iters][nblocks][2] residual sums
};
cudaError_t launch_batched_xupdate0(int kind, const BatchEpi* insts, const int4* work, int nwork, cudaStream_t st);
cudaError_t launch_batched_combine(int kind, const BatchEpi* insts, const int4* work, int nwork, int it, int last,
                                   cudaStream_t st);
// g of every image on (image, 32 x 32 tile) work items; every image with blur radius blur_r
cudaError_t launch_batched_grad(int blur_r, const BatchEpi* insts, const int4* work, int nwork, cudaStream_t st);
cudaError_t launch_batched_reduce(const BatchEpi* insts, int count, double* hist, int iters, cudaStream_t st);

// Batched balance (batched.cu): the balancing passes of many handles advance
// together, one phase-1 launch (launch_tma_gather_batched, q = d) and one epilogue
// launch per pass over the work items of every image that has not stopped.  Each
// image keeps its own plan, buffers and stopping rule (its BalanceCtl), so its
// result equals its own dsgnlm_balance bit for bit.
struct BatchBal {
    Cover cv;             // the image's phase-1 partial regions
    int H, W;
    int nbx, nblocks;     // epilogue blocks (kXH x kXW) per row and in all
    float* d[2];          // scaling of passes with parity 0 and 1 (each pass writes the other)
    float* t[2];          // K1 d of passes with parity 0 and 1
    float2* part;         // per epilogue block (max |d t - 1|, max d t)
    BalanceCtl* ctl;
};
// work: (image, block row, block column, -) items over every image's epilogue blocks;
// *stopped counts the images whose balance has stopped
cudaError_t launch_batched_balance_epilogue(const BatchBal* bb, const int4* work, int nwork, int parity,
                                            unsigned* stopped, cudaStream_t st);

}  // namespace dsg
