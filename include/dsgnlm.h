/*
 * dsgnlm.h -- C ABI of the GB300 (sm_103a) library for doubly stochastic nonlocal
 * means (DSG-NLM) and linearized plug-and-play ADMM.
 *
 * The method is that of Unni, Ghosh and Chaudhury, "Linearized ADMM and Fast
 * Nonlocal Denoising for Efficient Plug-and-Play Restoration": the denoiser is
 * W z with W the symmetric, doubly stochastic matrix obtained from the NLM kernel
 * by the hat window (Eq. S1), symmetric normalisation (Eq. S2) and the scaling
 * and diagonal closure of Eq. S3, computed without storing W as a matrix
 * (Algorithm 2); the outer solver is Algorithm 1.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Images are FP32, row-major [H][W] (row i, column j at i*W + j), contiguous.
 * - Pointers documented as "device" must be device (or managed) memory on the
 *   current CUDA device, 16-byte aligned for FP32/weight arrays.  "host" pointers
 *   are ordinary host memory.
 * - Buffers passed in are owned by the caller and are never freed by the library.
 *   A dsgnlm_t handle owns its weight planes and its scratch; dsgnlm_destroy frees
 *   them.
 * - All work is issued on the handle's CUDA stream (or the stream argument) and is
 *   asynchronous unless an entry point returns host values, in which case it
 *   synchronises that stream before returning.
 * - Errors are reported by the return code only; nothing aborts or prints.  After
 *   DSGNLM_ECUDA, dsgnlm_last_cuda_error() returns the CUDA error code.
 * - One handle must not be used from two host threads at once.
 */
#ifndef DSGNLM_H
#define DSGNLM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dsgnlm* dsgnlm_t;

typedef enum dsgnlm_status {
    DSGNLM_OK = 0,
    DSGNLM_EINVAL = 1,         /* bad argument: null pointer, size or radius out of range,
                                  misaligned pointer, unknown enum value */
    DSGNLM_ENOMEM = 2,         /* a device allocation failed */
    DSGNLM_ECUDA = 3,          /* a CUDA runtime call or launch failed */
    DSGNLM_NOT_BUILT = 4,      /* balance/apply/solve before dsgnlm_build */
    DSGNLM_NOT_BALANCED = 5,   /* apply/solve before dsgnlm_balance */
    DSGNLM_NOT_CONVERGED = 6,  /* balance made maxit updates with the residual above tol;
                                  W is still exactly symmetric and doubly stochastic */
    DSGNLM_STALLED = 7,        /* the balance residual stopped decreasing above tol (the
                                  FP32 floor of the scaling); W is still doubly stochastic */
    DSGNLM_TIMEOUT = 8         /* a bounded device-side wait gave up */
} dsgnlm_status;

/* storage type of the weight planes */
enum { DSGNLM_F32 = 0, DSGNLM_F16 = 1, DSGNLM_BF16 = 2 };

/* limits of the kernels (shared-memory tiles are sized from them) */
enum { DSGNLM_MAX_PATCH_R = 14, DSGNLM_MAX_SEARCH_R = 24 };
/* Update rules of the balance (dsgnlm_set_balance_scheme). */
enum { DSGNLM_BALANCE_SINKHORN = 0, DSGNLM_BALANCE_ACCELERATED = 1 };

/* ---------------------------------------------------------------------------
 * Denoiser handle
 * ------------------------------------------------------------------------- */

/* Create a handle whose work runs on `stream` (a cudaStream_t, NULL = legacy default
 * stream) and whose weight planes are stored as `weight_dtype` (DSGNLM_F32, _F16 or
 * _BF16; the arithmetic is FP32 in every case).  *out receives the handle. */
dsgnlm_status dsgnlm_create(dsgnlm_t* out, void* stream, int weight_dtype);

/* Release the handle and everything it owns.  Synchronises its stream first. */
void dsgnlm_destroy(dsgnlm_t h);

/* Rebind the handle to another stream. */
dsgnlm_status dsgnlm_set_stream(dsgnlm_t h, void* stream);

/* Weight build (Eq. NLM and Eq. S1; first aggregation of Algorithm 2; fast patch
 * distances of Sec. 3 whose cost does not grow with the patch size).
 *
 * guide      device, [H][W] FP32: the image the patches are taken from.
 * patch_r    patch radius: patches are N_p x N_p with N_p = 2*patch_r + 1 (0..14).
 * search_r   search radius N_s: the window is (2 N_s + 1)^2, clipped at the image
 *            border (0..24).
 * bandwidth  h > 0: k_{s,r} = exp(-||P_s - P_r||^2 / (2 N_p^2 h^2)).
 *
 * Patch pixels outside the image read the guide under half-sample symmetric
 * reflection.  For each of the n_h = 2 N_s (N_s + 1) offsets o of the half window
 * (o_y > 0, or o_y = 0 and o_x > 0) the handle stores the plane
 *     K1(s, s + o) = Lambda(o / (N_s + 1)) k_{s, s+o}   (0 where s + o is outside),
 * laid out [n_h][H][W] in the handle's weight dtype.  The other half of the window
 * follows from the symmetry K1(s, s - o) = K1(s - o, s) and the diagonal is 1.
 * (Re)allocates the planes if the size changed; clears any previous balance. */
dsgnlm_status dsgnlm_build(dsgnlm_t h, const float* guide, int H, int W,
                           int patch_r, int search_r, float bandwidth);

/* Balance (Eq. S2 iterated as symmetric Sinkhorn-Knopp, then Eq. S3; second
 * aggregation of Algorithm 2).
 *
 * From d = 1, repeats d <- sqrt(d / (K1 d)) until max_s |d_s (K1 d)_s - 1| <= tol
 * or `maxit` updates were made.  maxit = 1 gives d = g^{-1/2} (g the row sums of
 * K1), i.e. exactly the paper's one-shot normalisation.  Then m = max_s d_s (K1 d)_s
 * and the denoiser is W = diag(d) K1 diag(d) / m with the diagonal closed so that
 * every row sums to one (Eq. S3).  W is symmetric and doubly stochastic for any d.
 * The residual is reduced in FP64 from FP32 scalings; if it stops decreasing (three
 * passes without a 1% improvement) above tol the balance stops with STALLED.
 *
 * iters_out  host, optional: number of updates made.
 * resid_out  host, optional: the final residual max_s |d_s (K1 d)_s - 1|.
 * Synchronises the stream.  Returns OK, NOT_CONVERGED or STALLED (all leave a
 * usable W), NOT_BUILT, EINVAL (tol < 0, maxit < 0) or a CUDA error. */
dsgnlm_status dsgnlm_balance(dsgnlm_t h, double tol, int maxit,
                             int* iters_out, double* resid_out);

/* Update rule of this handle's balances (dsgnlm_balance, and its images in
 * dsgnlm_balance_batched).  DSGNLM_BALANCE_SINKHORN (the default): every pass is
 * the symmetric Sinkhorn step d <- sqrt(d / K1 d) (Eq. S2 iterated), so the scaling
 * after k updates is the oracle's after k updates.  DSGNLM_BALANCE_ACCELERATED
 * (search radii with the stencil kernel; others keep the plain step): the first
 * two passes are that step, later ones the heavy-ball step on log d,
 * d <- d (d K1 d)^(-a/2) (d / d_prev)^b with a = 4 / (1 + sqrt(1/2))^2 and
 * b = ((1 - sqrt(1/2)) / (1 + sqrt(1/2)))^2, which contracts the error about three
 * times faster per pass near the fixed point.  Its fixed point, d (K1 d) = 1, is
 * the plain step's, so a balance to a tolerance ends within that tolerance of the
 * same doubly stochastic W in fewer passes (9 instead of 17 to 1e-6 for the
 * 7x7 / 21x21 kernel of a 512x512 image); the stopping rule is unchanged.  (No
 * counterpart in the paper, which normalises once.)  EINVAL for another value. */
dsgnlm_status dsgnlm_set_balance_scheme(dsgnlm_t h, int scheme);

/* Balance `count` (1..96) built handles together: the passes of dsgnlm_balance, each
 * pass one phase-1 launch and one epilogue launch over the work items of every
 * image, each image's buffers and stopping rule kept.  With slices = 0 every image
 * also keeps its own offset schedule, so that its scaling, m, update count and
 * residual equal those of dsgnlm_balance on it, bit for bit; slices > 0 splits the
 * offsets of every image into that many slices (as lpnp_solve_batched_sched: a
 * batch fills the GPU by itself, and fewer slices read and write fewer partial
 * sums), which changes only the order of FP32 sums.  An image's items return at once
 * after the pass that stops it; the host reads the number of stopped images every
 * four passes.  All handles must be distinct, built on the stencil path (search
 * radius 1-8, 10 or 12) with the same search radius and weight dtype; the work runs
 * on hs[0]'s stream, after the other handles' streams are synchronised.
 *
 * hs          host array of count handles.
 * iters_out, resid_out, status_out
 *             host arrays of count entries, optional (NULL): per handle, the updates
 *             made, the final residual, and OK, NOT_CONVERGED or STALLED.
 * Synchronises the stream.  Returns OK (every handle is then balanced and usable),
 * EINVAL (bad count, tol or maxit, a handle repeated, off the stencil path or
 * mismatched), NOT_BUILT, TIMEOUT or a CUDA error. */
dsgnlm_status dsgnlm_balance_batched(dsgnlm_t* hs, int count, double tol, int maxit, int slices, int* iters_out,
                                     double* resid_out, int* status_out);

/* Apply y = W x (third aggregation of Algorithm 2).
 * x, y  device, [H][W] FP32; y must not alias x.  Asynchronous: a bounded device
 * wait that gives up during the call is reported by the next dsgnlm_sync (or by
 * the next balance or solve on the handle that reads the error word). */
dsgnlm_status dsgnlm_apply(dsgnlm_t h, const float* x, float* y);

/* Wait for the work queued on the handle's stream, then read and clear the handle's
 * device error word.  Returns TIMEOUT if a bounded wait of a stencil kernel gave up
 * since the word was last read (the outputs of that work are then invalid; the
 * handle stays usable), OK otherwise, or a CUDA error.  (No counterpart in the
 * paper: the asynchronous error report of this library.) */
dsgnlm_status dsgnlm_sync(dsgnlm_t h);

/* Test hook of the bounded waits (no counterpart in the paper).  In every phase-1
 * stencil launch of this handle, a consumer thread waits at most `cycles` GPU
 * clock cycles for a weight tile to land in shared memory; then the CTA sets the
 * handle's error word, stops, lets its copies in flight land and returns, so no
 * kernel waits without bound.  0 makes every consumer give up at its first wait
 * (the timeout path, without a fault or a hang); a negative value restores the
 * default of 4e9 cycles (about 2 s).  Releases the handle's recorded graphs when
 * the value changes (synchronises the stream).  EINVAL above the default. */
dsgnlm_status dsgnlm_set_wait_budget(dsgnlm_t h, long long cycles);

/* Diagnostics for tests: copy the weight planes ([n_h][H][W], weight dtype) to the
 * device buffer dst; copy the final scaling d ([H][W] FP32) to the device buffer
 * d_dst and m to *m_host.  dsgnlm_copy_scaling synchronises the stream. */
dsgnlm_status dsgnlm_copy_weights(dsgnlm_t h, void* dst);
dsgnlm_status dsgnlm_copy_scaling(dsgnlm_t h, float* d_dst, double* m_host);

/* Number of half-window offsets n_h of the current build (0 before a build). */
int dsgnlm_num_offsets(dsgnlm_t h);

/* ---------------------------------------------------------------------------
 * Forward models, measurements and guides (Sec. 4)
 * ------------------------------------------------------------------------- */

/* Super-resolution observation y = A x + n (Sec. 4.1): periodic blur by the
 * normalised (2 blur_r + 1)^2 Gaussian of std blur_sigma, keep pixels (2i, 2j),
 * add `noise`.  x device [H][W]; noise, y device [H/2][W/2]; H, W even.
 * noise may be NULL (y = A x). */
dsgnlm_status lpnp_sr_observe(const float* x, const float* noise, int H, int W,
                              float blur_sigma, int blur_r, float* y, void* stream);

/* lpnp_sr_observe with the blur boundary `boundary` (LPNP_BC_PERIODIC or
 * LPNP_BC_SYMMETRIC; the symmetric blur needs H, W >= 2 blur_r). */
dsgnlm_status lpnp_sr_observe_bc(const float* x, const float* noise, int H, int W, float blur_sigma, int blur_r,
                                 int boundary, float* y, void* stream);

/* Guide for super-resolution: 2x Keys cubic (a = -0.5) interpolation of y with
 * periodic wrap, low-resolution sample j at high-resolution 2j (the bicubic guide
 * of the F-DSG-NLM variant, Sec. 4).  y device [h][w]; guide device [2h][2w].
 * Asynchronous on `stream`.  EINVAL for null pointers or h, w < 1. */
dsgnlm_status lpnp_sr_guide(const float* y, int h, int w, float* guide, void* stream);

/* Single-photon measurement (Sec. 4.2): pixel i has K = k_side^2 sub-pixels; a
 * sub-pixel reads one iff its first photon arrival E ~ Exp(1) (`arrivals`) is
 * below the rate eta x_i / K, i.e. iff its Poisson count is >= 1.  The rate is
 * formed in FP32 as (eta * x_i) / K.
 * x device [H][W]; arrivals device FP32 and bits device uint8, [k_side H][k_side W]. */
dsgnlm_status lpnp_spi_observe(const float* x, const float* arrivals, int H, int W,
                               int k_side, float eta, uint8_t* bits, void* stream);

/* K1_i: number of ones among the k_side x k_side sub-pixels of pixel i (Sec. 4.2).
 * bits device uint8 in {0, 1}, [k_side H][k_side W]; counts device uint8 [H][W].
 * k_side in 1..15. */
dsgnlm_status lpnp_spi_counts(const uint8_t* bits, int H, int W, int k_side,
                              uint8_t* counts, void* stream);

/* Guide for single-photon imaging: per-pixel maximum-likelihood intensity
 * -(K/eta) log(1 - K1/K) clipped to [0, 1], then a 3x3 mean with symmetric
 * reflection.  counts device uint8 [H][W]; guide device [H][W]. */
dsgnlm_status lpnp_spi_guide(const uint8_t* counts, int H, int W, int K, float eta,
                             float* guide, void* stream);

/* Initial state of Algorithm 1: x = v = clip(guide, 0, 1), u = 0 (n pixels). */
dsgnlm_status lpnp_init(const float* guide, int n, float* x, float* v, float* u,
                        void* stream);

/* ---------------------------------------------------------------------------
 * Linearized plug-and-play ADMM (Algorithm 1)
 * ------------------------------------------------------------------------- */

enum { LPNP_SR2 = 0, LPNP_SPI = 1 };
enum { LPNP_C_NONE = 0, LPNP_C_NONNEG = 1, LPNP_C_BOX01 = 2 };
/* boundary of the SR blur: periodic (Sec. 4.1's main model) or half-sample
 * symmetric reflection (the standard-vs-linearized comparison of Sec. 4.1) */
enum { LPNP_BC_PERIODIC = 0, LPNP_BC_SYMMETRIC = 1 };

typedef struct lpnp_problem {
    int kind;              /* LPNP_SR2 (2x super-resolution) or LPNP_SPI */
    int H, W;              /* high-resolution image size (even for LPNP_SR2) */
    /* LPNP_SR2: f(x) = 1/2 ||y - A x||^2 (Eq. dataterm), grad f = A^T (A x - y) */
    const float* y;        /* device [H/2][W/2] observation */
    float blur_sigma;      /* std of the Gaussian blur */
    int blur_r;            /* blur radius (taps 2 r + 1 per axis), 0..8 */
    /* LPNP_SPI: f(x) = sum_i h(x_i) (Eq. obj), grad evaluated at max(x_i, spi_eps) */
    const uint8_t* counts; /* device [H][W] one-counts K1_i */
    int K;                 /* sub-pixels per pixel */
    float eta;             /* sensor gain */
    float spi_eps;         /* floor of x inside h' (h' is unbounded at 0) */
    int constraint;        /* LPNP_C_NONE, _NONNEG or _BOX01 (the set C of Pi_C) */
    float alpha;           /* linearization weight; > Lipschitz constant of grad f */
    dsgnlm_t den;          /* built and balanced denoiser (F-DSG-NLM: W fixed) */
    float* x;              /* device [H][W], in: initial x, out: final x */
    float* v;              /* device [H][W], in/out */
    float* u;              /* device [H][W], in/out (scaled multiplier) */
    double* resid_hist;    /* host [iters][2] or NULL: RMS primal ||x - v|| / sqrt(n)
                              and dual rho ||v - v_prev|| / sqrt(n) per iteration */
    int blur_boundary;     /* LPNP_SR2: LPNP_BC_PERIODIC or LPNP_BC_SYMMETRIC; the symmetric
                              blur needs H, W >= 2 blur_r and a denoiser on the stencil
                              path (search radius 1-8, 10 or 12) */
} lpnp_problem;

/* grad f(x) of the problem's data term (debug/tests).  x, grad device [H][W]. */
dsgnlm_status lpnp_gradient(const lpnp_problem* p, const float* x, float* grad);

/* Run `iters` iterations of Algorithm 1 with penalty rho > 0, mu = 1/(alpha + rho):
 *   x <- Pi_C(mu (alpha x + rho (v - u) - grad f(x)));  v <- W (x + u);  u <- u + x - v.
 * Uses p->den's handle stream.  Synchronises only if resid_hist is given.  On the
 * stencil path (and with profiling off, iters > 1) the kernel sequence is recorded as
 * a CUDA graph on the handle and replayed while the problem's buffers, sizes and
 * parameters are unchanged; the handle keeps two such graphs.  The observation (or
 * counts) is first copied into the handle, and after dsgnlm_balance the graphs read 1/m
 * on the device, so another image and W of the same size replay them. */
dsgnlm_status lpnp_solve(const lpnp_problem* p, float rho, int iters);

/* Standard PnP-ADMM for LPNP_SR2 (the comparison system of Sec. 4.1): the x-update
 * minimises f(x) + rho/2 ||x - (v - u)||^2 by `cg_iters` (>= 1) conjugate-gradient
 * steps on (A^T A + rho I) x = A^T y + rho (v - u), started from the current x, then
 * projects onto C; v <- W (x + u), u <- u + x - v as lpnp_solve.  alpha is unused.
 * The CG scalars stay on the device (no host round trips); synchronises only if
 * resid_hist is given.  EINVAL for SPI problems, cg_iters < 1, or a denoiser off
 * the stencil path. */
dsgnlm_status lpnp_solve_standard(const lpnp_problem* p, float rho, int iters, int cg_iters);

/* Algorithm 1 with W rebuilt from the denoiser input (Sec. 4): in each of the first
 * `adapt_iters` iterations (>= 1) the weights are built from z = x + u, after the
 * x-update, with the given patch radius, search radius and bandwidth (as
 * dsgnlm_build), then balanced to `tol` within `maxit` updates (as dsgnlm_balance;
 * a balance that ends NOT_CONVERGED or STALLED is accepted, W is still doubly
 * stochastic), and W z is formed; later iterations keep the last W.  adapt_iters >=
 * iters is A-DSG-NLM; a smaller value is the paper's F-DSG-NLM schedule (adapt for
 * about 15 iterations, then freeze).  p->den need not be built: its weights are
 * replaced, and on return it holds the last W, balanced.  search_r must be one the
 * stencil path supports (1-8, 10, 12), else DSGNLM_EINVAL; other errors as
 * lpnp_solve, dsgnlm_build and dsgnlm_balance.  Synchronises once per adaptation. */
dsgnlm_status lpnp_solve_adaptive(const lpnp_problem* p, float rho, int iters, int adapt_iters, int patch_r,
                                  int search_r, float bandwidth, double tol, int maxit);

/* Allocation-free super-resolution gradient: grad = A^T (A x - y) with the
 * PERIODIC blur, the same result as lpnp_gradient for a LPNP_SR2 problem whose
 * blur_boundary is LPNP_BC_PERIODIC (there is no symmetric-boundary form of this
 * call; such a problem needs lpnp_gradient), for callers that cannot
 * allocate device memory when they need it (a plugin whose host framework owns
 * every device allocation, a real-time loop that forbids allocation after
 * start-up).  The paper has no counterpart: this is a deployment variant.
 *
 * x, grad device [H][W]; y device [H/2][W/2]; H, W even; blur_sigma, blur_r as in
 * lpnp_problem, always with periodic wrap.
 * Its scratch, the low-resolution residual A x - y, lives in one static device
 * array of 1,048,576 floats (4 MiB) that every GPU loading the library keeps until
 * exit, so (H/2)(W/2) must not exceed 1,048,576 (e.g. 2048 x 2048); larger sizes
 * return DSGNLM_EINVAL before any work.  The call allocates nothing.  All calls on
 * a device share that array: calls that overlap on the GPU (other streams, other
 * host threads) race and must be serialised.  Every call overwrites the part it
 * reads, so no state carries over between calls.  The first call on a device
 * resolves the array's address (this may load the library's module onto the
 * device) and should come before any stream capture on that device.  The address
 * is kept for the life of the process: do not use this call on a device after
 * cudaDeviceReset or after its primary context was destroyed and created again
 * (the module may then sit at another address).
 * Asynchronous on `stream`. */
dsgnlm_status lpnp_sr_gradient_noalloc(const float* x, const float* y, int H, int W,
                                       float blur_sigma, int blur_r, float* grad, void* stream);

/* Batched Algorithm 1: `count` independent images (1..96) of any sizes advance
 * together; each iteration is one phase-1 launch and one combine/x-update launch
 * over a work-list of (image, tile) items of all images.  Same arguments and
 * results as calling lpnp_solve on each problem, image by image.  All problems
 * must have the same kind, and their denoisers (one distinct handle each, built
 * and balanced, all on a search radius with a TMA kernel) the same weight dtype
 * and search radius.  Work runs on probs[0].den's stream; the caller orders the
 * other handles' earlier work before it.  Synchronises only if a resid_hist is
 * given.  EINVAL for mixed batches or count out of range. */
dsgnlm_status lpnp_solve_batched(const lpnp_problem* probs, int count, float rho, int iters);

/* lpnp_solve_batched with an offset schedule: `slices` > 0 splits the window
 * offsets of every image into that many slices (phase-1 work items per tile);
 * 0 keeps each handle's own plan, which is sized for one image alone on the GPU.
 * Fewer slices mean fewer partial regions to combine; more mean more work items.
 * Results agree with the handles' own plans up to FP32 summation order.  The step
 * sequence of a batch is recorded into a CUDA graph on probs[0].den and replayed
 * while the batch (buffers, sizes, iters, schedule) is unchanged. */
dsgnlm_status lpnp_solve_batched_sched(const lpnp_problem* probs, int count, float rho, int iters, int slices);

/* Autotuner for the batched schedule (no counterpart in the paper): for each of
 * the `ncand` candidate slice counts (>= 0, as lpnp_solve_batched_sched), runs one
 * warm-up iteration and `trial_iters` timed iterations of the batch on copies of
 * the iterates (the problems' x, v, u are not modified; the weights are only read),
 * and returns the fastest candidate in *best_slices and, if ms_per_iter is not
 * NULL, the milliseconds per iteration of each candidate in ms_per_iter[ncand].
 * Allocates and frees three images per problem; synchronises. */
dsgnlm_status lpnp_tune_batched(const lpnp_problem* probs, int count, float rho, const int* candidates, int ncand,
                                int trial_iters, int* best_slices, float* ms_per_iter);

/* ---------------------------------------------------------------------------
 * Differentiable form: unrolled Algorithm 1 and its adjoint
 * ------------------------------------------------------------------------- */

typedef struct lpnp_tape* lpnp_tape_t;

/* A tape holds the checkpoints of one unrolled solve (every balancing scaling and
 * row sum, every iterate) for lpnp_backward.  Owned by the caller. */
dsgnlm_status lpnp_tape_create(lpnp_tape_t* out);
void lpnp_tape_destroy(lpnp_tape_t t);

/* Unrolled 2x super-resolution solve with every discrete choice fixed so that x_N is
 * differentiable in (y, guide, bandwidth, rho):
 *   K1 from `guide` (Eq. NLM, S1; radii and bandwidth as in dsgnlm_build) into `den`;
 *   exactly `balance_passes` passes d <- sqrt(d / K1 d) from d = 1 (Eq. S2 iterated,
 *   no tolerance stop), m = max_s d_s (K1 d)_s, W by Eq. S3;
 *   `iters` iterations of Algorithm 1 (box constraint [0,1], blur as in lpnp_problem)
 *   from x = v = clip(guide, 0, 1), u = 0.
 * y device [H/2][W/2]; guide device [H][W]; both must stay unchanged until
 * lpnp_backward.  x_out device [H][W] receives x_N.  Records the tape (replacing any
 * earlier recording).  `den` must not be rebuilt before the backward.  The shared
 * memory of the backward limits (4 ceil(iters / 2) + 2)(16 + N_s)(32 + 2 N_s) floats
 * (pair pass G) and (2 passes + 1)(16 + N_s)(32 + 2 N_s) floats to 220 KiB (EINVAL
 * otherwise).  m and 1/m are formed and read on the device, so the call queues all of
 * its work without waiting for the device (on an error it drains the stream first);
 * the handle reads m and 1/m back when a later call on it needs them on the host.
 * The iterations run their own kernels (the dual step of each also takes the next
 * x-step; the gradient it uses is formed beside the weight stream); every step, the
 * weight build included, is recorded once per configuration as a CUDA graph (on a
 * stream the tape owns) and replayed on the handle's stream. */
dsgnlm_status lpnp_unrolled_forward(lpnp_tape_t tape, dsgnlm_t den, const float* y, const float* guide, int H,
                                    int W, int patch_r, int search_r, float bandwidth, int balance_passes,
                                    float alpha, float rho, int iters, float blur_sigma, int blur_r, float* x_out);

/* Adjoint of the recorded solve for the cotangent x_bar of x_N (device [H][W]):
 * y_bar (device [H/2][W/2]) and guide_bar (device [H][W]) receive dL/dy and
 * dL/dguide; *h_bar and *rho_bar (host, optional) dL/dbandwidth and dL/drho.  The
 * derivative of the box projection and of the clip of the initial state is taken as
 * 1 strictly inside and 0 outside; m's derivative follows its first maximiser.
 * Synchronises the stream. */
dsgnlm_status lpnp_backward(lpnp_tape_t tape, const float* x_bar, float* y_bar, float* guide_bar, double* h_bar,
                            double* rho_bar);

/* Batched forms of the two calls above (Algorithm 1 unrolled, with Eq. S1-S3 for W;
 * the paper has no derivatives) for `count` images of one size and one parameter
 * set.  tapes[i] and dens[i] must be distinct.  y, guide, x_out (and x_bar, y_bar,
 * guide_bar) are host arrays of `count` device pointers with the layouts of the
 * single-image calls.  The images advance in lockstep: every step of the forward
 * (the weight build of all images included) and of the backward is one launch over
 * all images, queued on the first image's handle stream (dens[0], or the first tape's
 * handle for the backward) after the work already queued on the other handles'
 * streams; those streams then wait for the batch, so work queued on them afterwards
 * follows it.  Each call's launch sequence is recorded as a CUDA graph the first time
 * a configuration (sizes, radii, counts, buffers) is seen, on a stream the first tape
 * owns, and replayed on the handle's stream afterwards.  No image waits for the device
 * while it is queued (m and 1/m are formed and read on the device).  The forward
 * returns without waiting for the device; the backward synchronises the stream once,
 * at its end.  h_bar and rho_bar (host, optional) receive `count` per-image values.
 * Each handle's offset split (the slices of phase 1) is sized for `count` images at
 * once, so results equal the single-image calls up to the order in which W's partial
 * sums are added (bit for bit where the split is the same), and repeated calls give
 * identical results.  On an error the batch's streams are drained, the status of the
 * first failing image is returned and the tapes of the batch hold no usable
 * recording. */
dsgnlm_status lpnp_unrolled_forward_batched(lpnp_tape_t* tapes, dsgnlm_t* dens, int count, const float* const* y,
                                            const float* const* guide, int H, int W, int patch_r, int search_r,
                                            float bandwidth, int balance_passes, float alpha, float rho, int iters,
                                            float blur_sigma, int blur_r, float* const* x_out);
dsgnlm_status lpnp_backward_batched(lpnp_tape_t* tapes, int count, const float* const* x_bar, float* const* y_bar,
                                    float* const* guide_bar, double* h_bar, double* rho_bar);

/* ---------------------------------------------------------------------------
 * Misc
 * ------------------------------------------------------------------------- */

/* Per-kernel timing.  While enabled, the handle brackets each launch of the listed
 * kinds with CUDA events on its stream (DSGNLM_PROF_XUPDATE covers the data-term
 * kernels of one iteration of Algorithm 1).  Enabling (or re-enabling) clears the
 * records.  dsgnlm_profile_read synchronises the stream and returns the summed
 * event time in milliseconds and the number of timed launches of one kind. */
enum { DSGNLM_PROF_BUILD = 0, DSGNLM_PROF_BALANCE = 1, DSGNLM_PROF_APPLY = 2, DSGNLM_PROF_XUPDATE = 3 };
dsgnlm_status dsgnlm_profile_enable(dsgnlm_t h, int enable);
dsgnlm_status dsgnlm_profile_read(dsgnlm_t h, int kind, double* total_ms, int* launches);

/* Total number of kernels this library has launched in this process (a graph
 * replay counts each of its kernel nodes). */
uint64_t dsgnlm_launch_count(void);

/* Checked build.  The library built with -DDSGNLM_CHECKED (lib/libdsgnlm_checked.so)
 * tests the computed offsets of its gathers and scattered writes against the sizes of
 * the buffers they address: the weight planes the build writes, the phase-1 partial
 * regions (written by phase 1, read by every finish), the G planes and the window
 * partials of the adjoint.  A failed test sets a bit of a device word (1 weight planes,
 * 2 phase-1 partials, 8 G planes, 16 adjoint window partials, 0x80000000 the self
 * test) and skips the access, so an index error shows in the word instead of as a
 * fault.
 *   dsgnlm_is_checked: 1 in the checked build, 0 otherwise.
 *   dsgnlm_check_word: the OR of the words of every translation unit (0 in the normal
 *     build); with clear != 0 the words are reset.  Synchronises the device.
 *   dsgnlm_check_selftest: one thread tests `index` against `bound` with the checked
 *     build's test (bit 0x80000000) and touches no buffer; it checks the mechanism
 *     without an out-of-range access. */
int dsgnlm_is_checked(void);
dsgnlm_status dsgnlm_check_word(unsigned* word, int clear);
dsgnlm_status dsgnlm_check_selftest(long long index, long long bound);

/* CUDA error code (cudaError_t) of the most recent DSGNLM_ECUDA in this thread. */
int dsgnlm_last_cuda_error(void);

/* Static description of a status code. */
const char* dsgnlm_strerror(dsgnlm_status s);

#ifdef __cplusplus
}
#endif

#endif /* DSGNLM_H */
