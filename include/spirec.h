/*
 * spirec.h -- C ABI of the GB300 regularized spiral-MRI reconstruction library
 * (libspirec.so).
 *
 * The library minimises the criterion of section 3.3 of Boubertakh et al.,
 * "Regularized Reconstruction of MR Images from Spiral Acquisitions":
 *
 *     J(f) = ||s - H f||^2 + lambda1 Omega1(f) + lambda0 Omega0(f)
 *
 * with the exact, interpolation-free Fourier operator of Eq. ModDirect,
 *
 *     (H f)_l = (1/N) sum_{n,m=0}^{N-1} f[n][m] exp(+i 2 pi (kx_l m + ky_l n)),
 *
 * through the rewriting of section 3.4 (Eq. NewCritLS): the data enter once as
 * D = H^H s (Eq. AnnMatGD), the trajectory once as G (Eq. AnnMatG), and every
 * iteration of the Polak-Ribiere conjugate gradient runs in the image domain,
 * with H^H H applied as a zero-padded M x M FFT convolution by conj(G).
 *
 * Conventions (every entry point):
 *   - Images f[n][m] are N x N, row-major (f[n*N + m]); n is the row index and
 *     pairs with ky, m the column index and pairs with kx (Eq. ModDirect).
 *   - Complex arrays are interleaved (re, im) float32: an image is 2*N*N floats,
 *     a data vector 2*L floats.
 *   - Trajectories are float64 arrays kx[L], ky[L] in cycles/pixel, every value
 *     in [-0.5, 0.5] (section 2).
 *   - Gradients are dJ/dRe f + i dJ/dIm f, so the data-term gradient is
 *     2 (T f - D) with T = H^H H (section 3.4, Appendix B).
 *   - Every function returns a spirec_status; none aborts or traps the GPU.
 *     On failure spirec_last_error() gives a message (thread-local).
 *   - Functions without the _dev suffix take HOST pointers: the library copies
 *     inputs in and results out and returns after the copy-out finished.
 *     Functions with the _dev suffix take DEVICE pointers (current device),
 *     enqueue their work on the plan's stream and return without waiting; the
 *     caller keeps those buffers alive until spirec_sync() or a later
 *     stream-ordered use.
 *   - The caller owns every array it passes; the plan owns all device state it
 *     allocates (trajectory, G, the kernel spectrum, D, iterates, scratch) until
 *     spirec_plan_destroy().  A plan is not thread-safe: one host thread at a
 *     time.
 */
#ifndef SPIREC_H
#define SPIREC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct spirec_plan_s* spirec_plan;

typedef enum {
    SPIREC_OK = 0,
    SPIREC_EINVAL = -1,      /* bad argument: size, |k| > 0.5, NaN, unknown enum   */
    SPIREC_ENOMEM = -2,      /* device or host allocation failed                   */
    SPIREC_ECUDA = -3,       /* a CUDA runtime call failed                         */
    SPIREC_ESTATE = -4,      /* call out of order, e.g. solve before set_data      */
    SPIREC_EBUSY = -5,       /* resource budget exceeded                           */
    SPIREC_ETIMEOUT = -6,    /* a bounded device wait ran out                      */
    SPIREC_ENUMERIC = -7,    /* NaN or Inf met in the criterion                    */
    SPIREC_EUNSUPPORTED = -8 /* size or mode this build does not handle            */
} spirec_status;

/* Arithmetic of the trajectory contractions (G, D and H f).  The Toeplitz FFT,
 * the penalty and the CG vectors are FP32 in every mode; CG scalars are FP64.
 *   SPIREC_FP32         plain FP32 CUDA-core contraction.
 *   SPIREC_MIXED_FP16X3 tcgen05 tensor cores, each phase split into FP16 hi+lo,
 *                       products hi*hi + hi*lo + lo*hi, FP32 accumulation.
 *   SPIREC_MIXED_BF16X3 the same with BF16 hi+lo. */
typedef enum {
    SPIREC_FP32 = 0,
    SPIREC_MIXED_FP16X3 = 1,
    SPIREC_MIXED_BF16X3 = 2
} spirec_precision;

/* Penalty phi_alpha(r), r = |z| the modulus of a complex difference or pixel.
 *   HUBER       r^2 if r <= alpha, else 2 alpha r - alpha^2   (section 3.3)
 *   HYPERBOLIC  2 alpha (sqrt(alpha^2 + r^2) - alpha)         (not in the paper)
 *   QUADRATIC   r^2 (Hunt's phi, section 3.3)                              */
typedef enum {
    SPIREC_PHI_HUBER = 0,
    SPIREC_PHI_HYPERBOLIC = 1,
    SPIREC_PHI_QUADRATIC = 2
} spirec_phi;

/* Create a plan for an N x N image and L k-space samples.
 *   M          Toeplitz embedding grid side; 0 selects the smallest supported
 *              M >= 2N-1 (M = 2N for the usual sizes).  M must be >= 2N-1 and
 *              factor into 2, 3 and 5.  Sections 3.4 and Appendix B: the
 *              convolution by conj(G) is linear, so the FFT grid must hold the
 *              (2N-1)^2 lags without wrap-around.
 *   precision  spirec_precision.
 *   stream     cudaStream_t the plan orders its work after and before (NULL:
 *              the legacy default stream).  Internally the plan works on its
 *              own stream, joined to this one with events.
 *   kx, ky     optional HOST trajectory (L values each); NULL defers it to
 *              spirec_set_trajectory().
 * Allocates all device memory the plan needs; SPIREC_ENOMEM if that fails.
 * Valid sizes: 2 <= N <= 2048, 1 <= L <= 2^31. */
int spirec_plan_create(spirec_plan* out, int32_t N, int64_t L, int32_t M, int32_t precision,
                       void* stream, const double* kx, const double* ky);

/* Release every device resource of the plan.  NULL is accepted. */
int spirec_plan_destroy(spirec_plan plan);

/* Load a trajectory (L points) and build, once per trajectory:
 *   G_{u,v} = (1/N^2) sum_l exp(+i2pi(kx_l u + ky_l v)) for u in [0, N-1],
 *   v in [1-N, N-1] (Eq. AnnMatG; the other half is G_{-u,-v} = conj G_{u,v}),
 *   and the real spectrum of the M x M circulant that holds conj(G).
 * Each k is reduced exactly: it is stored as a 64-bit fixed-point fraction of a
 * cycle, so k * index mod 1 is exact before the trig call.
 * SPIREC_EINVAL if any |k| > 0.5 or a value is not finite.  Invalidates D.
 * The host variant checks the values on the host while the GPU builds G,
 * returns once the arrays are copied (the caller may then reuse them) and
 * reports a bad trajectory at once; the build itself completes in stream
 * order.  The _dev variant does not block and reports a bad trajectory
 * (SPIREC_EINVAL) at the plan's next host synchronisation: spirec_sync or
 * spirec_solve.  Either variant reports a tensor-core pipeline timeout
 * (SPIREC_ETIMEOUT) there too. */
int spirec_set_trajectory(spirec_plan plan, const double* kx, const double* ky);
int spirec_set_trajectory_dev(spirec_plan plan, const double* kx, const double* ky);

/* Load data s (2L floats) and compute, once per data set,
 *   D[n][m] = (1/N) sum_l s_l exp(-i2pi(kx_l m + ky_l n))   (Eq. AnnMatGD)
 * and ||s||^2 in FP64.  SPIREC_ESTATE without a trajectory.  The host variant
 * copies s on a side stream and returns once that copy is done (the caller
 * may then reuse s); D is computed in stream order after the trajectory's
 * work. */
int spirec_set_data(spirec_plan plan, const float* s);
int spirec_set_data_dev(spirec_plan plan, const float* s);

/* Set R(f) = lambda1 Omega1(f) + lambda0 Omega0(f) (section 3.3):
 *   Omega1 = sum phi_alpha1(|f[n+1][m]-f[n][m]|) + sum phi_alpha1(|f[n][m+1]-f[n][m]|)
 *            (free boundary: N(N-1) differences per direction),
 *   Omega0 = sum phi_alpha0(|f[n][m]|).
 * lambdas >= 0, alphas > 0 (alphas are unused by the quadratic phi). */
int spirec_set_reg(spirec_plan plan, double lambda1, double alpha1, double lambda0,
                   double alpha0, int32_t phi);

/* Run `iters` iterations of the plan's minimiser from x0 (spirec_set_minimiser;
 * for the half-quadratic one an iteration is one outer step).  The default is
 * the pseudo-conjugate gradient with the Polak-Ribiere correction (section 3.3):
 *   d0 = -grad J(x0); per iteration three majorize-minimize steps on
 *   h(t) = J(f + t d) from t = 0, f += t d, beta = max(0, Re<g',g'-g>/<g,g>),
 *   d = -g' + beta d, and d = -g' when Re<g', d> >= 0.
 * x0: 2N^2 floats or NULL (zeros).  x_out: 2N^2 floats.  J_hist: iters+1
 * doubles (J(x0), then J after each iteration) or NULL.  iters >= 0.
 * SPIREC_ESTATE before set_data and set_reg; SPIREC_ENUMERIC if J is not
 * finite at the end. */
int spirec_solve(spirec_plan plan, const float* x0, int32_t iters, float* x_out, double* J_hist);
/* Device-pointer variant; J_hist is a DEVICE array here.  The numeric check
 * is left to the caller (J_hist). */
int spirec_solve_dev(spirec_plan plan, const float* x0, int32_t iters, float* x_out,
                     double* J_hist);

/* ---- per-interleave kernel cache (series that reuse subsets of one set of
 * interleaves, e.g. dynamic imaging) ----
 * G (Eq. AnnMatG) is a sum over the samples, and the kernel spectrum is
 * linear in G, so the G and spectrum of a union of interleaves are the sums
 * of the interleaves' own.  A cache holds, for one (N, M, precision), the
 * fixed-point samples, G and spectrum of each of n interleaves; setting a
 * plan's trajectory from it copies the chosen samples and adds the cached G
 * and spectra (in the listed order) instead of building them. */
typedef struct spirec_kcache_s* spirec_kcache;
/* offsets: n + 1 increasing sample offsets into the HOST arrays kx, ky
 * (offsets[0] = 0, interleave i is [offsets[i], offsets[i+1])).  Builds every
 * interleave's G and spectrum with the plan machinery (synchronous).  Same
 * argument rules as spirec_plan_create; SPIREC_EINVAL for bad offsets or
 * trajectory values. */
int spirec_kcache_create(spirec_kcache* out, int32_t N, int32_t M, int32_t precision, int32_t n,
                         const int64_t* offsets, const double* kx, const double* ky, void* stream);
int spirec_kcache_destroy(spirec_kcache cache);
/* The plan's trajectory becomes interleaves which[0..count-1] of the cache,
 * concatenated in that order (their sample counts must add up to the plan's
 * L; 1 <= count <= 64; the plan's N and M equal the cache's, on the same
 * device).  Invalidates D, like spirec_set_trajectory. */
int spirec_set_trajectory_cached(spirec_plan plan, spirec_kcache cache, const int32_t* which, int32_t count);

/* How solve applies the normal operator H^H H to the direction each
 * iteration.  SPIREC_MODE_TOEPLITZ (the default, section 3.4 and Appendix B):
 * by the M x M zero-padded FFT convolution with the kernel spectrum built
 * once from G.  SPIREC_MODE_DIRECT (the original formulation, Eq. CritLS): by
 * the exact forward and adjoint NUDFT, T d = H^H (H d), every iteration (on
 * the tensor cores for the mixed precisions); the minimiser and its results
 * are the same up to rounding, the cost per iteration is that of two NUDFTs.
 * SPIREC_EINVAL for another value.  Takes effect at the next solve. */
#define SPIREC_MODE_TOEPLITZ 0
#define SPIREC_MODE_DIRECT 1
int spirec_set_mode(spirec_plan plan, int32_t mode);

/* Minimiser of spirec_solve.
 *   SPIREC_MIN_PRCG (default): Polak-Ribiere conjugate gradient (PR+, with a
 *     descent restart) and three majorize-minimize line-search steps per
 *     iteration (section 3.3); one T apply per iteration.
 *   SPIREC_MIN_HALF_QUADRATIC: the dual (half-quadratic) optimisation that
 *     section 5 names, multiplicative form: each of the solve's iters outer
 *     steps freezes the weights W_e = lambda_e phi'(r_e) / (2 r_e) at the
 *     iterate (r_e the modulus of an edge difference or a pixel), which makes
 *     a quadratic majorant of J touching it there, and takes inner_iters
 *     linear conjugate-gradient steps on its normal equations
 *     (T + sum_e W_e delta_e^H delta_e) f = D from the iterate (inner_iters T
 *     applies).  J never increases; J_hist[k] is J after k outer steps.
 *   SPIREC_MIN_NEWTON: the Newton-like method section 5 names, as truncated
 *     Newton: each outer step takes inner_iters linear conjugate-gradient
 *     steps from 0 on the Newton system Hess J(f) s = -grad J(f) (the exact
 *     Hessian: 2 T plus, per edge or pixel, lambda (b I + e z z^T) with
 *     b = phi'(r) / r, e = (phi''(r) - b) / r^2, z the difference at the
 *     iterate), then the three majorize-minimize line-search steps of
 *     SPIREC_MIN_PRCG along s (inner_iters T applies per outer step: T s is
 *     accumulated with s, so the line search needs no apply of its own).
 *     J never increases; J_hist[k] is J after k outer steps.
 * inner_iters: 1..1000 (ignored for SPIREC_MIN_PRCG).  Every minimiser works
 * in either mode; the half-quadratic and Newton ones run as a captured graph
 * of kernels, not in the persistent loop.  SPIREC_EINVAL for an unknown kind
 * or inner_iters out of range; SPIREC_ENOMEM if their 24 N^2-byte weight
 * buffer cannot be allocated. */
#define SPIREC_MIN_PRCG 0
#define SPIREC_MIN_HALF_QUADRATIC 1
#define SPIREC_MIN_NEWTON 2
int spirec_set_minimiser(spirec_plan plan, int32_t kind, int32_t inner_iters);

/* ---- operator access (device pointers, enqueued on the plan's stream) ---- */

/* y = H x (Eq. ModDirect): x 2N^2 floats, y 2L floats.  Needs a trajectory. */
int spirec_forward_dev(spirec_plan plan, const float* x, float* y);
/* x = H^H y: y 2L floats, x 2N^2 floats (Eq. AnnMatGD with s = y). */
int spirec_adjoint_dev(spirec_plan plan, const float* y, float* x);
/* Copy G's half: 2 * N * (2N-1) floats, entry (u, v) at [u*(2N-1) + v+N-1]. */
int spirec_gram_dev(spirec_plan plan, float* G);
/* Copy the real kernel spectrum, M*M floats, [ky*M + kx] (unnormalised DFT of
 * the circulant c[v mod M][u mod M] = conj G_{u,v}, divided by M^2). */
int spirec_kernel_spectrum_dev(spirec_plan plan, float* C);
/* Copy D (2N^2 floats).  Needs set_data. */
int spirec_data_adjoint_dev(spirec_plan plan, float* D);
/* Tx = H^H H x by the M x M zero-padded FFT (section 3.4): 2N^2 floats each. */
int spirec_toeplitz_dev(spirec_plan plan, const float* x, float* Tx);
/* J(x) through the rewritten form (Eq. NewCritLS plus R) and g = grad J(x)
 * (g: 2N^2 floats, device).  J is written to *J_host after a stream sync.
 * Needs set_data and set_reg. */
int spirec_objective_grad_dev(spirec_plan plan, const float* x, double* J_host, float* g);

/* ---- operator access (host pointers) ----
 * The input is copied to a plan buffer, the operator runs on the plan's
 * stream and the result is copied back; each call returns once the result is
 * in the caller's array and reports device-side errors as spirec_solve does.
 * The plan's scratch buffers are reused, so these calls do not overlap with
 * other work of the same plan (a plan is used by one host thread at a time). */

/* y = H x (Eq. ModDirect): x 2N^2 floats, y 2L floats.  SPIREC_ESTATE
 * without a trajectory. */
int spirec_forward(spirec_plan plan, const float* x, float* y);
/* x = H^H y (Eq. AnnMatGD with s = y; Appendix A): y 2L floats, x 2N^2
 * floats.  SPIREC_ESTATE without a trajectory. */
int spirec_adjoint(spirec_plan plan, const float* y, float* x);
/* Tx = H^H H x, the Toeplitz-block-Toeplitz Gram product by the M x M
 * zero-padded FFT convolution with conj(G) (section 3.4, Appendix B): 2N^2
 * floats each.  SPIREC_ESTATE without a trajectory. */
int spirec_gram_apply(spirec_plan plan, const float* x, float* Tx);
/* J(x) through the rewritten criterion (Eq. NewCritLS plus R, section 3.3)
 * into *J (may be NULL) and g = grad J(x) = 2 (T x - D) + grad R(x) into g
 * (2N^2 floats).  SPIREC_ESTATE before set_data and set_reg; SPIREC_ENUMERIC
 * if J is not finite. */
int spirec_objective_grad(spirec_plan plan, const float* x, double* J, float* g);

/* T x for callers that cannot allocate device memory: the same three-pass
 * zero-padded FFT as spirec_toeplitz_dev, but with no plan and no allocation
 * of any kind (no cudaMalloc, no cudaFree, no allocating library routine).
 * The paper has no counterpart; it exists for code that runs under a fixed
 * device-memory budget or must not grow its GPU footprint after start-up.
 *   x, Tx     device, 2N^2 floats each (images as everywhere in this header).
 *   spectrum  device, M*M floats: the real kernel spectrum in the layout
 *             spirec_kernel_spectrum_dev returns ([ky*M + kx]).
 *   N, M      2 <= N <= 512, 2N-1 <= M <= 1024, M a product of 2, 3 and 5;
 *             anything else returns SPIREC_EINVAL with a message.
 *   stream    cudaStream_t the work is enqueued on (NULL: legacy default).
 * Scratch is one file-scope device array of about 8.4 MB (the N x M rows, a
 * transposed spectrum and the twiddles), held by every GPU that loads the
 * library until the process exits.  The first call on a device looks up the
 * array's device address and sets kernel limits; make that first call before
 * any stream capture.  Every call shares the array: calls whose work overlaps
 * on the GPU (other streams, other threads) race and must be serialised by the
 * caller.  Returns after enqueueing; x and spectrum must stay valid until the
 * work has run. */
int spirec_toeplitz_noalloc(const float* x, const float* spectrum, float* Tx, int32_t N, int32_t M,
                            void* stream);

/* Wait for all work of the plan and report device-side errors raised since
 * the last trajectory upload (bad trajectory values, pipeline timeouts). */
int spirec_sync(spirec_plan plan);

/* Plan facts: any pointer may be NULL. */
int spirec_plan_info(spirec_plan plan, int32_t* N, int64_t* L, int32_t* M, int32_t* precision,
                     size_t* device_bytes);

/* Kernel timing with CUDA events recorded on the plan's own stream, for the
 * benchmark.  enable != 0 starts recording (and zeroes the totals).
 * spirec_timing_read returns, per stage, the summed milliseconds and launch
 * counts since enable: out_ms/out_count have SPIREC_NUM_STAGES entries in
 * the order gram, spectrum, adjoint_d, iterations.  Syncs the plan. */
#define SPIREC_NUM_STAGES 4
int spirec_timing(spirec_plan plan, int32_t enable);
int spirec_timing_read(spirec_plan plan, double* out_ms, int64_t* out_count);

/* ---- many reconstructions on one GPU ---- */

/* Solve n plans at once: each plan's solve is enqueued on its own stream (so
 * their kernels overlap on the device), then all are awaited.  x0 (array of
 * n DEVICE pointers, or NULL for zeros), x_out (n DEVICE pointers), J_hist
 * (n DEVICE pointers or NULL).  Trajectories and data are set per plan
 * beforehand (the _dev setters do not block).  Returns the first error. */
int spirec_batch_solve(const spirec_plan* plans, int32_t n, const float* const* x0, int32_t iters,
                       float* const* x_out, double* const* J_hist);

/* One reconstruction request; every pointer is HOST memory and is copied at
 * submission. */
typedef struct {
    int32_t N;           /* image side */
    int64_t L;           /* samples */
    const double* kx;    /* L values in [-0.5, 0.5] */
    const double* ky;
    const float* s;      /* 2L floats, interleaved complex */
    double lambda1, alpha1, lambda0, alpha0;
    int32_t phi;         /* spirec_phi */
    int32_t iters;       /* CG iterations */
} spirec_request;

typedef struct spirec_server_s* spirec_server;

/* A request loop with continuous batching: max_slots worker threads, each
 * with its own stream and resident plan (reused while requests keep the same
 * N and L).  A queued request is admitted, first come first served, when a
 * slot is idle and its device footprint fits hbm_budget_bytes next to the
 * plans already resident (idle workers release their plans when the head
 * request needs the room); admitted requests run concurrently and their
 * kernels overlap.  Solves on the persistent CG loop start only while the
 * loops already running leave room for all of their blocks on the device
 * (a cooperative launch needs every block resident at once); otherwise they
 * wait for a running loop to end.  Each result equals the result of the same request run
 * alone (launch shapes and summation orders depend only on its own sizes).
 * precision: spirec_precision of every plan. */
int spirec_server_create(spirec_server* out, size_t hbm_budget_bytes, int32_t max_slots, int32_t precision);
/* The device footprint the request loop reserves for a request of this shape
 * (its admission estimate: every buffer of the plan it creates, the host
 * upload buffer included) and, in *M (may be NULL), the grid side it plans
 * the request with.  Host-only.  The request loop is serving infrastructure;
 * no passage of the paper defines it.  SPIREC_EINVAL for N outside
 * [2, 2048], L < 1 or an unknown precision. */
int spirec_server_plan_bytes(int32_t N, int64_t L, int32_t precision, size_t* bytes, int32_t* M);
/* Queue a request; *ticket identifies it.  SPIREC_EBUSY if the request alone
 * exceeds the budget, SPIREC_EINVAL for bad fields (checked again on the GPU
 * path, e.g. |k| > 0.5, and then reported by spirec_server_wait). */
int spirec_server_submit(spirec_server srv, const spirec_request* req, uint64_t* ticket);
/* Wait up to timeout_ms for a request: x_out (2N^2 floats, host, may be
 * NULL), J (final criterion) and latency_s (submission to completion).
 * SPIREC_ETIMEOUT if not finished in time (the request stays queued and can
 * be waited for again); the request's own error status otherwise.  A ticket
 * can be collected once. */
int spirec_server_wait(spirec_server srv, uint64_t ticket, int32_t timeout_ms, float* x_out, double* J,
                       double* latency_s);
/* Latency percentiles (seconds) of the completed requests and the counts of
 * completed, failed and still queued requests; any pointer may be NULL. */
int spirec_server_stats(spirec_server srv, double* p50_s, double* p99_s, int64_t* completed, int64_t* failed,
                        int64_t* queued);
/* Finish the running requests, drop the queued ones, release everything. */
int spirec_server_destroy(spirec_server srv);

/* ------------------------------------------------------------- autotuning
 *
 * Launch parameters that change speed, not the arithmetic of a term: how the
 * sample sum of the contractions G (Eq. AnnMatG) and D = H^H y (Eq. AnnMatGD)
 * is split over the SMs, and how many image rows one block of the persistent
 * CG loop owns.  A split changes the grouping of the FP32 partial sums, so
 * results move within the contraction's rounding (never beyond the stated
 * tolerances); a row count changes the block order of the loop's reductions.
 * For one table, a shape always gets the same value: a solve gives the same
 * result alone and among other solves.
 *
 * The values live in one process-wide table keyed by (knob, N, M, precision,
 * L class, SM count), the L class being the smallest c with 2^c >= L (the
 * loop's key ignores L).  A shape without an entry uses the built-in
 * heuristic.  Knobs and their values:
 *   SPIREC_KNOB_GRAM_SPLIT     G: tensor-core paths, the number of CTAs the
 *                              stream-K schedule spreads the work over
 *                              (2..152, rounded down to even: the contraction
 *                              runs on CTA pairs); FP32 path, the number of
 *                              slices the samples are cut into (>= 1).
 *   SPIREC_KNOB_ADJOINT_SPLIT  the same for D and every other H^H y.
 *   SPIREC_KNOB_LOOP_ROWS      persistent CG loop: image rows per block.
 *   SPIREC_KNOB_GRAM_TILE      G, tensor-core paths: the tile shape, 1 = one
 *                              SM a tile of 128 output rows (MMA M = 128),
 *                              2 = a pair of SMs a tile of 256 rows (a cluster
 *                              of two CTAs, MMA M = 256 across the pair).
 *                              Without an entry: 2, except 1 where 256-row
 *                              tiles would leave a last tile half empty
 *                              beyond 256 rows (N = 384, 640, ...).
 *   SPIREC_KNOB_ADJOINT_TILE   the same for D and every other H^H y.
 * A value that does not fit the device or the plan at launch time (too many
 * CTAs for the split-K buffer, a loop shape whose blocks are not
 * co-resident) is clipped, or, for the loop, replaced by the heuristic. */
#define SPIREC_KNOB_GRAM_SPLIT 0
#define SPIREC_KNOB_ADJOINT_SPLIT 1
#define SPIREC_KNOB_LOOP_ROWS 2
#define SPIREC_KNOB_GRAM_TILE 3
#define SPIREC_KNOB_ADJOINT_TILE 4
#define SPIREC_NUM_KNOBS 5

/* Objectives: LATENCY minimises the time of one launch; THROUGHPUT the
 * SM-time (launch time x SMs the launch occupies), for many solves that share
 * the GPU (batched frames, the request loop). */
#define SPIREC_TUNE_LATENCY 0
#define SPIREC_TUNE_THROUGHPUT 1

/* Time every candidate value of each knob on the plan's own trajectory, data
 * and regularisation (all three set first: SPIREC_ESTATE otherwise) with CUDA
 * events on the plan's stream (one warm-up and the median of three runs),
 * store the best under the plan's key, and rebuild G, the spectrum and D with
 * it, so that the plan's state equals that of a new plan of the same shape.
 * The loop is timed over loop_iters iterations from x0 = 0 (>= 1; skipped in
 * direct mode and for M the loop does not handle); each contraction's tile
 * shape is chosen first (at the heuristic split), then its split.
 * chosen[SPIREC_NUM_KNOBS]
 * receives the stored values (0: knob not tuned); best_ms (may be NULL) the
 * median milliseconds of the winners.  Blocks the host until done. */
int spirec_autotune(spirec_plan plan, int32_t objective, int32_t loop_iters, int32_t* chosen, double* best_ms);

/* Set (value > 0) or remove (value == 0) a table entry.  sms == 0 means the
 * current device's SM count (needs a CUDA device; SPIREC_ECUDA otherwise).
 * SPIREC_EINVAL for an unknown knob or precision, N < 2, M < 2N - 1, L < 1,
 * sms < 0 or value < 0.  Host-only: no device work. */
int spirec_tune_set(int32_t knob, int32_t N, int32_t M, int32_t precision, int64_t L, int32_t sms, int32_t value);
/* The entry for a shape, 0 if none (arguments as spirec_tune_set). */
int spirec_tune_get(int32_t knob, int32_t N, int32_t M, int32_t precision, int64_t L, int32_t sms,
                    int32_t* value);
/* Number of entries; spirec_tune_clear removes them all. */
int spirec_tune_count(int64_t* count);
int spirec_tune_clear(void);
/* Write the table to a text file (one entry per line after a header line)
 * or add the entries of such a file to it (entries of the file replace equal
 * keys).  SPIREC_EINVAL for a file that cannot be opened or a malformed line;
 * a failed load leaves the table unchanged. */
int spirec_tune_save(const char* path);
int spirec_tune_load(const char* path);

/* Copy the plan's FP64 device scalars to the host (diagnostics; syncs the
 * plan).  out receives min(n, SPIREC_NUM_SCALARS) values in this order:
 * 0 ||s||^2, 1 q1, 2 q2, 3-5 line-search steps t1..t3, 6 <g,g>, 7 beta,
 * 8 J, 9 R, 16-25 nanoseconds block 0 of the persistent CG loop spent in the
 * iterations of its last solve, per phase: work, then barrier + reduction,
 * for the column pass, the row pass, the two further line-search steps and
 * the update, in that order. */
#define SPIREC_NUM_SCALARS 32
int spirec_plan_scalars(spirec_plan plan, double* out, int32_t n);

/* Number of CUDA kernels the plan has launched so far (a CUDA-graph replay
 * counts each of its kernel nodes).  Memory copies and sets are not kernels. */
int spirec_launch_count(spirec_plan plan, int64_t* count);

/* ---- failure injection, for tests of the error paths ----
 * No passage of the paper defines these: they let a test make each failure
 * the library reports happen, without faulting the GPU. */

/* Device allocations of plans succeed n more times, then fail with
 * SPIREC_ENOMEM (a plan creation that meets one releases what it had
 * allocated); n < 0, the default, injects nothing.  Process-wide. */
int spirec_inject_alloc_failure(int64_t n);

/* The kernels named by the bit mask (SPIREC_STALL_LOOP: the persistent CG
 * loop; SPIREC_STALL_CONTRACTION: the tensor-core contractions of G, D, H^H y
 * and H f) launched from now on first wait on a condition that nothing
 * fulfils, so that their bounded wait runs out (see spirec_set_wait_limit_ns)
 * and they end early as a real timeout would; 0 (the default) ends the
 * injection.  SPIREC_EINVAL for other bits.  Process-wide. */
#define SPIREC_STALL_LOOP 1
#define SPIREC_STALL_CONTRACTION 2
int spirec_inject_wait_stall(int32_t kernels);

/* Limit, in nanoseconds, of every bounded device wait in the kernels launched
 * from now on: the persistent CG loop's grid synchronisations and the
 * tensor-core contractions' pipeline waits.  0 restores the default, 2 s.
 * A wait that runs out ends its kernel early: the loop's blocks return at
 * their next synchronisation, a contraction's CTA waits (with a fixed 2 s
 * bound) for the copies and MMAs it issued, releases its tensor memory and
 * returns.  The plan then reports SPIREC_ETIMEOUT at its next host
 * synchronisation (spirec_solve, spirec_sync) until its trajectory is set
 * again; the results of that work are invalid.  Graphs captured earlier keep
 * the limit of their capture.  Process-wide. */
int spirec_set_wait_limit_ns(uint64_t ns);

/* Message of the last failure on this thread ("" if none). */
const char* spirec_last_error(void);

/* Library version string. */
const char* spirec_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SPIREC_H */
