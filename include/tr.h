/*
 * tr.h -- C ABI of libtr, the GB300 (sm_103a) implementation of the
 * per-iteration low-rank proximal step of the GNRHTC / GNHTC ADMM from
 * "Accelerating Large-Scale Regularized High-Order Tensor Recovery"
 * (arXiv 2506.09594).
 *
 * What one step computes (Alg. 5 with the pure-L prior, Gamma = {I}):
 *   1. L <- ((M - E + Y/mu) + (G - Lambda/mu)) / 2            (Eq. coef-tensor)
 *   2. G <- D_{Phi,tau}(L + Lambda/mu, L), tau = 1/mu         (Eq. L_prox, Alg. 4)
 *        = L^{-1}( per transformed face slice: randomized low-rank
 *          approximation, shrink singular values with Prox_{Phi,tau} )
 *   3. E <- Prox_{psi,lambda/mu}(H) on Omega, H off Omega,
 *        H = M - L + Y/mu                        (Eq. E_prox_ome / E_prox_ome1)
 *   4. Y += mu (M - L - E); Lambda += mu (L - G);
 *      mu <- min(mu_max, growth * mu)                  (Eq. lagrange11-22)
 *   5. five infinity-norm residuals                   (Eq. convercon)
 * The transform L is the orthonormal DCT-II along modes 3..d (Eq. trans,
 * Eq. orth with alpha = 1).
 *
 * Data layout (all tensors, device memory): the face-slice stack of an
 * order-d tensor n1 x n2 x n3 x ... x nd, i.e. X[j][i1][i2] row-major with
 * slice index j = i3 + n3*(i4 + n4*(...)) (i3 fastest; Sec. 2 face slice).
 * Element type is the problem's dtype (float or double).  N = n1*n2*n3*...*nd.
 *
 * Threading: a handle is used by one host thread at a time.  Calls enqueue
 * work on the handle's CUDA stream and return without synchronising unless
 * stated.
 *
 * Errors: every entry point returns a tr_status.  After any non-OK status
 * the handle stays valid; tr_last_error() describes the failure; a failed
 * tr_prox_step poisons the handle (further steps return TR_EINVAL) until
 * tr_set_state() installs a new iterate.
 */
#ifndef TR_H
#define TR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TR_OK = 0,
  TR_EINVAL = 1,        /* bad argument, unsupported shape, poisoned handle  */
  TR_ENOMEM = 2,        /* device allocation failed                          */
  TR_ECUDA = 3,         /* a CUDA runtime call failed                        */
  TR_ENUMERIC = 4,      /* NaN / Inf met in the iterate                      */
  TR_ETIMEOUT = 5,      /* a bounded device wait gave up                     */
  TR_ENOTCONV = 6,      /* tr_recover hit max_iter with tol > 0              */
  TR_EUNSUPPORTED = 7   /* option known but not built in this library        */
} tr_status;

typedef enum { TR_F32 = 0, TR_F64 = 1 } tr_dtype;

/* Phi (singular values, GNHTSVT) and psi (entries, GNHTT): Sec. 4.1 */
typedef enum { TR_PEN_L1 = 0, TR_PEN_MCP = 1 } tr_penalty;

/* h(.) of the noise term Upsilon (Eq. unified-regular11): none = GNHTC,
 * entrywise l1 = GNRHTC with entry-wise outliers.                         */
typedef enum { TR_NOISE_NONE = 0, TR_NOISE_L1 = 1 } tr_noise;

/* Low-rank engine inside GNHTSVT (Alg. 4). */
typedef enum {
  TR_LR_FULLSVD = 0,    /* deterministic branch: full SVD of every slice    */
  TR_LR_RSVD = 1,       /* per-slice Gaussian sketch + power iterations      */
  TR_LR_ADAPTIVE = 2,   /* per-slice fixed-accuracy block Lanczos (Alg. 3)  */
  TR_LR_LEARNED = 3,    /* per-slice sketch width predicted by an MLP        */
  TR_LR_TUCKER = 4      /* shared Tucker factors of modes 1, 2 (Alg. 1 +
                           Alg. 4 randomized branch): r = b = l, q Krylov
                           steps, (q + 1) l <= 32 and <= n1, n2; Gaussian
                           blocks per transformed slice (Philox streams 2
                           and 4, like the sketch's counters otherwise)    */
} tr_engine;

/* Operand precision of the slice contractions (accumulation is FP32).
 *   FP32:   SIMT FP32 FMA (the plain form).
 *   BF16:   tcgen05 tensor cores; the sketch and first power-iteration
 *           products in BF16, the last power product and B^T = Abar^T Q in
 *           split BF16 (x = hi + lo, three products: ~16-bit operands), so
 *           the final basis is refined at FP32-level accuracy (rel-F 1e-3).
 *   BF16X3: tcgen05 tensor cores, all four skinny products in split BF16
 *           (FP32-level accuracy, rel-F 1e-4).
 * The tensor-core forms need FP32 problems; TF32 is not built.             */
typedef enum { TR_PREC_FP32 = 0, TR_PREC_TF32 = 1, TR_PREC_BF16 = 2, TR_PREC_BF16X3 = 3 } tr_prec;

typedef struct tr_handle tr_handle;

/* The recovery problem: P_Omega(M) and Omega (Alg. 5 inputs). */
typedef struct {
  int order;               /* d >= 2, at most 8                              */
  int64_t dims[8];         /* n1, n2, n3, ..., nd                            */
  tr_dtype dtype;          /* element type of `observed` and of all state    */
  const void *observed;    /* device, N elements, face-slice layout; only
                              entries on Omega are read                      */
  const uint8_t *mask;     /* device, N bytes, 1 = observed (Omega), 0 = not */
} tr_problem;

/* Parameters (Alg. 5 input list; Sec. 6 parameter settings). */
typedef struct {
  tr_penalty phi;  double phi_theta, phi_gamma;  /* Phi: weight, MCP gamma  */
  tr_penalty psi;  double psi_theta, psi_gamma;  /* psi: weight, MCP gamma  */
  tr_noise noise;  double lambda;                /* lambda of Eq. orin_nonconvex */
  double mu0, mu_max, growth;                    /* mu^0, mu^max, vartheta   */
  double tol;                                    /* varpi; <= 0: fixed count */
  int max_iter;
  tr_engine engine;
  int rank, oversample;   /* sketch width l = rank + oversample (clamped to
                             min(n1, n2))                                    */
  int power_iters;        /* q                                              */
  double adapt_eps;       /* adaptive engine: relative accuracy epsilon      */
  int adapt_block;        /* adaptive engine: block size b                   */
  tr_prec prec;
  uint64_t seed;          /* Philox4x32-10 key of the Gaussian sketches      */
  const char *model_path; /* learned engine: rank-predictor weights file
                             (format under tr_set_model); NULL = a randomly
                             initialised predictor keyed by `seed`; unused
                             by the other engines                            */
} tr_params;

/* Per-step report (filled only when a non-NULL pointer is passed, which
 * synchronises the stream). */
typedef struct {
  int iter;               /* iterations completed so far                    */
  double mu;              /* mu used by this step                            */
  double tau;             /* 1/mu                                            */
  double res_inf[5];      /* ||dL||, ||dE||, ||L-G||, ||dG||, ||M-L-E||      */
  int max_rank;           /* max over slices of #(shrunk sigma > 0)          */
  int sum_rank;           /* sum over slices                                 */
  int fallback_slices;    /* learned engine: slices that fell back           */
  float ms;               /* device time of the step (0 if not timed)       */
} tr_step_info;

/* Fill `prm` with the defaults: Phi = psi = MCP (theta 1, gamma 4000),
 * entrywise l1 noise with lambda = 1/sqrt(max(n1,n2)) computed
 * at tr_init when lambda <= 0, mu0 = 1e-3, mu_max = 1e10, growth 1.1,
 * tol 1e-4, max_iter 100, RSVD engine, rank 10 + oversample 10, q = 1,
 * FP32 operands, seed 0.  (Sec. 6 parameter settings.)                     */
void tr_default_params(tr_params *prm);

/* Create a handle for one problem.  Copies nothing from `observed`/`mask`:
 * they are caller-owned and must stay valid until tr_free.  Allocates all
 * workspace (state L, E, Y, Lambda, G and transform-domain scratch) on the
 * current device and sets the iterate to zero with mu = mu0, t = 0 (Alg. 5
 * initialisation).  `cuda_stream` is a cudaStream_t (NULL = legacy default
 * stream).  Errors: TR_EINVAL (shape, dtype, pointers), TR_ENOMEM,
 * TR_EUNSUPPORTED (engine not built), TR_ECUDA.                             */
tr_status tr_init(tr_handle **h, const tr_problem *p, const tr_params *prm,
                  void *cuda_stream);

/* One ADMM iteration (steps 1-5 above) on the handle's state.  Asynchronous
 * unless `info` is non-NULL.  Errors: TR_EINVAL (poisoned), TR_ENUMERIC
 * (NaN/Inf in the tube pass's reduction: reported by this call when info is
 * non-NULL; a step without a report, graph replays included, copies its flag
 * to pinned host memory without synchronising, and a later call returns
 * TR_ENUMERIC once the copy has landed -- at the latest the first call after
 * the step has completed), TR_ECUDA.                                        */
tr_status tr_prox_step(tr_handle *h, tr_step_info *info);

/* Alg. 5 loop, stop test of Eq. convercon.  tol <= 0: max_iter steps (graph
 * replays when tr_graph_mode is on).  tol > 0: steps are enqueued without a
 * report and their residual maxima read back asynchronously; step k's five
 * maxima are complete after step k + 1 (its deferred inverse pass), so the
 * host checks step k after enqueuing step k + 2 and waits only for step
 * k + 1: the GPU never idles.  The loop stops at the first step whose maxima
 * are all <= tol; the iterate returned is at most two steps past it.  Then L
 * is copied to `L_out` (device, N elements, caller-owned; may be NULL) and
 * `last` (may be NULL) receives the returned iterate's residual maxima and
 * iteration count.  Returns TR_ENOTCONV when tol > 0 and neither a checked
 * step nor the returned iterate met tol within max_iter steps.             */
tr_status tr_recover(tr_handle *h, void *L_out, tr_step_info *last);

/* Copy the iterate out of / into the handle.  Each pointer is a device
 * buffer of N elements of the problem's dtype (NULL = skip that tensor).
 * tr_set_state clears the poisoned flag.  Both synchronise the stream.      */
tr_status tr_get_state(tr_handle *h, void *L, void *E, void *Y, void *Lam,
                       void *G, double *mu, int *t);
tr_status tr_set_state(tr_handle *h, const void *L, const void *E,
                       const void *Y, const void *Lam, const void *G,
                       double mu, int t);

/* Transform-domain building blocks of step 2, exposed for testing and for
 * callers that bring their own outer loop.  All pointers are device buffers
 * in the face-slice layout of the handle's problem.
 *   tr_transform_forward: dst = L(src)    (Eq. trans)
 *   tr_transform_inverse: dst = L^{-1}(src)
 *   tr_slice_prox: Gbar^<j> = the handle's engine applied to Abar^<j> with
 *     threshold tau, for every slice j, sketches drawn for iteration `t`
 *     (Philox counter word 2).  Abar and Gbar must not alias.               */
tr_status tr_transform_forward(tr_handle *h, const void *src, void *dst);
tr_status tr_transform_inverse(tr_handle *h, const void *src, void *dst);
tr_status tr_slice_prox(tr_handle *h, const void *Abar, void *Gbar,
                        double tau, int t);

/* The paper's own randomized GNHTSVT (Alg. 4, randomized branch) on the
 * transformed stack Abar: shared Tucker factors F1 (n1 x r1) and F2
 * (n2 x r2) of the two spatial modes from Alg. 1 (R-STHOSVD-BKI, processing
 * order (1, 2)): for each mode the block Krylov space
 * [A G, (A A^T) A G, ..., (A A^T)^q A G] of the mode unfolding A, an
 * orthonormal basis Z of it, the r top singular vectors U_r of
 * Z^T A A^T Z and F = Z U_r, the core truncated by F before the next mode.
 * Then every transformed slice is replaced by F1 Prox(F1^T Abar_j F2) F2^T
 * (the handle's Phi, theta, gamma; tau as given), written to Gbar.
 *   Abar, Gbar: device, (n, n1, n2) of the handle's shape and dtype; no alias.
 *   G1: device, column-major (n n2) x b1 Gaussian block of mode 1, row
 *       j n2 + i2 for slice j (a transform-domain draw: the transform of a
 *       spatial draw gives exactly the spatial form of Alg. 1).
 *   G2: device, column-major (n r1) x b2 Gaussian block of mode 2, row
 *       j r1 + a.
 *   F1_out, F2_out: device, column-major, optional (NULL: not written).
 * Needs 1 <= r1 <= min(n1, n2), r2 <= n2, r_k <= (q_k + 1) b_k <= 32 and
 * (q_k + 1) b_k <= the mode size.  Workspace is taken from the stream-ordered
 * allocator for the call.  Errors: TR_EINVAL (arguments), TR_EUNSUPPORTED
 * (Krylov spaces above 32 columns, panels beyond shared memory), TR_ECUDA. */
tr_status tr_slice_prox_tucker(tr_handle *h, const void *Abar, void *Gbar, double tau,
                               int r1, int r2, int b1, int b2, int q1, int q2,
                               const void *G1, const void *G2, void *F1_out, void *F2_out);

/* Point the handle at other observed data (device buffers of the same
 * shape, dtype and layout as at tr_init; caller-owned, valid until the next
 * call or tr_free).  Later steps read them; the iterate is kept.  For
 * streaming inputs: copy the next step's data into a second buffer on
 * another stream while a step runs.  Captured step graphs (tr_graph_mode)
 * are kept per (observed, mask) pair, two at a time, so alternating between
 * two buffer pairs replays without re-capturing.  Errors: TR_EINVAL (NULL).  */
tr_status tr_set_observed(tr_handle *h, const void *observed, const uint8_t *mask);

/* Enqueue on the handle's stream a copy of the residual maxima (Eq.
 * convercon) of the last enqueued step into res_host[0 .. 10): host memory,
 * caller-owned; pinned memory keeps the call asynchronous.  The values are
 * there once the stream has passed this point.
 *   res_host[0..5): the step's slots in tr_step_info.res_inf order.  A step
 *     without a report defers its inverse pass to the next step, so its
 *     ||L-G|| and ||dG|| slots are 0;
 *   res_host[5..10): ||L-G|| and ||dG|| (entries 7 and 8) of the step before,
 *     completed by this step's fused pass; the other entries are 0.
 * No host synchronisation, so a graph-replayed step can be followed by it.
 * Errors: TR_EINVAL (NULL), TR_ECUDA.                                        */
tr_status tr_read_residuals(tr_handle *h, double *res_host);

/* Per-slice singular values and kept ranks of the last slice pass (host
 * buffers: sigma n*l doubles, ranks n ints; either may be NULL).  `l` is
 * the sketch width in use.  Synchronises.                                   */
tr_status tr_last_slice_stats(tr_handle *h, double *sigma, int *ranks, int *l);

/* Instrumentation (not part of the method).
 *   tr_profile_enable: when max_steps > 0, the next max_steps calls of
 *     tr_prox_step record CUDA events on the handle's stream around the
 *     tube forward kernel, the slice pass and the tube inverse kernel
 *     (events are created here, outside any timed region); 0 disables.
 *   tr_profile_read: mean device milliseconds per recorded step of those
 *     three phases (ms[0..2]) and the number of recorded steps; synchronises.
 *   tr_kernel_launches: number of CUDA kernels this handle has launched.    */
tr_status tr_profile_enable(tr_handle *h, int max_steps);
tr_status tr_profile_read(tr_handle *h, double ms[3], int *steps);
tr_status tr_kernel_launches(const tr_handle *h, uint64_t *count);

/* Per-kernel device times of the fixed-width slice pass (the randomized
 * prox of Alg. 4 on every slice: sketch, 2 + 2q skinny products, 1 + 2q
 * panel QRs, the small SVD with the shrinkage of Def. gNtsvt, the rank-l
 * rebuild).  Instrumentation, not in the paper.  Runs `reps` eager passes of
 * the handle's engine settings (TR_LR_RSVD only, else TR_EUNSUPPORTED) on
 * the caller's device buffers Abar -> Gbar (n slices of n1 x n2, face-slice
 * layout, no alias) with threshold tau and Philox counter word t, all
 * kernels in order on the handle's stream (slice groups ignored), with a
 * CUDA event after every kernel; synchronises.  ms[k] (host, max_kernels
 * entries) receives the mean milliseconds of kernel k, names[k] (may be
 * NULL) a static label, *count the number of kernels.  Errors: TR_EINVAL,
 * TR_EUNSUPPORTED, TR_ECUDA.                                                */
tr_status tr_profile_slice_pass(tr_handle *h, const void *Abar, void *Gbar, double tau, int t,
                                int reps, double *ms, const char **names, int max_kernels,
                                int *count);

/* The slice pass of tr_slice_prox without any device allocation.  The paper
 * has no counterpart: this entry point exists for callers that cannot call
 * cudaMalloc -- a host thread on a latency-critical loop (allocation
 * synchronises the whole device), or code running inside another
 * framework's memory pool that owns all device memory.  It needs no handle:
 * the caller passes the transformed stack Abar (input) and Gbar (output),
 * both device buffers of n slices of n1 x n2 (face-slice layout, dtype
 * elements, must not alias); l (clamped to min(n1, n2)) is the sketch width,
 * q the power iterations, phi/theta/gamma/tau the shrinkage, seed and t the
 * Philox key and counter word of the sketches (as in tr_slice_prox).  Work
 * is enqueued on `cuda_stream` (a cudaStream_t, NULL = legacy stream).
 * Scratch comes from one fixed 16 MiB array compiled into the library and
 * kept on every GPU that loads it until exit; calls needing more return
 * TR_EUNSUPPORTED with the size in `err`.  The first call on a device looks
 * up that array's address (make it before any stream capture); later calls
 * look it up again, so the address stays valid across a device reset.  All
 * calls share the array: calls that overlap on the GPU race.  `err` (may be NULL)
 * receives a message of at most err_len bytes on failure.                  */
tr_status tr_slice_prox_noalloc(tr_dtype dtype, int n, int n1, int n2, const void *Abar,
                                void *Gbar, int l, int q, tr_penalty phi, double theta,
                                double gamma, double tau, uint64_t seed, int t,
                                void *cuda_stream, char *err, size_t err_len);

/* The paper's randomized GNHTSVT with the fixed-accuracy Tucker form
 * (Alg. "AD-RSTHOSVD-BLBP" with processing order (1, 2), then the core's
 * GNTSVT, Alg. 4 randomized branch) on the transformed stack Abar: per
 * spatial mode, the block Lanczos loop of Alg. 3 on the mode unfolding of
 * the current core (block size b, deflation tolerance delta_rel ||A||_F,
 * stop once the estimate E < eps^2 ||A||_F^2 or the basis reaches
 * min(rows, cols, max_rank) columns; max_rank 0: no cap) gives the factor,
 * the core is truncated by it; then every core slice gets Prox_{Phi,tau} of
 * its singular values (the exact per-slice prox) and Gbar_j = F1 Prox F2^T.
 * The Gaussian draws are Philox blocks per transformed slice: draw d of mode
 * m uses stream word 0x10000 m + 2 d with key seed and counter word t.  It
 * needs no handle: Abar and Gbar are device buffers of n slices of n1 x n2
 * (face-slice layout, dtype elements, no alias); `ranks` (host, 2 ints, may
 * be NULL) receives the two ranks found.  Work runs on `cuda_stream` and the
 * call synchronises it (the loop's decisions run on the host); workspace
 * comes from stream-ordered allocation (the core's prox included); a core
 * whose r1 x r2 slices exceed the slice kernels' shared memory, or with
 * min(r1, r2) > 96, gives TR_EUNSUPPORTED.
 * Errors: TR_EINVAL, TR_EUNSUPPORTED, TR_ENOMEM, TR_ECUDA; `err` (may be
 * NULL) receives a message of at most err_len bytes.                        */
tr_status tr_slice_prox_ad_tucker(tr_dtype dtype, int n, int n1, int n2, const void *Abar,
                                  void *Gbar, double tau, tr_penalty phi, double theta,
                                  double gamma, double eps, int b, double delta_rel, int max_rank,
                                  uint64_t seed, int t, int *ranks, void *cuda_stream, char *err,
                                  size_t err_len);

/* ---- Gradient-domain building blocks (GNHTCTV prior) -------------------
 * The operators of the gradient-domain model (Def. gradient tensor, Def.
 * GNHTCTV, Eq. coef-tensor, Eq. gnrhtc-L); they need no handle.  Tensors
 * are device buffers in the face-slice layout above, shape given by `order`
 * (2..8) and `dims` (host array n1, n2, n3, ...), dtype elements.  Work is
 * enqueued on `cuda_stream` (a cudaStream_t, NULL = legacy stream); `err`
 * (may be NULL) receives a message of at most err_len bytes on failure.
 *   tr_grad: dst = nabla_k(src) = src x_k D_{n_k}, the periodic forward
 *     difference (nabla_k X)[.., i_k, ..] = X[.., i_k + 1 mod n_k, ..] -
 *     X[.., i_k, ..], for mode k = `mode` (1..order); with adjoint != 0
 *     dst = nabla_k^T(src), the periodic backward difference.  src and dst
 *     must not alias.
 *   tr_gradient_solve: out = (I + sum_{k in Gamma} nabla_k^T nabla_k)^{-1} rhs,
 *     Gamma = the modes whose bit (k - 1) is set in `modes` (empty: a
 *     copy); the L-system of Eq. coef-tensor, solved as Eq. gnrhtc-L does by
 *     diagonalising every nabla_k^T nabla_k, here with the real Hartley
 *     basis (mode products with cas(2 pi a b / n)/sqrt(n)) instead of the
 *     complex FFT.  rhs and out must not alias.  Allocates its workspace
 *     (one tensor plus the Hartley matrices) with stream-ordered
 *     allocation.  Each mode in Gamma may have at most 2048 entries.
 * Errors: TR_EINVAL (dtype, shape, mode, pointers), TR_EUNSUPPORTED (mode
 * sizes or a tensor beyond one launch per product), TR_ENOMEM, TR_ECUDA.    */
tr_status tr_grad(tr_dtype dtype, int order, const int64_t *dims, int mode, int adjoint,
                  const void *src, void *dst, void *cuda_stream, char *err, size_t err_len);
tr_status tr_gradient_solve(tr_dtype dtype, int order, const int64_t *dims, uint32_t modes,
                            const void *rhs, void *out, void *cuda_stream, char *err,
                            size_t err_len);

/* ---- Gradient-domain prior, GNHTCTV (Alg. 5 with Gamma) -----------------
 * Alg. 5 on the model of Eq. equ_nonconvex with a set Gamma of gradient
 * directions (Def. GNHTCTV), gamma = |Gamma|.  One step:
 *   1. (I + sum_k nabla_k^T nabla_k) L = (M - E + Y/mu) + sum_k nabla_k^T (G_k - Lambda_k/mu)
 *      solved as tr_gradient_solve does          (Eq. coef-tensor, Eq. gnrhtc-L)
 *   2. G_k = D_{Phi, 1/(gamma mu)}(nabla_k L + Lambda_k/mu, L) by the
 *      per-slice randomized engine (sketch width rank + oversample,
 *      power_iters, Philox key seed, counter word t)            (Eq. L_prox)
 *   3. H = M - L + Y/mu; E = Prox_{psi, lambda/mu}(H) on Omega (0 with
 *      TR_NOISE_NONE), E = H off Omega              (Eq. E_prox_ome, E_prox_ome1)
 *   4. Y += mu (M - L - E); Lambda_k += mu (nabla_k L - G_k);
 *      mu = min(mu_max, growth mu)                        (Eq. lagrange11-22)
 *   5. res_inf = the infinity norms of L - L^t, E - E^t, nabla_k L - G_k and
 *      G_k - G_k^t (each the maximum over k), M - L - E      (Eq. convercon)
 * L is the orthonormal DCT-II along modes 3..d.
 *   tr_ctv_create: `problem` as for tr_init (order 3..8; observed and mask
 *     caller-owned, valid until tr_ctv_free); lambda <= 0 selects
 *     1/sqrt(max(n1, n2)).  Initialises L = E = Y = G_k = Lambda_k = 0,
 *     mu = mu0, t = 0.  Allocates about (7 + 2 |Gamma|) tensors plus an
 *     internal tr_init handle.
 *   tr_ctv_step: one iteration on the stream; with res_inf non-NULL (5
 *     doubles) it synchronises and returns the residuals of step 5.
 *   tr_ctv_get_state / tr_ctv_set_state: copy L, E, Y (N elements each) and
 *     G, Lambda (|Gamma| tensors back to back, modes ascending) out of /
 *     into the object (device buffers; NULL skips one); both synchronise.
 * Errors: TR_EINVAL, TR_EUNSUPPORTED (shapes the internal handle refuses),
 * TR_ENOMEM, TR_ECUDA.                                                      */
typedef struct tr_ctv tr_ctv;
typedef struct {
  uint32_t modes;                  /* Gamma: bit k - 1 set for mode k        */
  tr_penalty phi;  double phi_theta, phi_gamma;
  tr_penalty psi;  double psi_theta, psi_gamma;
  tr_noise noise;  double lambda;
  double mu0, mu_max, growth;
  int rank, oversample, power_iters;
  uint64_t seed;
  tr_prec prec;
} tr_ctv_params;

/* Defaults: Gamma = {1, 2}, Phi = psi = MCP (theta 1, gamma 4000), l1 noise,
 * lambda = 0 (automatic), mu0 = 1e-3, mu_max = 1e10, growth 1.1, rank 10 +
 * oversample 10, q = 1, seed 0, FP32 (Sec. 6 parameter settings).           */
void tr_ctv_default_params(tr_ctv_params *p);
tr_status tr_ctv_create(tr_ctv **c, const tr_problem *problem, const tr_ctv_params *prm,
                        void *cuda_stream, char *err, size_t err_len);
tr_status tr_ctv_step(tr_ctv *c, double *res_inf);
tr_status tr_ctv_get_state(tr_ctv *c, void *L, void *E, void *Y, void *G, void *Lam, double *mu,
                           int *t);
tr_status tr_ctv_set_state(tr_ctv *c, const void *L, const void *E, const void *Y, const void *G,
                           const void *Lam, double mu, int t);
const char *tr_ctv_last_error(const tr_ctv *c);
tr_status tr_ctv_free(tr_ctv *c);

/* ---- One-bit completion, GNOBHTC (Alg. 6) --------------------------------
 * Recovers L from m dithered one-bit samples q_k = sign(L*[s_k] + eps_k +
 * xi_k), xi_k ~ U[-theta, theta] (Prop. one-bitequ: theta q_k stands in for
 * the sample), by the ADMM of Alg. 6 on Eq. 1bittensorqqqq:
 *   1. L = clip((m mu Z + J1 - m Y) / (m mu + J2), -alpha, alpha), with
 *      J1 = sum_k theta q_k P_k and J2 = sum_k P_k (the L-subproblem is one
 *      box-constrained quadratic per entry)                      (Eq. 1bit-L)
 *   2. (I + sum_{i in Gamma} nabla_i^T nabla_i) Z =
 *      L + Y/mu + sum_i nabla_i^T (G_i - Lambda_i/mu)             (Eq. 1bit-Z)
 *   3. G_i = D_{Phi, lambda/(gamma mu)}(nabla_i Z + Lambda_i/mu, L), gamma =
 *      |Gamma|, by the per-slice randomized engine (sketch width rank +
 *      oversample, power_iters, Philox key seed, counter word t)  (Eq. 1bit-g)
 *   4. Y += mu (L - Z); Lambda_i += mu (nabla_i Z - G_i);
 *      mu = min(mu_max, growth mu)                          (Eq. 1bit-Y..MU)
 * L is the orthonormal DCT-II along modes 3..d, as for tr_init.
 *   tr_onebit_create: a problem of order 3..8 with sizes `dims` (host) and
 *     dtype; `idx` (device, m int64) holds the flat face-slice index of each
 *     sample, `sign` (device, m int8) its sign (> 0: +1, else -1); both are
 *     read once (J1, J2 are formed here) and may be freed afterwards.
 *     Initialises L = Z = Y = G_i = Lambda_i = 0, mu = mu0, t = 0 (Alg. 6).
 *     Allocates about (8 + 2 |Gamma|) tensors plus an internal tr_init
 *     handle.  An index outside the tensor gives TR_EINVAL.
 *   tr_onebit_step: one iteration on the stream; with rel_change non-NULL
 *     it synchronises and returns ||L^{t+1} - L^t||_F / ||L^t||_F (the stop
 *     quantity of Alg. 6; +inf when L^t = 0).
 *   tr_onebit_get_state / tr_onebit_set_state: copy L, Z, Y (N elements
 *     each) and G, Lambda (|Gamma| tensors back to back, modes ascending)
 *     out of / into the object (device buffers; NULL skips one); both
 *     synchronise.
 * Errors: TR_EINVAL, TR_EUNSUPPORTED (shapes the internal handle refuses,
 * more than 2^31 - 1 entries or samples), TR_ENOMEM, TR_ECUDA.              */
typedef struct tr_onebit tr_onebit;
typedef struct {
  uint32_t modes;                  /* Gamma: bit k - 1 set for mode k        */
  double lambda, theta, alpha;     /* lambda, dither half-width, ||L||_inf   */
  double mu0, mu_max, growth;      /* mu^0, mu^max, vartheta                 */
  double tol;                      /* varpi of the stop test                 */
  int max_iter;
  tr_penalty phi;  double phi_theta, phi_gamma;
  int rank, oversample, power_iters;
  uint64_t seed;
  tr_prec prec;
} tr_onebit_params;

/* Defaults: Gamma = {1, 2}, lambda = theta = alpha = 1, mu0 = 1e-6,
 * mu_max = 1e3, growth 1.05 (Alg. 6), tol 1e-5, max_iter 200, Phi = MCP
 * (theta 1, gamma 4000), rank 10 + oversample 10, q = 1, seed 0, FP32.      */
void tr_onebit_default_params(tr_onebit_params *p);
tr_status tr_onebit_create(tr_onebit **ob, tr_dtype dtype, int order, const int64_t *dims,
                           int64_t m, const int64_t *idx, const int8_t *sign,
                           const tr_onebit_params *prm, void *cuda_stream, char *err,
                           size_t err_len);
tr_status tr_onebit_step(tr_onebit *ob, double *rel_change);
tr_status tr_onebit_get_state(tr_onebit *ob, void *L, void *Z, void *Y, void *G, void *Lam,
                              double *mu, int *t);
tr_status tr_onebit_set_state(tr_onebit *ob, const void *L, const void *Z, const void *Y,
                              const void *G, const void *Lam, double mu, int t);
const char *tr_onebit_last_error(const tr_onebit *ob);
tr_status tr_onebit_free(tr_onebit *ob);

/* ---- Learned sketch widths (engine TR_LR_LEARNED) ----------------------
 * Not in the paper, which fixes one sketch rank (Alg. 1) or grows the basis
 * to an accuracy (Alg. 3) and leaves learned sketching to future work
 * (Sec. 7).  Per slice pass, for every transformed slice j:
 *   features F_j (TR_MLP_FEATURES floats, tr_features) of the previous pass;
 *   y_j = MLP(F_j) ~ log(1 + kept rank), an MLP 16 -> 128 -> 128 -> 128 -> 1
 *     with ReLU, FP16 weights, FP32 biases and accumulation;
 *   l_j = round_up(round(exp(y_j) - 1) + oversample, 8) clipped to
 *     [min(8, l_max), l_max], l_max = rank + oversample (tr_plan_widths);
 *   the randomized slice prox of TR_LR_RSVD with width l_j;
 *   certificate: if the kept rank exceeds l_j - oversample and l_j < l_max,
 *     slice j is recomputed at l_max (counted in fallback_slices).
 * The first pass of a handle (and the first after tr_set_state) has no
 * history and runs every slice at l_max.  Widths are planned and grouped on
 * the device, so a pass never synchronises the host and steady-state steps
 * can be replayed as a graph; the panels hold every width class at once
 * (n slices per class).
 *
 * MLP parameter vector (FP32, TR_MLP_PARAMS = 35329 values): for each layer
 * in order (16 -> 128, 128 -> 128, 128 -> 128, 128 -> 1) its weights W
 * (out x in, row-major) then its biases (out).                              */
#define TR_MLP_FEATURES 16
#define TR_MLP_PARAMS 35329

/* Number of MLP parameters (TR_MLP_PARAMS).                                */
int64_t tr_mlp_param_count(void);

/* Install predictor weights in a TR_LR_LEARNED handle: `params` is a host
 * array of `count` (= TR_MLP_PARAMS) floats.  Weights files (model_path)
 * hold the 8 bytes "TRRANK01", four little-endian int32 (16, 128, 3, 0),
 * one int64 count, then `count` float32 parameters.  The hidden layers'
 * weights are converted to FP16 here, once, for the slice passes' forward
 * evaluations.  Synchronises.
 * Errors: TR_EINVAL (not a learned handle, wrong count).                    */
tr_status tr_set_model(tr_handle *h, const float *params, int64_t count);

/* Sketch width used for every slice in the last slice pass (host buffer of
 * n ints; the RSVD engine reports l, the adaptive engine the basis size).
 * Synchronises.                                                             */
tr_status tr_last_slice_widths(tr_handle *h, int *widths);

/* Features of the handle's last slice pass as the learned engine would see
 * them before a pass with threshold parameter `tau` at iteration t (device
 * buffer of n x TR_MLP_FEATURES floats).  Works for every engine, so that
 * traces of the adaptive engine can train the predictor.  Errors: TR_EINVAL
 * when no slice pass has run yet.                                           */
tr_status tr_slice_features(tr_handle *h, double tau, int t, float *features);

/* Stateless building blocks (device pointers, work on `cuda_stream`).
 *   tr_features: F (n x 16) from the rows of `sig` (n rows of stride ldsig,
 *     dtype elements; row j holds width[j] singular values in any order),
 *     kept ranks `rank`, widths `width`, the current and previous shrink
 *     thresholds thr and thr0 and the run fraction tfrac:
 *       f0 = log(1 + rank)/log 129         f1 = log(w)/log 129
 *       f2 = clip(log(s1/thr), -8, 8)/8    f3 = clip(log(s1/thr0), -8, 8)/8
 *       f4..f9 = s_(i)/s1, i in {2,4,8,16,32,64} (i-th largest, 0 if i > w)
 *       f10..f12 = log(1 + #{s > x})/log 129 for x = thr, thr/2, 2 thr
 *       f13 = (w - #{s > thr})/w          f14 = clip(log(thr/thr0), -1, 1)
 *       f15 = clip(tfrac, 0, 1)
 *     with s1 = max s; s1 = 0 gives f2 = f3 = -1, f4..f9 = 0; a threshold
 *     <= 0 gives f2 (f3) = 1 and f14 = 0.  Negative or NaN s count as 0.
 *   tr_plan_widths: width[j] from yhat[j] as above (1 <= lmax <= 96), ids =
 *     slice ids stably sorted by width class (l - 1)/8, counts[c] per class
 *     (ceil(lmax/8) classes).
 *   tr_mlp_init: He-uniform weights U(-a, a), a = sqrt(6/fan_in), zero
 *     biases, from Philox4x32-10 keyed by `seed`.
 *   tr_mlp_forward: yhat (B) = MLP(X) for X (B x 16).
 *   tr_mlp_loss_grad: loss = (1/B) sum w_r (yhat_r - y_r)^2 with
 *     w_r = 1 + under_weight [yhat_r < y_r]; grad (TR_MLP_PARAMS floats) =
 *     dloss/dparams (the FP16 rounding of the weights passes the gradient
 *     straight through); `loss` (1 float) may be NULL.  Allocates its
 *     workspace with stream-ordered allocation.
 *   tr_mlp_adam: one Adam step (step >= 1) on params with moments m, v.
 *   tr_mlp_train: `steps` Adam steps on minibatches of `batch` rows drawn
 *     with replacement (Philox keyed by `seed`) from (X, y), n rows;
 *     loss_hist (steps floats) may be NULL.  Allocates its workspace with
 *     stream-ordered allocation.
 * Errors: TR_EINVAL (sizes), TR_ECUDA.                                      */
tr_status tr_features(tr_dtype dtype, int n, const void *sig, int ldsig, const int *rank,
                      const int *width, double thr, double thr0, double tfrac,
                      float *features, void *cuda_stream);
tr_status tr_plan_widths(int n, const float *yhat, int oversample, int lmax, int *width,
                         int *ids, int *counts, void *cuda_stream);
tr_status tr_mlp_init(float *params, uint64_t seed, void *cuda_stream);
tr_status tr_mlp_forward(const float *params, const float *X, int B, float *yhat,
                         void *cuda_stream);
tr_status tr_mlp_loss_grad(const float *params, const float *X, const float *y, int B,
                           double under_weight, float *grad, float *loss, void *cuda_stream);
tr_status tr_mlp_adam(float *params, const float *grad, float *m, float *v, int64_t count,
                      double lr, double beta1, double beta2, double eps, int step,
                      void *cuda_stream);
tr_status tr_mlp_train(float *params, const float *X, const float *y, int n, int batch,
                       int steps, double lr, double under_weight, uint64_t seed,
                       float *loss_hist, void *cuda_stream);

/* ---- Graph replay, tile autotuning and batches (not in the paper) ------
 * The penalty schedule (mu, the previous mu and the iteration index t of
 * the sketches' Philox counters) lives on the device and the last kernel of
 * a step advances it (mu <- min(growth mu, mu_max), t += 1), so the launch
 * sequence of a steady-state step -- a step taken without tr_step_info after
 * another such step -- is the same at every iteration.
 *
 * tr_graph_mode: when on, steady-state steps of this handle replay one
 *   captured CUDA graph (captured at the first such step, on a stream the
 *   handle owns, ordered after the handle's stream by events).  Results are
 *   identical to eager steps.
 * tr_set_tube_tile: tubes per block of the tube kernels (a power of two
 *   from 4 to 256; 0 = the default: the smallest of 32..256 whose tile gives
 *   each of the block's 256 threads a fibre of every transformed mode,
 *   halved until the tile fits).  Every tile computes the same values.
 *   Errors: TR_EINVAL (not a power of two in range or too large).
 * tr_set_slice_groups: split the RSVD slice pass into `groups` (1..4)
 *   contiguous slice ranges run on side streams, so that latency-bound
 *   kernels of one range overlap bandwidth-bound products of another.  Same
 *   values for every split.  Errors: TR_EINVAL (range), TR_EUNSUPPORTED
 *   (other engines).
 * tr_autotune: time every fitting tube tile on the transform kernel and
 *   (RSVD engine) every slice split on slice passes of L(M), using the
 *   handle's transform-domain scratch (`reps` runs each; the iterate is
 *   not touched -- a deferred inverse pass is completed first), install the
 *   fastest and cache them per shape class (dtype, n1, n2, transformed mode
 *   sizes, engine, sketch width, power steps, precision) for the process;
 *   reps = 0 reuses a cached choice when there is one.  `tile` and `groups`
 *   may be NULL.  Synchronises.                                               */
tr_status tr_graph_mode(tr_handle *h, int on);
tr_status tr_set_tube_tile(tr_handle *h, int tubes_per_block);
tr_status tr_set_slice_groups(tr_handle *h, int groups);
tr_status tr_autotune(tr_handle *h, int reps, int *tile, int *groups);

/* A batch: independent problems of any shapes, each with its own handle
 * (workspace, parameters, state), stepped together.  Problems are spread
 * over `nstreams` internal streams (<= 0: 8); each step of the batch is one
 * CUDA graph launch covering every problem's steady-state step (captured at
 * the first such step; eager launches otherwise, or when graph mode is off).
 *   tr_batch_create: problems[i] with params[i] (any engine);
 *     `cuda_stream` is the caller's stream, which every batch step is
 *     ordered after and before.
 *   tr_batch_step: one iteration of every problem; `infos` (NULL or nprob
 *     entries) requests the per-problem reports, which synchronises.
 *   tr_batch_handle: the handle of problem i (for tr_get_state and the
 *     other per-handle calls; do not tr_free it).
 *   tr_batch_autotune: tr_autotune on every problem (its tube tile and slice
 *     split, cached per shape class; `reps` as there), then the batch graph
 *     is captured afresh at the next steady-state step.  Values do not
 *     change.  Call it between steps; it synchronises.  Errors: as
 *     tr_autotune, for the first problem that fails.
 *   tr_batch_launches: kernels launched by the batch so far.
 *   tr_batch_last_error: message of the calling thread's last failed
 *     batch call.                                                          */
typedef struct tr_batch tr_batch;
tr_status tr_batch_create(tr_batch **b, int nprob, const tr_problem *problems,
                          const tr_params *params, int nstreams, void *cuda_stream);
tr_status tr_batch_step(tr_batch *b, tr_step_info *infos);
tr_status tr_batch_handle(tr_batch *b, int i, tr_handle **h);
tr_status tr_batch_graph_mode(tr_batch *b, int on);
tr_status tr_batch_autotune(tr_batch *b, int reps);
tr_status tr_batch_launches(const tr_batch *b, uint64_t *count);
tr_status tr_batch_free(tr_batch *b);
const char *tr_batch_last_error(void);

/* Release all workspace.  Safe on NULL.                                     */
tr_status tr_free(tr_handle *h);

/* Last error message for `h` (or, when h is NULL, for the calling thread's
 * last failed call that had no handle, such as tr_init).  The string is
 * owned by the library.                                                     */
const char *tr_last_error(const tr_handle *h);

#ifdef __cplusplus
}
#endif

#endif /* TR_H */
