// Internal declarations shared by the libtr translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "tr.h"

#define TR_MAX_TMODES 6
#define TR_MAX_NK 64          // largest transformed-mode size handled in registers
#define TR_MAX_L 96           // largest sketch width handled by the slice kernels
#define TR_MLP_IN 16          // rank-predictor features per slice
#define TR_MLP_HIDDEN 128     // units per hidden layer
#define TR_MLP_LAYERS 3       // hidden layers
#define TR_LEARNED_STREAMS 4  // streams the learned engine spreads width groups over

// The transformed modes 3..d of a problem as seen from the slice index j.
// Mode k (0-based among the transformed modes) has size dim[k] and stride
// stride[k] in j (stride[0] = 1, stride[k] = dim[0]*...*dim[k-1]).  Its
// forward matrix U (the orthonormal DCT-II, dim x dim, rows padded to nkpad
// columns with zeros) is at element offset off_fwd[k] of the matrix buffer;
// the inverse U^{-1} = U^T, folded by the cosine symmetry of U, at
// off_inv[k] (layout: transform_mats_layout).
struct TransformDesc {
  int nt;
  int nkpad;
  int dim[TR_MAX_TMODES];
  int stride[TR_MAX_TMODES];
  int off_fwd[TR_MAX_TMODES];
  int off_inv[TR_MAX_TMODES];
  int mats_len;   // elements in the matrix buffer (multiple of 4)
  int tp = 0;     // tubes per block (0: the largest of 32, 16, 8, 4 that fits)
};

// Scalars of one ADMM iteration used by the elementwise passes.
struct TubeScalars {
  double mu;          // mu^t
  double lam_over_mu; // lambda / mu^t  (threshold of GNHTT)
  int noise;          // tr_noise
  int psi;            // tr_penalty of GNHTT
  double psi_theta, psi_gamma;
  const double *dmu = nullptr;  // when set: mu^t = *dmu (device), lam_over_mu = lambda / mu^t
  double lambda = 0.0;
  int planes = 0;     // FP32: write Abar as BF16 planes (SliceWork::asplit)
};

// Device copy of the penalty schedule, so that a captured step stays valid
// from one iteration to the next: the step reads mu and t here, and its last
// kernel advances them (mu_prev <- mu, mu <- min(growth mu, mu_max), t += 1).
struct DevSched {
  double mu, mu_prev;
  int t, pad;
};
cudaError_t launch_schedule(DevSched *d, double growth, double mu_max, cudaStream_t s);

// Shrinkage of singular values in the slice pass.
struct ShrinkScalars {
  double tau;
  int phi;
  double theta, gamma;
  const double *dmu = nullptr;  // when set: tau = 1 / *dmu (device)
};

// Residual slots written with atomicMax on the bit pattern of a
// non-negative double.
enum { RES_DL = 0, RES_DE = 1, RES_LG = 2, RES_DG = 3, RES_CONS = 4, RES_COUNT = 5 };

// ---- programmatic dependent launch ----
// Kernels of a step launched with programmatic stream serialization may
// start while the previous kernel in the stream drains.  Each such kernel
// calls pdl_wait() before it touches memory (it returns once the previous
// grid has completed and its writes are visible) and pdl_trigger() after its
// last store; a grid is launched early only once every block of its
// predecessor has triggered or exited, so every predecessor block is already
// resident and nothing can wait on an unscheduled block.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// ---- tensor maps (tensor_map.cu) ----
// A 2D tensor map of `rows` rows of `cols` elements (FP32, or bytes when
// u8), rows `row_stride` elements apart, with boxes of box_cols x box_rows;
// cached by view.  False when the view breaks a tensor-copy rule (16-byte
// aligned base and row stride, box edge <= 256, box rows of 16-byte
// multiples) or the driver refuses it.
bool encode_tensor_2d(CUtensorMap *out, const void *base, bool u8, int64_t cols, int64_t rows,
                      int64_t row_stride, int box_cols, int box_rows);

// A 3D tensor map of FP32 elements (d0 contiguous, then d1 with element
// stride s1, then d2 with stride s2) with boxes of box0 x box1 x 1, the
// 128-byte swizzle when swizzle128 (then box0 * 4 must be 128); cached by
// view.  Elements past a dimension read as zeros.  False when the view
// breaks a tensor-copy rule or the driver refuses it.
bool encode_tensor_3d_f32(CUtensorMap *out, const void *base, int64_t d0, int64_t d1, int64_t d2,
                          int64_t s1, int64_t s2, int box0, int box1, bool swizzle128);
// The same for elements of esz bytes: 4 (FP32) or 2 (BF16); strides in
// elements, box0 * esz = 128 with the swizzle.
bool encode_tensor_3d(CUtensorMap *out, const void *base, int esz, int64_t d0, int64_t d1,
                      int64_t d2, int64_t s1, int64_t s2, int box0, int box1, bool swizzle128);

// ---- tube passes (tube_kernels.cu) ----
cudaError_t launch_tube_forward(tr_dtype dt, int64_t P, int n, const TransformDesc &td,
                                const void *mats, const void *M, const uint8_t *mask,
                                void *L, void *E, void *Y, const void *G, const void *Lam,
                                void *Abar, const TubeScalars &sc,
                                unsigned long long *res, int *flags, cudaStream_t s);
cudaError_t launch_tube_inverse(tr_dtype dt, int64_t P, int n, const TransformDesc &td,
                                const void *mats, const void *Gbar, const void *L,
                                void *G, void *Lam, double mu, const double *dmu,
                                unsigned long long *res, int *flags, cudaStream_t s);
cudaError_t launch_tube_fused(tr_dtype dt, int64_t P, int n, const TransformDesc &td,
                              const void *mats, const void *Gbar, double mu_prev,
                              const double *dmu_prev, const void *M, const uint8_t *mask, void *L,
                              void *E, void *Y, void *G, void *Lam, void *Abar,
                              const TubeScalars &sc, unsigned long long *res_prev,
                              unsigned long long *res, int *flags, cudaStream_t s);
cudaError_t launch_transform(tr_dtype dt, int64_t P, int n, const TransformDesc &td,
                             const void *mats, const void *src, void *dst, bool inverse,
                             cudaStream_t s);
int tube_tile_candidates(tr_dtype dt, int n, const TransformDesc &td, int *tps, int cap);
// Sets off_fwd, off_inv and mats_len from nt, dim and nkpad; returns HK, the
// padded half row length.  Forward rows: U[i][0..dim) at off_fwd + i nkpad.
// Folded inverse rows, m < ceil(dim/2): U[0][m], U[2][m], ... at
// off_inv + 2 HK m and U[1][m], U[3][m], ... at off_inv + 2 HK m + HK
// (zeros beyond dim).
int transform_mats_layout(TransformDesc &td);
size_t tube_smem_bytes(tr_dtype dt, int n, const TransformDesc &td, int *tp_out);

// ---- slice pass (slice_kernels.cu) ----
// Optional selection of slices for one launch: batch entry b (a block
// index) works on slice ids[b]; entries b >= *count exit at once.  Panels
// are indexed by b, the transformed tensors, Philox counters and per-slice
// statistics by the slice id.  Null pointers mean "all slices, in order".
struct SliceSel {
  const int *ids = nullptr;
  const int *count = nullptr;
};

// Optional per-kernel timing of one slice pass: mark() records an event
// after a kernel and labels it, so kernel k's device time is the interval
// between events k-1 and k (event 0 is recorded before the first kernel).
struct SliceProf {
  static constexpr int kMax = 40;
  cudaEvent_t ev[kMax] = {};
  const char *name[kMax] = {};
  int k = 0;
  void mark(cudaStream_t s, const char *nm) {
    if (k < kMax && ev[k]) {
      cudaEventRecord(ev[k], s);
      name[k++] = nm;
    }
  }
};

struct SliceWork {
  int n, n1, n2, l, q;
  uint64_t seed;
  void *Om;     // n * n2 * l, column-major per slice
  void *P1;     // n * n1 * l, column-major per slice (ld n1)
  void *P2;     // n * n2 * l, column-major per slice (ld n2)
  void *sig;    // singular values of B: row j (slice id) at sig + j * ldsig
  int *rank;    // kept rank per slice id
  int prec;     // tr_prec of the skinny products (FP32 problems only)
  int *err;     // device flag set by a tensor-core GEMM whose bounded wait expired
  SliceSel sel; // which slices this pass works on (default: all)
  int ldsig;    // row stride of sig (0: l); entries l..ldsig-1 are zeroed
  int *width;   // optional: sketch width used, per slice id
  const int *dt;  // optional: iteration index of the Philox counters (device)
  SliceProf *prof = nullptr;  // optional: per-kernel events (eager passes only)
  int nA = 0;   // slices in the Abar/Gbar arrays (0: n), the range of slice ids
  int asplit = 0;  // Abar is given as two BF16 planes (hi, then lo: x = hi + lo),
                   // FP32 problems in the BF16 and split-BF16 forms only
};
// Whether an n-slice stack of n1 x n2 slices with sketch width l can take its
// Abar as BF16 planes (n2 % 8 == 0, n1 % 4 == 0, l <= 64).
bool planes_ok(int64_t n, int n1, int n2, int l);
// FP32 x[0..count) -> BF16 planes: dst[i] = hi = bf16(x[i]), dst[count + i] =
// lo = bf16(x[i] - hi).
cudaError_t launch_split_planes(const float *x, void *dst, int64_t count, cudaStream_t s);
// Workspace of the fixed-accuracy engine (Alg. 3 per slice).
struct AdaptWork {
  int b, kcap;          // block size, basis cap (a multiple of b)
  double eps, delta_rel;
  void *Ucat, *Vcat, *X, *Lm, *Rm;
  double *E, *nrm2;
  int *active, *kept, *draws;
};
cudaError_t launch_slice_adaptive(tr_dtype dt, const SliceWork &w, const AdaptWork &aw,
                                  const void *Abar, void *Gbar, const ShrinkScalars &sh, int t,
                                  cudaStream_t s);
size_t adapt_smem_bytes(tr_dtype dt, int n1, int n2, int b, int kcap);
cudaError_t launch_slice_rsvd(tr_dtype dt, const SliceWork &w, const void *Abar, void *Gbar,
                              const ShrinkScalars &sh, int t, cudaStream_t s);
size_t slice_smem_limit_ok(tr_dtype dt, int n1, int n2, int l);
// Shared-Tucker randomized prox (Alg. 1 with processing order (1, 2), Alg. 4
// randomized branch) on a transformed stack; ws holds tucker_ws_bytes.
size_t tucker_ws_bytes(tr_dtype dt, int n, int n1, int n2, int r1, int r2, int b1, int b2, int q1,
                       int q2);
// g_blocks: G1, G2 are per-slice column-major blocks (k x b each) instead of
// one stacked matrix; sig (row stride r1) and rank receive the slice
// statistics when non-null.
cudaError_t launch_slice_tucker(tr_dtype dt, int n, int n1, int n2, int r1, int r2, int b1, int b2,
                                int q1, int q2, const void *Abar, void *Gbar, const void *G1,
                                const void *G2, void *ws, const ShrinkScalars &sh, void *F1_out,
                                void *F2_out, cudaStream_t s, bool g_blocks = false,
                                void *sig = nullptr, int *rank = nullptr);
// Columns of F (m x r, column-major) scaled by +-1 so that each column's
// entry of largest magnitude (the first one on ties) is positive: the sign
// convention of both Tucker forms' factors.
cudaError_t launch_canon_signs(tr_dtype dt, void *F, int m, int r, cudaStream_t s);
// n per-slice Gaussian blocks of per_slice elements (Philox4x32-10 counter
// (m/4, j, t, stream), Box-Muller; t from dt_dev when non-null).
cudaError_t launch_gaussian_blocks(tr_dtype dt, int n, int64_t per_slice, void *out, uint64_t seed,
                                   int t, const int *dt_dev, uint32_t stream, cudaStream_t s);

// ---- learned sketch widths and the rank-predictor MLP (learned.cu) ----
struct LearnedWork {
  int lmax = 0, p = 0;       // plain width (cap), oversampling
  int merge_min = 8;         // width groups with fewer slices join the next wider one
  float *params = nullptr;   // MLP parameters (FP32 master copy)
  void *w16 = nullptr;       // its hidden weights as FP16, packed once per model
  float *feat = nullptr;     // n x TR_MLP_IN features
  float *pred = nullptr;     // n predicted log(1 + rank)
  int *width = nullptr;      // sketch width used per slice (history of the last pass)
  int *ids = nullptr, *counts = nullptr;     // plan: slice ids sorted by width class
  int *fb_ids = nullptr, *fb_count = nullptr;
  int *gids = nullptr, *gcount = nullptr;    // width groups: C x n slice ids, C sizes
  bool have_hist = false;
  double thr_prev = 0.0;
  // the plain adaptive method (Alg. 3 per slice) as judge and fallback of
  // the learned widths: a sketch is kept when it meets Alg. 3's stop test
  // E_j = ||Abar_j||^2 - ||B_j||^2 < eps^2 ||Abar_j||^2, or kept rank <=
  // width - p, or width >= aw.kcap; else the adaptive engine recomputes the
  // slice (workspace aw, cap aw.kcap <= lmax)
  AdaptWork aw{};
  double *anorm2 = nullptr;  // ||Abar_j||_F^2 per slice
  int *iota = nullptr;       // 0, 1, ..., n-1
  cudaStream_t aux[TR_LEARNED_STREAMS] = {};
  cudaEvent_t fork = nullptr, join[TR_LEARNED_STREAMS] = {};
};
int64_t mlp_param_count();
size_t mlp_workspace_floats(int B);
cudaError_t launch_mlp_init(float *prm, uint64_t seed, cudaStream_t s);
cudaError_t launch_mlp_forward(const float *prm, const float *X, int B, float *yhat, float *H,
                               cudaStream_t s, const void *w16 = nullptr);
// The hidden layers' weights of prm as FP16 (mlp_pack_halves() halves).
size_t mlp_pack_halves();
cudaError_t launch_mlp_pack(const float *prm, void *w16, cudaStream_t s);
cudaError_t launch_mlp_loss_grad(const float *prm, const float *X, const float *y, int B,
                                 float under, float *work, float *yhat, float *grad, float *loss,
                                 cudaStream_t s);
cudaError_t launch_mlp_adam(float *prm, const float *g, float *m, float *v, int64_t n, double lr,
                            double b1, double b2, double eps, int step, cudaStream_t s);
cudaError_t launch_mlp_gather(const float *X, const float *y, int n, int B, int step,
                              uint64_t seed, float *Xb, float *yb, cudaStream_t s);
// Optional device schedule for the features: thresholds from mu and the
// previous mu, run fraction t / T (null d: the host values are used).
struct FeatSched {
  const DevSched *d = nullptr;
  int phi = 0;
  double theta = 1.0, gamma = 1.0;
  int T = 0;
};
cudaError_t launch_features(tr_dtype dt, int n, const void *sig, int ldsig, const int *rank,
                            const int *width, double thr, double thr0, double tfrac, float *F,
                            cudaStream_t s, FeatSched fs = FeatSched{});
int learned_panel_cols(int lmax);
int plan_classes(int lmax);
cudaError_t launch_plan(int n, const float *yhat, int p, int lmax, int *width, int *ids,
                        int *counts, cudaStream_t s);
cudaError_t launch_slice_learned(tr_dtype dt, const SliceWork &w, LearnedWork &lw,
                                 const void *Abar, void *Gbar, const ShrinkScalars &sh,
                                 double thr, int t, int T, FeatSched fs, cudaStream_t s,
                                 uint64_t *launches);
