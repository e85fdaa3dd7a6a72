// Internal declarations shared by the libtr translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "tr.h"

#define TR_MAX_TMODES 6
#define TR_MAX_NK 64          // largest transformed-mode size handled in registers
#define TR_MAX_L 96           // largest sketch width handled by the slice kernels

// The transformed modes 3..d of a problem as seen from the slice index j.
// Mode k (0-based among the transformed modes) has size dim[k] and stride
// stride[k] in j (stride[0] = 1, stride[k] = dim[0]*...*dim[k-1]).  Its
// forward matrix U (dim x dim, rows padded to nkpad columns with zeros) is at
// element offset off_fwd[k] of the matrix buffer, its inverse U^{-1} = U^T
// at off_inv[k].
struct TransformDesc {
  int nt;
  int nkpad;
  int dim[TR_MAX_TMODES];
  int stride[TR_MAX_TMODES];
  int off_fwd[TR_MAX_TMODES];
  int off_inv[TR_MAX_TMODES];
  int mats_len;   // elements in the matrix buffer (multiple of 4)
};

// Scalars of one ADMM iteration used by the elementwise passes.
struct TubeScalars {
  double mu;          // mu^t
  double lam_over_mu; // lambda / mu^t  (threshold of GNHTT)
  int noise;          // tr_noise
  int psi;            // tr_penalty of GNHTT
  double psi_theta, psi_gamma;
};

// Shrinkage of singular values in the slice pass.
struct ShrinkScalars {
  double tau;
  int phi;
  double theta, gamma;
};

// Residual slots written with atomicMax on the bit pattern of a
// non-negative double.
enum { RES_DL = 0, RES_DE = 1, RES_LG = 2, RES_DG = 3, RES_CONS = 4, RES_COUNT = 5 };

// ---- tube passes (tube_kernels.cu) ----
cudaError_t launch_tube_forward(tr_dtype dt, int64_t P, int n, const TransformDesc &td,
                                const void *mats, const void *M, const uint8_t *mask,
                                void *L, void *E, void *Y, const void *G, const void *Lam,
                                void *Abar, const TubeScalars &sc,
                                unsigned long long *res, int *flags, cudaStream_t s);
cudaError_t launch_tube_inverse(tr_dtype dt, int64_t P, int n, const TransformDesc &td,
                                const void *mats, const void *Gbar, const void *L,
                                void *G, void *Lam, double mu,
                                unsigned long long *res, int *flags, cudaStream_t s);
cudaError_t launch_tube_fused(tr_dtype dt, int64_t P, int n, const TransformDesc &td,
                              const void *mats, const void *Gbar, double mu_prev, const void *M,
                              const uint8_t *mask, void *L, void *E, void *Y, void *G, void *Lam,
                              void *Abar, const TubeScalars &sc, unsigned long long *res_prev,
                              unsigned long long *res, int *flags, cudaStream_t s);
cudaError_t launch_transform(tr_dtype dt, int64_t P, int n, const TransformDesc &td,
                             const void *mats, const void *src, void *dst, bool inverse,
                             cudaStream_t s);
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

struct SliceWork {
  int n, n1, n2, l, q;
  uint64_t seed;
  void *Om;     // n * n2 * l, column-major per slice
  void *P1;     // n * n1 * l, column-major per slice (ld n1)
  void *P2;     // n * n2 * l, column-major per slice (ld n2)
  void *sig;    // n * l singular values of B
  int *rank;    // n kept ranks
  int prec;     // tr_prec of the skinny products (FP32 problems only)
  int *err;     // device flag set by a tensor-core GEMM whose bounded wait expired
  SliceSel sel; // which slices this pass works on (default: all)
};
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
