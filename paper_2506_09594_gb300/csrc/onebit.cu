// One-bit completion (GNOBHTC), one ADMM iteration of Alg. 6 on the GPU.
//
// Model (Eq. 1bittensorqqqq): min (1/2m) sum_k (L[s_k] - theta q_k)^2
//   + (lambda/gamma) sum_{i in Gamma} ||G_i||_{Phi,L} + I{||L||_inf <= alpha}
//   s.t. Z = L, G_i = nabla_i(Z),
// with the augmented terms <Y, L - Z> + mu/2 ||L - Z||^2 and
// <Lambda_i, nabla_i Z - G_i> + mu/2 ||nabla_i Z - G_i||^2.  One iteration:
//   1. L = clip((m mu Z + J1 - m Y) / (m mu + J2), -alpha, alpha)   (Eq. 1bit-L)
//      with J1 = sum_k theta q_k P_k and J2 = sum_k P_k: the L-subproblem
//      separates into one box-constrained quadratic per entry;
//   2. (I + sum_i nabla_i^T nabla_i) Z = L + Y/mu + sum_i nabla_i^T (G_i - Lambda_i/mu)
//      (Eq. 1bit-Z, with the new L: Alg. 6 updates L first);
//   3. G_i = D_{Phi, lambda/(gamma mu)}(nabla_i Z + Lambda_i/mu, L)    (Eq. 1bit-g);
//   4. Y += mu (L - Z); Lambda_i += mu (nabla_i Z - G_i);
//      mu = min(mu_max, vartheta mu)                          (Eq. 1bit-Y..MU);
//   5. the stop quantity ||L^{t+1} - L^t||_F / ||L^t||_F of Alg. 6.
//
// Step 3 runs through the public entry points tr_transform_forward,
// tr_slice_prox and tr_transform_inverse of an internal handle (the
// randomized per-slice engine with its Philox sketches for iteration t);
// step 2 through fused stencil kernels and tr_gradient_solve.  J1 and J2 come from exact
// integer counts of the +1 and -1 samples per entry, so they do not depend
// on the order of the atomic updates.

#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <vector>

#include "ew_kernels.cuh"
#include "tr_internal.cuh"

struct tr_onebit {
  tr_dtype dtype = TR_F32;
  int order = 0;
  int64_t dims[8] = {0};
  int64_t S[8] = {0};             // flat stride of each mode
  int64_t N = 0, m = 0;
  int nmodes = 0;
  int modes[8] = {0};             // 1-based modes of Gamma, ascending
  tr_onebit_params prm{};
  cudaStream_t stream = nullptr;
  tr_handle *prox = nullptr;      // transform + per-slice prox of step 3
  size_t esz = 4;
  void *L = nullptr, *Z = nullptr, *Y = nullptr, *J1 = nullptr, *J2 = nullptr;
  void *G = nullptr, *Lam = nullptr;                 // nmodes tensors each, back to back
  void *R = nullptr, *Abar = nullptr, *Gbar = nullptr;
  uint8_t *mask = nullptr;        // the internal handle's (unread) mask
  double *acc = nullptr;          // device: sum (L' - L)^2, sum L^2
  double mu = 0.0;
  int t = 0;
  char err[256] = {0};
};

namespace {

tr_status ofail(tr_onebit *ob, char *buf, size_t len, tr_status st, const char *fmt, ...) {
  char tmp[256];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(tmp, sizeof tmp, fmt, ap);
  va_end(ap);
  if (ob) snprintf(ob->err, sizeof ob->err, "%s", tmp);
  if (buf && len) snprintf(buf, len, "%s", tmp);
  return st;
}

int ob_grid(int64_t N) {
  const int64_t blocks = (N + 255) / 256;
  return (int)(blocks < 152 * 32 ? (blocks < 1 ? 1 : blocks) : 152 * 32);
}

// Per-entry counts of the +1 and -1 samples; an index outside [0, N) sets
// *bad and is skipped.
__global__ void onebit_count_kernel(const int64_t *__restrict__ idx, const int8_t *__restrict__ sgn,
                                    int64_t m, int64_t N, int *pos, int *neg, int *bad) {
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m; k += step) {
    const int64_t e = idx[k];
    if (e < 0 || e >= N) {
      atomicExch(bad, 1);
      continue;
    }
    atomicAdd(sgn[k] > 0 ? pos + e : neg + e, 1);
  }
}

template <typename T>
__global__ void onebit_j_kernel(const int *__restrict__ pos, const int *__restrict__ neg, int64_t N,
                                T theta, T *J1, T *J2) {
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < N; f += step) {
    J1[f] = theta * (T)(pos[f] - neg[f]);
    J2[f] = (T)(pos[f] + neg[f]);
  }
}

// Step 1 in place on L, with the two sums of the stop quantity.
template <typename T>
__global__ void onebit_l_kernel(T *L, const T *__restrict__ Z, const T *__restrict__ Y,
                                const T *__restrict__ J1, const T *__restrict__ J2, int64_t N,
                                T m_mu, T m, T alpha, double *acc) {
  double d2 = 0.0, o2 = 0.0;
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < N; f += step) {
    const T old = L[f];
    T v = (m_mu * Z[f] + J1[f] - m * Y[f]) / (m_mu + J2[f]);
    v = v > alpha ? alpha : (v < -alpha ? -alpha : v);
    L[f] = v;
    d2 += (double)(v - old) * (double)(v - old);
    o2 += (double)old * (double)old;
  }
  for (int o = 16; o > 0; o >>= 1) {
    d2 += __shfl_xor_sync(0xffffffffu, d2, o);
    o2 += __shfl_xor_sync(0xffffffffu, o2, o);
  }
  __shared__ double s[2][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    s[0][warp] = d2;
    s[1][warp] = o2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a += s[0][w];
      b += s[1][w];
    }
    atomicAdd(acc, a);
    atomicAdd(acc + 1, b);
  }
}

void free_onebit(tr_onebit *ob) {
  if (ob->prox) tr_free(ob->prox);
  void *bufs[] = {ob->L, ob->Z, ob->Y, ob->J1, ob->J2, ob->G, ob->Lam,
                  ob->R, ob->Abar, ob->Gbar, ob->mask, ob->acc};
  for (void *p : bufs)
    if (p) cudaFree(p);
}

void *tensor(const tr_onebit *ob, void *base, int i) {
  return (char *)base + (size_t)i * (size_t)ob->N * ob->esz;
}

template <typename T>
tr_status onebit_step(tr_onebit *ob, double *rel) {
  cudaStream_t s = ob->stream;
  const int g = ob_grid(ob->N);
  const int64_t N = ob->N;
  const double mu = ob->mu;
  T *L = (T *)ob->L, *Z = (T *)ob->Z, *Y = (T *)ob->Y, *R = (T *)ob->R;
  char buf[256];
#define OB_CUDA(call)                                                                        \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess) return ofail(ob, nullptr, 0, TR_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)
#define OB_TR(call)                                                                          \
  do {                                                                                       \
    tr_status st_ = (call);                                                                  \
    if (st_ != TR_OK) return ofail(ob, nullptr, 0, st_, "%s: %s", #call, buf[0] ? buf : tr_last_error(ob->prox)); \
  } while (0)
  buf[0] = 0;
  // 1. L-update and the sums of the stop quantity
  OB_CUDA(cudaMemsetAsync(ob->acc, 0, 2 * sizeof(double), s));
  onebit_l_kernel<T><<<g, 256, 0, s>>>(L, Z, Y, (const T *)ob->J1, (const T *)ob->J2, N,
                                       (T)((double)ob->m * mu), (T)ob->m, (T)ob->prm.alpha,
                                       ob->acc);
  OB_CUDA(cudaGetLastError());
  // 2. Z-update: R = L + Y/mu + sum_i nabla_i^T (G_i - Lambda_i/mu); Z = solve(R)
  ew::axpby_kernel<T><<<g, 256, 0, s>>>(R, T(1), L, (T)(1.0 / mu), Y, N);
  OB_CUDA(cudaGetLastError());
  uint32_t mask = 0;
  for (int q = 0; q < ob->nmodes; ++q) {
    const int k = ob->modes[q];
    mask |= 1u << (k - 1);
    const T *Gi = (const T *)tensor(ob, ob->G, q), *Li = (const T *)tensor(ob, ob->Lam, q);
    ew::adj_grad_accum_kernel<T><<<g, 256, 0, s>>>(R, Gi, Li, (T)(1.0 / mu), N, ob->S[k - 1],
                                                  ob->dims[k - 1]);
    OB_CUDA(cudaGetLastError());
  }
  OB_TR(tr_gradient_solve(ob->dtype, ob->order, ob->dims, mask, R, Z, s, buf, sizeof buf));
  // 3. G-updates, tau = lambda / (gamma mu); 4. multipliers
  const double tau = ob->prm.lambda / ((double)ob->nmodes * mu);
  for (int q = 0; q < ob->nmodes; ++q) {
    const int k = ob->modes[q];
    T *Gi = (T *)tensor(ob, ob->G, q), *Li = (T *)tensor(ob, ob->Lam, q);
    const int64_t S = ob->S[k - 1], nk = ob->dims[k - 1];
    ew::grad_plus_kernel<T><<<g, 256, 0, s>>>(R, Z, Li, (T)(1.0 / mu), N, S, nk);   // prox input
    OB_CUDA(cudaGetLastError());
    OB_TR(tr_transform_forward(ob->prox, R, ob->Abar));
    OB_TR(tr_slice_prox(ob->prox, ob->Abar, ob->Gbar, tau, ob->t));
    OB_TR(tr_transform_inverse(ob->prox, ob->Gbar, Gi));
    ew::grad_multiplier_kernel<T><<<g, 256, 0, s>>>(Li, (T)mu, Z, Gi, N, S, nk);
    OB_CUDA(cudaGetLastError());
  }
  ew::multiplier_kernel<T><<<g, 256, 0, s>>>(Y, (T)mu, L, Z, N);
  OB_CUDA(cudaGetLastError());
#undef OB_CUDA
#undef OB_TR
  ob->mu = fmin(ob->prm.mu_max, ob->prm.growth * mu);
  ob->t += 1;
  if (rel) {
    double h[2] = {0.0, 0.0};
    cudaError_t e = cudaMemcpyAsync(h, ob->acc, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return ofail(ob, nullptr, 0, TR_ECUDA, "%s", cudaGetErrorString(e));
    *rel = h[1] > 0.0 ? sqrt(h[0] / h[1]) : INFINITY;
  }
  return TR_OK;
}

}  // namespace

extern "C" void tr_onebit_default_params(tr_onebit_params *p) {
  if (!p) return;
  memset(p, 0, sizeof *p);
  p->modes = 0b11;
  p->lambda = 1.0;
  p->theta = 1.0;
  p->alpha = 1.0;
  p->mu0 = 1e-6;
  p->mu_max = 1e3;
  p->growth = 1.05;
  p->tol = 1e-5;
  p->max_iter = 200;
  p->phi = TR_PEN_MCP;
  p->phi_theta = 1.0;
  p->phi_gamma = 4000.0;
  p->rank = 10;
  p->oversample = 10;
  p->power_iters = 1;
  p->seed = 0;
  p->prec = TR_PREC_FP32;
}

extern "C" tr_status tr_onebit_create(tr_onebit **out, tr_dtype dtype, int order,
                                      const int64_t *dims, int64_t m, const int64_t *idx,
                                      const int8_t *sign, const tr_onebit_params *prm,
                                      void *cuda_stream, char *err, size_t err_len) {
  if (err && err_len) err[0] = 0;
  if (!out || !prm || !dims || !idx || !sign || m < 1)
    return ofail(nullptr, err, err_len, TR_EINVAL, "null pointer or no samples");
  *out = nullptr;
  if (dtype != TR_F32 && dtype != TR_F64) return ofail(nullptr, err, err_len, TR_EINVAL, "bad dtype");
  if (order < 3 || order > 8)
    return ofail(nullptr, err, err_len, TR_EINVAL, "order must be 3..8 (slices need a transformed mode)");
  if (!(prm->mu0 > 0) || !(prm->growth >= 1.0) || !(prm->mu_max >= prm->mu0) ||
      !(prm->alpha > 0) || !(prm->theta > 0) || !(prm->lambda >= 0))
    return ofail(nullptr, err, err_len, TR_EINVAL,
                 "need mu0 > 0, growth >= 1, mu_max >= mu0, alpha > 0, theta > 0, lambda >= 0");
  if (prm->modes == 0 || (prm->modes >> order))
    return ofail(nullptr, err, err_len, TR_EINVAL, "Gamma must name at least one mode of the tensor");
  if (m > 0x7fffffff)
    return ofail(nullptr, err, err_len, TR_EUNSUPPORTED, "at most 2^31 - 1 samples");
  tr_onebit *ob = new (std::nothrow) tr_onebit();
  if (!ob) return ofail(nullptr, err, err_len, TR_ENOMEM, "host allocation failed");
  ob->dtype = dtype;
  ob->order = order;
  ob->N = 1;
  for (int k = 0; k < order; ++k) {
    if (dims[k] < 1) {
      delete ob;
      return ofail(nullptr, err, err_len, TR_EINVAL, "empty mode");
    }
    ob->dims[k] = dims[k];
    ob->N *= dims[k];
  }
  if (ob->N > 0x7fffffff) {
    delete ob;
    return ofail(nullptr, err, err_len, TR_EUNSUPPORTED, "at most 2^31 - 1 entries (int counts)");
  }
  ob->m = m;
  for (int k = 1; k <= order; ++k) {
    ob->S[k - 1] = ew::mode_stride(ob->dims, k);
    if (prm->modes & (1u << (k - 1))) ob->modes[ob->nmodes++] = k;
  }
  ob->prm = *prm;
  ob->stream = (cudaStream_t)cuda_stream;
  ob->esz = dtype == TR_F64 ? 8 : 4;
  ob->mu = prm->mu0;
  const size_t T = (size_t)ob->N * ob->esz;
  cudaError_t e = cudaSuccess;
  void **single[] = {&ob->L, &ob->Z, &ob->Y, &ob->J1, &ob->J2, &ob->R, &ob->Abar, &ob->Gbar};
  for (void **p : single)
    if (e == cudaSuccess) e = cudaMalloc(p, T);
  if (e == cudaSuccess) e = cudaMalloc(&ob->G, T * ob->nmodes);
  if (e == cudaSuccess) e = cudaMalloc(&ob->Lam, T * ob->nmodes);
  if (e == cudaSuccess) e = cudaMalloc((void **)&ob->mask, (size_t)ob->N);
  if (e == cudaSuccess) e = cudaMalloc((void **)&ob->acc, 2 * sizeof(double));
  if (e != cudaSuccess) {
    free_onebit(ob);
    delete ob;
    return ofail(nullptr, err, err_len, e == cudaErrorMemoryAllocation ? TR_ENOMEM : TR_ECUDA,
                 "workspace: %s", cudaGetErrorString(e));
  }
  cudaStream_t s = ob->stream;
  // Alg. 6 initialisation: G_i = Z = Lambda_i = Y = 0 (and L = 0)
  void *zero[] = {ob->L, ob->Z, ob->Y};
  for (void *p : zero)
    if (e == cudaSuccess) e = cudaMemsetAsync(p, 0, T, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(ob->G, 0, T * ob->nmodes, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(ob->Lam, 0, T * ob->nmodes, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(ob->mask, 0, (size_t)ob->N, s);
  // J1, J2 from the samples
  int *counts = nullptr, *bad = nullptr;
  if (e == cudaSuccess) e = cudaMallocAsync((void **)&counts, 2 * (size_t)ob->N * sizeof(int), s);
  if (e == cudaSuccess) e = cudaMallocAsync((void **)&bad, sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(counts, 0, 2 * (size_t)ob->N * sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, sizeof(int), s);
  int hbad = 0;
  if (e == cudaSuccess) {
    onebit_count_kernel<<<ob_grid(m), 256, 0, s>>>(idx, sign, m, ob->N, counts, counts + ob->N, bad);
    if (dtype == TR_F32)
      onebit_j_kernel<float><<<ob_grid(ob->N), 256, 0, s>>>(counts, counts + ob->N, ob->N,
                                                            (float)prm->theta, (float *)ob->J1,
                                                            (float *)ob->J2);
    else
      onebit_j_kernel<double><<<ob_grid(ob->N), 256, 0, s>>>(counts, counts + ob->N, ob->N,
                                                             prm->theta, (double *)ob->J1,
                                                             (double *)ob->J2);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  if (counts) cudaFreeAsync(counts, s);
  if (bad) cudaFreeAsync(bad, s);
  if (e != cudaSuccess || hbad) {
    free_onebit(ob);
    delete ob;
    if (hbad) return ofail(nullptr, err, err_len, TR_EINVAL, "a sample index is outside the tensor");
    return ofail(nullptr, err, err_len, TR_ECUDA, "samples: %s", cudaGetErrorString(e));
  }
  // the internal handle: transform and randomized per-slice prox of step 3
  tr_problem pb{};
  pb.order = order;
  for (int k = 0; k < order; ++k) pb.dims[k] = dims[k];
  pb.dtype = dtype;
  pb.observed = ob->L;
  pb.mask = ob->mask;
  tr_params hp;
  tr_default_params(&hp);
  hp.phi = prm->phi;
  hp.phi_theta = prm->phi_theta;
  hp.phi_gamma = prm->phi_gamma;
  hp.engine = TR_LR_RSVD;
  hp.rank = prm->rank;
  hp.oversample = prm->oversample;
  hp.power_iters = prm->power_iters;
  hp.seed = prm->seed;
  hp.prec = prm->prec;
  const tr_status st = tr_init(&ob->prox, &pb, &hp, cuda_stream);
  if (st != TR_OK) {
    const tr_status r = ofail(nullptr, err, err_len, st, "prox handle: %s", tr_last_error(nullptr));
    ob->prox = nullptr;
    free_onebit(ob);
    delete ob;
    return r;
  }
  *out = ob;
  return TR_OK;
}

extern "C" tr_status tr_onebit_step(tr_onebit *ob, double *rel_change) {
  if (!ob) return TR_EINVAL;
  return ob->dtype == TR_F32 ? onebit_step<float>(ob, rel_change) : onebit_step<double>(ob, rel_change);
}

extern "C" tr_status tr_onebit_get_state(tr_onebit *ob, void *L, void *Z, void *Y, void *G,
                                         void *Lam, double *mu, int *t) {
  if (!ob) return TR_EINVAL;
  const size_t T = (size_t)ob->N * ob->esz;
  const void *src[] = {ob->L, ob->Z, ob->Y, ob->G, ob->Lam};
  void *dst[] = {L, Z, Y, G, Lam};
  const size_t bytes[] = {T, T, T, T * ob->nmodes, T * ob->nmodes};
  for (int i = 0; i < 5; ++i) {
    if (!dst[i]) continue;
    const cudaError_t e = cudaMemcpyAsync(dst[i], src[i], bytes[i], cudaMemcpyDeviceToDevice, ob->stream);
    if (e != cudaSuccess) return ofail(ob, nullptr, 0, TR_ECUDA, "%s", cudaGetErrorString(e));
  }
  if (mu) *mu = ob->mu;
  if (t) *t = ob->t;
  const cudaError_t e = cudaStreamSynchronize(ob->stream);
  return e == cudaSuccess ? TR_OK : ofail(ob, nullptr, 0, TR_ECUDA, "%s", cudaGetErrorString(e));
}

extern "C" tr_status tr_onebit_set_state(tr_onebit *ob, const void *L, const void *Z,
                                         const void *Y, const void *G, const void *Lam, double mu,
                                         int t) {
  if (!ob || !(mu > 0) || t < 0) return TR_EINVAL;
  const size_t T = (size_t)ob->N * ob->esz;
  const void *src[] = {L, Z, Y, G, Lam};
  void *dst[] = {ob->L, ob->Z, ob->Y, ob->G, ob->Lam};
  const size_t bytes[] = {T, T, T, T * ob->nmodes, T * ob->nmodes};
  for (int i = 0; i < 5; ++i) {
    if (!src[i]) continue;
    const cudaError_t e = cudaMemcpyAsync(dst[i], src[i], bytes[i], cudaMemcpyDeviceToDevice, ob->stream);
    if (e != cudaSuccess) return ofail(ob, nullptr, 0, TR_ECUDA, "%s", cudaGetErrorString(e));
  }
  ob->mu = mu;
  ob->t = t;
  const cudaError_t e = cudaStreamSynchronize(ob->stream);
  return e == cudaSuccess ? TR_OK : ofail(ob, nullptr, 0, TR_ECUDA, "%s", cudaGetErrorString(e));
}

extern "C" const char *tr_onebit_last_error(const tr_onebit *ob) { return ob ? ob->err : ""; }

extern "C" tr_status tr_onebit_free(tr_onebit *ob) {
  if (!ob) return TR_OK;
  if (ob->stream) cudaStreamSynchronize(ob->stream);
  else cudaDeviceSynchronize();
  free_onebit(ob);
  delete ob;
  return TR_OK;
}
