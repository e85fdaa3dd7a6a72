// The gradient-domain prior (GNHTCTV): one ADMM iteration of Alg. 5 with a
// set Gamma of gradient directions, on the GPU.
//
// Model (Eq. equ_nonconvex): min (1/gamma) sum_{k in Gamma} ||G_k||_{Phi,L}
//   + lambda Upsilon(P_Omega(E))  s.t. G_k = nabla_k(L), L + E = M,
// gamma = |Gamma|.  One iteration, in Alg. 5's order:
//   1. (I + sum_k nabla_k^T nabla_k) L = (M - E + Y/mu) + sum_k nabla_k^T (G_k - Lambda_k/mu)
//                                              (Eq. coef-tensor, Eq. gnrhtc-L)
//   2. G_k = D_{Phi, 1/(gamma mu)}(nabla_k L + Lambda_k/mu, L)      (Eq. L_prox)
//   3. H = M - L + Y/mu; E = Prox_{psi, lambda/mu}(H) on Omega (0 when
//      noise-free), E = H off Omega                 (Eq. E_prox_ome, E_prox_ome1)
//   4. Y += mu (M - L - E); Lambda_k += mu (nabla_k L - G_k);
//      mu = min(mu_max, vartheta mu)                      (Eq. lagrange11-22)
//   5. the infinity norms of L - L^t, E - E^t, nabla_k L - G_k and G_k - G_k^t
//      (each the maximum over k) and M - L - E               (Eq. convercon)
// The periodic differences are applied on the fly inside fused stencil
// kernels; the linear solve runs through tr_gradient_solve; step 2 through the
// public entry points tr_transform_forward, tr_slice_prox (the randomized
// per-slice engine with the Philox sketches of iteration t) and
// tr_transform_inverse of an internal handle.

#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>

#include "ew_kernels.cuh"
#include "tr_internal.cuh"

struct tr_ctv {
  tr_dtype dtype = TR_F32;
  int order = 0;
  int64_t dims[8] = {0};
  int64_t S[8] = {0};              // flat stride of each mode
  int64_t N = 0;
  int nmodes = 0;
  int modes[8] = {0};              // 1-based modes of Gamma, ascending
  tr_ctv_params prm{};
  cudaStream_t stream = nullptr;
  tr_handle *prox = nullptr;
  size_t esz = 4;
  const void *M = nullptr;         // caller-owned observed values
  const uint8_t *mask = nullptr;   // caller-owned Omega
  void *L = nullptr, *E = nullptr, *Y = nullptr, *G = nullptr, *Lam = nullptr;
  void *R = nullptr, *W = nullptr, *Abar = nullptr, *Gbar = nullptr;
  unsigned long long *res = nullptr;   // device: the five maxima (double bits)
  double mu = 0.0;
  int t = 0;
  char err[256] = {0};
};

namespace {

tr_status cfail(tr_ctv *c, char *buf, size_t len, tr_status st, const char *fmt, ...) {
  char tmp[256];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(tmp, sizeof tmp, fmt, ap);
  va_end(ap);
  if (c) snprintf(c->err, sizeof c->err, "%s", tmp);
  if (buf && len) snprintf(buf, len, "%s", tmp);
  return st;
}

// Prox_{psi,mu}(v) of Eq. equ_gst1 for psi = l1 (kind 0) or MCP (kind 1):
// l1 soft threshold at mu theta; MCP with gamma > mu: 0 up to mu theta,
// (|v| - mu theta)/(1 - mu/gamma) with the sign of v up to gamma theta, v
// beyond; MCP with gamma <= mu: hard threshold at theta sqrt(gamma mu).
template <typename T>
__device__ T prox_scalar(T v, T mu, int kind, T theta, T gamma) {
  const T a = fabs(v);
  const T sgn = v > T(0) ? T(1) : (v < T(0) ? T(-1) : T(0));
  if (kind == 0) return a > mu * theta ? sgn * (a - mu * theta) : T(0);
  if (gamma > mu) {
    if (a > gamma * theta) return v;
    if (a <= mu * theta) return T(0);
    return sgn * (a - mu * theta) / (T(1) - mu / gamma);
  }
  return a > theta * sqrt(gamma * mu) ? v : T(0);
}

// R = M - E + Y/mu
template <typename T>
__global__ void ctv_rhs_kernel(T *R, const T *__restrict__ M, const T *__restrict__ E,
                               const T *__restrict__ Y, T inv_mu, int64_t N) {
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < N; f += step)
    R[f] = M[f] - E[f] + Y[f] * inv_mu;
}

// L = Lnew, with max |Lnew - L| into res[0].
template <typename T>
__global__ void ctv_commit_l_kernel(T *L, const T *__restrict__ Lnew, int64_t N,
                                    unsigned long long *res) {
  double m = 0.0;
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < N; f += step) {
    const T v = Lnew[f];
    m = fmax(m, fabs((double)v - (double)L[f]));
    L[f] = v;
  }
  ew::block_max_to(m, res);
}

// G_k = Gnew and Lambda_k += mu (D - Gnew), D = nabla_k L computed on the
// fly; max |Gnew - G_k| into res[3] and max |D - Gnew| into res[2].
template <typename T>
__global__ void ctv_commit_g_kernel(T *G, T *Lam, const T *__restrict__ Gnew, const T *__restrict__ L,
                                    T mu, int64_t N, int64_t S, int64_t nk, unsigned long long *res) {
  double m2 = 0.0, m3 = 0.0;
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < N; f += step) {
    const T g = Gnew[f], d = L[ew::fwd_neighbour(f, S, nk)] - L[f];
    m3 = fmax(m3, fabs((double)g - (double)G[f]));
    m2 = fmax(m2, fabs((double)d - (double)g));
    G[f] = g;
    Lam[f] += mu * (d - g);
  }
  ew::block_max_to(m2, res + 2);
  ew::block_max_to(m3, res + 3);
}

// Steps 3 and 4 for E and Y, with res[1] = max |E - E^t| and
// res[4] = max |M - L - E|.
template <typename T>
__global__ void ctv_e_kernel(T *E, T *Y, const T *__restrict__ M, const uint8_t *__restrict__ mask,
                             const T *__restrict__ L, T mu, T lam_mu, int noise, int psi,
                             T psi_theta, T psi_gamma, int64_t N, unsigned long long *res) {
  double m1 = 0.0, m4 = 0.0;
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < N; f += step) {
    const T Mf = M[f], Lf = L[f], Yf = Y[f];
    const T H = Mf - Lf + Yf / mu;
    T e = H;
    if (mask[f]) e = noise == 0 ? T(0) : prox_scalar<T>(H, lam_mu, psi, psi_theta, psi_gamma);
    m1 = fmax(m1, fabs((double)e - (double)E[f]));
    const T r = Mf - Lf - e;
    m4 = fmax(m4, fabs((double)r));
    E[f] = e;
    Y[f] = Yf + mu * r;
  }
  ew::block_max_to(m1, res + 1);
  ew::block_max_to(m4, res + 4);
}

void free_ctv(tr_ctv *c) {
  if (c->prox) tr_free(c->prox);
  void *bufs[] = {c->L, c->E, c->Y, c->G, c->Lam, c->R, c->W, c->Abar, c->Gbar, c->res};
  for (void *p : bufs)
    if (p) cudaFree(p);
}

void *slot(const tr_ctv *c, void *base, int i) {
  return (char *)base + (size_t)i * (size_t)c->N * c->esz;
}

template <typename T>
tr_status ctv_step(tr_ctv *c, double *res_out) {
  cudaStream_t s = c->stream;
  const int g = ew::grid(c->N);
  const int64_t N = c->N;
  const double mu = c->mu;
  T *L = (T *)c->L, *E = (T *)c->E, *Y = (T *)c->Y, *R = (T *)c->R, *W = (T *)c->W;
  const T *M = (const T *)c->M;
  char buf[256];
  buf[0] = 0;
#define CV_CUDA(call)                                                                        \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess) return cfail(c, nullptr, 0, TR_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)
#define CV_TR(call)                                                                          \
  do {                                                                                       \
    tr_status st_ = (call);                                                                  \
    if (st_ != TR_OK) return cfail(c, nullptr, 0, st_, "%s: %s", #call, buf[0] ? buf : tr_last_error(c->prox)); \
  } while (0)
  CV_CUDA(cudaMemsetAsync(c->res, 0, 5 * sizeof(unsigned long long), s));
  // 1. L-update: R = (M - E + Y/mu) + sum_k nabla_k^T (G_k - Lambda_k/mu)
  ctv_rhs_kernel<T><<<g, 256, 0, s>>>(R, M, E, Y, (T)(1.0 / mu), N);
  CV_CUDA(cudaGetLastError());
  uint32_t bits = 0;
  for (int q = 0; q < c->nmodes; ++q) {
    const int k = c->modes[q];
    bits |= 1u << (k - 1);
    const T *Gk = (const T *)slot(c, c->G, q), *Lk = (const T *)slot(c, c->Lam, q);
    ew::adj_grad_accum_kernel<T><<<g, 256, 0, s>>>(R, Gk, Lk, (T)(1.0 / mu), N, c->S[k - 1],
                                                  c->dims[k - 1]);
    CV_CUDA(cudaGetLastError());
  }
  CV_TR(tr_gradient_solve(c->dtype, c->order, c->dims, bits, R, W, s, buf, sizeof buf));
  ctv_commit_l_kernel<T><<<g, 256, 0, s>>>(L, W, N, c->res);
  CV_CUDA(cudaGetLastError());
  // 2. G-updates, tau = 1/(gamma mu); 4. their multipliers
  const double tau = 1.0 / ((double)c->nmodes * mu);
  for (int q = 0; q < c->nmodes; ++q) {
    const int k = c->modes[q];
    T *Gk = (T *)slot(c, c->G, q), *Lk = (T *)slot(c, c->Lam, q);
    const int64_t S = c->S[k - 1], nk = c->dims[k - 1];
    ew::grad_plus_kernel<T><<<g, 256, 0, s>>>(R, L, Lk, (T)(1.0 / mu), N, S, nk);   // nabla_k L + Lambda_k/mu
    CV_CUDA(cudaGetLastError());
    CV_TR(tr_transform_forward(c->prox, R, c->Abar));
    CV_TR(tr_slice_prox(c->prox, c->Abar, c->Gbar, tau, c->t));
    CV_TR(tr_transform_inverse(c->prox, c->Gbar, R));                             // R = G_k new
    ctv_commit_g_kernel<T><<<g, 256, 0, s>>>(Gk, Lk, R, L, (T)mu, N, S, nk, c->res);
    CV_CUDA(cudaGetLastError());
  }
  // 3. E-update and 4. Y-update
  const tr_ctv_params &p = c->prm;
  ctv_e_kernel<T><<<g, 256, 0, s>>>(E, Y, M, c->mask, L, (T)mu, (T)(p.lambda / mu),
                                    p.noise == TR_NOISE_NONE ? 0 : 1, p.psi == TR_PEN_L1 ? 0 : 1,
                                    (T)p.psi_theta, (T)p.psi_gamma, N, c->res);
  CV_CUDA(cudaGetLastError());
#undef CV_CUDA
#undef CV_TR
  c->mu = fmin(p.mu_max, p.growth * mu);
  c->t += 1;
  if (res_out) {
    unsigned long long h[5];
    cudaError_t e = cudaMemcpyAsync(h, c->res, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cfail(c, nullptr, 0, TR_ECUDA, "%s", cudaGetErrorString(e));
    for (int i = 0; i < 5; ++i) {
      double v;
      memcpy(&v, &h[i], sizeof v);
      res_out[i] = v;
    }
  }
  return TR_OK;
}

}  // namespace

extern "C" void tr_ctv_default_params(tr_ctv_params *p) {
  if (!p) return;
  memset(p, 0, sizeof *p);
  p->modes = 0b11;
  p->phi = TR_PEN_MCP;
  p->phi_theta = 1.0;
  p->phi_gamma = 4000.0;
  p->psi = TR_PEN_MCP;
  p->psi_theta = 1.0;
  p->psi_gamma = 4000.0;
  p->noise = TR_NOISE_L1;
  p->lambda = 0.0;
  p->mu0 = 1e-3;
  p->mu_max = 1e10;
  p->growth = 1.1;
  p->rank = 10;
  p->oversample = 10;
  p->power_iters = 1;
  p->seed = 0;
  p->prec = TR_PREC_FP32;
}

extern "C" tr_status tr_ctv_create(tr_ctv **out, const tr_problem *pb, const tr_ctv_params *prm,
                                   void *cuda_stream, char *err, size_t err_len) {
  if (err && err_len) err[0] = 0;
  if (!out || !pb || !prm) return cfail(nullptr, err, err_len, TR_EINVAL, "null pointer");
  *out = nullptr;
  if (pb->dtype != TR_F32 && pb->dtype != TR_F64)
    return cfail(nullptr, err, err_len, TR_EINVAL, "bad dtype");
  if (pb->order < 3 || pb->order > 8)
    return cfail(nullptr, err, err_len, TR_EINVAL, "order must be 3..8");
  if (!pb->observed || !pb->mask)
    return cfail(nullptr, err, err_len, TR_EINVAL, "observed and mask are required");
  if (prm->modes == 0 || (prm->modes >> pb->order))
    return cfail(nullptr, err, err_len, TR_EINVAL, "Gamma must name at least one mode of the tensor");
  if (!(prm->mu0 > 0) || !(prm->growth >= 1.0) || !(prm->mu_max >= prm->mu0) || prm->lambda < 0)
    return cfail(nullptr, err, err_len, TR_EINVAL, "need mu0 > 0, growth >= 1, mu_max >= mu0, lambda >= 0");
  if ((prm->phi != TR_PEN_L1 && prm->phi != TR_PEN_MCP) || (prm->psi != TR_PEN_L1 && prm->psi != TR_PEN_MCP) ||
      (prm->noise != TR_NOISE_NONE && prm->noise != TR_NOISE_L1))
    return cfail(nullptr, err, err_len, TR_EINVAL, "bad penalty or noise model");
  tr_ctv *c = new (std::nothrow) tr_ctv();
  if (!c) return cfail(nullptr, err, err_len, TR_ENOMEM, "host allocation failed");
  c->dtype = pb->dtype;
  c->order = pb->order;
  c->N = 1;
  for (int k = 0; k < pb->order; ++k) {
    if (pb->dims[k] < 1) {
      delete c;
      return cfail(nullptr, err, err_len, TR_EINVAL, "empty mode");
    }
    c->dims[k] = pb->dims[k];
    c->N *= pb->dims[k];
  }
  for (int k = 1; k <= pb->order; ++k) {
    c->S[k - 1] = ew::mode_stride(c->dims, k);
    if (prm->modes & (1u << (k - 1))) c->modes[c->nmodes++] = k;
  }
  c->prm = *prm;
  if (c->prm.lambda <= 0.0) {   // lambda = 1/sqrt(max(n1, n2)), as tr_init's default
    const double mx = (double)(c->dims[0] > c->dims[1] ? c->dims[0] : c->dims[1]);
    c->prm.lambda = 1.0 / sqrt(mx);
  }
  c->stream = (cudaStream_t)cuda_stream;
  c->esz = pb->dtype == TR_F64 ? 8 : 4;
  c->mu = prm->mu0;
  c->M = pb->observed;
  c->mask = pb->mask;
  // the internal handle: transform and randomized per-slice prox of step 2
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
  tr_status st = tr_init(&c->prox, pb, &hp, cuda_stream);
  if (st != TR_OK) {
    const tr_status r = cfail(nullptr, err, err_len, st, "prox handle: %s", tr_last_error(nullptr));
    c->prox = nullptr;
    delete c;
    return r;
  }
  const size_t T = (size_t)c->N * c->esz;
  cudaError_t e = cudaSuccess;
  void **single[] = {&c->L, &c->E, &c->Y, &c->R, &c->W, &c->Abar, &c->Gbar};
  for (void **p : single)
    if (e == cudaSuccess) e = cudaMalloc(p, T);
  if (e == cudaSuccess) e = cudaMalloc(&c->G, T * c->nmodes);
  if (e == cudaSuccess) e = cudaMalloc(&c->Lam, T * c->nmodes);
  if (e == cudaSuccess) e = cudaMalloc((void **)&c->res, 5 * sizeof(unsigned long long));
  // Alg. 5 initialisation: L = E = Y = G_k = Lambda_k = 0
  void *zero[] = {c->L, c->E, c->Y};
  for (void *p : zero)
    if (e == cudaSuccess) e = cudaMemsetAsync(p, 0, T, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->G, 0, T * c->nmodes, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->Lam, 0, T * c->nmodes, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    free_ctv(c);
    delete c;
    return cfail(nullptr, err, err_len, e == cudaErrorMemoryAllocation ? TR_ENOMEM : TR_ECUDA,
                 "workspace: %s", cudaGetErrorString(e));
  }
  *out = c;
  return TR_OK;
}

extern "C" tr_status tr_ctv_step(tr_ctv *c, double *res_inf) {
  if (!c) return TR_EINVAL;
  return c->dtype == TR_F32 ? ctv_step<float>(c, res_inf) : ctv_step<double>(c, res_inf);
}

extern "C" tr_status tr_ctv_get_state(tr_ctv *c, void *L, void *E, void *Y, void *G, void *Lam,
                                      double *mu, int *t) {
  if (!c) return TR_EINVAL;
  const size_t T = (size_t)c->N * c->esz;
  const void *src[] = {c->L, c->E, c->Y, c->G, c->Lam};
  void *dst[] = {L, E, Y, G, Lam};
  const size_t bytes[] = {T, T, T, T * c->nmodes, T * c->nmodes};
  for (int i = 0; i < 5; ++i) {
    if (!dst[i]) continue;
    const cudaError_t e = cudaMemcpyAsync(dst[i], src[i], bytes[i], cudaMemcpyDeviceToDevice, c->stream);
    if (e != cudaSuccess) return cfail(c, nullptr, 0, TR_ECUDA, "%s", cudaGetErrorString(e));
  }
  if (mu) *mu = c->mu;
  if (t) *t = c->t;
  const cudaError_t e = cudaStreamSynchronize(c->stream);
  return e == cudaSuccess ? TR_OK : cfail(c, nullptr, 0, TR_ECUDA, "%s", cudaGetErrorString(e));
}

extern "C" tr_status tr_ctv_set_state(tr_ctv *c, const void *L, const void *E, const void *Y,
                                      const void *G, const void *Lam, double mu, int t) {
  if (!c || !(mu > 0) || t < 0) return TR_EINVAL;
  const size_t T = (size_t)c->N * c->esz;
  const void *src[] = {L, E, Y, G, Lam};
  void *dst[] = {c->L, c->E, c->Y, c->G, c->Lam};
  const size_t bytes[] = {T, T, T, T * c->nmodes, T * c->nmodes};
  for (int i = 0; i < 5; ++i) {
    if (!src[i]) continue;
    const cudaError_t e = cudaMemcpyAsync(dst[i], src[i], bytes[i], cudaMemcpyDeviceToDevice, c->stream);
    if (e != cudaSuccess) return cfail(c, nullptr, 0, TR_ECUDA, "%s", cudaGetErrorString(e));
  }
  c->mu = mu;
  c->t = t;
  const cudaError_t e = cudaStreamSynchronize(c->stream);
  return e == cudaSuccess ? TR_OK : cfail(c, nullptr, 0, TR_ECUDA, "%s", cudaGetErrorString(e));
}

extern "C" const char *tr_ctv_last_error(const tr_ctv *c) { return c ? c->err : ""; }

extern "C" tr_status tr_ctv_free(tr_ctv *c) {
  if (!c) return TR_OK;
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  free_ctv(c);
  delete c;
  return TR_OK;
}
