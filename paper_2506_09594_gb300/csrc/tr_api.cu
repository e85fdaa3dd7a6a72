// C ABI of libtr (include/tr.h): handle life cycle, one ADMM iteration of
// Alg. 5 (pure-L form) as a sequence of launches on the caller's stream,
// the recovery loop, and state import/export.

#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <vector>

#include "tr_internal.cuh"

struct tr_handle {
  // problem
  int order = 0;
  int64_t n1 = 0, n2 = 0, n = 0, P = 0, N = 0;
  tr_dtype dtype = TR_F32;
  size_t esz = 4;
  const void *M = nullptr;
  const uint8_t *mask = nullptr;
  tr_params prm{};
  cudaStream_t stream = nullptr;
  TransformDesc td{};
  // device buffers
  void *mats = nullptr;                       // transform matrices
  void *L = nullptr, *E = nullptr, *Y = nullptr, *Lam = nullptr, *G = nullptr;
  void *Abar = nullptr, *Gbar = nullptr;      // transform-domain scratch
  SliceWork sw{};
  AdaptWork aw{};                             // fixed-accuracy engine workspace
  LearnedWork lw{};                           // learned-width engine state
  int *width = nullptr;                       // sketch width per slice, last pass
  bool have_pass = false;                     // a slice pass has run
  double thr_last = 0.0;                      // its shrink threshold
  unsigned long long *res = nullptr;          // RES_COUNT slots
  unsigned long long *res_prev = nullptr;     // slots for a deferred inverse pass
  int *flags = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // instrumentation
  std::vector<cudaEvent_t> prof_ev;   // 4 per profiled step
  int prof_cap = 0, prof_used = 0;
  uint64_t launches = 0;
  // host state
  double mu = 0.0;
  int t = 0;
  // The inverse pass of the last step is deferred and fused into the next
  // step's forward pass when `pending` is set (steps taken without info).
  bool pending = false;
  double mu_prev = 0.0;
  bool poisoned = false;
  char err[512] = {0};
};

static char g_init_err[512] = {0};

static tr_status fail(tr_handle *h, tr_status st, const char *fmt, ...) {
  char *buf = h ? h->err : g_init_err;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, 512, fmt, ap);
  va_end(ap);
  return st;
}

#define TR_CUDA(h, call)                                                                   \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return fail((h), e_ == cudaErrorMemoryAllocation ? TR_ENOMEM : TR_ECUDA, "%s: %s (%s:%d)", \
                  #call, cudaGetErrorString(e_), __FILE__, __LINE__);                      \
  } while (0)

extern "C" void tr_default_params(tr_params *p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
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
  p->tol = 1e-4;
  p->max_iter = 100;
  p->engine = TR_LR_RSVD;
  p->rank = 10;
  p->oversample = 10;
  p->power_iters = 1;
  p->adapt_eps = 0.01;
  p->adapt_block = 10;
  p->prec = TR_PREC_FP32;
  p->seed = 0;
  p->model_path = nullptr;
}

// Orthonormal DCT-II: U[k][m] = s_k cos(pi (2m+1) k / (2n)), s_0 = sqrt(1/n),
// s_k = sqrt(2/n); U U^T = I, so U^{-1} = U^T (Eq. orth with alpha = 1).
static void dct2_matrix(int n, std::vector<double> &U) {
  U.assign((size_t)n * n, 0.0);
  const double pi = 3.14159265358979323846;
  for (int k = 0; k < n; ++k) {
    const double s = k == 0 ? sqrt(1.0 / n) : sqrt(2.0 / n);
    for (int m = 0; m < n; ++m) U[(size_t)k * n + m] = s * cos(pi * (2.0 * m + 1.0) * k / (2.0 * n));
  }
}

static void free_profile(tr_handle *h) {
  for (cudaEvent_t e : h->prof_ev) cudaEventDestroy(e);
  h->prof_ev.clear();
  h->prof_cap = h->prof_used = 0;
}

static void free_all(tr_handle *h) {
  free_profile(h);
  LearnedWork &lw = h->lw;
  void *lbufs[] = {lw.params, lw.feat, lw.pred, lw.ids, lw.counts, lw.fb_ids, lw.fb_count};
  for (void *b : lbufs)
    if (b) cudaFree(b);
  if (lw.h_counts) cudaFreeHost(lw.h_counts);
  for (int i = 0; i < TR_LEARNED_STREAMS; ++i) {
    if (lw.aux[i]) cudaStreamDestroy(lw.aux[i]);
    if (lw.join[i]) cudaEventDestroy(lw.join[i]);
  }
  if (lw.fork) cudaEventDestroy(lw.fork);
  if (h->width) cudaFree(h->width);
  void *bufs[] = {h->mats, h->L, h->E, h->Y, h->Lam, h->G, h->Abar, h->Gbar,
                  h->sw.Om, h->sw.P1, h->sw.P2, h->sw.sig, h->sw.rank, h->sw.err,
                  h->aw.Ucat, h->aw.Vcat, h->aw.X, h->aw.Lm, h->aw.Rm, h->aw.E, h->aw.nrm2,
                  h->aw.active, h->aw.kept, h->aw.draws, h->res,
                  h->res_prev, h->flags};
  for (void *b : bufs)
    if (b) cudaFree(b);
  if (h->ev0) cudaEventDestroy(h->ev0);
  if (h->ev1) cudaEventDestroy(h->ev1);
}

// Weights file: "TRRANK01", int32 16, 128, 3, 0, int64 count, count float32.
static bool read_model(const char *path, std::vector<float> &w, char *err, size_t errlen) {
  FILE *f = fopen(path, "rb");
  if (!f) {
    snprintf(err, errlen, "cannot open model file %s", path);
    return false;
  }
  char magic[8];
  int32_t dims[4];
  int64_t count = 0;
  bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, "TRRANK01", 8) == 0 &&
            fread(dims, 4, 4, f) == 4 && dims[0] == TR_MLP_IN && dims[1] == TR_MLP_HIDDEN &&
            dims[2] == TR_MLP_LAYERS && fread(&count, 8, 1, f) == 1 && count == mlp_param_count();
  if (ok) {
    w.resize((size_t)count);
    ok = fread(w.data(), 4, (size_t)count, f) == (size_t)count;
  }
  fclose(f);
  if (!ok) snprintf(err, errlen, "model file %s: bad header or size", path);
  return ok;
}

// Smallest singular value the shrink keeps nonzero: tau theta (l1, and MCP
// with gamma > tau), theta sqrt(gamma tau) (MCP hard-threshold regime).
static double shrink_threshold(const tr_params &p, double tau) {
  if (p.phi == TR_PEN_L1 || p.phi_gamma > tau) return tau * p.phi_theta;
  return p.phi_theta * sqrt(p.phi_gamma * tau);
}

static int sketch_width(const tr_handle *h) {
  int64_t l = (int64_t)h->prm.rank + h->prm.oversample;
  if (l > h->n1) l = h->n1;
  if (l > h->n2) l = h->n2;
  if (l < 1) l = 1;
  return (int)l;
}

extern "C" tr_status tr_init(tr_handle **out, const tr_problem *p, const tr_params *prm,
                             void *cuda_stream) {
  if (!out || !p || !prm) return fail(nullptr, TR_EINVAL, "tr_init: NULL argument");
  *out = nullptr;
  if (p->order < 2 || p->order > 8) return fail(nullptr, TR_EINVAL, "order %d not in [2, 8]", p->order);
  if (p->order - 2 > TR_MAX_TMODES)
    return fail(nullptr, TR_EUNSUPPORTED, "at most %d transformed modes", TR_MAX_TMODES);
  if (p->dtype != TR_F32 && p->dtype != TR_F64) return fail(nullptr, TR_EINVAL, "bad dtype");
  if (!p->observed || !p->mask) return fail(nullptr, TR_EINVAL, "observed/mask must be device pointers");
  for (int i = 0; i < p->order; ++i)
    if (p->dims[i] < 1) return fail(nullptr, TR_EINVAL, "dims[%d] = %lld < 1", i, (long long)p->dims[i]);
  if (prm->engine != TR_LR_RSVD && prm->engine != TR_LR_ADAPTIVE && prm->engine != TR_LR_LEARNED)
    return fail(nullptr, TR_EUNSUPPORTED, "engine %d not built", (int)prm->engine);
  if (prm->engine == TR_LR_ADAPTIVE &&
      (prm->adapt_block < 1 || prm->adapt_block > 32 || !(prm->adapt_eps > 0)))
    return fail(nullptr, TR_EINVAL, "adaptive engine: need 1 <= adapt_block <= 32, adapt_eps > 0");
  if (prm->prec != TR_PREC_FP32 && prm->prec != TR_PREC_BF16 && prm->prec != TR_PREC_BF16X3)
    return fail(nullptr, TR_EUNSUPPORTED, "precision %d not built", (int)prm->prec);
  if (prm->prec != TR_PREC_FP32 && p->dtype != TR_F32)
    return fail(nullptr, TR_EUNSUPPORTED, "tensor-core precisions need an FP32 problem");
  if (!(prm->mu0 > 0) || !(prm->growth >= 1.0) || !(prm->mu_max >= prm->mu0))
    return fail(nullptr, TR_EINVAL, "need mu0 > 0, growth >= 1, mu_max >= mu0");
  if (prm->power_iters < 0 || prm->rank < 0 || prm->oversample < 0)
    return fail(nullptr, TR_EINVAL, "negative rank/oversample/power_iters");

  tr_handle *h = new (std::nothrow) tr_handle();
  if (!h) return fail(nullptr, TR_ENOMEM, "host allocation failed");
  h->order = p->order;
  h->n1 = p->dims[0];
  h->n2 = p->dims[1];
  h->n = 1;
  for (int i = 2; i < p->order; ++i) h->n *= p->dims[i];
  h->P = h->n1 * h->n2;
  h->N = h->P * h->n;
  h->dtype = p->dtype;
  h->esz = p->dtype == TR_F64 ? 8 : 4;
  h->M = p->observed;
  h->mask = p->mask;
  h->prm = *prm;
  h->stream = (cudaStream_t)cuda_stream;
  if (h->prm.lambda <= 0.0) {
    const double mx = (double)(h->n1 > h->n2 ? h->n1 : h->n2);
    // Sec. 6 sets xi / sqrt(max(n1,n2) n3..nd) for the FFT (rho = n3..nd); with
    // the orthonormal DCT (rho = 1) the same balance is xi / sqrt(max(n1,n2)).
    h->prm.lambda = 1.0 / sqrt(mx);
  }
  if (h->n1 > 65535 * 64LL || h->n > 65535) {
    tr_status st = fail(nullptr, TR_EUNSUPPORTED, "too many slices (%lld) for one launch", (long long)h->n);
    delete h;
    return st;
  }

  // transform description and matrices
  TransformDesc &td = h->td;
  td.nt = p->order - 2;
  int maxd = 1;
  for (int k = 0; k < td.nt; ++k) {
    td.dim[k] = (int)p->dims[k + 2];
    if (td.dim[k] > maxd) maxd = td.dim[k];
  }
  if (maxd > TR_MAX_NK) {
    tr_status st = fail(nullptr, TR_EUNSUPPORTED, "transformed mode of size %d > %d", maxd, TR_MAX_NK);
    delete h;
    return st;
  }
  td.nkpad = ((maxd + 7) / 8) * 8;
  int stride = 1, off = 0;
  for (int k = 0; k < td.nt; ++k) {
    td.stride[k] = stride;
    stride *= td.dim[k];
    td.off_fwd[k] = off;
    off += td.dim[k] * td.nkpad;
    td.off_inv[k] = off;
    off += td.dim[k] * td.nkpad;
  }
  td.mats_len = ((off + 3) / 4) * 4;
  if (td.mats_len == 0) td.mats_len = 4;
  int tp = 0;
  if (tube_smem_bytes(h->dtype, (int)h->n, td, &tp) == 0 || tp == 0) {
    tr_status st = fail(nullptr, TR_EUNSUPPORTED, "%lld slices do not fit a tube tile", (long long)h->n);
    delete h;
    return st;
  }
  int l = sketch_width(h);
  if (prm->engine == TR_LR_ADAPTIVE) {
    // basis cap: rank + oversample rounded up to whole blocks, within min(n1, n2)
    const int b = prm->adapt_block;
    const int mn = (int)(h->n1 < h->n2 ? h->n1 : h->n2);
    int kcap = ((prm->rank + prm->oversample + b - 1) / b) * b;
    if (kcap > (mn / b) * b) kcap = (mn / b) * b;
    if (kcap < b || adapt_smem_bytes(h->dtype, (int)h->n1, (int)h->n2, b, kcap) > 227 * 1024) {
      tr_status st = fail(nullptr, TR_EUNSUPPORTED, "adaptive engine: block %d does not fit", b);
      delete h;
      return st;
    }
    l = kcap;
    h->aw.b = b;
    h->aw.kcap = kcap;
    h->aw.eps = prm->adapt_eps;
    h->aw.delta_rel = p->dtype == TR_F64 ? 1e-11 : 1e-5;
  }
  if (l > TR_MAX_L || !slice_smem_limit_ok(h->dtype, (int)h->n1, (int)h->n2, l)) {
    tr_status st = fail(nullptr, TR_EUNSUPPORTED, "slice panels %lld x %d exceed shared memory",
                        (long long)(h->n1 > h->n2 ? h->n1 : h->n2), l);
    delete h;
    return st;
  }

  std::vector<double> hm((size_t)td.mats_len, 0.0), U;
  for (int k = 0; k < td.nt; ++k) {
    const int d = td.dim[k];
    dct2_matrix(d, U);
    for (int i = 0; i < d; ++i)
      for (int m = 0; m < d; ++m) {
        hm[(size_t)td.off_fwd[k] + (size_t)i * td.nkpad + m] = U[(size_t)i * d + m];
        hm[(size_t)td.off_inv[k] + (size_t)i * td.nkpad + m] = U[(size_t)m * d + i];
      }
  }

  const size_t bytes = (size_t)h->N * h->esz;
  auto cleanup = [&](tr_status st) {
    free_all(h);
    snprintf(g_init_err, sizeof g_init_err, "%s", h->err);
    delete h;
    return st;
  };
#define INIT_CUDA(call)                                                                \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) {                                                           \
      fail(h, e_ == cudaErrorMemoryAllocation ? TR_ENOMEM : TR_ECUDA, "%s: %s", #call, \
           cudaGetErrorString(e_));                                                    \
      return cleanup(e_ == cudaErrorMemoryAllocation ? TR_ENOMEM : TR_ECUDA);          \
    }                                                                                  \
  } while (0)

  INIT_CUDA(cudaMalloc(&h->mats, (size_t)td.mats_len * h->esz));
  if (h->dtype == TR_F64) {
    INIT_CUDA(cudaMemcpy(h->mats, hm.data(), hm.size() * 8, cudaMemcpyHostToDevice));
  } else {
    std::vector<float> hf(hm.begin(), hm.end());
    INIT_CUDA(cudaMemcpy(h->mats, hf.data(), hf.size() * 4, cudaMemcpyHostToDevice));
  }
  void **state[] = {&h->L, &h->E, &h->Y, &h->Lam, &h->G, &h->Abar, &h->Gbar};
  for (void **b : state) INIT_CUDA(cudaMalloc(b, bytes));
  for (int i = 0; i < 5; ++i) INIT_CUDA(cudaMemsetAsync(*state[i], 0, bytes, h->stream));

  SliceWork &sw = h->sw;
  sw.n = (int)h->n;
  sw.n1 = (int)h->n1;
  sw.n2 = (int)h->n2;
  sw.l = l;
  sw.q = prm->power_iters;
  sw.seed = prm->seed;
  // the learned engine packs width groups into the panels, each group's
  // region rounded up to 64 elements
  const size_t slack = prm->engine == TR_LR_LEARNED ? (size_t)64 * plan_classes(l) : 0;
  INIT_CUDA(cudaMalloc(&sw.Om, ((size_t)h->n * h->n2 * l + slack) * h->esz));
  INIT_CUDA(cudaMalloc(&sw.P1, ((size_t)h->n * h->n1 * l + slack) * h->esz));
  INIT_CUDA(cudaMalloc(&sw.P2, ((size_t)h->n * h->n2 * l + slack) * h->esz));
  INIT_CUDA(cudaMalloc((void **)&h->width, (size_t)h->n * sizeof(int)));
  sw.width = h->width;
  sw.ldsig = l;
  INIT_CUDA(cudaMalloc(&sw.sig, (size_t)h->n * l * h->esz));
  INIT_CUDA(cudaMalloc((void **)&sw.rank, (size_t)h->n * sizeof(int)));
  INIT_CUDA(cudaMalloc((void **)&h->res, RES_COUNT * sizeof(unsigned long long)));
  INIT_CUDA(cudaMalloc((void **)&h->res_prev, RES_COUNT * sizeof(unsigned long long)));
  INIT_CUDA(cudaMalloc((void **)&h->flags, sizeof(int)));
  INIT_CUDA(cudaMalloc((void **)&sw.err, sizeof(int)));
  INIT_CUDA(cudaMemsetAsync(sw.err, 0, sizeof(int), h->stream));
  sw.prec = (int)prm->prec;
  INIT_CUDA(cudaMemsetAsync(sw.rank, 0, (size_t)h->n * sizeof(int), h->stream));
  if (prm->engine == TR_LR_ADAPTIVE) {
    AdaptWork &aw = h->aw;
    const size_t mx = (size_t)(h->n1 > h->n2 ? h->n1 : h->n2);
    INIT_CUDA(cudaMalloc(&aw.Ucat, (size_t)h->n * h->n1 * aw.kcap * h->esz));
    INIT_CUDA(cudaMalloc(&aw.Vcat, (size_t)h->n * h->n2 * (aw.kcap + aw.b) * h->esz));
    INIT_CUDA(cudaMalloc(&aw.X, (size_t)h->n * mx * aw.b * h->esz));
    INIT_CUDA(cudaMalloc(&aw.Lm, (size_t)h->n * aw.b * aw.b * h->esz));
    INIT_CUDA(cudaMalloc(&aw.Rm, (size_t)h->n * aw.b * aw.b * h->esz));
    INIT_CUDA(cudaMalloc((void **)&aw.E, (size_t)h->n * sizeof(double)));
    INIT_CUDA(cudaMalloc((void **)&aw.nrm2, (size_t)h->n * sizeof(double)));
    INIT_CUDA(cudaMalloc((void **)&aw.active, (size_t)h->n * sizeof(int)));
    INIT_CUDA(cudaMalloc((void **)&aw.kept, (size_t)h->n * sizeof(int)));
    INIT_CUDA(cudaMalloc((void **)&aw.draws, (size_t)h->n * sizeof(int)));
  }
  if (prm->engine == TR_LR_LEARNED) {
    LearnedWork &lw = h->lw;
    lw.lmax = l;
    lw.p = prm->oversample;
    const int C = plan_classes(l);
    INIT_CUDA(cudaMalloc((void **)&lw.params, (size_t)mlp_param_count() * sizeof(float)));
    INIT_CUDA(cudaMalloc((void **)&lw.feat, (size_t)h->n * TR_MLP_IN * sizeof(float)));
    INIT_CUDA(cudaMalloc((void **)&lw.pred, (size_t)h->n * sizeof(float)));
    INIT_CUDA(cudaMalloc((void **)&lw.ids, (size_t)h->n * sizeof(int)));
    INIT_CUDA(cudaMalloc((void **)&lw.counts, (size_t)C * sizeof(int)));
    INIT_CUDA(cudaMalloc((void **)&lw.fb_ids, (size_t)h->n * sizeof(int)));
    INIT_CUDA(cudaMalloc((void **)&lw.fb_count, sizeof(int)));
    INIT_CUDA(cudaMallocHost((void **)&lw.h_counts, ((TR_MAX_L + 7) / 8 + 1) * sizeof(int)));
    lw.width = h->width;
    for (int i = 0; i < TR_LEARNED_STREAMS; ++i) {
      INIT_CUDA(cudaStreamCreateWithFlags(&lw.aux[i], cudaStreamNonBlocking));
      INIT_CUDA(cudaEventCreateWithFlags(&lw.join[i], cudaEventDisableTiming));
    }
    INIT_CUDA(cudaEventCreateWithFlags(&lw.fork, cudaEventDisableTiming));
    if (prm->model_path) {
      std::vector<float> w;
      if (!read_model(prm->model_path, w, h->err, sizeof h->err))
        return cleanup(TR_EINVAL);
      INIT_CUDA(cudaMemcpy(lw.params, w.data(), w.size() * sizeof(float), cudaMemcpyHostToDevice));
    } else {
      INIT_CUDA(launch_mlp_init(lw.params, prm->seed, h->stream));
    }
  }
  INIT_CUDA(cudaEventCreate(&h->ev0));
  INIT_CUDA(cudaEventCreate(&h->ev1));
  INIT_CUDA(cudaStreamSynchronize(h->stream));
#undef INIT_CUDA
  h->mu = prm->mu0;
  h->t = 0;
  *out = h;
  return TR_OK;
}

static tr_status slice_pass(tr_handle *h, const void *Abar, void *Gbar, double tau, int t) {
  ShrinkScalars sh{tau, (int)h->prm.phi, h->prm.phi_theta, h->prm.phi_gamma};
  const double thr = shrink_threshold(h->prm, tau);
  if (h->prm.engine == TR_LR_ADAPTIVE) {
    TR_CUDA(h, launch_slice_adaptive(h->dtype, h->sw, h->aw, Abar, Gbar, sh, t, h->stream));
    const uint64_t nblk = (uint64_t)(h->aw.kcap / h->aw.b);
    h->launches += 1 + 4 * nblk - 2 + 3;   // init, per block GEMM+U (+GEMM+V), B GEMM, SVD, rebuild
    // the width of an adaptive slice is its basis size
    TR_CUDA(h, cudaMemcpyAsync(h->width, h->aw.kept, (size_t)h->n * sizeof(int),
                               cudaMemcpyDeviceToDevice, h->stream));
  } else if (h->prm.engine == TR_LR_LEARNED) {
    cudaError_t e = launch_slice_learned(h->dtype, h->sw, h->lw, Abar, Gbar, sh, thr, t,
                                         h->prm.max_iter, h->stream, &h->launches);
    if (e != cudaSuccess)
      return fail(h, TR_ECUDA, "learned slice pass: %s", cudaGetErrorString(e));
  } else {
    TR_CUDA(h, launch_slice_rsvd(h->dtype, h->sw, Abar, Gbar, sh, t, h->stream));
    h->launches += 7 + 4 * (uint64_t)h->sw.q;   // sketch, 2 + 2q GEMM, 1 + 2q QR, SVD core, rebuild
  }
  h->have_pass = true;
  h->thr_last = thr;
  return TR_OK;
}

static tr_status read_info(tr_handle *h, double mu_used, tr_step_info *info) {
  unsigned long long r[RES_COUNT];
  int flag = 0;
  TR_CUDA(h, cudaMemcpyAsync(r, h->res, sizeof r, cudaMemcpyDeviceToHost, h->stream));
  TR_CUDA(h, cudaMemcpyAsync(&flag, h->flags, sizeof flag, cudaMemcpyDeviceToHost, h->stream));
  std::vector<int> ranks((size_t)h->n);
  TR_CUDA(h, cudaMemcpyAsync(ranks.data(), h->sw.rank, ranks.size() * sizeof(int),
                             cudaMemcpyDeviceToHost, h->stream));
  TR_CUDA(h, cudaStreamSynchronize(h->stream));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, h->ev0, h->ev1);
  info->iter = h->t;
  info->mu = mu_used;
  info->tau = 1.0 / mu_used;
  for (int i = 0; i < RES_COUNT; ++i) {
    double v;
    memcpy(&v, &r[i], sizeof v);
    info->res_inf[i] = v;
  }
  int mx = 0;
  long long sum = 0;
  for (int v : ranks) {
    mx = v > mx ? v : mx;
    sum += v;
  }
  info->max_rank = mx;
  info->sum_rank = (int)sum;
  info->fallback_slices = h->prm.engine == TR_LR_LEARNED ? h->lw.last_fallback : 0;
  info->ms = ms;
  int tc_err = 0;
  TR_CUDA(h, cudaMemcpy(&tc_err, h->sw.err, sizeof tc_err, cudaMemcpyDeviceToHost));
  if (tc_err) {
    h->poisoned = true;
    return fail(h, TR_ETIMEOUT, "a tensor-core GEMM gave up waiting for its MMAs");
  }
  if (flag) {
    h->poisoned = true;
    return fail(h, TR_ENUMERIC, "NaN or Inf in the iterate at iteration %d", h->t);
  }
  return TR_OK;
}

// Run the deferred inverse pass (G = L^{-1}(Gbar), Lambda update) of the
// last step, so that the handle's state is the complete iterate.
static tr_status finalize(tr_handle *h) {
  if (!h->pending) return TR_OK;
  cudaError_t e = launch_tube_inverse(h->dtype, h->P, (int)h->n, h->td, h->mats, h->Gbar, h->L,
                                      h->G, h->Lam, h->mu_prev, h->res_prev, h->flags, h->stream);
  if (e != cudaSuccess) {
    h->poisoned = true;
    return fail(h, TR_ECUDA, "tube inverse: %s", cudaGetErrorString(e));
  }
  h->launches += 1;
  h->pending = false;
  return TR_OK;
}

extern "C" tr_status tr_prox_step(tr_handle *h, tr_step_info *info) {
  if (!h) return TR_EINVAL;
  if (h->poisoned) return fail(h, TR_EINVAL, "handle poisoned by an earlier failure; call tr_set_state");
  const double mu = h->mu;
  TubeScalars sc{mu, h->prm.lambda / mu, (int)h->prm.noise, (int)h->prm.psi, h->prm.psi_theta,
                 h->prm.psi_gamma};
  auto guard = [&](tr_status st) {
    if (st != TR_OK) h->poisoned = true;
    return st;
  };
  if (info) TR_CUDA(h, cudaEventRecord(h->ev0, h->stream));
  cudaEvent_t *pev = nullptr;
  if (h->prof_used < h->prof_cap) pev = &h->prof_ev[(size_t)4 * h->prof_used++];
  cudaError_t e = cudaMemsetAsync(h->res, 0, RES_COUNT * sizeof(unsigned long long), h->stream);
  if (e == cudaSuccess && pev) e = cudaEventRecord(pev[0], h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->flags, 0, sizeof(int), h->stream);
  if (e == cudaSuccess) {
    if (h->pending)
      e = launch_tube_fused(h->dtype, h->P, (int)h->n, h->td, h->mats, h->Gbar, h->mu_prev, h->M,
                            h->mask, h->L, h->E, h->Y, h->G, h->Lam, h->Abar, sc, h->res_prev,
                            h->res, h->flags, h->stream);
    else
      e = launch_tube_forward(h->dtype, h->P, (int)h->n, h->td, h->mats, h->M, h->mask, h->L,
                              h->E, h->Y, h->G, h->Lam, h->Abar, sc, h->res, h->flags, h->stream);
  }
  h->pending = false;
  if (e == cudaSuccess && pev) e = cudaEventRecord(pev[1], h->stream);
  if (e != cudaSuccess)
    return guard(fail(h, TR_ECUDA, "tube forward: %s", cudaGetErrorString(e)));
  h->launches += 1;
  tr_status st = slice_pass(h, h->Abar, h->Gbar, 1.0 / mu, h->t);
  if (st != TR_OK) return guard(st);
  if (pev) e = cudaEventRecord(pev[2], h->stream);
  if (info) {
    if (e == cudaSuccess)
      e = launch_tube_inverse(h->dtype, h->P, (int)h->n, h->td, h->mats, h->Gbar, h->L, h->G,
                              h->Lam, mu, h->res, h->flags, h->stream);
    if (e != cudaSuccess)
      return guard(fail(h, TR_ECUDA, "tube inverse: %s", cudaGetErrorString(e)));
    h->launches += 1;
  } else {
    h->pending = true;
    h->mu_prev = mu;
  }
  if (e == cudaSuccess && pev) e = cudaEventRecord(pev[3], h->stream);
  if (e != cudaSuccess) return guard(fail(h, TR_ECUDA, "event: %s", cudaGetErrorString(e)));
  if (info) TR_CUDA(h, cudaEventRecord(h->ev1, h->stream));
  h->t += 1;
  double next = h->prm.growth * mu;
  h->mu = next < h->prm.mu_max ? next : h->prm.mu_max;
  if (info) return guard(read_info(h, mu, info));
  return TR_OK;
}

extern "C" tr_status tr_recover(tr_handle *h, void *L_out, tr_step_info *last) {
  if (!h) return TR_EINVAL;
  tr_step_info info{};
  const bool check = h->prm.tol > 0.0;
  bool converged = false;
  for (int it = 0; it < h->prm.max_iter; ++it) {
    tr_status st = tr_prox_step(h, (check || (last && it == h->prm.max_iter - 1)) ? &info : nullptr);
    if (st != TR_OK) return st;
    if (check) {
      double mx = 0;
      for (double v : info.res_inf) mx = v > mx ? v : mx;
      if (mx <= h->prm.tol) {
        converged = true;
        break;
      }
    }
  }
  {
    tr_status fs = finalize(h);
    if (fs != TR_OK) return fs;
  }
  if (L_out) {
    TR_CUDA(h, cudaMemcpyAsync(L_out, h->L, (size_t)h->N * h->esz, cudaMemcpyDeviceToDevice, h->stream));
    TR_CUDA(h, cudaStreamSynchronize(h->stream));
  }
  if (last) *last = info;
  if (check && !converged) return fail(h, TR_ENOTCONV, "max_iter %d reached", h->prm.max_iter);
  return TR_OK;
}

extern "C" tr_status tr_get_state(tr_handle *h, void *L, void *E, void *Y, void *Lam, void *G,
                                  double *mu, int *t) {
  if (!h) return TR_EINVAL;
  {
    tr_status fs = finalize(h);
    if (fs != TR_OK) return fs;
  }
  const size_t bytes = (size_t)h->N * h->esz;
  void *dst[] = {L, E, Y, Lam, G};
  void *src[] = {h->L, h->E, h->Y, h->Lam, h->G};
  for (int i = 0; i < 5; ++i)
    if (dst[i]) TR_CUDA(h, cudaMemcpyAsync(dst[i], src[i], bytes, cudaMemcpyDeviceToDevice, h->stream));
  TR_CUDA(h, cudaStreamSynchronize(h->stream));
  if (mu) *mu = h->mu;
  if (t) *t = h->t;
  return TR_OK;
}

extern "C" tr_status tr_set_state(tr_handle *h, const void *L, const void *E, const void *Y,
                                  const void *Lam, const void *G, double mu, int t) {
  if (!h) return TR_EINVAL;
  if (!(mu > 0) || t < 0) return fail(h, TR_EINVAL, "need mu > 0 and t >= 0");
  const size_t bytes = (size_t)h->N * h->esz;
  const void *src[] = {L, E, Y, Lam, G};
  void *dst[] = {h->L, h->E, h->Y, h->Lam, h->G};
  for (int i = 0; i < 5; ++i)
    if (src[i]) TR_CUDA(h, cudaMemcpyAsync(dst[i], src[i], bytes, cudaMemcpyDeviceToDevice, h->stream));
  TR_CUDA(h, cudaStreamSynchronize(h->stream));
  h->mu = mu;
  h->t = t;
  h->poisoned = false;
  h->pending = false;
  h->lw.have_hist = false;
  return TR_OK;
}

extern "C" tr_status tr_transform_forward(tr_handle *h, const void *src, void *dst) {
  if (!h || !src || !dst) return TR_EINVAL;
  TR_CUDA(h, launch_transform(h->dtype, h->P, (int)h->n, h->td, h->mats, src, dst, false, h->stream));
  return TR_OK;
}

extern "C" tr_status tr_transform_inverse(tr_handle *h, const void *src, void *dst) {
  if (!h || !src || !dst) return TR_EINVAL;
  TR_CUDA(h, launch_transform(h->dtype, h->P, (int)h->n, h->td, h->mats, src, dst, true, h->stream));
  return TR_OK;
}

extern "C" tr_status tr_slice_prox(tr_handle *h, const void *Abar, void *Gbar, double tau, int t) {
  if (!h || !Abar || !Gbar) return TR_EINVAL;
  if (Abar == Gbar) return fail(h, TR_EINVAL, "Abar and Gbar must not alias");
  if (!(tau >= 0) || t < 0) return fail(h, TR_EINVAL, "need tau >= 0, t >= 0");
  return slice_pass(h, Abar, Gbar, tau, t);
}

extern "C" tr_status tr_last_slice_stats(tr_handle *h, double *sigma, int *ranks, int *l) {
  if (!h) return TR_EINVAL;
  const int ll = h->sw.l;
  if (l) *l = ll;
  if (sigma) {
    const size_t cnt = (size_t)h->n * ll;
    if (h->dtype == TR_F64) {
      TR_CUDA(h, cudaMemcpyAsync(sigma, h->sw.sig, cnt * 8, cudaMemcpyDeviceToHost, h->stream));
      TR_CUDA(h, cudaStreamSynchronize(h->stream));
    } else {
      std::vector<float> tmp(cnt);
      TR_CUDA(h, cudaMemcpyAsync(tmp.data(), h->sw.sig, cnt * 4, cudaMemcpyDeviceToHost, h->stream));
      TR_CUDA(h, cudaStreamSynchronize(h->stream));
      for (size_t i = 0; i < cnt; ++i) sigma[i] = tmp[i];
    }
  }
  if (ranks) {
    TR_CUDA(h, cudaMemcpyAsync(ranks, h->sw.rank, (size_t)h->n * sizeof(int), cudaMemcpyDeviceToHost,
                               h->stream));
    TR_CUDA(h, cudaStreamSynchronize(h->stream));
  }
  return TR_OK;
}

extern "C" tr_status tr_profile_enable(tr_handle *h, int max_steps) {
  if (!h || max_steps < 0) return TR_EINVAL;
  TR_CUDA(h, cudaStreamSynchronize(h->stream));
  free_profile(h);
  if (max_steps == 0) return TR_OK;
  h->prof_ev.resize((size_t)4 * max_steps, nullptr);
  for (auto &e : h->prof_ev) TR_CUDA(h, cudaEventCreate(&e));
  h->prof_cap = max_steps;
  h->prof_used = 0;
  return TR_OK;
}

extern "C" tr_status tr_profile_read(tr_handle *h, double ms[3], int *steps) {
  if (!h || !ms) return TR_EINVAL;
  TR_CUDA(h, cudaStreamSynchronize(h->stream));
  double acc[3] = {0, 0, 0};
  for (int s = 0; s < h->prof_used; ++s) {
    for (int k = 0; k < 3; ++k) {
      float v = 0.f;
      TR_CUDA(h, cudaEventElapsedTime(&v, h->prof_ev[(size_t)4 * s + k], h->prof_ev[(size_t)4 * s + k + 1]));
      acc[k] += v;
    }
  }
  for (int k = 0; k < 3; ++k) ms[k] = h->prof_used ? acc[k] / h->prof_used : 0.0;
  if (steps) *steps = h->prof_used;
  return TR_OK;
}

extern "C" tr_status tr_kernel_launches(const tr_handle *h, uint64_t *count) {
  if (!h || !count) return TR_EINVAL;
  *count = h->launches;
  return TR_OK;
}

extern "C" int64_t tr_mlp_param_count(void) { return mlp_param_count(); }

extern "C" tr_status tr_set_model(tr_handle *h, const float *params, int64_t count) {
  if (!h || !params) return TR_EINVAL;
  if (h->prm.engine != TR_LR_LEARNED) return fail(h, TR_EINVAL, "not a learned-engine handle");
  if (count != mlp_param_count())
    return fail(h, TR_EINVAL, "expected %lld parameters, got %lld", (long long)mlp_param_count(),
                (long long)count);
  TR_CUDA(h, cudaMemcpyAsync(h->lw.params, params, (size_t)count * sizeof(float),
                             cudaMemcpyHostToDevice, h->stream));
  TR_CUDA(h, cudaStreamSynchronize(h->stream));
  return TR_OK;
}

extern "C" tr_status tr_last_slice_widths(tr_handle *h, int *widths) {
  if (!h || !widths) return TR_EINVAL;
  TR_CUDA(h, cudaMemcpyAsync(widths, h->width, (size_t)h->n * sizeof(int), cudaMemcpyDeviceToHost,
                             h->stream));
  TR_CUDA(h, cudaStreamSynchronize(h->stream));
  return TR_OK;
}

extern "C" tr_status tr_slice_features(tr_handle *h, double tau, int t, float *features) {
  if (!h || !features) return TR_EINVAL;
  if (!h->have_pass) return fail(h, TR_EINVAL, "no slice pass has run yet");
  if (!(tau >= 0) || t < 0) return fail(h, TR_EINVAL, "need tau >= 0, t >= 0");
  const double T = h->prm.max_iter > 0 ? (double)h->prm.max_iter : 1.0;
  TR_CUDA(h, launch_features(h->dtype, (int)h->n, h->sw.sig, h->sw.ldsig, h->sw.rank, h->width,
                             shrink_threshold(h->prm, tau), h->thr_last, (double)t / T, features,
                             h->stream));
  h->launches += 1;
  return TR_OK;
}

#define TR_STATELESS(call)                                                              \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return fail(nullptr, e_ == cudaErrorMemoryAllocation ? TR_ENOMEM : TR_ECUDA,      \
                  "%s: %s", #call, cudaGetErrorString(e_));                             \
  } while (0)

extern "C" tr_status tr_features(tr_dtype dtype, int n, const void *sig, int ldsig, const int *rank,
                                 const int *width, double thr, double thr0, double tfrac,
                                 float *features, void *stream) {
  if (n < 0 || (n > 0 && (!sig || !rank || !width || !features)) || ldsig < 1 ||
      (dtype != TR_F32 && dtype != TR_F64))
    return fail(nullptr, TR_EINVAL, "tr_features: bad arguments");
  TR_STATELESS(launch_features(dtype, n, sig, ldsig, rank, width, thr, thr0, tfrac, features,
                               (cudaStream_t)stream));
  return TR_OK;
}

extern "C" tr_status tr_plan_widths(int n, const float *yhat, int oversample, int lmax, int *width,
                                    int *ids, int *counts, void *stream) {
  if (n < 0 || oversample < 0 || lmax < 1 || lmax > TR_MAX_L || !counts ||
      (n > 0 && (!yhat || !width || !ids)))
    return fail(nullptr, TR_EINVAL, "tr_plan_widths: bad arguments");
  TR_STATELESS(launch_plan(n, yhat, oversample, lmax, width, ids, counts, (cudaStream_t)stream));
  return TR_OK;
}

extern "C" tr_status tr_mlp_init(float *params, uint64_t seed, void *stream) {
  if (!params) return fail(nullptr, TR_EINVAL, "tr_mlp_init: NULL params");
  TR_STATELESS(launch_mlp_init(params, seed, (cudaStream_t)stream));
  return TR_OK;
}

extern "C" tr_status tr_mlp_forward(const float *params, const float *X, int B, float *yhat,
                                    void *stream) {
  if (B < 0 || (B > 0 && (!params || !X || !yhat)))
    return fail(nullptr, TR_EINVAL, "tr_mlp_forward: bad arguments");
  TR_STATELESS(launch_mlp_forward(params, X, B, yhat, nullptr, (cudaStream_t)stream));
  return TR_OK;
}

extern "C" tr_status tr_mlp_loss_grad(const float *params, const float *X, const float *y, int B,
                                      double under_weight, float *grad, float *loss, void *stream) {
  if (B < 1 || !params || !X || !y || !grad || !(under_weight >= 0))
    return fail(nullptr, TR_EINVAL, "tr_mlp_loss_grad: bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  float *work = nullptr;
  const size_t nf = mlp_workspace_floats(B) + (size_t)B;
  TR_STATELESS(cudaMallocAsync((void **)&work, nf * sizeof(float), s));
  cudaError_t e = launch_mlp_loss_grad(params, X, y, B, (float)under_weight, work,
                                       work + mlp_workspace_floats(B), grad, loss, s);
  cudaFreeAsync(work, s);
  TR_STATELESS(e);
  return TR_OK;
}

extern "C" tr_status tr_mlp_adam(float *params, const float *grad, float *m, float *v,
                                 int64_t count, double lr, double beta1, double beta2, double eps,
                                 int step, void *stream) {
  if (count < 0 || step < 1 || (count > 0 && (!params || !grad || !m || !v)) ||
      !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) || !(eps > 0))
    return fail(nullptr, TR_EINVAL, "tr_mlp_adam: bad arguments");
  TR_STATELESS(launch_mlp_adam(params, grad, m, v, count, lr, beta1, beta2, eps, step,
                               (cudaStream_t)stream));
  return TR_OK;
}

extern "C" tr_status tr_mlp_train(float *params, const float *X, const float *y, int n, int batch,
                                  int steps, double lr, double under_weight, uint64_t seed,
                                  float *loss_hist, void *stream) {
  if (!params || !X || !y || n < 1 || batch < 1 || steps < 0 || !(under_weight >= 0))
    return fail(nullptr, TR_EINVAL, "tr_mlp_train: bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t P = mlp_param_count();
  const size_t nw = mlp_workspace_floats(batch);
  const size_t total = nw + (size_t)batch /* yhat */ + (size_t)batch * TR_MLP_IN + batch +
                       3 * (size_t)P;
  float *buf = nullptr;
  TR_STATELESS(cudaMallocAsync((void **)&buf, total * sizeof(float), s));
  float *work = buf, *yhat = work + nw, *Xb = yhat + batch, *yb = Xb + (size_t)batch * TR_MLP_IN;
  float *grad = yb + batch, *m = grad + P, *v = m + P;
  cudaError_t e = cudaMemsetAsync(m, 0, 2 * (size_t)P * sizeof(float), s);
  for (int it = 0; it < steps && e == cudaSuccess; ++it) {
    e = launch_mlp_gather(X, y, n, batch, it, seed, Xb, yb, s);
    if (e == cudaSuccess)
      e = launch_mlp_loss_grad(params, Xb, yb, batch, (float)under_weight, work, yhat, grad,
                               loss_hist ? loss_hist + it : nullptr, s);
    if (e == cudaSuccess) e = launch_mlp_adam(params, grad, m, v, P, lr, 0.9, 0.999, 1e-8, it + 1, s);
  }
  cudaFreeAsync(buf, s);
  TR_STATELESS(e);
  return TR_OK;
}

extern "C" tr_status tr_free(tr_handle *h) {
  if (!h) return TR_OK;
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  free_all(h);
  delete h;
  return TR_OK;
}

extern "C" const char *tr_last_error(const tr_handle *h) { return h ? h->err : g_init_err; }
