// C ABI of libtr (include/tr.h): handle life cycle, one ADMM iteration of
// Alg. 5 (pure-L form) as a sequence of launches on the caller's stream,
// the recovery loop, and state import/export.

#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <new>
#include <vector>

#include "tr_internal.cuh"

constexpr int kSideStreams = 4;

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
  // the steps' tube passes write Abar as BF16 planes (hi, lo) for the
  // tensor-core products (FP32 problems, BF16 forms, fixed-width engine)
  bool abar_planes = false;
  double thr_last = 0.0;                      // its shrink threshold
  DevSched *sched = nullptr;                  // device copy of mu, mu_prev, t
  // the RSVD slice pass split into `slice_groups` independent slice ranges on
  // side streams, so latency-bound kernels of one range overlap the
  // bandwidth-bound products of another (tr_set_slice_groups, tr_autotune)
  int slice_groups = 1;
  // shared-Tucker engine (TR_LR_TUCKER): workspace and the two Gaussian blocks
  void *tk_ws = nullptr, *tk_g1 = nullptr, *tk_g2 = nullptr;
  int *iota = nullptr;                        // 0, 1, ..., n-1 (slice ids of the ranges)
  cudaStream_t side[kSideStreams] = {};
  cudaEvent_t side_fork = nullptr, side_join[kSideStreams] = {};
  // graph replay of steady-state steps (tr_graph_mode)
  // Captured steps are kept per observed-data pair (tr_set_observed), so that
  // double-buffered inputs replay two graphs instead of re-capturing.
  bool graph_on = false;
  cudaStream_t gstream = nullptr;
  struct GraphSlot {
    const void *M = nullptr;
    const uint8_t *mask = nullptr;
    cudaGraphExec_t exec = nullptr;
  } gx[2];
  int gx_next = 0;
  cudaEvent_t gev_in = nullptr, gev_out = nullptr;
  uint64_t graph_kernels = 0;                 // kernels in one replay
  unsigned long long *res = nullptr;          // RES_COUNT slots
  unsigned long long *res_prev = nullptr;     // slots for a deferred inverse pass
  int *flags = nullptr;
  // pinned host copy of `flags`, written by every step (replays included)
  // without a host synchronisation; a later call reads it
  volatile int *flags_host = nullptr;
  // pinned ring of residual reads for tr_recover's lagged stop test
  double *rec_ring = nullptr;
  cudaEvent_t rec_ev[3] = {};
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

// Messages of failed calls that have no handle, one per calling host thread.
static thread_local char g_init_err[512] = {0};

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
  void *lbufs[] = {lw.params, lw.w16, lw.feat, lw.pred, lw.ids, lw.counts, lw.fb_ids,
                   lw.fb_count, lw.gids, lw.gcount, lw.anorm2, lw.iota};
  for (void *b : lbufs)
    if (b) cudaFree(b);
  for (int i = 0; i < TR_LEARNED_STREAMS; ++i) {
    if (lw.aux[i]) cudaStreamDestroy(lw.aux[i]);
    if (lw.join[i]) cudaEventDestroy(lw.join[i]);
  }
  if (lw.fork) cudaEventDestroy(lw.fork);
  if (h->width) cudaFree(h->width);
  if (h->sched) cudaFree(h->sched);
  if (h->tk_ws) cudaFree(h->tk_ws);
  if (h->tk_g1) cudaFree(h->tk_g1);
  if (h->tk_g2) cudaFree(h->tk_g2);
  if (h->iota) cudaFree(h->iota);
  for (int i = 0; i < kSideStreams; ++i) {
    if (h->side[i]) cudaStreamDestroy(h->side[i]);
    if (h->side_join[i]) cudaEventDestroy(h->side_join[i]);
  }
  if (h->side_fork) cudaEventDestroy(h->side_fork);
  for (auto &g : h->gx)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  if (h->gstream) cudaStreamDestroy(h->gstream);
  if (h->gev_in) cudaEventDestroy(h->gev_in);
  if (h->gev_out) cudaEventDestroy(h->gev_out);
  void *bufs[] = {h->mats, h->L, h->E, h->Y, h->Lam, h->G, h->Abar, h->Gbar,
                  h->sw.Om, h->sw.P1, h->sw.P2, h->sw.sig, h->sw.rank, h->sw.err,
                  h->aw.Ucat, h->aw.Vcat, h->aw.X, h->aw.Lm, h->aw.Rm, h->aw.E, h->aw.nrm2,
                  h->aw.active, h->aw.kept, h->aw.draws, h->res,
                  h->res_prev, h->flags};
  for (void *b : bufs)
    if (b) cudaFree(b);
  if (h->ev0) cudaEventDestroy(h->ev0);
  if (h->ev1) cudaEventDestroy(h->ev1);
  if (h->flags_host) cudaFreeHost((void *)h->flags_host);
  if (h->rec_ring) cudaFreeHost(h->rec_ring);
  for (cudaEvent_t e : h->rec_ev)
    if (e) cudaEventDestroy(e);
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
  if (prm->engine != TR_LR_RSVD && prm->engine != TR_LR_ADAPTIVE && prm->engine != TR_LR_LEARNED &&
      prm->engine != TR_LR_TUCKER)
    return fail(nullptr, TR_EUNSUPPORTED, "engine %d not built", (int)prm->engine);
  if ((prm->engine == TR_LR_ADAPTIVE || prm->engine == TR_LR_LEARNED) &&
      (prm->adapt_block < 1 || prm->adapt_block > 32 || !(prm->adapt_eps > 0)))
    return fail(nullptr, TR_EINVAL,
                "adaptive and learned engines: need 1 <= adapt_block <= 32, adapt_eps > 0");
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
  int stride = 1;
  for (int k = 0; k < td.nt; ++k) {
    td.stride[k] = stride;
    stride *= td.dim[k];
  }
  const int hk = transform_mats_layout(td);
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
  if (prm->engine == TR_LR_LEARNED) {
    // the adaptive judge and fallback: cap = the plain width rounded down to
    // whole blocks (so its singular values fit the rows of l_max)
    const int b = prm->adapt_block;
    const int mn = (int)(h->n1 < h->n2 ? h->n1 : h->n2);
    int kcap = (l / b) * b;
    if (kcap > (mn / b) * b) kcap = (mn / b) * b;
    if (kcap < b || adapt_smem_bytes(h->dtype, (int)h->n1, (int)h->n2, b, kcap) > 227 * 1024) {
      tr_status st = fail(nullptr, TR_EUNSUPPORTED,
                          "learned engine: adaptive fallback block %d does not fit width %d", b, l);
      delete h;
      return st;
    }
    h->aw.b = b;
    h->aw.kcap = kcap;
    h->aw.eps = prm->adapt_eps;
    h->aw.delta_rel = p->dtype == TR_F64 ? 1e-11 : 1e-5;
  }
  if (prm->engine == TR_LR_TUCKER) {
    const int64_t L = (int64_t)(prm->power_iters + 1) * l;
    if (L > 32 || L > h->n1 || L > h->n2) {
      tr_status st = fail(nullptr, TR_EUNSUPPORTED,
                          "shared-Tucker engine: (q + 1) l = %lld above 32 or a mode size",
                          (long long)L);
      delete h;
      return st;
    }
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
        // column m of U, even rows then odd rows, for the folded inverse
        if (2 * m + 1 <= d)
          hm[(size_t)td.off_inv[k] + (size_t)m * 2 * hk + (i & 1) * hk + i / 2] = U[(size_t)i * d + m];
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
  // the learned engine gives every width class its own panel region able to
  // hold all n slices at the class width
  const size_t pcols = prm->engine == TR_LR_LEARNED ? (size_t)learned_panel_cols(l) : (size_t)l;
  INIT_CUDA(cudaMalloc(&sw.Om, (size_t)h->n * h->n2 * pcols * h->esz));
  INIT_CUDA(cudaMalloc(&sw.P1, (size_t)h->n * h->n1 * pcols * h->esz));
  INIT_CUDA(cudaMalloc(&sw.P2, (size_t)h->n * h->n2 * pcols * h->esz));
  INIT_CUDA(cudaMalloc((void **)&h->width, (size_t)h->n * sizeof(int)));
  sw.width = h->width;
  sw.ldsig = l;
  INIT_CUDA(cudaMalloc(&sw.sig, (size_t)h->n * l * h->esz));
  INIT_CUDA(cudaMalloc((void **)&sw.rank, (size_t)h->n * sizeof(int)));
  INIT_CUDA(cudaMalloc((void **)&h->res, RES_COUNT * sizeof(unsigned long long)));
  INIT_CUDA(cudaMalloc((void **)&h->res_prev, RES_COUNT * sizeof(unsigned long long)));
  INIT_CUDA(cudaMalloc((void **)&h->flags, sizeof(int)));
  {
    void *fh = nullptr;
    INIT_CUDA(cudaHostAlloc(&fh, sizeof(int), cudaHostAllocDefault));
    h->flags_host = static_cast<volatile int *>(fh);
    *h->flags_host = 0;
  }
  INIT_CUDA(cudaMalloc((void **)&sw.err, sizeof(int)));
  INIT_CUDA(cudaMemsetAsync(sw.err, 0, sizeof(int), h->stream));
  sw.prec = (int)prm->prec;
  h->abar_planes = p->dtype == TR_F32 && prm->engine == TR_LR_RSVD &&
                   (prm->prec == TR_PREC_BF16 || prm->prec == TR_PREC_BF16X3) &&
                   planes_ok(h->n, (int)h->n1, (int)h->n2, l);
  INIT_CUDA(cudaMemsetAsync(sw.rank, 0, (size_t)h->n * sizeof(int), h->stream));
  if (prm->engine == TR_LR_ADAPTIVE || prm->engine == TR_LR_LEARNED) {
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
  if (prm->engine == TR_LR_TUCKER) {
    // r = b = l on both spatial modes, q = power_iters Krylov steps
    const int q = prm->power_iters;
    INIT_CUDA(cudaMalloc(&h->tk_ws, tucker_ws_bytes(h->dtype, (int)h->n, (int)h->n1, (int)h->n2, l,
                                                   l, l, l, q, q)));
    INIT_CUDA(cudaMalloc(&h->tk_g1, (size_t)h->n * h->n2 * l * h->esz));
    INIT_CUDA(cudaMalloc(&h->tk_g2, (size_t)h->n * l * l * h->esz));
  }
  if (prm->engine == TR_LR_LEARNED) {
    LearnedWork &lw = h->lw;
    lw.lmax = l;
    lw.p = prm->oversample;
    const int C = plan_classes(l);
    INIT_CUDA(cudaMalloc((void **)&lw.params, (size_t)mlp_param_count() * sizeof(float)));
    INIT_CUDA(cudaMalloc(&lw.w16, mlp_pack_halves() * 2));
    INIT_CUDA(cudaMalloc((void **)&lw.feat, (size_t)h->n * TR_MLP_IN * sizeof(float)));
    INIT_CUDA(cudaMalloc((void **)&lw.pred, (size_t)h->n * sizeof(float)));
    INIT_CUDA(cudaMalloc((void **)&lw.ids, (size_t)h->n * sizeof(int)));
    INIT_CUDA(cudaMalloc((void **)&lw.counts, (size_t)C * sizeof(int)));
    INIT_CUDA(cudaMalloc((void **)&lw.fb_ids, (size_t)h->n * sizeof(int)));
    INIT_CUDA(cudaMalloc((void **)&lw.fb_count, sizeof(int)));
    INIT_CUDA(cudaMalloc((void **)&lw.gids, (size_t)C * h->n * sizeof(int)));
    INIT_CUDA(cudaMalloc((void **)&lw.gcount, (size_t)C * sizeof(int)));
    INIT_CUDA(cudaMalloc((void **)&lw.anorm2, (size_t)h->n * sizeof(double)));
    INIT_CUDA(cudaMalloc((void **)&lw.iota, (size_t)h->n * sizeof(int)));
    {
      std::vector<int> ids((size_t)h->n);
      for (size_t i = 0; i < ids.size(); ++i) ids[i] = (int)i;
      INIT_CUDA(cudaMemcpy(lw.iota, ids.data(), ids.size() * sizeof(int), cudaMemcpyHostToDevice));
    }
    lw.aw = h->aw;
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
    INIT_CUDA(launch_mlp_pack(lw.params, lw.w16, h->stream));
  }
  INIT_CUDA(cudaMalloc((void **)&h->sched, sizeof(DevSched)));
  {
    const DevSched d0{prm->mu0, prm->mu0, 0, 0};
    INIT_CUDA(cudaMemcpy(h->sched, &d0, sizeof d0, cudaMemcpyHostToDevice));
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

// One slice pass.  `sched`: take tau = 1/mu and the iteration index from the
// device schedule (a step) rather than from the arguments (tr_slice_prox).
static tr_status slice_pass(tr_handle *h, const void *Abar, void *Gbar, double tau, int t,
                            bool sched = false, bool planes = false) {
  ShrinkScalars sh{tau, (int)h->prm.phi, h->prm.phi_theta, h->prm.phi_gamma};
  if (sched) sh.dmu = &h->sched->mu;
  h->sw.dt = sched ? &h->sched->t : nullptr;
  const double thr = shrink_threshold(h->prm, tau);
  if (h->prm.engine == TR_LR_ADAPTIVE) {
    TR_CUDA(h, launch_slice_adaptive(h->dtype, h->sw, h->aw, Abar, Gbar, sh, t, h->stream));
    const uint64_t nblk = (uint64_t)(h->aw.kcap / h->aw.b);
    h->launches += 1 + 4 * nblk - 2 + 3;   // init, per block GEMM+U (+GEMM+V), B GEMM, SVD, rebuild
    // the width of an adaptive slice is its basis size
    TR_CUDA(h, cudaMemcpyAsync(h->width, h->aw.kept, (size_t)h->n * sizeof(int),
                               cudaMemcpyDeviceToDevice, h->stream));
  } else if (h->prm.engine == TR_LR_LEARNED) {
    FeatSched fs;
    if (sched) {   // a step: thresholds and t from the device schedule
      fs.d = h->sched;
      fs.phi = (int)h->prm.phi;
      fs.theta = h->prm.phi_theta;
      fs.gamma = h->prm.phi_gamma;
      fs.T = h->prm.max_iter;
    }
    cudaError_t e = launch_slice_learned(h->dtype, h->sw, h->lw, Abar, Gbar, sh, thr, t,
                                         h->prm.max_iter, fs, h->stream, &h->launches);
    if (e != cudaSuccess)
      return fail(h, TR_ECUDA, "learned slice pass: %s", cudaGetErrorString(e));
  } else if (h->prm.engine == TR_LR_TUCKER) {
    // Gaussian blocks per transformed slice (Philox streams 2 and 4), then
    // the shared-Tucker prox with r = b = l and q Krylov steps per mode
    const int l = h->sw.l, q = h->prm.power_iters, n = (int)h->n;
    TR_CUDA(h, launch_gaussian_blocks(h->dtype, n, (int64_t)h->n2 * l, h->tk_g1, h->prm.seed, t,
                                      h->sw.dt, 2u, h->stream));
    TR_CUDA(h, launch_gaussian_blocks(h->dtype, n, (int64_t)l * l, h->tk_g2, h->prm.seed, t,
                                      h->sw.dt, 4u, h->stream));
    cudaError_t e = launch_slice_tucker(h->dtype, n, (int)h->n1, (int)h->n2, l, l, l, l, q, q, Abar,
                                        Gbar, h->tk_g1, h->tk_g2, h->tk_ws, sh, nullptr, nullptr,
                                        h->stream, true, h->sw.sig, h->sw.rank);
    if (e != cudaSuccess) return fail(h, TR_ECUDA, "tucker slice pass: %s", cudaGetErrorString(e));
    h->launches += 2 + 2 * (7 + 3 * (uint64_t)q) + 7;
  } else if (h->slice_groups > 1) {
    // contiguous slice ranges on side streams; each range's panels sit at
    // its own offset of the workspace (same width, so no overlap)
    const int G = h->slice_groups, n = (int)h->n;
    TR_CUDA(h, cudaEventRecord(h->side_fork, h->stream));
    for (int g = 0; g < G; ++g) TR_CUDA(h, cudaStreamWaitEvent(h->side[g], h->side_fork, 0));
    int start = 0;
    for (int g = 0; g < G; ++g) {
      const int cnt = n / G + (g < n % G ? 1 : 0);
      SliceWork gw = h->sw;
      gw.asplit = planes;
      gw.n = cnt;
      gw.sel.ids = h->iota + start;
      gw.Om = (char *)h->sw.Om + (size_t)start * h->n2 * h->sw.l * h->esz;
      gw.P1 = (char *)h->sw.P1 + (size_t)start * h->n1 * h->sw.l * h->esz;
      gw.P2 = (char *)h->sw.P2 + (size_t)start * h->n2 * h->sw.l * h->esz;
      gw.nA = (int)h->n;
      if (cnt > 0) {
        TR_CUDA(h, launch_slice_rsvd(h->dtype, gw, Abar, Gbar, sh, t, h->side[g]));
        h->launches += 7 + 4 * (uint64_t)h->sw.q;
      }
      start += cnt;
    }
    for (int g = 0; g < G; ++g) {
      TR_CUDA(h, cudaEventRecord(h->side_join[g], h->side[g]));
      TR_CUDA(h, cudaStreamWaitEvent(h->stream, h->side_join[g], 0));
    }
  } else {
    SliceWork sw = h->sw;
    sw.asplit = planes;
    TR_CUDA(h, launch_slice_rsvd(h->dtype, sw, Abar, Gbar, sh, t, h->stream));
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
  info->fallback_slices = 0;
  if (h->prm.engine == TR_LR_LEARNED && h->lw.fb_count)
    TR_CUDA(h, cudaMemcpy(&info->fallback_slices, h->lw.fb_count, sizeof(int),
                          cudaMemcpyDeviceToHost));
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
  // the inverse pass's residual slots: ||L - G|| and ||dG|| of the last step
  cudaError_t e = cudaMemsetAsync(h->res_prev, 0, RES_COUNT * sizeof(unsigned long long), h->stream);
  if (e == cudaSuccess)
    e = launch_tube_inverse(h->dtype, h->P, (int)h->n, h->td, h->mats, h->Gbar, h->L,
                                      h->G, h->Lam, h->mu_prev, &h->sched->mu_prev, h->res_prev,
                                      h->flags, h->stream);
  if (e != cudaSuccess) {
    h->poisoned = true;
    return fail(h, TR_ECUDA, "tube inverse: %s", cudaGetErrorString(e));
  }
  h->launches += 1;
  h->pending = false;
  return TR_OK;
}

// Enqueue one iteration on h->stream.  pending: fuse the deferred inverse
// pass of the last step into this step's forward pass; with_inverse: finish
// the step now (needed for the residuals of tr_step_info), otherwise defer
// it.  mu^t and t come from the device schedule, which the last kernel
// advances, so the enqueued work is the same for every steady-state step.
static tr_status enqueue_step(tr_handle *h, bool pending, bool with_inverse, cudaEvent_t *pev) {
  const double mu = h->mu;
  TubeScalars sc{mu, h->prm.lambda / mu, (int)h->prm.noise, (int)h->prm.psi, h->prm.psi_theta,
                 h->prm.psi_gamma};
  sc.dmu = &h->sched->mu;
  sc.lambda = h->prm.lambda;
  sc.planes = h->abar_planes ? 1 : 0;
  cudaError_t e = cudaMemsetAsync(h->res, 0, RES_COUNT * sizeof(unsigned long long), h->stream);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(h->res_prev, 0, RES_COUNT * sizeof(unsigned long long), h->stream);
  if (e == cudaSuccess && pev) e = cudaEventRecord(pev[0], h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->flags, 0, sizeof(int), h->stream);
  if (e == cudaSuccess) {
    if (pending)
      e = launch_tube_fused(h->dtype, h->P, (int)h->n, h->td, h->mats, h->Gbar, h->mu_prev,
                            &h->sched->mu_prev, h->M, h->mask, h->L, h->E, h->Y, h->G, h->Lam,
                            h->Abar, sc, h->res_prev, h->res, h->flags, h->stream);
    else
      e = launch_tube_forward(h->dtype, h->P, (int)h->n, h->td, h->mats, h->M, h->mask, h->L,
                              h->E, h->Y, h->G, h->Lam, h->Abar, sc, h->res, h->flags, h->stream);
  }
  // the NaN/Inf flag of this tube pass goes to pinned host memory, so that
  // steps without a report (graph replays) are checked by a later call
  if (e == cudaSuccess)
    e = cudaMemcpyAsync((void *)h->flags_host, h->flags, sizeof(int), cudaMemcpyDeviceToHost,
                        h->stream);
  if (e == cudaSuccess && pev) e = cudaEventRecord(pev[1], h->stream);
  if (e != cudaSuccess) return fail(h, TR_ECUDA, "tube forward: %s", cudaGetErrorString(e));
  h->launches += 1;
  tr_status st = slice_pass(h, h->Abar, h->Gbar, 1.0 / mu, h->t, true, h->abar_planes);
  if (st != TR_OK) return st;
  if (pev) e = cudaEventRecord(pev[2], h->stream);
  if (with_inverse) {
    if (e == cudaSuccess)
      e = launch_tube_inverse(h->dtype, h->P, (int)h->n, h->td, h->mats, h->Gbar, h->L, h->G,
                              h->Lam, mu, &h->sched->mu, h->res, h->flags, h->stream);
    if (e != cudaSuccess) return fail(h, TR_ECUDA, "tube inverse: %s", cudaGetErrorString(e));
    h->launches += 1;
  }
  if (e == cudaSuccess && pev) e = cudaEventRecord(pev[3], h->stream);
  if (e == cudaSuccess) e = launch_schedule(h->sched, h->prm.growth, h->prm.mu_max, h->stream);
  if (e != cudaSuccess) return fail(h, TR_ECUDA, "schedule: %s", cudaGetErrorString(e));
  h->launches += 1;
  return TR_OK;
}

// Host mirror of the schedule kernel (same double arithmetic).
static void advance_host(tr_handle *h, bool deferred) {
  h->pending = deferred;
  h->mu_prev = h->mu;
  h->t += 1;
  const double next = h->prm.growth * h->mu;
  h->mu = next < h->prm.mu_max ? next : h->prm.mu_max;
}

// Capture one steady-state step (pending, deferred inverse) on the private
// stream; the graph is replayed for every later step of that kind.
static tr_status capture_step(tr_handle *h) {
  cudaStream_t user = h->stream;
  h->stream = h->gstream;
  const uint64_t before = h->launches;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(h->gstream, cudaStreamCaptureModeRelaxed);
  tr_status st = TR_OK;
  if (e == cudaSuccess) {
    st = enqueue_step(h, true, false, nullptr);
    cudaError_t e2 = cudaStreamEndCapture(h->gstream, &g);
    if (st == TR_OK && e2 != cudaSuccess) st = fail(h, TR_ECUDA, "capture: %s", cudaGetErrorString(e2));
  } else {
    st = fail(h, TR_ECUDA, "capture: %s", cudaGetErrorString(e));
  }
  h->stream = user;
  h->graph_kernels = h->launches - before;
  h->launches = before;
  if (st == TR_OK) {
    tr_handle::GraphSlot &slot = h->gx[h->gx_next];
    if (slot.exec) {
      cudaGraphExecDestroy(slot.exec);
      slot.exec = nullptr;
    }
    e = cudaGraphInstantiate(&slot.exec, g, 0);
    if (e != cudaSuccess) {
      slot.exec = nullptr;
      st = fail(h, TR_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    } else {
      slot.M = h->M;
      slot.mask = h->mask;
      h->gx_next ^= 1;
    }
  }
  if (g) cudaGraphDestroy(g);
  return st;
}

// Forget every captured step (their kernels hold settings that changed).
static tr_status drop_graphs(tr_handle *h) {
  bool any = false;
  for (auto &g : h->gx) any |= g.exec != nullptr;
  if (!any) return TR_OK;
  TR_CUDA(h, cudaStreamSynchronize(h->gstream));
  for (auto &g : h->gx) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g = tr_handle::GraphSlot{};
  }
  return TR_OK;
}

static cudaGraphExec_t find_graph(tr_handle *h) {
  for (auto &g : h->gx)
    if (g.exec && g.M == h->M && g.mask == h->mask) return g.exec;
  return nullptr;
}

static tr_status replay_step(tr_handle *h) {
  cudaGraphExec_t exec = find_graph(h);
  if (!exec) {
    tr_status st = capture_step(h);
    if (st != TR_OK) return st;
    exec = find_graph(h);
  }
  TR_CUDA(h, cudaEventRecord(h->gev_in, h->stream));
  TR_CUDA(h, cudaStreamWaitEvent(h->gstream, h->gev_in, 0));
  TR_CUDA(h, cudaGraphLaunch(exec, h->gstream));
  TR_CUDA(h, cudaEventRecord(h->gev_out, h->gstream));
  TR_CUDA(h, cudaStreamWaitEvent(h->stream, h->gev_out, 0));
  h->launches += h->graph_kernels;
  return TR_OK;
}

extern "C" tr_status tr_prox_step(tr_handle *h, tr_step_info *info) {
  if (!h) return TR_EINVAL;
  if (h->poisoned) return fail(h, TR_EINVAL, "handle poisoned by an earlier failure; call tr_set_state");
  if (*h->flags_host) {   // an earlier step without a report met NaN or Inf
    h->poisoned = true;
    return fail(h, TR_ENUMERIC, "NaN or Inf in the iterate, found after iteration %d", h->t);
  }
  const double mu = h->mu;
  auto guard = [&](tr_status st) {
    if (st != TR_OK) h->poisoned = true;
    return st;
  };
  cudaEvent_t *pev = nullptr;
  if (h->prof_used < h->prof_cap) pev = &h->prof_ev[(size_t)4 * h->prof_used++];
  if (!info && !pev && h->graph_on && h->pending) {
    tr_status st = replay_step(h);
    if (st != TR_OK) return guard(st);
    h->thr_last = shrink_threshold(h->prm, 1.0 / mu);
    advance_host(h, true);
    return TR_OK;
  }
  if (info) TR_CUDA(h, cudaEventRecord(h->ev0, h->stream));
  tr_status st = enqueue_step(h, h->pending, info != nullptr, pev);
  if (st != TR_OK) return guard(st);
  if (info) TR_CUDA(h, cudaEventRecord(h->ev1, h->stream));
  advance_host(h, info == nullptr);
  if (info) return guard(read_info(h, mu, info));
  return TR_OK;
}

extern "C" tr_status tr_graph_mode(tr_handle *h, int on) {
  if (!h) return TR_EINVAL;
  if (on && !h->gstream) {
    TR_CUDA(h, cudaStreamCreateWithFlags(&h->gstream, cudaStreamNonBlocking));
    TR_CUDA(h, cudaEventCreateWithFlags(&h->gev_in, cudaEventDisableTiming));
    TR_CUDA(h, cudaEventCreateWithFlags(&h->gev_out, cudaEventDisableTiming));
  }
  h->graph_on = on != 0;
  return TR_OK;
}

// The complete residual vector (Eq. convercon) of step k: its own slots
// from the read after step k, its deferred ||L - G|| and ||dG|| from the read
// after step k + 1 (tr_read_residuals layout).
static double residual_max(const double *own, const double *next) {
  double mx = 0.0;
  for (int i = 0; i < RES_COUNT; ++i) {
    const double v = (i == RES_LG || i == RES_DG) ? next[RES_COUNT + i] : own[i];
    mx = v > mx ? v : mx;
  }
  return mx;
}

extern "C" tr_status tr_recover(tr_handle *h, void *L_out, tr_step_info *last) {
  if (!h) return TR_EINVAL;
  tr_step_info info{};
  const bool check = h->prm.tol > 0.0;
  bool converged = false;
  if (!check) {
    for (int it = 0; it < h->prm.max_iter; ++it) {
      tr_status st = tr_prox_step(h, (last && it == h->prm.max_iter - 1) ? &info : nullptr);
      if (st != TR_OK) return st;
    }
    tr_status fs = finalize(h);
    if (fs != TR_OK) return fs;
    if (L_out) {
      TR_CUDA(h, cudaMemcpyAsync(L_out, h->L, (size_t)h->N * h->esz, cudaMemcpyDeviceToDevice,
                                 h->stream));
      TR_CUDA(h, cudaStreamSynchronize(h->stream));
    }
    if (last) *last = info;
    return TR_OK;
  } else {
    // Steps are enqueued without a report (graph replays when tr_graph_mode
    // is on), each followed by an asynchronous read of its residuals into a
    // pinned ring of three.  Step k's residuals are complete once step k + 1
    // has run, so after enqueuing step k + 2 the host waits only for step
    // k + 1's read: the GPU always has a step queued.  The loop stops at the
    // first step whose residuals all meet tol; the iterate returned is then
    // at most two steps past it.
    if (!h->rec_ring) {
      TR_CUDA(h, cudaHostAlloc((void **)&h->rec_ring, 3 * 2 * RES_COUNT * sizeof(double),
                               cudaHostAllocDefault));
      for (auto &e : h->rec_ev) TR_CUDA(h, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    int done = 0;   // steps enqueued
    for (int it = 0; it < h->prm.max_iter && !converged; ++it) {
      tr_status st = tr_prox_step(h, nullptr);
      if (st != TR_OK) return st;
      st = tr_read_residuals(h, h->rec_ring + 2 * RES_COUNT * (it % 3));
      if (st != TR_OK) return st;
      TR_CUDA(h, cudaEventRecord(h->rec_ev[it % 3], h->stream));
      done = it + 1;
      if (it >= 2) {
        const int k = it - 2;   // the step whose residuals are now complete
        TR_CUDA(h, cudaEventSynchronize(h->rec_ev[(k + 1) % 3]));
        if (*h->flags_host) {
          h->poisoned = true;
          return fail(h, TR_ENUMERIC, "NaN or Inf in the iterate, found after iteration %d", h->t);
        }
        const double mx = residual_max(h->rec_ring + 2 * RES_COUNT * (k % 3),
                                       h->rec_ring + 2 * RES_COUNT * ((k + 1) % 3));
        if (mx <= h->prm.tol) converged = true;
      }
    }
    (void)done;
  }
  {
    tr_status fs = finalize(h);
    if (fs != TR_OK) return fs;
  }
  TR_CUDA(h, cudaStreamSynchronize(h->stream));
  if (*h->flags_host) {
    h->poisoned = true;
    return fail(h, TR_ENUMERIC, "NaN or Inf in the iterate, found after iteration %d", h->t);
  }
  {
    // the residuals of the returned iterate: its own slots and the deferred
    // ones its finalising inverse pass wrote
    unsigned long long r[RES_COUNT], rp[RES_COUNT];
    TR_CUDA(h, cudaMemcpy(r, h->res, sizeof r, cudaMemcpyDeviceToHost));
    TR_CUDA(h, cudaMemcpy(rp, h->res_prev, sizeof rp, cudaMemcpyDeviceToHost));
    double mx = 0.0;
    for (int i = 0; i < RES_COUNT; ++i) {
      double v, vp;
      memcpy(&v, &r[i], sizeof v);
      memcpy(&vp, &rp[i], sizeof vp);
      if (i == RES_LG || i == RES_DG) v = v > vp ? v : vp;
      info.res_inf[i] = v;
      mx = v > mx ? v : mx;
    }
    info.iter = h->t;
    info.mu = h->mu_prev;
    info.tau = 1.0 / h->mu_prev;
    if (mx <= h->prm.tol) converged = true;
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
  {
    const DevSched d{mu, mu, t, 0};
    TR_CUDA(h, cudaMemcpyAsync(h->sched, &d, sizeof d, cudaMemcpyHostToDevice, h->stream));
    TR_CUDA(h, cudaStreamSynchronize(h->stream));
  }
  h->mu = mu;
  h->mu_prev = mu;
  h->t = t;
  h->poisoned = false;
  h->pending = false;
  h->lw.have_hist = false;
  *h->flags_host = 0;
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

extern "C" tr_status tr_slice_prox_tucker(tr_handle *h, const void *Abar, void *Gbar, double tau,
                                          int r1, int r2, int b1, int b2, int q1, int q2,
                                          const void *G1, const void *G2, void *F1_out,
                                          void *F2_out) {
  if (!h || !Abar || !Gbar || !G1 || !G2) return TR_EINVAL;
  if (Abar == Gbar) return fail(h, TR_EINVAL, "Abar and Gbar must not alias");
  if (!(tau >= 0)) return fail(h, TR_EINVAL, "need tau >= 0");
  const int n1 = (int)h->n1, n2 = (int)h->n2, L1 = (q1 + 1) * b1, L2 = (q2 + 1) * b2;
  if (r1 < 1 || r2 < 1 || b1 < 1 || b2 < 1 || q1 < 0 || q2 < 0)
    return fail(h, TR_EINVAL, "need ranks, blocks >= 1 and Krylov steps >= 0");
  if (r1 > n1 || r1 > n2 || r2 > n2 || L1 < r1 || L2 < r2 || L1 > n1 || L2 > n2)
    return fail(h, TR_EINVAL, "need r1 <= min(n1, n2), r2 <= n2, r <= (q+1) b <= mode size");
  if (L1 > 32 || L2 > 32 || !slice_smem_limit_ok(h->dtype, n1, n2, r1))
    return fail(h, TR_EUNSUPPORTED, "Krylov spaces above 32 columns are not built");
  const size_t bytes = tucker_ws_bytes(h->dtype, (int)h->n, n1, n2, r1, r2, b1, b2, q1, q2);
  void *ws = nullptr;
  TR_CUDA(h, cudaMallocAsync(&ws, bytes, h->stream));
  ShrinkScalars sh{tau, (int)h->prm.phi, h->prm.phi_theta, h->prm.phi_gamma};
  cudaError_t e = launch_slice_tucker(h->dtype, (int)h->n, n1, n2, r1, r2, b1, b2, q1, q2, Abar,
                                      Gbar, G1, G2, ws, sh, F1_out, F2_out, h->stream);
  cudaError_t e2 = cudaFreeAsync(ws, h->stream);
  if (e != cudaSuccess) return fail(h, TR_ECUDA, "tucker prox: %s", cudaGetErrorString(e));
  if (e2 != cudaSuccess) return fail(h, TR_ECUDA, "tucker workspace: %s", cudaGetErrorString(e2));
  return TR_OK;
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

extern "C" tr_status tr_profile_slice_pass(tr_handle *h, const void *Abar, void *Gbar, double tau,
                                           int t, int reps, double *ms, const char **names,
                                           int max_kernels, int *count) {
  if (!h || !Abar || !Gbar || !ms || !count || reps < 1 || max_kernels < 1) return TR_EINVAL;
  if (Abar == Gbar) return fail(h, TR_EINVAL, "Abar and Gbar must not alias");
  if (!(tau >= 0) || t < 0) return fail(h, TR_EINVAL, "need tau >= 0, t >= 0");
  if (h->prm.engine != TR_LR_RSVD)
    return fail(h, TR_EUNSUPPORTED, "per-kernel profile of the fixed-width engine only");
  SliceProf prof;
  for (int i = 0; i < SliceProf::kMax; ++i) {
    if (cudaEventCreate(&prof.ev[i]) != cudaSuccess) {
      for (int k = 0; k < i; ++k) cudaEventDestroy(prof.ev[k]);
      return fail(h, TR_ECUDA, "event creation failed");
    }
  }
  ShrinkScalars sh{tau, (int)h->prm.phi, h->prm.phi_theta, h->prm.phi_gamma};
  SliceWork w = h->sw;
  w.dt = nullptr;
  w.prof = &prof;
  // a handle whose steps hand the slice pass BF16 planes is profiled on the
  // same path: the FP32 Abar is split into the handle's Abar first
  if (h->abar_planes && Abar != h->Abar) {
    cudaError_t e = launch_split_planes((const float *)Abar, h->Abar, h->n * h->P, h->stream);
    if (e != cudaSuccess) {
      for (int i = 0; i < SliceProf::kMax; ++i) cudaEventDestroy(prof.ev[i]);
      return fail(h, TR_ECUDA, "split planes: %s", cudaGetErrorString(e));
    }
    Abar = h->Abar;
    w.asplit = 1;
  }
  std::vector<double> acc(SliceProf::kMax, 0.0);
  int nk = 0;
  tr_status st = TR_OK;
  for (int r = 0; r < reps && st == TR_OK; ++r) {
    prof.k = 0;
    prof.mark(h->stream, "start");
    cudaError_t e = launch_slice_rsvd(h->dtype, w, Abar, Gbar, sh, t, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
      st = fail(h, TR_ECUDA, "profiled slice pass: %s", cudaGetErrorString(e));
      break;
    }
    h->launches += (uint64_t)(prof.k - 1);
    nk = prof.k - 1;
    for (int k = 1; k < prof.k; ++k) {
      float v = 0.f;
      cudaEventElapsedTime(&v, prof.ev[k - 1], prof.ev[k]);
      acc[k] += v;
    }
  }
  if (st == TR_OK) {
    const int m = nk < max_kernels ? nk : max_kernels;
    for (int k = 0; k < m; ++k) {
      ms[k] = acc[k + 1] / reps;
      if (names) names[k] = prof.name[k + 1];
    }
    *count = m;
  }
  for (int i = 0; i < SliceProf::kMax; ++i) cudaEventDestroy(prof.ev[i]);
  return st;
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
  TR_CUDA(h, launch_mlp_pack(h->lw.params, h->lw.w16, h->stream));
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

// ---- autotuner -------------------------------------------------------------
// Two launch choices per shape class, each timed with CUDA events on the
// handle's own buffers: the tube tile (tubes per block) on the transform
// kernel, and (RSVD engine) the number of slice ranges the slice pass is
// split into, on a slice pass of L(M) -- the observed data -- held in the
// transform-domain scratch.  Every candidate computes the same values: a
// tile only partitions tubes among blocks, a range split only partitions
// slices among streams.  Choices are cached per process.
struct TuneKey {
  int dt, n, nt, dims[TR_MAX_TMODES];
  int64_t n1, n2;
  int engine, l, q, prec;
  bool operator==(const TuneKey &o) const {
    if (dt != o.dt || n != o.n || nt != o.nt || n1 != o.n1 || n2 != o.n2 ||
        engine != o.engine || l != o.l || q != o.q || prec != o.prec)
      return false;
    for (int k = 0; k < nt; ++k)
      if (dims[k] != o.dims[k]) return false;
    return true;
  }
};
struct TuneChoice {
  int tp, groups;
};
static std::vector<std::pair<TuneKey, TuneChoice>> g_tune_cache;
static std::mutex g_tune_mu;
extern "C" tr_status tr_set_slice_groups(tr_handle *h, int groups);

// Mean milliseconds of `reps` runs of `body` on the handle's stream.
template <typename F>
static tr_status time_ms(tr_handle *h, int reps, float &ms, F body) {
  TR_CUDA(h, cudaEventRecord(h->ev0, h->stream));
  for (int i = 0; i < reps; ++i) {
    tr_status st = body(i);
    if (st != TR_OK) return st;
  }
  TR_CUDA(h, cudaEventRecord(h->ev1, h->stream));
  TR_CUDA(h, cudaEventSynchronize(h->ev1));
  TR_CUDA(h, cudaEventElapsedTime(&ms, h->ev0, h->ev1));
  ms /= reps;
  return TR_OK;
}

extern "C" tr_status tr_autotune(tr_handle *h, int reps, int *tile, int *groups) {
  if (!h || reps < 0) return TR_EINVAL;
  TuneKey key{(int)h->dtype, (int)h->n, h->td.nt, {0}, h->n1, h->n2, (int)h->prm.engine,
              h->sw.l, h->sw.q, h->sw.prec};
  for (int k = 0; k < h->td.nt; ++k) key.dims[k] = h->td.dim[k];
  if (reps == 0) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (auto &kv : g_tune_cache)
      if (kv.first == key) {
        h->td.tp = kv.second.tp;
        if (tile) *tile = kv.second.tp;
        if (groups) *groups = kv.second.groups;
        return tr_set_slice_groups(h, kv.second.groups);
      }
  }
  const int r = reps > 0 ? reps : 3;
  {
    tr_status fs = finalize(h);   // the scratch below may hold a deferred step's Gbar
    if (fs != TR_OK) return fs;
  }
  // tube tile
  int cand[8];
  const int nc = tube_tile_candidates(h->dtype, (int)h->n, h->td, cand, 8);
  if (nc == 0) return fail(h, TR_EUNSUPPORTED, "no tube tile fits");
  float best = 0.f;
  int best_tp = cand[0];
  // The tile is timed on the transform kernel.  For FP32 problems whose
  // position count allows it, only tiles of a multiple of 16 tubes are
  // candidates: the fused pass prefetches its streams into L2 only with those
  // (a mask row of the tile must be a 16-byte multiple), which the transform
  // kernel's timing cannot see (200 against 340 us on 400 slices of 200 x 200).
  const bool pf_tiles = h->dtype == TR_F32 && h->P % 16 == 0;
  bool any = false;
  for (int c = 0; c < nc; ++c) {
    if (pf_tiles && cand[c] % 16 != 0) continue;
    TransformDesc td = h->td;
    td.tp = cand[c];
    TR_CUDA(h, launch_transform(h->dtype, h->P, (int)h->n, td, h->mats, h->Abar, h->Gbar, false,
                                h->stream));
    float ms = 0.f;
    tr_status st = time_ms(h, r, ms, [&](int i) -> tr_status {
      TR_CUDA(h, launch_transform(h->dtype, h->P, (int)h->n, td, h->mats, h->Abar, h->Gbar,
                                  (i & 1) != 0, h->stream));
      return TR_OK;
    });
    if (st != TR_OK) return st;
    h->launches += 1 + (uint64_t)r;
    if (!any || ms < best) {
      best = ms;
      best_tp = cand[c];
      any = true;
    }
  }
  h->td.tp = best_tp;
  // slice ranges
  int best_g = 1;
  if (h->prm.engine == TR_LR_RSVD) {
    if (h->abar_planes) {   // the steps' form: Abar as BF16 planes
      TR_CUDA(h, launch_transform(h->dtype, h->P, (int)h->n, h->td, h->mats, h->M, h->Gbar, false,
                                  h->stream));
      TR_CUDA(h, launch_split_planes((const float *)h->Gbar, h->Abar, h->n * h->P, h->stream));
      h->launches += 2;
    } else {
      TR_CUDA(h, launch_transform(h->dtype, h->P, (int)h->n, h->td, h->mats, h->M, h->Abar, false,
                                  h->stream));
      h->launches += 1;
    }
    const double tau = 1.0 / h->mu;
    float bestg = 0.f;
    for (int G = 1; G <= kSideStreams; G *= 2) {
      if (G > 1 && G > h->n) break;
      tr_status st = tr_set_slice_groups(h, G);
      if (st != TR_OK) return st;
      const bool pl = h->abar_planes;
      if ((st = slice_pass(h, h->Abar, h->Gbar, tau, h->t, false, pl)) != TR_OK) return st;
      float ms = 0.f;
      st = time_ms(h, r, ms,
                   [&](int) { return slice_pass(h, h->Abar, h->Gbar, tau, h->t, false, pl); });
      if (st != TR_OK) return st;
      if (G == 1 || ms < bestg) {
        bestg = ms;
        best_g = G;
      }
    }
    tr_status st = tr_set_slice_groups(h, best_g);
    if (st != TR_OK) return st;
  }
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    bool found = false;
    for (auto &kv : g_tune_cache)
      if (kv.first == key) {
        kv.second = TuneChoice{best_tp, best_g};
        found = true;
      }
    if (!found) g_tune_cache.push_back({key, TuneChoice{best_tp, best_g}});
  }
  {   // a captured step holds the old choices
    tr_status st = drop_graphs(h);
    if (st != TR_OK) return st;
  }
  if (tile) *tile = best_tp;
  if (groups) *groups = best_g;
  return TR_OK;
}

extern "C" tr_status tr_read_residuals(tr_handle *h, double *res_host) {
  if (!h || !res_host) return TR_EINVAL;
  // the slots hold the bit patterns of non-negative doubles (atomicMax)
  static_assert(sizeof(double) == sizeof(unsigned long long), "64-bit slots");
  TR_CUDA(h, cudaMemcpyAsync(res_host, h->res, RES_COUNT * sizeof(double), cudaMemcpyDeviceToHost,
                             h->stream));
  TR_CUDA(h, cudaMemcpyAsync(res_host + RES_COUNT, h->res_prev, RES_COUNT * sizeof(double),
                             cudaMemcpyDeviceToHost, h->stream));
  return TR_OK;
}

extern "C" tr_status tr_set_observed(tr_handle *h, const void *observed, const uint8_t *mask) {
  if (!h || !observed || !mask) return TR_EINVAL;
  h->M = observed;
  h->mask = mask;   // captured steps are looked up by these pointers
  return TR_OK;
}

extern "C" tr_status tr_set_tube_tile(tr_handle *h, int tp) {
  if (!h) return TR_EINVAL;
  if (tp != 0) {
    int cand[8];
    const int nc = tube_tile_candidates(h->dtype, (int)h->n, h->td, cand, 8);
    bool ok = false;
    for (int c = 0; c < nc; ++c) ok = ok || cand[c] == tp;
    if (!ok) return fail(h, TR_EINVAL, "tube tile %d does not fit", tp);
  }
  TR_CUDA(h, cudaStreamSynchronize(h->stream));
  h->td.tp = tp;
  return drop_graphs(h);
}

extern "C" tr_status tr_set_slice_groups(tr_handle *h, int groups) {
  if (!h) return TR_EINVAL;
  if (groups < 1 || groups > kSideStreams)
    return fail(h, TR_EINVAL, "slice groups %d not in [1, %d]", groups, kSideStreams);
  if (groups > 1 && h->prm.engine != TR_LR_RSVD)
    return fail(h, TR_EUNSUPPORTED, "slice groups apply to the RSVD engine");
  if (groups > 1 && !h->iota) {
    std::vector<int> ids((size_t)h->n);
    for (size_t j = 0; j < ids.size(); ++j) ids[j] = (int)j;
    TR_CUDA(h, cudaMalloc((void **)&h->iota, ids.size() * sizeof(int)));
    TR_CUDA(h, cudaMemcpy(h->iota, ids.data(), ids.size() * sizeof(int), cudaMemcpyHostToDevice));
    for (int i = 0; i < kSideStreams; ++i) {
      TR_CUDA(h, cudaStreamCreateWithFlags(&h->side[i], cudaStreamNonBlocking));
      TR_CUDA(h, cudaEventCreateWithFlags(&h->side_join[i], cudaEventDisableTiming));
    }
    TR_CUDA(h, cudaEventCreateWithFlags(&h->side_fork, cudaEventDisableTiming));
  }
  TR_CUDA(h, cudaStreamSynchronize(h->stream));
  h->slice_groups = groups;
  return drop_graphs(h);
}

// ---- batches of independent problems ----------------------------------------
struct tr_batch {
  std::vector<tr_handle *> hs;
  std::vector<cudaStream_t> pool;
  std::vector<cudaEvent_t> join;
  cudaStream_t stream = nullptr;      // caller's stream
  cudaStream_t cap = nullptr;         // private stream the batch graph runs on
  cudaEvent_t fork = nullptr, done = nullptr;
  cudaGraphExec_t gexec = nullptr;
  uint64_t graph_kernels = 0;
  uint64_t launches = 0;
  bool graph_on = true;
};

static thread_local char g_batch_err[512] = {0};

static tr_status batch_fail(tr_status st, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_batch_err, sizeof g_batch_err, fmt, ap);
  va_end(ap);
  return st;
}

extern "C" tr_status tr_batch_free(tr_batch *b) {
  if (!b) return TR_OK;
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (cudaStream_t s : b->pool) cudaStreamSynchronize(s);
  if (b->cap) cudaStreamSynchronize(b->cap);
  for (tr_handle *h : b->hs) tr_free(h);
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  for (cudaStream_t s : b->pool) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->join) cudaEventDestroy(e);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->done) cudaEventDestroy(b->done);
  delete b;
  return TR_OK;
}

extern "C" tr_status tr_batch_create(tr_batch **out, int nprob, const tr_problem *probs,
                                     const tr_params *prms, int nstreams, void *cuda_stream) {
  if (!out || nprob < 1 || !probs || !prms) return batch_fail(TR_EINVAL, "tr_batch_create: bad arguments");
  *out = nullptr;
  tr_batch *b = new (std::nothrow) tr_batch();
  if (!b) return batch_fail(TR_ENOMEM, "host allocation failed");
  b->stream = (cudaStream_t)cuda_stream;
  const int S = nstreams < 1 ? 8 : (nstreams > 32 ? 32 : nstreams);
  auto bail = [&](tr_status st) {
    tr_batch_free(b);
    return st;
  };
#define BATCH_CUDA(call)                                                                 \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return bail(batch_fail(e_ == cudaErrorMemoryAllocation ? TR_ENOMEM : TR_ECUDA, "%s: %s", \
                             #call, cudaGetErrorString(e_)));                            \
  } while (0)
  for (int i = 0; i < S && i < nprob; ++i) {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    BATCH_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    b->pool.push_back(st);
    BATCH_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    b->join.push_back(ev);
  }
  BATCH_CUDA(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
  BATCH_CUDA(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
  BATCH_CUDA(cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming));
  for (int i = 0; i < nprob; ++i) {
    tr_handle *h = nullptr;
    tr_status st = tr_init(&h, &probs[i], &prms[i], b->pool[(size_t)i % b->pool.size()]);
    if (st != TR_OK) return bail(batch_fail(st, "problem %d: %s", i, g_init_err));
    b->hs.push_back(h);
  }
#undef BATCH_CUDA
  *out = b;
  return TR_OK;
}

extern "C" tr_status tr_batch_handle(tr_batch *b, int i, tr_handle **h) {
  if (!b || !h || i < 0 || i >= (int)b->hs.size()) return batch_fail(TR_EINVAL, "tr_batch_handle: bad index");
  *h = b->hs[(size_t)i];
  return TR_OK;
}

extern "C" tr_status tr_batch_graph_mode(tr_batch *b, int on) {
  if (!b) return TR_EINVAL;
  b->graph_on = on != 0;
  return TR_OK;
}

extern "C" tr_status tr_batch_autotune(tr_batch *b, int reps) {
  if (!b || reps < 0) return batch_fail(TR_EINVAL, "tr_batch_autotune: bad arguments");
  // every problem's streams idle before its scratch is used for timing
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->cap);
  for (cudaStream_t s : b->pool)
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return batch_fail(TR_ECUDA, "tr_batch_autotune: %s", cudaGetErrorString(e));
  // the batch graph holds the earlier launch shapes: dropped before any
  // problem is retuned, so that a failure part way leaves no stale graph
  if (b->gexec) {
    cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
  }
  for (size_t i = 0; i < b->hs.size(); ++i) {
    tr_status st = tr_autotune(b->hs[i], reps, nullptr, nullptr);
    if (st != TR_OK) return batch_fail(st, "problem %zu: %s", i, b->hs[i]->err);
  }
  return TR_OK;
}

extern "C" tr_status tr_batch_launches(const tr_batch *b, uint64_t *count) {
  if (!b || !count) return TR_EINVAL;
  uint64_t c = b->launches;
  for (const tr_handle *h : b->hs) c += h->launches;
  *count = c;
  return TR_OK;
}

// Fork every pool stream from `from`, join them back into `to`.
static cudaError_t batch_fork(tr_batch *b, cudaStream_t from) {
  cudaError_t e = cudaEventRecord(b->fork, from);
  for (cudaStream_t s : b->pool)
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->fork, 0);
  return e;
}
static cudaError_t batch_join(tr_batch *b, cudaStream_t to) {
  cudaError_t e = cudaSuccess;
  for (size_t k = 0; k < b->pool.size() && e == cudaSuccess; ++k) {
    e = cudaEventRecord(b->join[k], b->pool[k]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(to, b->join[k], 0);
  }
  return e;
}

static tr_status batch_capture(tr_batch *b) {
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return batch_fail(TR_ECUDA, "capture: %s", cudaGetErrorString(e));
  tr_status st = TR_OK;
  if ((e = batch_fork(b, b->cap)) != cudaSuccess) st = batch_fail(TR_ECUDA, "fork: %s", cudaGetErrorString(e));
  uint64_t kernels = 0;
  for (size_t i = 0; i < b->hs.size() && st == TR_OK; ++i) {
    tr_handle *h = b->hs[i];
    const uint64_t before = h->launches;
    st = enqueue_step(h, true, false, nullptr);
    if (st != TR_OK) batch_fail(st, "problem %zu: %s", i, h->err);
    kernels += h->launches - before;
    h->launches = before;
  }
  if (st == TR_OK && (e = batch_join(b, b->cap)) != cudaSuccess)
    st = batch_fail(TR_ECUDA, "join: %s", cudaGetErrorString(e));
  cudaError_t e2 = cudaStreamEndCapture(b->cap, &g);
  if (st == TR_OK && e2 != cudaSuccess) st = batch_fail(TR_ECUDA, "capture: %s", cudaGetErrorString(e2));
  if (st == TR_OK && (e = cudaGraphInstantiate(&b->gexec, g, 0)) != cudaSuccess)
    st = batch_fail(TR_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
  if (g) cudaGraphDestroy(g);
  b->graph_kernels = kernels;
  return st;
}

extern "C" tr_status tr_batch_step(tr_batch *b, tr_step_info *infos) {
  if (!b) return TR_EINVAL;
  for (size_t i = 0; i < b->hs.size(); ++i)
    if (b->hs[i]->poisoned) return batch_fail(TR_EINVAL, "problem %zu is poisoned", i);
  cudaError_t e;
  bool all_pending = true;
  for (tr_handle *h : b->hs) all_pending = all_pending && h->pending;
  if (!infos && b->graph_on && all_pending) {
    // one graph launch runs the whole iteration of every problem
    if (!b->gexec) {
      tr_status st = batch_capture(b);
      if (st != TR_OK) return st;
    }
    if ((e = cudaEventRecord(b->fork, b->stream)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(b->cap, b->fork, 0)) != cudaSuccess ||
        (e = cudaGraphLaunch(b->gexec, b->cap)) != cudaSuccess ||
        (e = cudaEventRecord(b->done, b->cap)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(b->stream, b->done, 0)) != cudaSuccess)
      return batch_fail(TR_ECUDA, "graph launch: %s", cudaGetErrorString(e));
    for (cudaStream_t s : b->pool)
      if ((e = cudaStreamWaitEvent(s, b->done, 0)) != cudaSuccess)
        return batch_fail(TR_ECUDA, "graph launch: %s", cudaGetErrorString(e));
    b->launches += b->graph_kernels;
    for (tr_handle *h : b->hs) {
      h->thr_last = shrink_threshold(h->prm, 1.0 / h->mu);
      h->have_pass = true;
      advance_host(h, true);
    }
    return TR_OK;
  }
  if ((e = batch_fork(b, b->stream)) != cudaSuccess)
    return batch_fail(TR_ECUDA, "fork: %s", cudaGetErrorString(e));
  for (size_t i = 0; i < b->hs.size(); ++i) {
    tr_status st = tr_prox_step(b->hs[i], infos ? &infos[i] : nullptr);
    if (st != TR_OK) return batch_fail(st, "problem %zu: %s", i, b->hs[i]->err);
  }
  if ((e = batch_join(b, b->stream)) != cudaSuccess)
    return batch_fail(TR_ECUDA, "join: %s", cudaGetErrorString(e));
  return TR_OK;
}

extern "C" const char *tr_batch_last_error(void) { return g_batch_err; }

extern "C" tr_status tr_free(tr_handle *h) {
  if (!h) return TR_OK;
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  free_all(h);
  delete h;
  return TR_OK;
}

extern "C" const char *tr_last_error(const tr_handle *h) { return h ? h->err : g_init_err; }
