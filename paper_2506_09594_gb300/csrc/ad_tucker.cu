// Fixed-accuracy Tucker compression (Alg. "AD-RSTHOSVD-BLBP", processing
// order (1, 2)) followed by the core's GNTSVT (Alg. 4, randomized branch),
// on a transformed stack: tr_slice_prox_ad_tucker.
//
// Per mode, with A the mode unfolding of the current core C (n slices of
// p1 x p2; mode 1: A is p1 x (n p2), column j p2 + i2; mode 2: A is
// p2 x (n p1), column j p1 + i1), the block Lanczos loop of Alg. 3:
//   V = orth(G); E = ||A||_F^2;
//   repeat: [U, R] = defl-QR(A V - U_prev L, delta); E -= ||R||^2;
//           V' = A^T U - V R^T, reorthogonalised against V^{v};
//           [V', L^T] = defl-QR(V', delta); E -= ||L||^2;
//           refill V' with Gaussian columns (orthogonalised against V^{v})
//           when deflation kept fewer than b;
//   until E < eps^2 ||A||_F^2, the basis reaches its cap, or V' is empty;
// then F = U^{v} with the sign convention of the shared-Tucker form (each
// column's entry of largest magnitude positive: mode 2's draws act on
// C x_1 F1^T, so under a rank cap F2 depends on F1's signs) and
// C <- C x_mode F^T.  Finally every slice of the core gets
// the per-slice prox, and Gbar_j = F1 Prox(C_j) F2^T.
//
// GPU form.  A V and A^T U never form the unfolding: they are per-slice
// strided GEMMs (A V adds a sum over the slices).  defl-QR is column-pivoted
// classical Gram-Schmidt with one reorthogonalisation pass (pivot = the
// column of largest residual norm, the rule of the pivoted Householder QR;
// stop once that norm is below delta; R = Q^T A): column norms and dot
// products are multi-CTA reductions in double, the pivot choice runs on the
// host.  orth() of a Gaussian draw (the first V block and the refills) is
// the same Gram-Schmidt taking the columns in order, which gives the columns
// of the unpivoted Householder QR up to sign, so a rank cap keeps the same
// directions as that form.  Gaussian draws are the per-slice Philox blocks of the sketch kernel
// (stream 0x10000 m + 2 d for draw d of mode m), gathered into a stacked
// column-major panel.  The core's prox is the slice pass at full width
// (exact) on this call's own workspace.  Panels are column-major.

#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "sgemm.cuh"
#include "tr_internal.cuh"

namespace {

tr_status afail(char *buf, size_t len, tr_status st, const char *fmt, ...) {
  if (buf && len) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, len, fmt, ap);
    va_end(ap);
  }
  return st;
}

int agrid(int64_t N) {
  const int64_t blocks = (N + 255) / 256;
  return (int)(blocks < 152 * 32 ? (blocks < 1 ? 1 : blocks) : 152 * 32);
}

// out[i] = sum_o in[o M + i]
template <typename T>
__global__ void batch_sum_kernel(T *out, const T *__restrict__ in, int64_t M, int64_t nb) {
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += step) {
    T s = T(0);
    for (int64_t o = 0; o < nb; ++o) s += in[o * M + i];
    out[i] = s;
  }
}

// out[c] += sum_r W[r + c ld] * V[r + c ldv] for c < k (V = W: squared norms).
template <typename T>
__global__ void col_dots_kernel(const T *__restrict__ W, int64_t ld, const T *__restrict__ V,
                                int64_t ldv, int64_t rows, int k, double *out) {
  const int c = blockIdx.y;
  double acc = 0.0;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows;
       r += (int64_t)gridDim.x * blockDim.x)
    acc += (double)W[r + c * ld] * (double)V[r + c * ldv];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ double s[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) s[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s[w];
    atomicAdd(out + c, t);
  }
  (void)k;
}

// out[c] += sum_r W[r + c ld] q[r] for c < k.
template <typename T>
__global__ void col_dot_vec_kernel(const T *__restrict__ W, int64_t ld, const T *__restrict__ q,
                                   int64_t rows, double *out) {
  const int c = blockIdx.y;
  double acc = 0.0;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows;
       r += (int64_t)gridDim.x * blockDim.x)
    acc += (double)W[r + c * ld] * (double)q[r];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ double s[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) s[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s[w];
    atomicAdd(out + c, t);
  }
}

// W[r + c ld] -= q[r] coef[c] for c < k.
template <typename T>
__global__ void rank1_kernel(T *W, int64_t ld, const T *__restrict__ q, const double *coef,
                             int64_t rows, int k) {
  const int64_t total = rows * k;
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += step) {
    const int64_t r = e % rows;
    const int c = (int)(e / rows);
    W[r + c * ld] -= q[r] * (T)coef[c];
  }
}

// q[r] -= sum_i Q[r + i rows] coef[i] for i < s.
template <typename T>
__global__ void gemv_sub_kernel(T *q, const T *__restrict__ Q, int64_t rows, int s,
                                const double *coef) {
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += step) {
    double acc = 0.0;
    for (int i = 0; i < s; ++i) acc += (double)Q[r + i * rows] * coef[i];
    q[r] = (T)((double)q[r] - acc);
  }
}

// dst = src * scale
template <typename T>
__global__ void scale_kernel(T *dst, const T *__restrict__ src, int64_t rows, double scale) {
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += step)
    dst[r] = (T)((double)src[r] * scale);
}

// out[(j p + i) + c ld] = in[j p cols + c p + i]: per-slice column-major
// blocks (p x cols) stacked into one column-major panel.
template <typename T>
__global__ void gather_slices_kernel(T *out, int64_t ld, const T *__restrict__ in, int64_t n,
                                     int64_t p, int64_t cols) {
  const int64_t total = n * p * cols;
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += step) {
    const int64_t i = e % p, c = (e / p) % cols, j = e / (p * cols);
    out[(j * p + i) + c * ld] = in[e];
  }
}

// out[0] += sum X^2
template <typename T>
__global__ void sumsq_kernel(const T *__restrict__ X, int64_t N, double *out) {
  double acc = 0.0;
  for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < N;
       f += (int64_t)gridDim.x * blockDim.x)
    acc += (double)X[f] * (double)X[f];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ double s[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) s[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s[w];
    atomicAdd(out, t);
  }
}

struct Ctx {
  cudaStream_t s;
  double *dscr;            // device doubles (>= 64)
  double *hscr;            // host copy
  cudaError_t e = cudaSuccess;
};

// Read `k` doubles of dscr to the host (synchronises).
bool fetch(Ctx &x, int k) {
  if (x.e != cudaSuccess) return false;
  x.e = cudaMemcpyAsync(x.hscr, x.dscr, k * sizeof(double), cudaMemcpyDeviceToHost, x.s);
  if (x.e == cudaSuccess) x.e = cudaStreamSynchronize(x.s);
  return x.e == cudaSuccess;
}

dim3 red_grid(int64_t rows, int k) {
  const int64_t bx = std::min<int64_t>((rows + 255) / 256, 64);
  return dim3((unsigned)(bx < 1 ? 1 : bx), (unsigned)k);
}

// defl-QR of the panel W (rows x k, ld rows; overwritten with residuals),
// whose original is Worig: the Gram-Schmidt columns go to Q (ld rows,
// columns 0..s-1) and R = Q^T Worig (s x k, ld s) to Rout.  pivot: the next
// column is the one of largest residual norm and the loop stops once that
// norm is below delta; otherwise the columns are taken in order (orth()),
// stopping at a zero residual.  Returns s.
template <typename T>
int defl_qr(Ctx &x, T *W, const T *Worig, int64_t rows, int k, double delta, bool pivot, T *Q,
            T *Rout) {
  std::vector<char> used(k, 0);
  int s = 0;
  for (int step = 0; step < k && x.e == cudaSuccess; ++step) {
    int j = step;
    if (pivot) {
      x.e = cudaMemsetAsync(x.dscr, 0, k * sizeof(double), x.s);
      col_dots_kernel<T><<<red_grid(rows, k), 256, 0, x.s>>>(W, rows, W, rows, rows, k, x.dscr);
      if (x.e == cudaSuccess) x.e = cudaGetLastError();
      if (!fetch(x, k)) break;
      j = -1;
      double best = -1.0;
      for (int c = 0; c < k; ++c)
        if (!used[c] && x.hscr[c] > best) {
          best = x.hscr[c];
          j = c;
        }
      if (j < 0 || !(sqrt(std::max(best, 0.0)) >= delta)) break;
    }
    used[j] = 1;
    T *q = Q + (int64_t)s * rows;
    x.e = cudaMemcpyAsync(q, W + (int64_t)j * rows, rows * sizeof(T), cudaMemcpyDeviceToDevice, x.s);
    if (s > 0 && x.e == cudaSuccess) {   // second pass against the columns kept so far
      x.e = cudaMemsetAsync(x.dscr, 0, s * sizeof(double), x.s);
      col_dot_vec_kernel<T><<<red_grid(rows, s), 256, 0, x.s>>>(Q, rows, q, rows, x.dscr);
      gemv_sub_kernel<T><<<agrid(rows), 256, 0, x.s>>>(q, Q, rows, s, x.dscr);
      if (x.e == cudaSuccess) x.e = cudaGetLastError();
    }
    if (x.e != cudaSuccess) break;
    x.e = cudaMemsetAsync(x.dscr, 0, sizeof(double), x.s);
    col_dots_kernel<T><<<red_grid(rows, 1), 256, 0, x.s>>>(q, rows, q, rows, rows, 1, x.dscr);
    if (x.e == cudaSuccess) x.e = cudaGetLastError();
    if (!fetch(x, 1)) break;
    const double nq = sqrt(x.hscr[0]);
    if (!(nq > 0)) break;
    scale_kernel<T><<<agrid(rows), 256, 0, x.s>>>(q, q, rows, 1.0 / nq);
    // remaining columns lose their component along q
    x.e = cudaMemsetAsync(x.dscr, 0, k * sizeof(double), x.s);
    col_dot_vec_kernel<T><<<red_grid(rows, k), 256, 0, x.s>>>(W, rows, q, rows, x.dscr);
    if (x.e == cudaSuccess) x.e = cudaGetLastError();
    rank1_kernel<T><<<agrid(rows * k), 256, 0, x.s>>>(W, rows, q, x.dscr, rows, k);
    if (x.e == cudaSuccess) x.e = cudaGetLastError();
    ++s;
  }
  if (s > 0 && x.e == cudaSuccess) {   // R = Q^T Worig (s x k, column-major, ld s)
    sg::GemmArgs g{};
    g.A = Q; g.ax = rows; g.ab = 1;           // Q^T: (i, b) at b + i rows
    g.B = Worig; g.bb = 1; g.by = rows;
    g.C = Rout; g.cx = 1; g.cy = s;
    g.X = s; g.Y = k; g.K = rows;
    x.e = sg::gemm<T>(g, 1, x.s);
  }
  return s;
}

// Sum of squares of the s x k matrix at R (host copy).
template <typename T>
double sumsq_host(Ctx &x, const T *R, int64_t count) {
  std::vector<T> h((size_t)count);
  if (count == 0 || x.e != cudaSuccess) return 0.0;
  x.e = cudaMemcpyAsync(h.data(), R, count * sizeof(T), cudaMemcpyDeviceToHost, x.s);
  if (x.e == cudaSuccess) x.e = cudaStreamSynchronize(x.s);
  double s = 0.0;
  for (const T &v : h) s += (double)v * (double)v;
  return s;
}

struct Mode {
  int mode;               // 1 or 2
  int64_t n, p1, p2;      // current core shape
  int64_t rows, cols;     // unfolding shape
};

// out (rows x k, ld rows) = A V for V (cols x k, ld ldv); tmp holds n rows k.
template <typename T>
cudaError_t unfold_times(const Mode &m, const T *C, const T *V, int64_t ldv, int k, T *tmp, T *out,
                         cudaStream_t s) {
  sg::GemmArgs g{};
  g.A = C;
  g.B = V;
  g.C = tmp;
  g.ao = m.p1 * m.p2;
  if (m.mode == 1) {   // C_j (p1 x p2) V_j (p2 x k), V_j at rows j p2
    g.ax = m.p2; g.ab = 1;
    g.bo = m.p2; g.bb = 1; g.by = ldv;
    g.co = m.p1 * k; g.cx = 1; g.cy = m.p1;
    g.X = m.p1; g.Y = k; g.K = m.p2;
  } else {             // C_j^T (p2 x p1) V_j (p1 x k), V_j at rows j p1
    g.ax = 1; g.ab = m.p2;
    g.bo = m.p1; g.bb = 1; g.by = ldv;
    g.co = m.p2 * k; g.cx = 1; g.cy = m.p2;
    g.X = m.p2; g.Y = k; g.K = m.p1;
  }
  cudaError_t e = sg::gemm<T>(g, m.n, s);
  if (e != cudaSuccess) return e;
  batch_sum_kernel<T><<<agrid(m.rows * k), 256, 0, s>>>(out, tmp, m.rows * k, m.n);
  return cudaGetLastError();
}

// out (cols x k, ld cols) = A^T U for U (rows x k, ld rows).
template <typename T>
cudaError_t unfold_t_times(const Mode &m, const T *C, const T *U, int k, T *out, cudaStream_t s) {
  sg::GemmArgs g{};
  g.A = C;
  g.B = U;
  g.C = out;
  g.ao = m.p1 * m.p2;
  g.bo = 0; g.bb = 1; g.by = m.rows;
  if (m.mode == 1) {   // (C_j^T U)[i2][c] at row j p2 + i2
    g.ax = 1; g.ab = m.p2;
    g.co = m.p2; g.cx = 1; g.cy = m.cols;
    g.X = m.p2; g.Y = k; g.K = m.p1;
  } else {             // (C_j U)[i1][c] at row j p1 + i1
    g.ax = m.p2; g.ab = 1;
    g.co = m.p1; g.cx = 1; g.cy = m.cols;
    g.X = m.p1; g.Y = k; g.K = m.p2;
  }
  return sg::gemm<T>(g, m.n, s);
}

// C (rows_a x k_c, ld lc) = A (rows_a x K, ld la) B (K x k_c, ld lb), one matrix.
template <typename T>
cudaError_t matmul(const T *A, int64_t la, const T *B, int64_t lb, T *C, int64_t lc, int64_t M,
                   int64_t N, int64_t K, bool transA, cudaStream_t s) {
  sg::GemmArgs g{};
  g.A = A; g.B = B; g.C = C;
  if (transA) { g.ax = la; g.ab = 1; }   // A^T: element (x, b) at b + x la
  else { g.ax = 1; g.ab = la; }          // A: element (x, b) at x + b la
  g.bb = 1; g.by = lb;
  g.cx = 1; g.cy = lc;
  g.X = M; g.Y = N; g.K = K;
  return sg::gemm<T>(g, 1, s);
}

template <typename T>
__global__ void sub_kernel(T *X, const T *__restrict__ Y, int64_t rows, int k, int64_t ldx,
                           int64_t ldy) {
  const int64_t total = rows * k;
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += step) {
    const int64_t r = e % rows;
    const int c = (int)(e / rows);
    X[r + c * ldx] -= Y[r + c * ldy];
  }
}

struct Panels {
  void *Ucat, *Vcat, *P, *P0, *Vn, *Vn0, *tmp, *X, *R, *Lt, *L, *G, *Gs;
};

// One mode: the factor F (rows x r) into Ucat; returns r, or -1 on error.
template <typename T>
int blbp_mode(Ctx &x, const Mode &m, const T *C, double eps, int b, double delta_rel, int64_t cap,
              int64_t capV, uint64_t seed, int t, const Panels &pn, char *err, size_t err_len,
              double *E_out) {
  cudaStream_t s = x.s;
  T *Ucat = (T *)pn.Ucat, *Vcat = (T *)pn.Vcat, *P = (T *)pn.P, *P0 = (T *)pn.P0;
  T *Vn = (T *)pn.Vn, *Vn0 = (T *)pn.Vn0, *tmp = (T *)pn.tmp, *X = (T *)pn.X;
  T *R = (T *)pn.R, *Lt = (T *)pn.Lt, *L = (T *)pn.L, *G = (T *)pn.G, *Gs = (T *)pn.Gs;
  const int64_t rows = m.rows, cols = m.cols;
  x.e = cudaMemsetAsync(x.dscr, 0, sizeof(double), s);
  sumsq_kernel<T><<<agrid(m.n * m.p1 * m.p2), 256, 0, s>>>(C, m.n * m.p1 * m.p2, x.dscr);
  if (!fetch(x, 1)) return -1;
  const double normA2 = x.hscr[0];
  const double delta = delta_rel * sqrt(normA2);
  double E = normA2;
  *E_out = 0.0;
  if (normA2 == 0.0) return 0;
  const uint32_t base = m.mode == 1 ? 0x10000u : 0x20000u;
  int draw = 0;
  const int64_t per = cols / m.n;   // rows of each slice's share of V
  auto gauss = [&](int k, T *dst) -> bool {   // dst (cols x k, ld cols)
    x.e = launch_gaussian_blocks(sizeof(T) == 8 ? TR_F64 : TR_F32, (int)m.n, per * k, Gs, seed, t,
                                 nullptr, base + 2u * (uint32_t)draw, s);
    ++draw;
    if (x.e != cudaSuccess) return false;
    gather_slices_kernel<T><<<agrid(cols * k), 256, 0, s>>>(dst, cols, Gs, m.n, per, k);
    x.e = cudaGetLastError();
    return x.e == cudaSuccess;
  };
  // V = orth(G): Gram-Schmidt of the first draw (all b columns kept)
  const int b0 = (int)std::min<int64_t>(b, cols);
  if (!gauss(b0, G)) return -1;
  x.e = cudaMemcpyAsync(Vn0, G, cols * b0 * sizeof(T), cudaMemcpyDeviceToDevice, s);
  int kv = defl_qr<T>(x, G, Vn0, cols, b0, 0.0, false, Vcat, R);
  if (x.e != cudaSuccess) return -1;
  int64_t vcols = kv, vstart = 0, ucols = 0, ustart = 0;
  int sprev = 0;       // columns of U_prev
  int lcols = 0;       // L is sprev x kv (ld sprev), first lcols columns nonzero
  while (true) {
    // P = A V - U_prev L
    x.e = unfold_times<T>(m, C, Vcat + vstart * cols, cols, kv, tmp, P, s);
    if (x.e == cudaSuccess && sprev > 0 && lcols > 0) {
      x.e = matmul<T>(Ucat + ustart * rows, rows, L, sprev, X, rows, rows, lcols, sprev, false, s);
      if (x.e == cudaSuccess) {
        sub_kernel<T><<<agrid(rows * lcols), 256, 0, s>>>(P, X, rows, lcols, rows, rows);
        x.e = cudaGetLastError();
      }
    }
    if (x.e != cudaSuccess) return -1;
    x.e = cudaMemcpyAsync(P0, P, rows * kv * sizeof(T), cudaMemcpyDeviceToDevice, s);
    const int su = defl_qr<T>(x, P, P0, rows, kv, delta, true, Ucat + ucols * rows, R);
    if (x.e != cudaSuccess) return -1;
    const int64_t uadd = su;
    E -= sumsq_host<T>(x, R, (int64_t)su * kv);
    // V' = A^T U - V R^T, then against V^{v}
    int sv = 0;
    if (su > 0) {
      x.e = unfold_t_times<T>(m, C, Ucat + ucols * rows, su, Vn, s);
      if (x.e != cudaSuccess) return -1;
      // X = V R^T (cols x su): R is su x kv (ld su), so R^T's (b, y) is R[y + b su]
      sg::GemmArgs g{};
      g.A = Vcat + vstart * cols; g.ax = 1; g.ab = cols;
      g.B = R; g.bb = su; g.by = 1;
      g.C = X; g.cx = 1; g.cy = cols;
      g.X = cols; g.Y = su; g.K = kv;
      x.e = sg::gemm<T>(g, 1, s);
      if (x.e == cudaSuccess) {
        sub_kernel<T><<<agrid(cols * su), 256, 0, s>>>(Vn, X, cols, su, cols, cols);
        x.e = cudaGetLastError();
      }
      // Vn -= Vcat (Vcat^T Vn)
      if (x.e == cudaSuccess)
        x.e = matmul<T>(Vcat, cols, Vn, cols, Lt, vcols, vcols, su, cols, true, s);   // Lt: coef
      if (x.e == cudaSuccess)
        x.e = matmul<T>(Vcat, cols, Lt, vcols, X, cols, cols, su, vcols, false, s);
      if (x.e == cudaSuccess) {
        sub_kernel<T><<<agrid(cols * su), 256, 0, s>>>(Vn, X, cols, su, cols, cols);
        x.e = cudaGetLastError();
      }
      if (x.e == cudaSuccess)
        x.e = cudaMemcpyAsync(Vn0, Vn, cols * su * sizeof(T), cudaMemcpyDeviceToDevice, s);
      if (x.e != cudaSuccess) return -1;
      if (vcols + su > capV)
        return afail(err, err_len, TR_EUNSUPPORTED, "V basis above %lld columns", (long long)capV),
               -2;
      sv = defl_qr<T>(x, Vn, Vn0, cols, su, delta, true, Vcat + vcols * cols, Lt);   // Lt: sv x su
      if (x.e != cudaSuccess) return -1;
      E -= sumsq_host<T>(x, Lt, (int64_t)sv * su);
    }
    const int64_t new_vstart = vcols;
    vcols += sv;
    // L = Lt^T (su x sv, ld su)
    if (sv > 0) {
      std::vector<T> h((size_t)sv * su), ht((size_t)su * sv);
      x.e = cudaMemcpyAsync(h.data(), Lt, h.size() * sizeof(T), cudaMemcpyDeviceToHost, s);
      if (x.e == cudaSuccess) x.e = cudaStreamSynchronize(s);
      for (int i = 0; i < sv; ++i)
        for (int c = 0; c < su; ++c) ht[c + (size_t)i * su] = h[i + (size_t)c * sv];
      if (x.e == cudaSuccess)
        x.e = cudaMemcpyAsync(L, ht.data(), ht.size() * sizeof(T), cudaMemcpyHostToDevice, s);
      if (x.e == cudaSuccess) x.e = cudaStreamSynchronize(s);
      if (x.e != cudaSuccess) return -1;
    }
    int knext = sv;
    if (sv < b && vcols < cols) {   // refill with Gaussian columns against V^{v}
      const int want = b - sv;
      if (!gauss(want, G)) return -1;
      x.e = matmul<T>(Vcat, cols, G, cols, X, vcols, vcols, want, cols, true, s);
      if (x.e == cudaSuccess) x.e = matmul<T>(Vcat, cols, X, vcols, Vn, cols, cols, want, vcols, false, s);
      if (x.e == cudaSuccess) {
        sub_kernel<T><<<agrid(cols * want), 256, 0, s>>>(G, Vn, cols, want, cols, cols);
        x.e = cudaGetLastError();
      }
      if (x.e == cudaSuccess)
        x.e = cudaMemcpyAsync(Vn0, G, cols * want * sizeof(T), cudaMemcpyDeviceToDevice, s);
      if (x.e != cudaSuccess) return -1;
      const int keep = (int)std::max<int64_t>(0, std::min<int64_t>(want, cols - vcols));
      if (vcols + want > capV)
        return afail(err, err_len, TR_EUNSUPPORTED, "V basis above %lld columns", (long long)capV),
               -2;
      int sr = defl_qr<T>(x, G, Vn0, cols, want, 0.0, false, Vcat + vcols * cols, X);
      if (x.e != cudaSuccess) return -1;
      sr = std::min(sr, keep);
      vcols += sr;
      knext += sr;
    }
    ucols += uadd;
    ustart = ucols - uadd;
    sprev = (int)uadd;
    lcols = sv;
    vstart = new_vstart;
    kv = knext;
    if (E < eps * eps * normA2 || ucols >= cap || kv == 0) break;
  }
  *E_out = E;
  return (int)std::min<int64_t>(ucols, cap);
}

// C' = C x_mode F^T: mode 1 C'_j = F^T C_j (r x p2); mode 2 C'_j = C_j F (p1 x r).
template <typename T>
cudaError_t truncate_core(const Mode &m, const T *C, const T *F, int64_t r, T *out, cudaStream_t s) {
  sg::GemmArgs g{};
  g.ao = m.p1 * m.p2;
  if (m.mode == 1) {
    g.A = F; g.ax = m.rows; g.ab = 1;                 // F^T: (a, i1) at i1 + a rows
    g.B = C; g.bo = m.p1 * m.p2; g.bb = m.p2; g.by = 1;
    g.C = out; g.co = r * m.p2; g.cx = m.p2; g.cy = 1;
    g.X = r; g.Y = m.p2; g.K = m.p1;
    g.ao = 0;
  } else {
    g.A = C; g.ax = m.p2; g.ab = 1;
    g.B = F; g.bb = 1; g.by = m.rows;                 // F: (i2, a) at i2 + a rows
    g.C = out; g.co = m.p1 * r; g.cx = r; g.cy = 1;
    g.X = m.p1; g.Y = r; g.K = m.p2;
  }
  return sg::gemm<T>(g, m.n, s);
}

template <typename T>
tr_status ad_tucker(tr_dtype dt, int n, int n1, int n2, const T *Abar, T *Gbar, double tau,
                    tr_penalty phi, double theta, double gamma, double eps, int b, double delta_rel,
                    int max_rank, uint64_t seed, int t, int *ranks, cudaStream_t s, char *err,
                    size_t err_len) {
  const size_t esz = sizeof(T);
  const int64_t N = (int64_t)n * n1 * n2;
  // sizes for the larger of the two modes
  const int64_t rows_max = std::max<int64_t>(n1, n2);
  const int64_t cols_max = (int64_t)n * std::max<int64_t>(n1, n2);
  const int64_t cap_max = std::min<int64_t>(rows_max, max_rank > 0 ? max_rank : rows_max);
  // V basis columns: the loop keeps at most about cols of them (a capped run
  // about b (cap + 4)), and the block being appended may pass that by b
  // before deflation trims it
  const int64_t capV = std::min<int64_t>(cols_max, (int64_t)b * (cap_max + 4)) + b;
  std::vector<void *> allocs;
  cudaError_t e = cudaSuccess;
  auto alloc = [&](size_t bytes) -> void * {
    void *p = nullptr;
    if (e == cudaSuccess) e = cudaMallocAsync(&p, std::max<size_t>(bytes, 16), s);
    if (p) allocs.push_back(p);
    return p;
  };
  Panels pn{};
  pn.Ucat = alloc(rows_max * (cap_max + b) * esz);   // a last block may pass the cap
  pn.Vcat = alloc(cols_max * capV * esz);
  pn.P = alloc(rows_max * b * esz);
  pn.P0 = alloc(rows_max * b * esz);
  pn.Vn = alloc(cols_max * b * esz);
  pn.Vn0 = alloc(cols_max * b * esz);
  pn.tmp = alloc((size_t)n * rows_max * b * esz);
  pn.X = alloc(std::max<int64_t>(cols_max, rows_max) * std::max<int64_t>(b, capV) * esz);
  pn.R = alloc((size_t)b * b * esz);
  pn.Lt = alloc(std::max<int64_t>((int64_t)b * b, capV * b) * esz);
  pn.L = alloc((size_t)b * b * esz);
  pn.G = alloc(cols_max * b * esz);
  pn.Gs = alloc(cols_max * b * esz);
  void *F1 = alloc(n1 * cap_max * esz), *C1 = alloc(N * esz), *C2 = alloc(N * esz);
  void *Ct = alloc(N * esz), *Tb = alloc(N * esz);
  double *dscr = (double *)alloc(64 * sizeof(double));
  std::vector<double> hscr(64);
  tr_status st = TR_OK;
  auto finish = [&](tr_status r) {
    for (void *p : allocs) cudaFreeAsync(p, s);
    return r;
  };
  if (e != cudaSuccess)
    return finish(afail(err, err_len, e == cudaErrorMemoryAllocation ? TR_ENOMEM : TR_ECUDA,
                        "workspace: %s", cudaGetErrorString(e)));
  Ctx x{s, dscr, hscr.data()};
  double E1 = 0.0, E2 = 0.0;
  // mode 1 on Abar
  Mode m1{1, n, n1, n2, n1, (int64_t)n * n2};
  const int64_t cap1 = std::min<int64_t>(std::min<int64_t>(m1.rows, m1.cols),
                                         max_rank > 0 ? max_rank : m1.rows);
  int r1 = blbp_mode<T>(x, m1, Abar, eps, b, delta_rel, cap1, capV, seed, t, pn, err, err_len, &E1);
  if (r1 == -2) return finish(TR_EUNSUPPORTED);
  if (r1 < 0 || x.e != cudaSuccess)
    return finish(afail(err, err_len, TR_ECUDA, "mode 1: %s", cudaGetErrorString(x.e)));
  if (r1 == 0) {
    e = cudaMemsetAsync(Gbar, 0, N * esz, s);
    if (ranks) ranks[0] = ranks[1] = 0;
    return finish(e == cudaSuccess ? TR_OK : TR_ECUDA);
  }
  e = cudaMemcpyAsync(F1, pn.Ucat, n1 * r1 * esz, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = launch_canon_signs(dt, F1, n1, r1, s);
  if (e == cudaSuccess) e = truncate_core<T>(m1, Abar, (const T *)F1, r1, (T *)C1, s);
  // mode 2 on the core (n x r1 x n2)
  Mode m2{2, n, r1, n2, n2, (int64_t)n * r1};
  const int64_t cap2 = std::min<int64_t>(std::min<int64_t>(m2.rows, m2.cols),
                                         max_rank > 0 ? max_rank : m2.rows);
  int r2 = e == cudaSuccess ? blbp_mode<T>(x, m2, (const T *)C1, eps, b, delta_rel, cap2, capV,
                                           seed, t, pn, err, err_len, &E2)
                            : -1;
  if (r2 == -2) return finish(TR_EUNSUPPORTED);
  if (r2 < 0 || x.e != cudaSuccess || e != cudaSuccess)
    return finish(afail(err, err_len, TR_ECUDA, "mode 2: %s",
                        cudaGetErrorString(x.e != cudaSuccess ? x.e : e)));
  if (ranks) {
    ranks[0] = r1;
    ranks[1] = r2;
  }
  if (r2 == 0) {
    e = cudaMemsetAsync(Gbar, 0, N * esz, s);
    return finish(e == cudaSuccess ? TR_OK : TR_ECUDA);
  }
  const T *F2 = (const T *)pn.Ucat;
  e = launch_canon_signs(dt, pn.Ucat, n2, r2, s);
  if (e == cudaSuccess) e = truncate_core<T>(m2, (const T *)C1, F2, r2, (T *)C2, s);
  // the core's prox at full width (exact): slices r1 x r2, on workspace of
  // this call's own (sketch, two panels, singular values, ranks)
  if (e == cudaSuccess) {
    const int l = std::min(r1, r2);
    if (l > TR_MAX_L || !slice_smem_limit_ok(dt, r1, r2, l))
      return finish(afail(err, err_len, TR_EUNSUPPORTED,
                          "core slices of %dx%d exceed the slice kernels' shared memory", r1, r2));
    SliceWork w{};
    w.n = n;
    w.n1 = r1;
    w.n2 = r2;
    w.l = l;
    w.q = 1;
    w.seed = seed;
    w.Om = alloc((size_t)n * r2 * l * esz);
    w.P1 = alloc((size_t)n * r1 * l * esz);
    w.P2 = alloc((size_t)n * r2 * l * esz);
    w.sig = alloc((size_t)n * l * esz);
    w.rank = (int *)alloc((size_t)n * sizeof(int));
    if (e != cudaSuccess)
      return finish(afail(err, err_len, e == cudaErrorMemoryAllocation ? TR_ENOMEM : TR_ECUDA,
                          "core workspace: %s", cudaGetErrorString(e)));
    ShrinkScalars sh{tau, (int)phi, theta, gamma};
    e = launch_slice_rsvd(dt, w, C2, Ct, sh, t, s);
  }
  // Gbar_j = F1 Ct_j F2^T: T_j = Ct_j F2^T (r1 x n2), then F1 T_j
  if (e == cudaSuccess) {
    sg::GemmArgs g{};
    g.A = Ct; g.ao = (int64_t)r1 * r2; g.ax = r2; g.ab = 1;
    g.B = F2; g.bb = n2; g.by = 1;                   // F2^T: (c, i2) at i2 + c n2
    g.C = Tb; g.co = (int64_t)r1 * n2; g.cx = n2; g.cy = 1;
    g.X = r1; g.Y = n2; g.K = r2;
    e = sg::gemm<T>(g, n, s);
  }
  if (e == cudaSuccess) {
    sg::GemmArgs g{};
    g.A = F1; g.ax = 1; g.ab = n1;                   // F1: (i1, a) at i1 + a n1
    g.B = Tb; g.bo = (int64_t)r1 * n2; g.bb = n2; g.by = 1;
    g.C = Gbar; g.co = (int64_t)n1 * n2; g.cx = n2; g.cy = 1;
    g.X = n1; g.Y = n2; g.K = r1;
    e = sg::gemm<T>(g, n, s);
  }
  if (e != cudaSuccess) return finish(afail(err, err_len, TR_ECUDA, "%s", cudaGetErrorString(e)));
  return finish(TR_OK);
}

}  // namespace

extern "C" tr_status tr_slice_prox_ad_tucker(tr_dtype dtype, int n, int n1, int n2,
                                             const void *Abar, void *Gbar, double tau,
                                             tr_penalty phi, double theta, double gamma, double eps,
                                             int b, double delta_rel, int max_rank, uint64_t seed,
                                             int t, int *ranks, void *cuda_stream, char *err,
                                             size_t err_len) {
  if (err && err_len) err[0] = 0;
  if (dtype != TR_F32 && dtype != TR_F64) return afail(err, err_len, TR_EINVAL, "bad dtype");
  if (n < 1 || n1 < 1 || n2 < 1 || b < 1 || b > 32 || t < 0 || !(tau >= 0) || !(eps > 0) ||
      !(delta_rel >= 0) || max_rank < 0)
    return afail(err, err_len, TR_EINVAL,
                 "need n, n1, n2 >= 1, 1 <= b <= 32, t >= 0, tau >= 0, eps > 0, delta_rel >= 0");
  if (!Abar || !Gbar || Abar == Gbar)
    return afail(err, err_len, TR_EINVAL, "Abar and Gbar must be distinct device pointers");
  if (phi != TR_PEN_L1 && phi != TR_PEN_MCP) return afail(err, err_len, TR_EINVAL, "bad penalty");
  if (n > 65535) return afail(err, err_len, TR_EUNSUPPORTED, "at most 65535 slices per call");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (dtype == TR_F32)
    return ad_tucker<float>(dtype, n, n1, n2, (const float *)Abar, (float *)Gbar, tau, phi, theta,
                            gamma, eps, b, delta_rel, max_rank, seed, t, ranks, s, err, err_len);
  return ad_tucker<double>(dtype, n, n1, n2, (const double *)Abar, (double *)Gbar, tau, phi, theta,
                           gamma, eps, b, delta_rel, max_rank, seed, t, ranks, s, err, err_len);
}
