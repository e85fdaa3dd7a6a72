// Building blocks of the gradient-domain prior (Def. gradient tensor,
// Eq. coef-tensor, Eq. gnrhtc-L): the difference operator nabla_k, its
// adjoint, and the solve of (I + sum_{k in Gamma} nabla_k^T nabla_k) X = R.
//
// Layout: the face-slice stack of an order-d tensor, flat index
// f = (j n1 + i1) n2 + i2 with j = i3 + n3 (i4 + n4 (...)).  Mode k then has
// the flat stride S_1 = n2, S_2 = 1, S_k = n1 n2 n3 ... n_{k-1} (k >= 3), and
// the coordinate i_k = (f / S_k) mod n_k.
//
// nabla_k(X) = X x_k D_{n_k}, D_n the row circulant of (-1, 1, 0, ..., 0):
// a periodic forward difference along mode k; nabla_k^T the periodic
// backward difference x_{i-1} - x_i.
//
// The solve.  nabla_k^T nabla_k is a symmetric circulant along mode k.  The
// real Hartley matrix H_n[a][b] = cas(2 pi a b / n) / sqrt(n), cas = cos + sin,
// is symmetric, orthogonal and its own inverse, and it diagonalises every
// symmetric circulant of size n; the eigenvalue of D_n^T D_n at index a is
// 2 - 2 cos(2 pi a / n).  So
//     X = (prod_k H_k) diag(1 / (1 + sum_k lambda_k)) (prod_k H_k) R,
// the mode products taken along every k in Gamma.  This equals the FFT form
// of Eq. gnrhtc-L in real arithmetic.  Each mode product is a batched GEMM:
// for k != 2, out[o][a][c] = sum_b H[a][b] in[o][b][c] with c < S_k; for the
// contiguous mode 2, out[r][a] = sum_b in[r][b] H[b][a].

#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include <mutex>
#include <vector>

#include "sgemm.cuh"
#include "tr_internal.cuh"

namespace {

tr_status gfail(char *buf, size_t len, tr_status st, const char *fmt, ...) {
  if (buf && len) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, len, fmt, ap);
    va_end(ap);
  }
  return st;
}

constexpr int kGradMaxMode = 2048;   // largest mode size of the solve (H is n x n)

struct Shape {
  int order;
  int64_t n[8];      // n1, n2, n3, ...
  int64_t S[8];      // flat stride of each mode
  int64_t N;
};

bool make_shape(int order, const int64_t *dims, Shape &s) {
  if (order < 2 || order > 8 || !dims) return false;
  s.order = order;
  s.N = 1;
  for (int k = 0; k < order; ++k) {
    if (dims[k] < 1 || dims[k] > (int64_t(1) << 31)) return false;
    s.n[k] = dims[k];
    if (s.N > (int64_t(1) << 40) / dims[k]) return false;
    s.N *= dims[k];
  }
  s.S[0] = s.n[1];
  s.S[1] = 1;
  int64_t stride = s.n[0] * s.n[1];
  for (int k = 2; k < order; ++k) {
    s.S[k] = stride;
    stride *= s.n[k];
  }
  return true;
}

// dst[f] = src[f'] - src[f], f' the periodic neighbour of f along the mode
// (forward: i_k + 1; adjoint: i_k - 1).
template <typename T>
__global__ void grad_kernel(const T *__restrict__ src, T *__restrict__ dst, int64_t N, int64_t S,
                            int64_t nk, int adjoint) {
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < N; f += step) {
    const int64_t i = (f / S) % nk;
    int64_t g;
    if (!adjoint)
      g = (i == nk - 1) ? f - (nk - 1) * S : f + S;
    else
      g = (i == 0) ? f + (nk - 1) * S : f - S;
    dst[f] = src[g] - src[f];
  }
}

// X[f] /= 1 + sum over the modes in Gamma of lambda_k[i_k].
struct ScaleModes {
  int count;
  int64_t S[8], n[8];           // stride and size of each mode
  const void *lam[8];           // its eigenvalue table (n entries)
};

template <typename T>
__global__ void eig_scale_kernel(T *X, int64_t N, ScaleModes m) {
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < N; f += step) {
    T den = T(1);
    for (int q = 0; q < m.count; ++q) den += ((const T *)m.lam[q])[(f / m.S[q]) % m.n[q]];
    X[f] = X[f] / den;
  }
}

// The Hartley matrix H_n (n x n, row-major) followed by the eigenvalues
// 2 - 2 cos(2 pi a / n) of D_n^T D_n, computed in double, stored as T.
template <typename T>
void hartley_tables(int64_t n, T *out) {
  const double two_pi = 6.283185307179586476925286766559;
  const double inv_sqrt = 1.0 / sqrt((double)n);
  for (int64_t a = 0; a < n; ++a) {
    for (int64_t b = 0; b < n; ++b) {
      const double ang = two_pi * (double)((a * b) % n) / (double)n;
      out[a * n + b] = (T)((cos(ang) + sin(ang)) * inv_sqrt);
    }
    out[n * n + a] = (T)(2.0 - 2.0 * cos(two_pi * (double)a / (double)n));
  }
}

// Device copies of the tables, built once per (device, element size, n) and
// kept until the process exits (at most kTableCacheEntries of them; later
// sizes are built per call).
struct TableEntry {
  int dev;
  size_t esz;
  int64_t n;
  void *ptr;
};
constexpr int kTableCacheEntries = 32;
std::mutex g_table_mu;
TableEntry g_tables[kTableCacheEntries];
int g_table_count = 0;

template <typename T>
const T *cached_tables(int64_t n) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lock(g_table_mu);
  for (int i = 0; i < g_table_count; ++i)
    if (g_tables[i].dev == dev && g_tables[i].esz == sizeof(T) && g_tables[i].n == n)
      return (const T *)g_tables[i].ptr;
  if (g_table_count == kTableCacheEntries) return nullptr;
  std::vector<T> host((size_t)(n * n + n));
  hartley_tables<T>(n, host.data());
  void *d = nullptr;
  if (cudaMalloc(&d, host.size() * sizeof(T)) != cudaSuccess) return nullptr;
  if (cudaMemcpy(d, host.data(), host.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(d);
    return nullptr;
  }
  g_tables[g_table_count++] = TableEntry{dev, sizeof(T), n, d};
  return (const T *)d;
}

int grid_for(int64_t N) {
  const int64_t blocks = (N + 255) / 256;
  return (int)(blocks < 152 * 32 ? (blocks < 1 ? 1 : blocks) : 152 * 32);
}

// One Hartley mode product dst = H_k x_k src (H at Hdev, n_k x n_k row-major).
template <typename T>
cudaError_t hartley_product(const Shape &s, int k, const T *Hdev, const T *src, T *dst,
                            cudaStream_t st) {
  const int64_t m = s.n[k], S = s.S[k];
  sg::GemmArgs g;
  dim3 grid;
  if (k == 1) {   // mode 2, contiguous: out[r][a] = sum_b in[r][b] H[b][a]
    g = sg::GemmArgs{src, Hdev, dst, 0, m, 1, 0, m, 1, 0, m, 1, s.N / m, m, m};
    grid = dim3((unsigned)((g.Y + sg::kBY - 1) / sg::kBY), (unsigned)((g.X + sg::kBX - 1) / sg::kBX), 1);
  } else {        // out[o][a][c] = sum_b H[a][b] in[o][b][c]
    g = sg::GemmArgs{Hdev, src, dst, 0, m, 1, m * S, S, 1, m * S, S, 1, m, S, m};
    grid = dim3((unsigned)((g.Y + sg::kBY - 1) / sg::kBY), (unsigned)((g.X + sg::kBX - 1) / sg::kBX),
                (unsigned)(s.N / (m * S)));
  }
  sg::strided_gemm_kernel<T><<<grid, sg::kGemmThreads, 0, st>>>(g);
  return cudaGetLastError();
}

// Grid limits of every product of the solve (blocks in y and z <= 65535).
bool solve_grid_ok(const Shape &s, uint32_t modes) {
  for (int k = 0; k < s.order; ++k) {
    if (!(modes & (1u << k))) continue;
    const int64_t m = s.n[k], S = s.S[k];
    if (k == 1) {
      if ((s.N / m + sg::kBX - 1) / sg::kBX > 65535) return false;
    } else {
      if ((m + sg::kBX - 1) / sg::kBX > 65535 || s.N / (m * S) > 65535) return false;
      if ((S + sg::kBY - 1) / sg::kBY > 0x7fffffff) return false;
    }
  }
  return true;
}

template <typename T>
tr_status gradient_solve(const Shape &s, uint32_t modes, const T *rhs, T *out, cudaStream_t st,
                         char *err, size_t err_len) {
  int ks[8], nm = 0;
  for (int k = 0; k < s.order; ++k)
    if (modes & (1u << k)) ks[nm++] = k;
  const size_t esz = sizeof(T);
  if (nm == 0) {
    const cudaError_t e = cudaMemcpyAsync(out, rhs, (size_t)s.N * esz, cudaMemcpyDeviceToDevice, st);
    return e == cudaSuccess ? TR_OK : gfail(err, err_len, TR_ECUDA, "%s", cudaGetErrorString(e));
  }
  // per mode: its cached tables, or tables built for this call
  const T *tab[8];
  size_t own_off[8], own_total = 0;
  for (int q = 0; q < nm; ++q) {
    const int64_t n = s.n[ks[q]];
    tab[q] = cached_tables<T>(n);
    own_off[q] = own_total;
    if (!tab[q]) own_total += (size_t)(n * n + n);
  }
  void *own = nullptr, *tmp = nullptr;
  cudaError_t e = cudaSuccess;
  if (own_total) e = cudaMallocAsync(&own, own_total * esz, st);
  if (e == cudaSuccess) e = cudaMallocAsync(&tmp, (size_t)s.N * esz, st);
  if (e != cudaSuccess) {
    if (own) cudaFreeAsync(own, st);
    return gfail(err, err_len, e == cudaErrorMemoryAllocation ? TR_ENOMEM : TR_ECUDA,
                 "workspace: %s", cudaGetErrorString(e));
  }
  std::vector<T> host(own_total);
  for (int q = 0; q < nm; ++q) {
    if (tab[q]) continue;
    hartley_tables<T>(s.n[ks[q]], host.data() + own_off[q]);
    tab[q] = (const T *)own + own_off[q];
  }
  // pageable source: the call returns once the host buffer has been staged
  if (own_total) e = cudaMemcpyAsync(own, host.data(), own_total * esz, cudaMemcpyHostToDevice, st);
  T *buf[2] = {(T *)tmp, out};    // product p (0-based) writes buf[p % 2]; 2 nm products end in out
  const T *cur = rhs;
  int p = 0;
  for (int q = 0; q < nm && e == cudaSuccess; ++q, ++p) {
    e = hartley_product<T>(s, ks[q], tab[q], cur, buf[p % 2], st);
    cur = buf[p % 2];
  }
  if (e == cudaSuccess) {
    ScaleModes sm{};
    sm.count = nm;
    for (int q = 0; q < nm; ++q) {
      sm.S[q] = s.S[ks[q]];
      sm.n[q] = s.n[ks[q]];
      sm.lam[q] = tab[q] + s.n[ks[q]] * s.n[ks[q]];
    }
    eig_scale_kernel<T><<<grid_for(s.N), 256, 0, st>>>((T *)cur, s.N, sm);
    e = cudaGetLastError();
  }
  for (int q = 0; q < nm && e == cudaSuccess; ++q, ++p) {
    e = hartley_product<T>(s, ks[q], tab[q], cur, buf[p % 2], st);
    cur = buf[p % 2];
  }
  cudaFreeAsync(tmp, st);
  if (own) cudaFreeAsync(own, st);
  if (e != cudaSuccess) return gfail(err, err_len, TR_ECUDA, "%s", cudaGetErrorString(e));
  return TR_OK;
}

}  // namespace

extern "C" tr_status tr_grad(tr_dtype dtype, int order, const int64_t *dims, int mode, int adjoint,
                             const void *src, void *dst, void *cuda_stream, char *err,
                             size_t err_len) {
  if (err && err_len) err[0] = 0;
  Shape s;
  if (dtype != TR_F32 && dtype != TR_F64) return gfail(err, err_len, TR_EINVAL, "bad dtype");
  if (!make_shape(order, dims, s)) return gfail(err, err_len, TR_EINVAL, "bad order or dims");
  if (mode < 1 || mode > order) return gfail(err, err_len, TR_EINVAL, "mode must be in 1..order");
  if (!src || !dst || src == dst)
    return gfail(err, err_len, TR_EINVAL, "src and dst must be distinct device pointers");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int64_t S = s.S[mode - 1], nk = s.n[mode - 1];
  if (dtype == TR_F32)
    grad_kernel<float><<<grid_for(s.N), 256, 0, st>>>((const float *)src, (float *)dst, s.N, S, nk,
                                                      adjoint ? 1 : 0);
  else
    grad_kernel<double><<<grid_for(s.N), 256, 0, st>>>((const double *)src, (double *)dst, s.N, S,
                                                       nk, adjoint ? 1 : 0);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? TR_OK : gfail(err, err_len, TR_ECUDA, "%s", cudaGetErrorString(e));
}

extern "C" tr_status tr_gradient_solve(tr_dtype dtype, int order, const int64_t *dims,
                                       uint32_t modes, const void *rhs, void *out,
                                       void *cuda_stream, char *err, size_t err_len) {
  if (err && err_len) err[0] = 0;
  Shape s;
  if (dtype != TR_F32 && dtype != TR_F64) return gfail(err, err_len, TR_EINVAL, "bad dtype");
  if (!make_shape(order, dims, s)) return gfail(err, err_len, TR_EINVAL, "bad order or dims");
  if (modes >> order) return gfail(err, err_len, TR_EINVAL, "modes names a mode beyond the order");
  if (!rhs || !out || rhs == out)
    return gfail(err, err_len, TR_EINVAL, "rhs and out must be distinct device pointers");
  for (int k = 0; k < order; ++k)
    if ((modes & (1u << k)) && s.n[k] > kGradMaxMode)
      return gfail(err, err_len, TR_EUNSUPPORTED, "mode %d has size %lld > %d", k + 1,
                   (long long)s.n[k], kGradMaxMode);
  if (!solve_grid_ok(s, modes))
    return gfail(err, err_len, TR_EUNSUPPORTED, "tensor too large for one launch per product");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (dtype == TR_F32)
    return gradient_solve<float>(s, modes, (const float *)rhs, (float *)out, st, err, err_len);
  return gradient_solve<double>(s, modes, (const double *)rhs, (double *)out, st, err, err_len);
}
