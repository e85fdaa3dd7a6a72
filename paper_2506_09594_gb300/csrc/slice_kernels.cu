// Slice pass: the per-transformed-face-slice randomized low-rank prox inside
// GNHTSVT (Alg. 4; sketch and power steps as in Alg. 1, applied per slice).
// For every slice Abar^<j> (n1 x n2, row-major):
//   Y = Abar Omega                      Gaussian sketch, Omega n2 x l
//   q times: Q = qr(Y); W = qr(Abar^T Q); Y = Abar W
//   Q = qr(Y);  B^T = Abar^T Q           (B = Q^T Abar, l x n2)
//   B^T = Qb R;  R = Ur S Vr^T           (QR, then one-sided Jacobi SVD of R)
//   C = Vr diag(Prox_{Phi,tau}(S)) Ur^T  (l x l)
//   Gbar^<j> = (Q C) Qb^T               = Q Uhat diag(prox(S)) V^T of B
// Panels (n x l) live column-major in global workspace; the small l x l
// factors live in shared memory.
//
// The Gaussian sketch uses Philox4x32-10 (Salmon et al., SC'11) with counter
// (m/4, j, t, stream) and key (seed lo, seed hi), Box-Muller (1958) on word
// pairs, element m = c*n2 + k of the column-major n2 x l sketch taking
// output m mod 4.

#include <float.h>
#include <math.h>

#include "tr_internal.cuh"

namespace {

// ---------------------------------------------------------------- Philox
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t hi_a = __umulhi(0xD2511F53u, c[0]), lo_a = 0xD2511F53u * c[0];
    const uint32_t hi_b = __umulhi(0xCD9E8D57u, c[2]), lo_b = 0xCD9E8D57u * c[2];
    const uint32_t n0 = hi_b ^ c[1] ^ k0, n2 = hi_a ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo_b;
    c[2] = n2;
    c[3] = lo_a;
  }
}

__device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, float &z0, float &z1) {
  const float u1 = ((float)a + 0.5f) * 2.3283064365386963e-10f;   // (a + 1/2) / 2^32
  const float u2 = ((float)b + 0.5f) * 2.3283064365386963e-10f;
  const float r = sqrtf(-2.0f * logf(u1));
  float s, c;
  sincospif(2.0f * u2, &s, &c);
  z0 = r * c;
  z1 = r * s;
}

__device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, double &z0, double &z1) {
  const double u1 = ((double)a + 0.5) * 2.3283064365386963e-10;
  const double u2 = ((double)b + 0.5) * 2.3283064365386963e-10;
  const double r = sqrt(-2.0 * log(u1));
  double s, c;
  sincospi(2.0 * u2, &s, &c);
  z0 = r * c;
  z1 = r * s;
}

template <typename T>
__global__ void sketch_kernel(int64_t per_slice, T *__restrict__ Om, uint32_t k0, uint32_t k1,
                              uint32_t t, uint32_t stream) {
  const int j = blockIdx.y;
  const int64_t ngroups = (per_slice + 3) / 4;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ngroups;
       g += (int64_t)gridDim.x * blockDim.x) {
    uint32_t c[4] = {(uint32_t)g, (uint32_t)j, t, stream};
    philox4x32_10(c, k0, k1);
    T z[4];
    box_muller(c[0], c[1], z[0], z[1]);
    box_muller(c[2], c[3], z[2], z[3]);
    T *dst = Om + (int64_t)j * per_slice;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int64_t m = 4 * g + i;
      if (m < per_slice) dst[m] = z[i];
    }
  }
}

// ------------------------------------------------------ batched SIMT GEMM
// C[b](M x N) = A[b](M x K) B[b](K x N) with element strides, so transposes
// and column/row-major operands are expressed by the strides alone.
struct GemmArgs {
  int M, N, K;
  const void *A;
  int64_t sAb, sAi, sAk;
  const void *B;
  int64_t sBb, sBk, sBn;
  void *C;
  int64_t sCb, sCi, sCn;
};

template <typename T, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
bgemm_kernel(GemmArgs g) {
  constexpr int NT = (BM / TM) * (BN / TN);
  __shared__ __align__(16) T As[BK][BM + 4];
  __shared__ __align__(16) T Bs[BK][BN + 4];
  const int tid = threadIdx.x;
  const int tx = tid % (BN / TN), ty = tid / (BN / TN);
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int64_t b = blockIdx.z;
  const T *A = (const T *)g.A + b * g.sAb;
  const T *B = (const T *)g.B + b * g.sBb;
  T *C = (T *)g.C + b * g.sCb;
  const bool a_kc = g.sAk == 1;
  const bool b_nc = g.sBn == 1;
  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int jn = 0; jn < TN; ++jn) acc[i][jn] = T(0);

  // Register prefetch: the next K-tile is loaded from global memory while the
  // current one is multiplied out of shared memory.
  constexpr int NA = (BM * BK + NT - 1) / NT, NB = (BK * BN + NT - 1) / NT;
  T ra[NA], rb[NB];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int r = 0; r < NA; ++r) {
      const int e = tid + r * NT;
      int i, k;
      if (a_kc) { i = e / BK; k = e % BK; } else { i = e % BM; k = e / BM; }
      const int gi = m0 + i, gk = k0 + k;
      ra[r] = (e < BM * BK && gi < g.M && gk < g.K) ? A[gi * g.sAi + gk * g.sAk] : T(0);
    }
#pragma unroll
    for (int r = 0; r < NB; ++r) {
      const int e = tid + r * NT;
      int k, nn;
      if (b_nc) { k = e / BN; nn = e % BN; } else { k = e % BK; nn = e / BK; }
      const int gk = k0 + k, gn = n0 + nn;
      rb[r] = (e < BK * BN && gk < g.K && gn < g.N) ? B[gk * g.sBk + gn * g.sBn] : T(0);
    }
  };
  auto stash = [&]() {
#pragma unroll
    for (int r = 0; r < NA; ++r) {
      const int e = tid + r * NT;
      if (e >= BM * BK) break;
      int i, k;
      if (a_kc) { i = e / BK; k = e % BK; } else { i = e % BM; k = e / BM; }
      As[k][i] = ra[r];
    }
#pragma unroll
    for (int r = 0; r < NB; ++r) {
      const int e = tid + r * NT;
      if (e >= BK * BN) break;
      int k, nn;
      if (b_nc) { k = e / BN; nn = e % BN; } else { k = e % BK; nn = e / BK; }
      Bs[k][nn] = rb[r];
    }
  };
  fetch(0);
  for (int k0 = 0; k0 < g.K; k0 += BK) {
    __syncthreads();
    stash();
    __syncthreads();
    if (k0 + BK < g.K) fetch(k0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[TM], bb[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty * TM + i];
#pragma unroll
      for (int jn = 0; jn < TN; ++jn) bb[jn] = Bs[kk][tx * TN + jn];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int jn = 0; jn < TN; ++jn) acc[i][jn] = fma(a[i], bb[jn], acc[i][jn]);
    }
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int row = m0 + ty * TM + i;
    if (row >= g.M) continue;
#pragma unroll
    for (int jn = 0; jn < TN; ++jn) {
      const int col = n0 + tx * TN + jn;
      if (col < g.N) C[row * g.sCi + col * g.sCn] = acc[i][jn];
    }
  }
}

template <typename T>
cudaError_t bgemm(const GemmArgs &g, int batch, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0 || batch <= 0) return cudaSuccess;
  if (g.N <= 32) {
    dim3 grid((g.M + 63) / 64, (g.N + 31) / 32, batch);
    bgemm_kernel<T, 64, 32, 32, 4, 2><<<grid, 256, 0, s>>>(g);
  } else {
    dim3 grid((g.M + 63) / 64, (g.N + 63) / 64, batch);
    bgemm_kernel<T, 64, 64, 16, 4, 4><<<grid, 256, 0, s>>>(g);
  }
  return cudaGetLastError();
}

// -------------------------------------------------- block Householder QR
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// In-place Householder QR of the m x l panel P (column-major, leading dim
// ld, l <= m) in shared memory.  Reflector k is H_k = I - tau_k v v^T with
// v = (1, P[k+1:m, k]); R is left in the upper triangle (LAPACK geqr2
// convention: H_k x = beta e_1, beta = -sign(x_0) ||x||).
template <typename T>
__device__ void block_qr_factor(T *P, int m, int l, int ld, T *tau) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int k = 0; k < l; ++k) {
    if (warp == 0) {
      T *col = P + (size_t)k * ld;
      T ss = T(0);
      for (int i = k + 1 + lane; i < m; i += 32) ss = fma(col[i], col[i], ss);
      ss = warp_sum(ss);
      const T x0 = col[k];
      T beta = x0, tk = T(0), scale = T(0);
      if (ss > T(0)) {
        const T nrm = sqrt(fma(x0, x0, ss));
        beta = x0 >= T(0) ? -nrm : nrm;
        tk = (beta - x0) / beta;
        scale = T(1) / (x0 - beta);
      }
      __syncwarp();
      for (int i = k + 1 + lane; i < m; i += 32) col[i] *= scale;
      if (lane == 0) {
        col[k] = beta;
        tau[k] = tk;
      }
    }
    __syncthreads();
    const T tk = tau[k];
    const T *v = P + (size_t)k * ld;
    for (int c = k + 1 + warp; c < l; c += nw) {
      T *col = P + (size_t)c * ld;
      const T ck = col[k];
      T s = T(0);
      for (int i = k + 1 + lane; i < m; i += 32) s = fma(v[i], col[i], s);
      s = warp_sum(s) + ck;
      const T w = tk * s;
      for (int i = k + 1 + lane; i < m; i += 32) col[i] = fma(-w, v[i], col[i]);
      if (lane == 0) col[k] = ck - w;
    }
    __syncthreads();
  }
}

// Overwrite the factored panel with the thin Q = H_0 ... H_{l-1} [I; 0]
// (LAPACK org2r order: backwards, each column formed after its trailing
// columns).
template <typename T>
__device__ void block_qr_form_q(T *P, int m, int l, int ld, const T *tau) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int k = l - 1; k >= 0; --k) {
    const T tk = tau[k];
    const T *v = P + (size_t)k * ld;
    for (int c = k + 1 + warp; c < l; c += nw) {
      T *col = P + (size_t)c * ld;
      const T ck = col[k];
      T s = T(0);
      for (int i = k + 1 + lane; i < m; i += 32) s = fma(v[i], col[i], s);
      s = warp_sum(s) + ck;
      const T w = tk * s;
      for (int i = k + 1 + lane; i < m; i += 32) col[i] = fma(-w, v[i], col[i]);
      if (lane == 0) col[k] = ck - w;
    }
    __syncthreads();
    T *colk = P + (size_t)k * ld;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      if (i < k) colk[i] = T(0);
      else if (i == k) colk[i] = T(1) - tk;
      else colk[i] = -tk * colk[i];
    }
    __syncthreads();
  }
}

template <typename T>
__global__ void qr_kernel(int m, int l, T *__restrict__ P, int64_t sP) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *panel = reinterpret_cast<T *>(smem_raw);
  T *tau = panel + (size_t)m * l;
  T *Pj = P + (int64_t)blockIdx.x * sP;
  for (int e = threadIdx.x; e < m * l; e += blockDim.x) panel[e] = Pj[e];
  __syncthreads();
  block_qr_factor(panel, m, l, m, tau);
  block_qr_form_q(panel, m, l, m, tau);
  for (int e = threadIdx.x; e < m * l; e += blockDim.x) Pj[e] = panel[e];
}

// ------------------------------------------------------ one-sided Jacobi
// Hestenes one-sided Jacobi on the l x l matrix W (column-major): rotate
// column pairs until all are mutually orthogonal, accumulating the
// rotations in J, so that W_in J = W_out.  Pairs follow the round-robin
// (circle) ordering so that l/2 disjoint pairs rotate concurrently, one
// warp per pair.
template <typename T>
__device__ void block_jacobi(T *W, T *J, int l, int *flag, T tol, int max_sweeps) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int lp = l + (l & 1);
  if (lp < 2) return;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) *flag = 0;
    __syncthreads();
    for (int r = 0; r < lp - 1; ++r) {
      for (int pi = warp; pi < lp / 2; pi += nw) {
        int a, b;
        if (pi == 0) { a = lp - 1; b = r; }
        else { a = (r + pi) % (lp - 1); b = (r - pi + lp - 1) % (lp - 1); }
        const int p = a < b ? a : b, q = a < b ? b : a;
        if (q >= l) continue;
        T *wp = W + (size_t)p * l, *wq = W + (size_t)q * l;
        T al = T(0), be = T(0), ga = T(0);
        for (int i = lane; i < l; i += 32) {
          const T x = wp[i], y = wq[i];
          al = fma(x, x, al);
          be = fma(y, y, be);
          ga = fma(x, y, ga);
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        if (ga != T(0) && fabs(ga) > tol * sqrt(al * be)) {
          const T zeta = (be - al) / (T(2) * ga);
          const T t = (zeta >= T(0) ? T(1) : T(-1)) / (fabs(zeta) + hypot(T(1), zeta));
          const T c = T(1) / sqrt(fma(t, t, T(1)));
          const T s = c * t;
          for (int i = lane; i < l; i += 32) {
            const T x = wp[i], y = wq[i];
            wp[i] = c * x - s * y;
            wq[i] = s * x + c * y;
          }
          T *jp = J + (size_t)p * l, *jq = J + (size_t)q * l;
          for (int i = lane; i < l; i += 32) {
            const T x = jp[i], y = jq[i];
            jp[i] = c * x - s * y;
            jq[i] = s * x + c * y;
          }
          if (lane == 0) *flag = 1;
        }
      }
      __syncthreads();
    }
    const int any = *flag;
    __syncthreads();
    if (!any) break;
  }
}

template <typename T>
__device__ __forceinline__ T prox_sv(T s, const ShrinkScalars &sh) {
  // Prox_{Phi,tau} on a singular value s >= 0 (Def. gNtsvt, Eq. equ_gst1).
  const T tau = T(sh.tau), th = T(sh.theta), ga = T(sh.gamma);
  if (sh.phi == TR_PEN_L1) {
    const T r = s - tau * th;
    return r > T(0) ? r : T(0);
  }
  if (ga > tau) {
    if (s <= tau * th) return T(0);
    if (s > ga * th) return s;
    return (s - tau * th) / (T(1) - tau / ga);
  }
  return s > th * sqrt(ga * tau) ? s : T(0);
}

// Per slice: QR of B^T (P2), Jacobi SVD of R, shrink, core C, then
// P1 <- P1 C (= Q C) and P2 <- Qb, ready for Gbar = P1 P2^T.
template <typename T>
__global__ void svd_core_kernel(int n1, int n2, int l, T *__restrict__ P1, int64_t sP1,
                                T *__restrict__ P2, int64_t sP2, ShrinkScalars sh,
                                T *__restrict__ sig_out, int *__restrict__ rank_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int mx = n1 > n2 ? n1 : n2;
  T *panel = reinterpret_cast<T *>(smem_raw);
  T *W = panel + (size_t)mx * l;
  T *J = W + l * l;
  T *C = J + l * l;
  T *tau = C + l * l;
  T *ratio = tau + l;
  int *flag = reinterpret_cast<int *>(ratio + l);
  const int j = blockIdx.x;
  T *P1j = P1 + (int64_t)j * sP1;
  T *P2j = P2 + (int64_t)j * sP2;

  for (int e = threadIdx.x; e < n2 * l; e += blockDim.x) panel[e] = P2j[e];
  __syncthreads();
  block_qr_factor(panel, n2, l, n2, tau);
  for (int e = threadIdx.x; e < l * l; e += blockDim.x) {
    const int r = e % l, c = e / l;
    W[e] = r <= c ? panel[(size_t)c * n2 + r] : T(0);
    J[e] = r == c ? T(1) : T(0);
  }
  __syncthreads();
  block_qr_form_q(panel, n2, l, n2, tau);
  for (int e = threadIdx.x; e < n2 * l; e += blockDim.x) P2j[e] = panel[e];
  // Rotate only while a pair's cosine exceeds max(l, 8) * eps: below that the
  // computed inner product is rounding noise (an l-term dot product).
  const T eps = sizeof(T) == 4 ? T(FLT_EPSILON) : T(DBL_EPSILON);
  const T tol = T(l > 8 ? l : 8) * eps;
  block_jacobi(W, J, l, flag, tol, sizeof(T) == 4 ? 16 : 30);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int i = warp; i < l; i += nw) {
    T ss = T(0);
    for (int r = lane; r < l; r += 32) ss = fma(W[(size_t)i * l + r], W[(size_t)i * l + r], ss);
    ss = warp_sum(ss);
    if (lane == 0) {
      const T sg = sqrt(ss);
      const T sp = prox_sv(sg, sh);
      ratio[i] = sg > T(0) ? sp / sg : T(0);
      sig_out[(int64_t)j * l + i] = sg;
      tau[i] = sp;   // reuse tau[] for the shrunk values
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int k = 0;
    for (int i = 0; i < l; ++i) k += tau[i] > T(0);
    rank_out[j] = k;
  }
  // C[a][b] = sum_i J[a][i] ratio_i W[b][i]   (column-major C[a + b*l])
  for (int e = threadIdx.x; e < l * l; e += blockDim.x) {
    const int a = e % l, b = e / l;
    T acc = T(0);
    for (int i = 0; i < l; ++i) acc = fma(J[(size_t)i * l + a] * ratio[i], W[(size_t)i * l + b], acc);
    C[e] = acc;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n1 * l; e += blockDim.x) panel[e] = P1j[e];
  __syncthreads();
  for (int e = threadIdx.x; e < n1 * l; e += blockDim.x) {
    const int r = e % n1, b = e / n1;
    T acc = T(0);
    for (int a = 0; a < l; ++a) acc = fma(panel[(size_t)a * n1 + r], C[a + (size_t)b * l], acc);
    P1j[e] = acc;
  }
}

template <typename T>
size_t qr_smem(int m, int l) {
  return sizeof(T) * ((size_t)m * l + l);
}

template <typename T>
size_t svd_smem(int n1, int n2, int l) {
  const int mx = n1 > n2 ? n1 : n2;
  return sizeof(T) * ((size_t)mx * l + 3 * (size_t)l * l + 2 * (size_t)l) + 16;
}

constexpr size_t kSliceSmemMax = 227 * 1024;

template <typename T>
cudaError_t run_qr(int m, int l, T *P, int n, cudaStream_t s) {
  const size_t smem = qr_smem<T>(m, l);
  cudaError_t e = cudaFuncSetAttribute(qr_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  qr_kernel<T><<<n, 256, smem, s>>>(m, l, P, (int64_t)m * l);
  return cudaGetLastError();
}

template <typename T>
cudaError_t run_rsvd(const SliceWork &w, const T *Abar, T *Gbar, const ShrinkScalars &sh, int t,
                     cudaStream_t s) {
  const int n = w.n, n1 = w.n1, n2 = w.n2, l = w.l;
  const int64_t sA = (int64_t)n1 * n2;
  T *Om = (T *)w.Om, *P1 = (T *)w.P1, *P2 = (T *)w.P2;
  cudaError_t e;
  // Omega for every slice
  {
    const int64_t per = (int64_t)n2 * l;
    const int64_t groups = (per + 3) / 4;
    dim3 grid((unsigned)((groups + 255) / 256), n);
    sketch_kernel<T><<<grid, 256, 0, s>>>(per, Om, (uint32_t)(w.seed & 0xffffffffu),
                                          (uint32_t)(w.seed >> 32), (uint32_t)t, 0u);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  // Y = Abar X (X: n2 x l column-major panel with batch stride sX)
  auto gemm_AX = [&](const T *X, T *Y) {
    GemmArgs g{n1, l, n2, Abar, sA, n2, 1, X, (int64_t)n2 * l, 1, n2, Y, (int64_t)n1 * l, 1, n1};
    return bgemm<T>(g, n, s);
  };
  // W = Abar^T Q (Q: n1 x l)
  auto gemm_AtX = [&](const T *X, T *Wt) {
    GemmArgs g{n2, l, n1, Abar, sA, 1, n2, X, (int64_t)n1 * l, 1, n1, Wt, (int64_t)n2 * l, 1, n2};
    return bgemm<T>(g, n, s);
  };
  if ((e = gemm_AX(Om, P1)) != cudaSuccess) return e;
  for (int it = 0; it < w.q; ++it) {
    if ((e = run_qr<T>(n1, l, P1, n, s)) != cudaSuccess) return e;
    if ((e = gemm_AtX(P1, P2)) != cudaSuccess) return e;
    if ((e = run_qr<T>(n2, l, P2, n, s)) != cudaSuccess) return e;
    if ((e = gemm_AX(P2, P1)) != cudaSuccess) return e;
  }
  if ((e = run_qr<T>(n1, l, P1, n, s)) != cudaSuccess) return e;
  if ((e = gemm_AtX(P1, P2)) != cudaSuccess) return e;
  {
    const size_t smem = svd_smem<T>(n1, n2, l);
    if ((e = cudaFuncSetAttribute(svd_core_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)) != cudaSuccess)
      return e;
    const int lp = l + (l & 1);
    int threads = 32 * (lp / 2 > 8 ? lp / 2 : 8);
    if (threads > 1024) threads = 1024;
    svd_core_kernel<T><<<n, threads, smem, s>>>(n1, n2, l, P1, (int64_t)n1 * l, P2,
                                                (int64_t)n2 * l, sh, (T *)w.sig, w.rank);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  // Gbar = Z Qb^T : (n1 x l) (l x n2), row-major output
  GemmArgs g{n1, n2, l, P1, (int64_t)n1 * l, 1, n1, P2, (int64_t)n2 * l, n2, 1, Gbar, sA, n2, 1};
  return bgemm<T>(g, n, s);
}

}  // namespace

cudaError_t launch_slice_rsvd(tr_dtype dt, const SliceWork &w, const void *Abar, void *Gbar,
                              const ShrinkScalars &sh, int t, cudaStream_t s) {
  if (dt == TR_F64) return run_rsvd<double>(w, (const double *)Abar, (double *)Gbar, sh, t, s);
  return run_rsvd<float>(w, (const float *)Abar, (float *)Gbar, sh, t, s);
}

size_t slice_smem_limit_ok(tr_dtype dt, int n1, int n2, int l) {
  const int mx = n1 > n2 ? n1 : n2;
  const size_t a = dt == TR_F64 ? svd_smem<double>(n1, n2, l) : svd_smem<float>(n1, n2, l);
  const size_t b = dt == TR_F64 ? qr_smem<double>(mx, l) : qr_smem<float>(mx, l);
  return (a <= kSliceSmemMax && b <= kSliceSmemMax) ? 1 : 0;
}
