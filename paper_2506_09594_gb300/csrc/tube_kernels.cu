// Tube passes: the elementwise ADMM updates fused with the transform L along
// modes 3..d (Eq. trans).  A CTA owns TP consecutive (i1, i2) positions of
// every face slice (a "tube tile", TP x n elements), staged once in shared
// memory: loads and stores are coalesced rows of TP elements per slice, and
// each mode product runs on fibres held in registers.
//
// Forward pass (Alg. 5 steps L, E, Y and the start of the G step):
//   L1 = ((M - E + Y/mu) + (G - Lambda/mu)) / 2          Eq. coef-tensor, nabla = I
//   H  = M - L1 + Y/mu;  E1 = Prox_{psi,lambda/mu}(H) on Omega, H off Omega
//                                                         Eq. E_prox_ome(1), GNHTT
//   Y1 = Y + mu (M - L1 - E1)                             Eq. lagrange11
//   Abar = L(L1 + Lambda/mu)                              input of Eq. L_prox
// Inverse pass (end of the G step and the Lambda update):
//   G1 = L^{-1}(Gbar);  Lambda1 = Lambda + mu (L1 - G1)   Eq. lagrange11-22
// Both passes reduce their share of the Eq. convercon infinity norms.

#include <math.h>

#include "tr_internal.cuh"

namespace {

constexpr int kTubeThreads = 256;

template <typename T>
__device__ __forceinline__ T prox_scalar(T v, T thr, int kind, T theta, T gamma) {
  // Prox_{psi,thr}(v), Eq. equ_gst1, for psi = theta|x| (l1) or MCP.
  T a = fabs(v);
  T sgn = v < T(0) ? T(-1) : T(1);
  if (kind == TR_PEN_L1) {
    T r = a - thr * theta;
    return r > T(0) ? sgn * r : T(0);
  }
  if (gamma > thr) {
    if (a <= thr * theta) return T(0);
    if (a > gamma * theta) return v;
    return sgn * (a - thr * theta) / (T(1) - thr / gamma);
  }
  return a > theta * sqrt(gamma * thr) ? v : T(0);
}

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long *slot, double v) {
  atomicMax(slot, (unsigned long long)__double_as_longlong(v));
}

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide max of up to 3 values, one atomic per value per CTA.
template <typename T, int K>
__device__ void block_max_to_global(T (&v)[K], unsigned long long *const (&slot)[K]) {
  __shared__ T red[K][32];
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    T w = warp_max(v[k]);
    if (lane == 0) red[k][warp] = w;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      T w = lane < nw ? red[k][lane] : T(0);
      w = warp_max(w);
      if (lane == 0) atomic_max_nonneg(slot[k], (double)w);
    }
  }
}

// Apply the mode products of the transform (or its inverse) to a tube tile
// held in shared memory as tile[j * TP + p].  A fibre is the n_k elements of
// one position p that differ only in mode k; a thread loads its fibre into
// registers, multiplies by the n_k x n_k matrix (rows zero-padded to NK) and
// writes the result back in place.
template <typename T, int NK>
__device__ void tile_transform(T *tile, int n, int TP, const T *mats, const TransformDesc &td,
                               bool inverse) {
  for (int mi = 0; mi < td.nt; ++mi) {
    const int k = inverse ? td.nt - 1 - mi : mi;
    const int nk = td.dim[k], st = td.stride[k];
    const T *U = mats + (inverse ? td.off_inv[k] : td.off_fwd[k]);
    const int nfib = n / nk;
    for (int w = threadIdx.x; w < nfib * TP; w += blockDim.x) {
      const int p = w % TP, f = w / TP;
      const int base = (f % st) + (f / st) * (st * nk);
      T x[NK];
#pragma unroll
      for (int m = 0; m < NK; ++m) x[m] = (m < nk) ? tile[(base + m * st) * TP + p] : T(0);
      for (int i = 0; i < nk; ++i) {
        const T *Ui = U + i * NK;
        T acc = T(0);
#pragma unroll
        for (int m = 0; m < NK; ++m) acc = fma(Ui[m], x[m], acc);
        tile[(base + i * st) * TP + p] = acc;
      }
    }
    __syncthreads();
  }
}

template <typename T>
__device__ __forceinline__ void load_mats(T *dst, const T *src, int len) {
  for (int i = threadIdx.x; i < len; i += blockDim.x) dst[i] = src[i];
}

template <typename T, int NK>
__global__ void __launch_bounds__(kTubeThreads)
tube_forward_kernel(int64_t P, int n, int TP, TransformDesc td, const T *__restrict__ mats_g,
                    const T *__restrict__ M, const uint8_t *__restrict__ mask, T *__restrict__ L,
                    T *__restrict__ E, T *__restrict__ Y, const T *__restrict__ G,
                    const T *__restrict__ Lam, T *__restrict__ Abar, TubeScalars sc,
                    unsigned long long *res, int *flags) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *mats = reinterpret_cast<T *>(smem_raw);
  T *tile = mats + td.mats_len;
  load_mats(mats, mats_g, td.mats_len);

  const T mu = T(sc.mu), imu = T(1.0 / sc.mu), thr = T(sc.lam_over_mu);
  const T th = T(sc.psi_theta), ga = T(sc.psi_gamma);
  const int64_t p0 = (int64_t)blockIdx.x * TP;
  T rL = 0, rE = 0, rC = 0;
  int bad = 0;
  for (int e = threadIdx.x; e < n * TP; e += blockDim.x) {
    const int j = e / TP, p = e % TP;
    const int64_t pos = p0 + p;
    T a = T(0);
    if (pos < P) {
      const int64_t idx = (int64_t)j * P + pos;
      const bool om = mask[idx] != 0;
      const T m = om ? M[idx] : T(0);
      const T l0 = L[idx], e0 = E[idx], y0 = Y[idx], g0 = G[idx], la = Lam[idx];
      const T l1 = T(0.5) * ((m - e0 + y0 * imu) + (g0 - la * imu));
      const T h = m - l1 + y0 * imu;
      T e1;
      if (om) e1 = (sc.noise == TR_NOISE_NONE) ? T(0) : prox_scalar(h, thr, sc.psi, th, ga);
      else e1 = h;
      const T y1 = y0 + mu * (m - l1 - e1);
      a = l1 + la * imu;
      L[idx] = l1;
      E[idx] = e1;
      Y[idx] = y1;
      rL = fmax(rL, fabs(l1 - l0));
      rE = fmax(rE, fabs(e1 - e0));
      rC = fmax(rC, fabs(m - l1 - e1));
      bad |= !(isfinite(a) && isfinite(e1) && isfinite(y1));
    }
    tile[j * TP + p] = a;
  }
  __syncthreads();
  tile_transform<T, NK>(tile, n, TP, mats, td, false);
  for (int e = threadIdx.x; e < n * TP; e += blockDim.x) {
    const int j = e / TP, p = e % TP;
    const int64_t pos = p0 + p;
    if (pos < P) Abar[(int64_t)j * P + pos] = tile[j * TP + p];
  }
  if (bad) atomicOr(flags, 1);
  T v[3] = {rL, rE, rC};
  unsigned long long *const slots[3] = {res + RES_DL, res + RES_DE, res + RES_CONS};
  block_max_to_global<T, 3>(v, slots);
}

template <typename T, int NK>
__global__ void __launch_bounds__(kTubeThreads)
tube_inverse_kernel(int64_t P, int n, int TP, TransformDesc td, const T *__restrict__ mats_g,
                    const T *__restrict__ Gbar, const T *__restrict__ L, T *__restrict__ G,
                    T *__restrict__ Lam, double mu_d, unsigned long long *res, int *flags) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *mats = reinterpret_cast<T *>(smem_raw);
  T *tile = mats + td.mats_len;
  load_mats(mats, mats_g, td.mats_len);
  const int64_t p0 = (int64_t)blockIdx.x * TP;
  for (int e = threadIdx.x; e < n * TP; e += blockDim.x) {
    const int j = e / TP, p = e % TP;
    const int64_t pos = p0 + p;
    tile[j * TP + p] = pos < P ? Gbar[(int64_t)j * P + pos] : T(0);
  }
  __syncthreads();
  tile_transform<T, NK>(tile, n, TP, mats, td, true);
  const T mu = T(mu_d);
  T rLG = 0, rG = 0;
  int bad = 0;
  for (int e = threadIdx.x; e < n * TP; e += blockDim.x) {
    const int j = e / TP, p = e % TP;
    const int64_t pos = p0 + p;
    if (pos < P) {
      const int64_t idx = (int64_t)j * P + pos;
      const T g1 = tile[j * TP + p];
      const T l1 = L[idx], g0 = G[idx], la = Lam[idx];
      const T la1 = la + mu * (l1 - g1);
      G[idx] = g1;
      Lam[idx] = la1;
      rLG = fmax(rLG, fabs(l1 - g1));
      rG = fmax(rG, fabs(g1 - g0));
      bad |= !(isfinite(g1) && isfinite(la1));
    }
  }
  if (bad) atomicOr(flags, 1);
  T v[2] = {rLG, rG};
  unsigned long long *const slots[2] = {res + RES_LG, res + RES_DG};
  block_max_to_global<T, 2>(v, slots);
}

template <typename T, int NK>
__global__ void __launch_bounds__(kTubeThreads)
transform_kernel(int64_t P, int n, int TP, TransformDesc td, const T *__restrict__ mats_g,
                 const T *__restrict__ src, T *__restrict__ dst, int inverse) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *mats = reinterpret_cast<T *>(smem_raw);
  T *tile = mats + td.mats_len;
  load_mats(mats, mats_g, td.mats_len);
  const int64_t p0 = (int64_t)blockIdx.x * TP;
  for (int e = threadIdx.x; e < n * TP; e += blockDim.x) {
    const int j = e / TP, p = e % TP;
    const int64_t pos = p0 + p;
    tile[j * TP + p] = pos < P ? src[(int64_t)j * P + pos] : T(0);
  }
  __syncthreads();
  tile_transform<T, NK>(tile, n, TP, mats, td, inverse != 0);
  for (int e = threadIdx.x; e < n * TP; e += blockDim.x) {
    const int j = e / TP, p = e % TP;
    const int64_t pos = p0 + p;
    if (pos < P) dst[(int64_t)j * P + pos] = tile[j * TP + p];
  }
}

template <typename T>
size_t tube_smem_for(int n, const TransformDesc &td, int TP) {
  return sizeof(T) * ((size_t)td.mats_len + (size_t)n * TP);
}

constexpr size_t kSmemBudget = 200 * 1024;

template <typename T>
int pick_tp(int n, const TransformDesc &td) {
  int tp = 32;
  while (tp > 4 && tube_smem_for<T>(n, td, tp) > kSmemBudget) tp >>= 1;
  return tube_smem_for<T>(n, td, tp) > kSmemBudget ? 0 : tp;
}

// Dispatch on the padded fibre length NK (a multiple of 8, at most 64).
template <typename T, template <typename, int> class Launcher, typename... Args>
cudaError_t dispatch_nk(int nkpad, Args... args) {
  switch (nkpad) {
    case 8: return Launcher<T, 8>::run(args...);
    case 16: return Launcher<T, 16>::run(args...);
    case 24: return Launcher<T, 24>::run(args...);
    case 32: return Launcher<T, 32>::run(args...);
    case 40: return Launcher<T, 40>::run(args...);
    case 48: return Launcher<T, 48>::run(args...);
    case 56: return Launcher<T, 56>::run(args...);
    case 64: return Launcher<T, 64>::run(args...);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T, int NK>
struct FwdLauncher {
  static cudaError_t run(int64_t P, int n, const TransformDesc &td, const void *mats,
                         const void *M, const uint8_t *mask, void *L, void *E, void *Y,
                         const void *G, const void *Lam, void *Abar, const TubeScalars &sc,
                         unsigned long long *res, int *flags, cudaStream_t s) {
    int tp = pick_tp<T>(n, td);
    if (!tp) return cudaErrorInvalidValue;
    size_t smem = tube_smem_for<T>(n, td, tp);
    auto k = tube_forward_kernel<T, NK>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int64_t grid = (P + tp - 1) / tp;
    k<<<(unsigned)grid, kTubeThreads, smem, s>>>(P, n, tp, td, (const T *)mats, (const T *)M, mask,
                                                (T *)L, (T *)E, (T *)Y, (const T *)G,
                                                (const T *)Lam, (T *)Abar, sc, res, flags);
    return cudaGetLastError();
  }
};

template <typename T, int NK>
struct InvLauncher {
  static cudaError_t run(int64_t P, int n, const TransformDesc &td, const void *mats,
                         const void *Gbar, const void *L, void *G, void *Lam, double mu,
                         unsigned long long *res, int *flags, cudaStream_t s) {
    int tp = pick_tp<T>(n, td);
    if (!tp) return cudaErrorInvalidValue;
    size_t smem = tube_smem_for<T>(n, td, tp);
    auto k = tube_inverse_kernel<T, NK>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int64_t grid = (P + tp - 1) / tp;
    k<<<(unsigned)grid, kTubeThreads, smem, s>>>(P, n, tp, td, (const T *)mats, (const T *)Gbar,
                                                (const T *)L, (T *)G, (T *)Lam, mu, res, flags);
    return cudaGetLastError();
  }
};

template <typename T, int NK>
struct XfLauncher {
  static cudaError_t run(int64_t P, int n, const TransformDesc &td, const void *mats,
                         const void *src, void *dst, bool inverse, cudaStream_t s) {
    int tp = pick_tp<T>(n, td);
    if (!tp) return cudaErrorInvalidValue;
    size_t smem = tube_smem_for<T>(n, td, tp);
    auto k = transform_kernel<T, NK>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int64_t grid = (P + tp - 1) / tp;
    k<<<(unsigned)grid, kTubeThreads, smem, s>>>(P, n, tp, td, (const T *)mats, (const T *)src,
                                                (T *)dst, inverse ? 1 : 0);
    return cudaGetLastError();
  }
};

}  // namespace

cudaError_t launch_tube_forward(tr_dtype dt, int64_t P, int n, const TransformDesc &td,
                                const void *mats, const void *M, const uint8_t *mask, void *L,
                                void *E, void *Y, const void *G, const void *Lam, void *Abar,
                                const TubeScalars &sc, unsigned long long *res, int *flags,
                                cudaStream_t s) {
  if (dt == TR_F64)
    return dispatch_nk<double, FwdLauncher>(td.nkpad, P, n, td, mats, M, mask, L, E, Y, G, Lam,
                                            Abar, sc, res, flags, s);
  return dispatch_nk<float, FwdLauncher>(td.nkpad, P, n, td, mats, M, mask, L, E, Y, G, Lam, Abar,
                                         sc, res, flags, s);
}

cudaError_t launch_tube_inverse(tr_dtype dt, int64_t P, int n, const TransformDesc &td,
                                const void *mats, const void *Gbar, const void *L, void *G,
                                void *Lam, double mu, unsigned long long *res, int *flags,
                                cudaStream_t s) {
  if (dt == TR_F64)
    return dispatch_nk<double, InvLauncher>(td.nkpad, P, n, td, mats, Gbar, L, G, Lam, mu, res,
                                            flags, s);
  return dispatch_nk<float, InvLauncher>(td.nkpad, P, n, td, mats, Gbar, L, G, Lam, mu, res, flags,
                                         s);
}

cudaError_t launch_transform(tr_dtype dt, int64_t P, int n, const TransformDesc &td,
                             const void *mats, const void *src, void *dst, bool inverse,
                             cudaStream_t s) {
  if (dt == TR_F64)
    return dispatch_nk<double, XfLauncher>(td.nkpad, P, n, td, mats, src, dst, inverse, s);
  return dispatch_nk<float, XfLauncher>(td.nkpad, P, n, td, mats, src, dst, inverse, s);
}

size_t tube_smem_bytes(tr_dtype dt, int n, const TransformDesc &td, int *tp_out) {
  int tp = dt == TR_F64 ? pick_tp<double>(n, td) : pick_tp<float>(n, td);
  if (tp_out) *tp_out = tp;
  if (!tp) return 0;
  return dt == TR_F64 ? tube_smem_for<double>(n, td, tp) : tube_smem_for<float>(n, td, tp);
}
