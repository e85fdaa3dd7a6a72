// Tube passes: the elementwise ADMM updates fused with the transform L along
// modes 3..d (Eq. trans).  A CTA owns TP consecutive (i1, i2) positions of
// every face slice (a "tube tile", TP x n elements) staged once in shared
// memory; global traffic is coalesced 16-byte packs of VEC consecutive
// positions, UNR packs per thread in flight, and each mode product runs on
// fibres held in registers.
//
// Forward pass (first half of Alg. 5 iteration t):
//   L1 = ((M - E + Y/mu) + (G - Lambda/mu)) / 2          Eq. coef-tensor, nabla = I
//   H  = M - L1 + Y/mu;  E1 = Prox_{psi,lambda/mu}(H) on Omega, H off Omega
//                                                         Eq. E_prox_ome(1), GNHTT
//   Y1 = Y + mu (M - L1 - E1)                             Eq. lagrange11
//   Abar = L(L1 + Lambda/mu)                              input of Eq. L_prox
// Inverse pass (second half):
//   G1 = L^{-1}(Gbar);  Lambda1 = Lambda + mu (L1 - G1)   Eq. lagrange11-22
// Fused pass: the inverse pass of iteration t-1 followed, in the same tile,
// by the forward pass of iteration t (G and Lambda of t-1 never leave the
// SM before the forward pass uses them).
// All three reduce their share of the Eq. convercon infinity norms.

#include <math.h>
#include <stdint.h>

#include <initializer_list>

#include <cuda_bf16.h>

#include "tr_internal.cuh"

namespace {

constexpr int kTubeThreads = 256;
constexpr int kUnroll = 1;

// CTAs per SM the register budget must allow: three for the common small
// fibres in FP32 (three 256-thread CTAs keep ~80 KB of loads in flight per
// SM), no constraint for long fibres or FP64.
template <typename T, int NK>
constexpr int tube_min_blocks() { return (sizeof(T) == 4 && NK <= 32) ? 3 : 1; }

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

// ---- packs of VEC consecutive elements (16-byte vectors when VEC > 1)
template <typename T, int VEC>
struct Pk {
  T v[VEC];
};

template <typename T, int VEC>
__device__ __forceinline__ Pk<T, VEC> ld(const T *p) {
  Pk<T, VEC> r;
  if constexpr (VEC == 1) {
    r.v[0] = *p;
  } else if constexpr (sizeof(T) == 4) {
    const float4 x = *reinterpret_cast<const float4 *>(p);
    r.v[0] = x.x; r.v[1] = x.y; r.v[2] = x.z; r.v[3] = x.w;
  } else {
    const double2 x = *reinterpret_cast<const double2 *>(p);
    r.v[0] = x.x; r.v[1] = x.y;
  }
  return r;
}

template <typename T, int VEC>
__device__ __forceinline__ void st(T *p, const Pk<T, VEC> &r) {
  if constexpr (VEC == 1) {
    *p = r.v[0];
  } else if constexpr (sizeof(T) == 4) {
    *reinterpret_cast<float4 *>(p) = make_float4(r.v[0], r.v[1], r.v[2], r.v[3]);
  } else {
    *reinterpret_cast<double2 *>(p) = make_double2(r.v[0], r.v[1]);
  }
}

template <int VEC>
__device__ __forceinline__ Pk<uint8_t, VEC> ldm(const uint8_t *p) {
  Pk<uint8_t, VEC> r;
  if constexpr (VEC == 1) {
    r.v[0] = *p;
  } else if constexpr (VEC == 4) {
    const uchar4 x = *reinterpret_cast<const uchar4 *>(p);
    r.v[0] = x.x; r.v[1] = x.y; r.v[2] = x.z; r.v[3] = x.w;
  } else {
    const uchar2 x = *reinterpret_cast<const uchar2 *>(p);
    r.v[0] = x.x; r.v[1] = x.y;
  }
  return r;
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

// Block-wide max of K values, one atomic per value per CTA.
template <typename T, int K>
__device__ void block_max_to_global(const T (&v)[K], unsigned long long *const (&slot)[K]) {
  __shared__ T red[K][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const T w = warp_max(v[k]);
    if (lane == 0) red[k][warp] = w;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      T w = lane < nw ? red[k][lane] : T(0);
      w = warp_max(w);
      if (lane == 0 && slot[k]) atomic_max_nonneg(slot[k], (double)w);
    }
  }
}

// Dot product of a matrix row (shared memory, NK entries, 16-byte aligned:
// rows are padded to a multiple of 8) with a register fibre.  The row is read
// with 16-byte shared loads, which every lane of a warp reads at the same
// address (broadcast), so a row costs NK/4 (float) or NK/2 (double) load
// instructions instead of NK.
template <int NK>
__device__ __forceinline__ float row_dot(const float *Ui, const float (&x)[NK]) {
  const float4 *U4 = reinterpret_cast<const float4 *>(Ui);
  float acc = 0.f;
#pragma unroll
  for (int m = 0; m < NK / 4; ++m) {
    const float4 u = U4[m];
    acc = fmaf(u.x, x[4 * m], acc);
    acc = fmaf(u.y, x[4 * m + 1], acc);
    acc = fmaf(u.z, x[4 * m + 2], acc);
    acc = fmaf(u.w, x[4 * m + 3], acc);
  }
  return acc;
}
template <int NK>
__device__ __forceinline__ double row_dot(const double *Ui, const double (&x)[NK]) {
  const double2 *U2 = reinterpret_cast<const double2 *>(Ui);
  double acc = 0.0;
#pragma unroll
  for (int m = 0; m < NK / 2; ++m) {
    const double2 u = U2[m];
    acc = fma(u.x, x[2 * m], acc);
    acc = fma(u.y, x[2 * m + 1], acc);
  }
  return acc;
}

// Mode products of the transform (or its inverse) on a tube tile in shared
// memory, tile[j * TP + p].  A fibre is the n_k elements of one position p
// that differ only in mode k; a thread reads its fibre into registers,
// applies the n_k x n_k matrix and writes the result back in place.
//
// The transform is the orthonormal DCT-II along every mode, whose matrix
// obeys C[k][n-1-m] = (-1)^k C[k][m] (the cosines are symmetric about the
// centre of the fibre).  With h = ceil(n/2) the forward product folds the
// fibre into s_m = x_m + x_{n-1-m}, d_m = x_m - x_{n-1-m} (m < h; the centre
// of an odd fibre enters both as x_m) and takes
//   y_k = sum_{m<h} C[k][m] s_m (k even),   y_k = sum_{m<h} C[k][m] d_m (k odd),
// the inverse x = C^T y the even-k and odd-k sums E_m, O_m of C[k][m] y_k
// with x_m = E_m + O_m and x_{n-1-m} = E_m - O_m: half the multiply-adds of
// the plain matrix-vector product, the same values up to rounding.
//   Forward rows: row k of C at off_fwd + k NK (entries m >= h meet zeros).
//   Inverse rows: row m < h at off_inv + 2 HK m holds C[0][m], C[2][m], ...
//   (HK entries) and then C[1][m], C[3][m], ... (HK entries).
template <int NK>
__host__ __device__ constexpr int half_k() {
  return ((NK / 2 + 3) / 4) * 4;
}

template <typename T, int NK>
__device__ void tile_transform(T *tile, int n, int TP, const T *mats, const TransformDesc &td,
                               bool inverse) {
  static_assert(NK % 4 == 0, "rows padded to a multiple of 4");
  constexpr int HK = half_k<NK>();
  for (int mi = 0; mi < td.nt; ++mi) {
    const int k = inverse ? td.nt - 1 - mi : mi;
    const int nk = td.dim[k], stp = td.stride[k], h = (nk + 1) / 2;
    const T *U = mats + (inverse ? td.off_inv[k] : td.off_fwd[k]);
    const int nfib = n / nk;
    const int lgtp = 31 - __clz(TP);   // TP is a power of two
    for (int w = threadIdx.x; w < nfib * TP; w += blockDim.x) {
      const int p = w & (TP - 1), f = w >> lgtp;
      T *fib = tile + ((f % stp) + (f / stp) * (stp * nk)) * TP + p;
      const int step = stp * TP;
      T a[HK], b[HK];
      if (!inverse) {
#pragma unroll
        for (int m = 0; m < HK; ++m) {
          if (m < h) {
            const T x0 = fib[m * step];
            if (2 * m + 1 == nk) {
              a[m] = x0;
              b[m] = x0;
            } else {
              const T x1 = fib[(nk - 1 - m) * step];
              a[m] = x0 + x1;
              b[m] = x0 - x1;
            }
          } else {
            a[m] = T(0);
            b[m] = T(0);
          }
        }
        for (int i = 0; i < nk; i += 2) {
          fib[i * step] = row_dot<HK>(U + i * NK, a);
          if (i + 1 < nk) fib[(i + 1) * step] = row_dot<HK>(U + (i + 1) * NK, b);
        }
      } else {
#pragma unroll
        for (int i = 0; i < HK; ++i) {
          a[i] = (2 * i < nk) ? fib[2 * i * step] : T(0);
          b[i] = (2 * i + 1 < nk) ? fib[(2 * i + 1) * step] : T(0);
        }
        for (int m = 0; m < h; ++m) {
          const T e = row_dot<HK>(U + m * 2 * HK, a), o = row_dot<HK>(U + m * 2 * HK + HK, b);
          fib[m * step] = e + o;
          if (2 * m + 1 != nk) fib[(nk - 1 - m) * step] = e - o;
        }
      }
    }
    __syncthreads();
  }
}

template <typename T>
__device__ __forceinline__ void load_mats(T *dst, const T *src, int len) {
  for (int i = threadIdx.x; i < len; i += blockDim.x) dst[i] = src[i];
}

// Pack e of the tile -> (slice j, first position p within the tile).
struct PackIdx {
  int j, p;
};
// per_row = TP / VEC is a power of two (tiles hold 2^k tubes): shifts, not
// divisions
__device__ __forceinline__ PackIdx pack_idx(int e, int per_row, int VEC) {
  const int lg = 31 - __clz(per_row);
  return {e >> lg, (e & (per_row - 1)) * VEC};
}

// Copy a tile of a slice-major array into shared memory (zero beyond P).
template <typename T, int VEC>
__device__ void tile_load(T *tile, const T *__restrict__ src, int64_t P, int n, int TP,
                          int64_t p0) {
  // one array only: four packs per thread in flight
  constexpr int U = 4;
  const int per_row = TP / VEC, total = n * per_row;
  for (int e0 = threadIdx.x; e0 < total; e0 += kTubeThreads * U) {
    Pk<T, VEC> v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * kTubeThreads;
      const PackIdx q = pack_idx(e, per_row, VEC);
      if (e < total && p0 + q.p < P) v[u] = ld<T, VEC>(src + (int64_t)q.j * P + p0 + q.p);
      else
#pragma unroll
        for (int i = 0; i < VEC; ++i) v[u].v[i] = T(0);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * kTubeThreads;
      if (e < total) {
        const PackIdx q = pack_idx(e, per_row, VEC);
        st<T, VEC>(tile + q.j * TP + q.p, v[u]);
      }
    }
  }
}

template <typename T, int VEC>
__device__ void tile_store(T *__restrict__ dst, const T *tile, int64_t P, int n, int TP,
                           int64_t p0) {
  const int per_row = TP / VEC, total = n * per_row;
  for (int e = threadIdx.x; e < total; e += kTubeThreads) {
    const PackIdx q = pack_idx(e, per_row, VEC);
    if (p0 + q.p < P) st<T, VEC>(dst + (int64_t)q.j * P + p0 + q.p, ld<T, VEC>(tile + q.j * TP + q.p));
  }
}

// The tile as Abar's BF16 planes: hi = bf16(x) at j P + p, lo = bf16(x - hi)
// at n P + j P + p (x - hi is exact in FP32).  FP32 only.
template <typename T, int VEC>
__device__ void tile_store_planes(T *__restrict__ dst, const T *tile, int64_t P, int n, int TP,
                                  int64_t p0) {
  if constexpr (sizeof(T) == 4) {
    __nv_bfloat16 *hi_p = reinterpret_cast<__nv_bfloat16 *>(dst);
    __nv_bfloat16 *lo_p = hi_p + (int64_t)n * P;
    const int per_row = TP / VEC, total = n * per_row;
    for (int e = threadIdx.x; e < total; e += kTubeThreads) {
      const PackIdx q = pack_idx(e, per_row, VEC);
      if (p0 + q.p >= P) continue;
      const Pk<T, VEC> x = ld<T, VEC>(tile + q.j * TP + q.p);
      const int64_t o = (int64_t)q.j * P + p0 + q.p;
      if constexpr (VEC == 4) {
        __nv_bfloat162 h[2], l[2];
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          h[i] = __floats2bfloat162_rn(x.v[2 * i], x.v[2 * i + 1]);
          const float2 f = __bfloat1622float2(h[i]);
          l[i] = __floats2bfloat162_rn(x.v[2 * i] - f.x, x.v[2 * i + 1] - f.y);
        }
        *reinterpret_cast<uint2 *>(hi_p + o) = *reinterpret_cast<const uint2 *>(h);
        *reinterpret_cast<uint2 *>(lo_p + o) = *reinterpret_cast<const uint2 *>(l);
      } else {
#pragma unroll
        for (int i = 0; i < VEC; ++i) {
          const __nv_bfloat16 h = __float2bfloat16_rn(x.v[i]);
          hi_p[o + i] = h;
          lo_p[o + i] = __float2bfloat16_rn(x.v[i] - __bfloat162float(h));
        }
      }
    }
  }
}

template <typename T, int VEC>
__device__ __forceinline__ void store_abar(T *__restrict__ Abar, const T *tile, int64_t P, int n,
                                           int TP, int64_t p0, int planes) {
  if (sizeof(T) == 4 && planes) tile_store_planes<T, VEC>(Abar, tile, P, n, TP, p0);
  else tile_store<T, VEC>(Abar, tile, P, n, TP, p0);
}

// Scalars of the forward update with mu^t taken from the device schedule
// when the launch carries one.
__device__ __forceinline__ TubeScalars resolve(const TubeScalars &sc) {
  TubeScalars r = sc;
  if (sc.dmu) {
    r.mu = *sc.dmu;
    r.lam_over_mu = sc.lambda / r.mu;
  }
  return r;
}

// The forward update's scalars in the element type, formed once per block
// (the double-precision division and conversions stay out of the element
// loop: FP64 issues slowly on this part).
template <typename T>
struct FwdK {
  T mu, imu, thr, th, ga;
  int noise, psi;
};
template <typename T>
__device__ __forceinline__ FwdK<T> fwd_scalars(const TubeScalars &sc) {
  return FwdK<T>{T(sc.mu), T(1.0 / sc.mu), T(sc.lam_over_mu), T(sc.psi_theta), T(sc.psi_gamma),
                 sc.noise, sc.psi};
}

// The forward elementwise update on a pack; `gv` holds G^t (from global
// memory or from the fused inverse), `la` Lambda^t.
template <typename T, int VEC>
__device__ __forceinline__ void forward_pack(const Pk<T, VEC> &m_, const Pk<uint8_t, VEC> &om,
                                             const Pk<T, VEC> &l0, const Pk<T, VEC> &e0,
                                             const Pk<T, VEC> &y0, const Pk<T, VEC> &gv,
                                             const Pk<T, VEC> &la, const FwdK<T> &sc,
                                             Pk<T, VEC> &l1, Pk<T, VEC> &e1, Pk<T, VEC> &y1,
                                             Pk<T, VEC> &a, T &rL, T &rE, T &rC, int &bad) {
  const T mu = sc.mu, imu = sc.imu, thr = sc.thr, th = sc.th, ga = sc.ga;
#pragma unroll
  for (int i = 0; i < VEC; ++i) {
    const bool o = om.v[i] != 0;
    const T m = o ? m_.v[i] : T(0);
    // (M - E + Y/mu) + (G - Lambda/mu) summed as (M - E + G) + (Y - Lambda)/mu:
    // Y/mu and Lambda/mu grow large and nearly cancel (Lambda -> Y at a KKT
    // point), so subtracting the multipliers first avoids that cancellation.
    const T l = T(0.5) * ((m - e0.v[i] + gv.v[i]) + (y0.v[i] - la.v[i]) * imu);
    const T h = m - l + y0.v[i] * imu;
    T e;
    if (o) e = (sc.noise == TR_NOISE_NONE) ? T(0) : prox_scalar(h, thr, sc.psi, th, ga);
    else e = h;
    const T y = y0.v[i] + mu * (m - l - e);
    l1.v[i] = l;
    e1.v[i] = e;
    y1.v[i] = y;
    a.v[i] = l + la.v[i] * imu;
    rL = fmax(rL, fabs(l - l0.v[i]));
    rE = fmax(rE, fabs(e - e0.v[i]));
    rC = fmax(rC, fabs(m - l - e));
    bad |= !(isfinite(a.v[i]) && isfinite(e) && isfinite(y));
  }
}

template <typename T, int NK, int VEC>
__global__ void __launch_bounds__(kTubeThreads, tube_min_blocks<T, NK>())
tube_forward_kernel(int64_t P, int n, int TP, TransformDesc td, const T *__restrict__ mats_g,
                    const T *__restrict__ M, const uint8_t *__restrict__ mask, T *__restrict__ L,
                    T *__restrict__ E, T *__restrict__ Y, const T *__restrict__ G,
                    const T *__restrict__ Lam, T *__restrict__ Abar, TubeScalars sc,
                    unsigned long long *res, int *flags) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *mats = reinterpret_cast<T *>(smem_raw);
  T *tile = mats + td.mats_len;
  load_mats(mats, mats_g, td.mats_len);
  const int64_t p0 = (int64_t)blockIdx.x * TP;
  const int per_row = TP / VEC, total = n * per_row;
  const FwdK<T> scr = fwd_scalars<T>(resolve(sc));
  T rL = 0, rE = 0, rC = 0;
  int bad = 0;
  for (int e0 = threadIdx.x; e0 < total; e0 += kTubeThreads * kUnroll) {
    Pk<T, VEC> m[kUnroll], l0[kUnroll], ee[kUnroll], y0[kUnroll], g0[kUnroll], la[kUnroll];
    Pk<uint8_t, VEC> om[kUnroll];
    bool in[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int e = e0 + u * kTubeThreads;
      const PackIdx q = pack_idx(e, per_row, VEC);
      in[u] = e < total && p0 + q.p < P;
      if (in[u]) {
        const int64_t idx = (int64_t)q.j * P + p0 + q.p;
        m[u] = ld<T, VEC>(M + idx);
        om[u] = ldm<VEC>(mask + idx);
        l0[u] = ld<T, VEC>(L + idx);
        ee[u] = ld<T, VEC>(E + idx);
        y0[u] = ld<T, VEC>(Y + idx);
        g0[u] = ld<T, VEC>(G + idx);
        la[u] = ld<T, VEC>(Lam + idx);
      }
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int e = e0 + u * kTubeThreads;
      if (e >= total) continue;
      const PackIdx q = pack_idx(e, per_row, VEC);
      Pk<T, VEC> a;
      if (in[u]) {
        const int64_t idx = (int64_t)q.j * P + p0 + q.p;
        Pk<T, VEC> l1, e1, y1;
        forward_pack<T, VEC>(m[u], om[u], l0[u], ee[u], y0[u], g0[u], la[u], scr, l1, e1, y1, a,
                             rL, rE, rC, bad);
        st<T, VEC>(L + idx, l1);
        st<T, VEC>(E + idx, e1);
        st<T, VEC>(Y + idx, y1);
      } else {
#pragma unroll
        for (int i = 0; i < VEC; ++i) a.v[i] = T(0);
      }
      st<T, VEC>(tile + q.j * TP + q.p, a);
    }
  }
  __syncthreads();
  tile_transform<T, NK>(tile, n, TP, mats, td, false);
  store_abar<T, VEC>(Abar, tile, P, n, TP, p0, sc.planes);
  if (bad) atomicOr(flags, 1);
  const T v[3] = {rL, rE, rC};
  unsigned long long *const slots[3] = {res + RES_DL, res + RES_DE, res + RES_CONS};
  block_max_to_global<T, 3>(v, slots);
}

template <typename T, int NK, int VEC>
__global__ void __launch_bounds__(kTubeThreads, tube_min_blocks<T, NK>())
tube_inverse_kernel(int64_t P, int n, int TP, TransformDesc td, const T *__restrict__ mats_g,
                    const T *__restrict__ Gbar, const T *__restrict__ L, T *__restrict__ G,
                    T *__restrict__ Lam, double mu_d, const double *dmu,
                    unsigned long long *res, int *flags) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *mats = reinterpret_cast<T *>(smem_raw);
  T *tile = mats + td.mats_len;
  load_mats(mats, mats_g, td.mats_len);
  const int64_t p0 = (int64_t)blockIdx.x * TP;
  tile_load<T, VEC>(tile, Gbar, P, n, TP, p0);
  __syncthreads();
  tile_transform<T, NK>(tile, n, TP, mats, td, true);
  const T mu = T(dmu ? *dmu : mu_d);
  const int per_row = TP / VEC, total = n * per_row;
  T rLG = 0, rG = 0;
  int bad = 0;
  constexpr int U = 2;
  for (int e0 = threadIdx.x; e0 < total; e0 += kTubeThreads * U) {
    Pk<T, VEC> l1[U], g0[U], la[U];
    bool in[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * kTubeThreads;
      const PackIdx q = pack_idx(e, per_row, VEC);
      in[u] = e < total && p0 + q.p < P;
      if (in[u]) {
        const int64_t idx = (int64_t)q.j * P + p0 + q.p;
        l1[u] = ld<T, VEC>(L + idx);
        g0[u] = ld<T, VEC>(G + idx);
        la[u] = ld<T, VEC>(Lam + idx);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (!in[u]) continue;
      const int e = e0 + u * kTubeThreads;
      const PackIdx q = pack_idx(e, per_row, VEC);
      const int64_t idx = (int64_t)q.j * P + p0 + q.p;
      const Pk<T, VEC> g1 = ld<T, VEC>(tile + q.j * TP + q.p);
      Pk<T, VEC> la1;
#pragma unroll
      for (int i = 0; i < VEC; ++i) {
        la1.v[i] = la[u].v[i] + mu * (l1[u].v[i] - g1.v[i]);
        rLG = fmax(rLG, fabs(l1[u].v[i] - g1.v[i]));
        rG = fmax(rG, fabs(g1.v[i] - g0[u].v[i]));
        bad |= !(isfinite(g1.v[i]) && isfinite(la1.v[i]));
      }
      st<T, VEC>(G + idx, g1);
      st<T, VEC>(Lam + idx, la1);
    }
  }
  if (bad) atomicOr(flags, 1);
  const T v[2] = {rLG, rG};
  unsigned long long *const slots[2] = {res + RES_LG, res + RES_DG};
  block_max_to_global<T, 2>(v, slots);
}

// Inverse pass of iteration t-1 (mu_prev) + forward pass of iteration t (sc).
// ---- L2 prefetch of the fused pass's streams (FP32) -------------------------
// Tensor maps of the slice-major arrays (n rows of P positions) with boxes of
// TP positions x 1024 / TP rows: the rows that one iteration of the fused
// kernel's main loop reads (256 threads x 4 positions).  Thread 0 prefetches
// the Gbar tile and the first row chunk of M, L, E, Y, G, Lambda and the
// mask into L2 before the inverse transform, then one chunk per iteration,
// kPrefetchAhead ahead of the loads (no shared memory and no wait:
// cp.async.bulk.prefetch.tensor only warms L2).  One chunk ahead measured
// best (200 us against 213 us without prefetch on 400 slices of 200 x 200;
// three ahead 210 us, six ahead 245 us).
struct TubeMaps {
  CUtensorMap gbar, m, l, e, y, g, lam, mask;
};

constexpr int kPrefetchAhead = 1;

__device__ __forceinline__ void l2_prefetch_2d(const CUtensorMap *map, int x, int y) {
  asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(x), "r"(y)
               : "memory");
}

__device__ __forceinline__ void prefetch_chunk(const TubeMaps &tm, int p0, int row0) {
  l2_prefetch_2d(&tm.m, p0, row0);
  l2_prefetch_2d(&tm.l, p0, row0);
  l2_prefetch_2d(&tm.e, p0, row0);
  l2_prefetch_2d(&tm.y, p0, row0);
  l2_prefetch_2d(&tm.g, p0, row0);
  l2_prefetch_2d(&tm.lam, p0, row0);
  l2_prefetch_2d(&tm.mask, p0, row0);
}

template <typename T, int NK, int VEC, bool PF>
__global__ void __launch_bounds__(kTubeThreads, tube_min_blocks<T, NK>())
tube_fused_kernel(int64_t P, int n, int TP, TransformDesc td, const T *__restrict__ mats_g,
                  const T *__restrict__ Gbar, double mu_prev, const double *dmu_prev,
                  const T *__restrict__ M,
                  const uint8_t *__restrict__ mask, T *__restrict__ L, T *__restrict__ E,
                  T *__restrict__ Y, T *__restrict__ G, T *__restrict__ Lam,
                  T *__restrict__ Abar, TubeScalars sc, unsigned long long *res_prev,
                  unsigned long long *res, int *flags, const __grid_constant__ TubeMaps tm,
                  int RBG, int nbox) {
  pdl_wait();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *mats = reinterpret_cast<T *>(smem_raw);
  T *tile = mats + td.mats_len;
  const int64_t p0 = (int64_t)blockIdx.x * TP;
  const int rows_it = kTubeThreads * kUnroll / (TP / VEC);   // rows per main-loop iteration
  const int nit = (n + rows_it - 1) / rows_it;
  if (PF && threadIdx.x == 0) {
    for (int b = 0; b < nbox; ++b) l2_prefetch_2d(&tm.gbar, (int)p0, b * RBG);
    for (int c = 0; c < kPrefetchAhead && c < nit; ++c) prefetch_chunk(tm, (int)p0, c * rows_it);
  }
  load_mats(mats, mats_g, td.mats_len);
  tile_load<T, VEC>(tile, Gbar, P, n, TP, p0);
  __syncthreads();
  tile_transform<T, NK>(tile, n, TP, mats, td, true);
  const T mup = T(dmu_prev ? *dmu_prev : mu_prev);
  const FwdK<T> scr = fwd_scalars<T>(resolve(sc));
  const int per_row = TP / VEC, total = n * per_row;
  T rLG = 0, rG = 0, rL = 0, rE = 0, rC = 0;
  int bad = 0;
  for (int e0 = threadIdx.x, it = 0; e0 < total; e0 += kTubeThreads * kUnroll, ++it) {
    if (PF && threadIdx.x == 0 && it + kPrefetchAhead < nit)
      prefetch_chunk(tm, (int)p0, (it + kPrefetchAhead) * rows_it);
    Pk<T, VEC> m[kUnroll], l0[kUnroll], ee[kUnroll], y0[kUnroll], g0[kUnroll], la[kUnroll];
    Pk<uint8_t, VEC> om[kUnroll];
    bool in[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int e = e0 + u * kTubeThreads;
      const PackIdx q = pack_idx(e, per_row, VEC);
      in[u] = e < total && p0 + q.p < P;
      if (in[u]) {
        const int64_t idx = (int64_t)q.j * P + p0 + q.p;
        m[u] = ld<T, VEC>(M + idx);
        om[u] = ldm<VEC>(mask + idx);
        l0[u] = ld<T, VEC>(L + idx);
        ee[u] = ld<T, VEC>(E + idx);
        y0[u] = ld<T, VEC>(Y + idx);
        g0[u] = ld<T, VEC>(G + idx);
        la[u] = ld<T, VEC>(Lam + idx);
      }
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int e = e0 + u * kTubeThreads;
      if (e >= total) continue;
      const PackIdx q = pack_idx(e, per_row, VEC);
      Pk<T, VEC> a;
      if (in[u]) {
        const int64_t idx = (int64_t)q.j * P + p0 + q.p;
        const Pk<T, VEC> g1 = ld<T, VEC>(tile + q.j * TP + q.p);   // G^t
        Pk<T, VEC> la1;                                            // Lambda^t
#pragma unroll
        for (int i = 0; i < VEC; ++i) {
          la1.v[i] = la[u].v[i] + mup * (l0[u].v[i] - g1.v[i]);
          rLG = fmax(rLG, fabs(l0[u].v[i] - g1.v[i]));
          rG = fmax(rG, fabs(g1.v[i] - g0[u].v[i]));
        }
        Pk<T, VEC> l1, e1, y1;
        forward_pack<T, VEC>(m[u], om[u], l0[u], ee[u], y0[u], g1, la1, scr, l1, e1, y1, a, rL,
                             rE, rC, bad);
        st<T, VEC>(G + idx, g1);
        st<T, VEC>(Lam + idx, la1);
        st<T, VEC>(L + idx, l1);
        st<T, VEC>(E + idx, e1);
        st<T, VEC>(Y + idx, y1);
      } else {
#pragma unroll
        for (int i = 0; i < VEC; ++i) a.v[i] = T(0);
      }
      st<T, VEC>(tile + q.j * TP + q.p, a);
    }
  }
  __syncthreads();
  tile_transform<T, NK>(tile, n, TP, mats, td, false);
  store_abar<T, VEC>(Abar, tile, P, n, TP, p0, sc.planes);
  if (bad) atomicOr(flags, 1);
  const T v[5] = {rLG, rG, rL, rE, rC};
  unsigned long long *const slots[5] = {res_prev + RES_LG, res_prev + RES_DG, res + RES_DL,
                                        res + RES_DE, res + RES_CONS};
  block_max_to_global<T, 5>(v, slots);
  pdl_trigger();
}

template <typename T, int NK, int VEC>
__global__ void __launch_bounds__(kTubeThreads, tube_min_blocks<T, NK>())
transform_kernel(int64_t P, int n, int TP, TransformDesc td, const T *__restrict__ mats_g,
                 const T *__restrict__ src, T *__restrict__ dst, int inverse) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *mats = reinterpret_cast<T *>(smem_raw);
  T *tile = mats + td.mats_len;
  load_mats(mats, mats_g, td.mats_len);
  const int64_t p0 = (int64_t)blockIdx.x * TP;
  tile_load<T, VEC>(tile, src, P, n, TP, p0);
  __syncthreads();
  tile_transform<T, NK>(tile, n, TP, mats, td, inverse != 0);
  tile_store<T, VEC>(dst, tile, P, n, TP, p0);
}

template <typename T>
size_t tube_smem_for(int n, const TransformDesc &td, int TP) {
  return sizeof(T) * ((size_t)td.mats_len + (size_t)n * TP);
}

constexpr size_t kSmemBudget = 200 * 1024;

// Default tubes per block: a mode product has n / n_k fibres per tube, so a
// tile of TP tubes gives the block's threads (n / n_k) TP fibres; take the
// smallest power of two from 32 up to kMaxTP that gives every thread at least
// one fibre of every mode, then halve while the tile does not fit.
constexpr int kMaxTP = 256;

template <typename T>
int pick_tp(int n, const TransformDesc &td) {
  int nfib = n;
  for (int k = 0; k < td.nt; ++k) nfib = n / td.dim[k] < nfib ? n / td.dim[k] : nfib;
  if (nfib < 1) nfib = 1;
  int tp = 32;
  while (tp < kMaxTP && nfib * tp < kTubeThreads) tp <<= 1;
  while (tp > 4 && tube_smem_for<T>(n, td, tp) > kSmemBudget) tp >>= 1;
  return tube_smem_for<T>(n, td, tp) > kSmemBudget ? 0 : tp;
}

// Vector width usable for every pointer of a launch: 16-byte packs need
// P % VEC == 0 and 16-byte aligned bases (mask: VEC-byte aligned).
template <typename T>
int pick_vec(int64_t P, int tp, std::initializer_list<const void *> ptrs, const void *mask) {
  constexpr int V = 16 / sizeof(T);
  if (P % V != 0 || tp % V != 0) return 1;
  for (const void *p : ptrs)
    if (p && ((uintptr_t)p % 16) != 0) return 1;
  if (mask && ((uintptr_t)mask % V) != 0) return 1;
  return V;
}

template <typename K>
cudaError_t prep(K kern, size_t smem) {
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

// Dispatch on (NK, VEC) at run time.
template <typename T, template <typename, int, int> class Launcher, typename... Args>
cudaError_t dispatch(int nkpad, int vec, Args... args) {
  constexpr int V = 16 / sizeof(T);
#define TR_CASE(NKV)                                                                         \
  case NKV:                                                                                  \
    return vec == V ? Launcher<T, NKV, V>::run(args...) : Launcher<T, NKV, 1>::run(args...);
  switch (nkpad) {
    TR_CASE(8)
    TR_CASE(16)
    TR_CASE(24)
    TR_CASE(32)
    TR_CASE(40)
    TR_CASE(48)
    TR_CASE(56)
    TR_CASE(64)
    default: return cudaErrorInvalidValue;
  }
#undef TR_CASE
}

struct TubeLaunch {
  int64_t P;
  int n, tp;
  size_t smem;
  unsigned grid;
};

template <typename T>
bool tube_geometry(int64_t P, int n, const TransformDesc &td, TubeLaunch &g) {
  g.P = P;
  g.n = n;
  g.tp = pick_tp<T>(n, td);
  if (!g.tp) return false;
  if (td.tp > 0 && td.tp <= kMaxTP && (td.tp & (td.tp - 1)) == 0 &&
      tube_smem_for<T>(n, td, td.tp) <= kSmemBudget)
    g.tp = td.tp;
  if ((g.tp & (g.tp - 1)) != 0) return false;   // the kernels index tiles with shifts
  g.smem = tube_smem_for<T>(n, td, g.tp);
  g.grid = (unsigned)((P + g.tp - 1) / g.tp);
  return true;
}

template <typename T, int NK, int VEC>
struct FwdLauncher {
  static cudaError_t run(const TubeLaunch &g, const TransformDesc &td, const void *mats,
                         const void *M, const uint8_t *mask, void *L, void *E, void *Y,
                         const void *G, const void *Lam, void *Abar, const TubeScalars &sc,
                         unsigned long long *res, int *flags, cudaStream_t s) {
    auto k = tube_forward_kernel<T, NK, VEC>;
    cudaError_t e = prep(k, g.smem);
    if (e != cudaSuccess) return e;
    k<<<g.grid, kTubeThreads, g.smem, s>>>(g.P, g.n, g.tp, td, (const T *)mats, (const T *)M, mask,
                                          (T *)L, (T *)E, (T *)Y, (const T *)G, (const T *)Lam,
                                          (T *)Abar, sc, res, flags);
    return cudaGetLastError();
  }
};

template <typename T, int NK, int VEC>
struct InvLauncher {
  static cudaError_t run(const TubeLaunch &g, const TransformDesc &td, const void *mats,
                         const void *Gbar, const void *L, void *G, void *Lam, double mu,
                         const double *dmu, unsigned long long *res, int *flags,
                         cudaStream_t s) {
    auto k = tube_inverse_kernel<T, NK, VEC>;
    cudaError_t e = prep(k, g.smem);
    if (e != cudaSuccess) return e;
    k<<<g.grid, kTubeThreads, g.smem, s>>>(g.P, g.n, g.tp, td, (const T *)mats, (const T *)Gbar,
                                          (const T *)L, (T *)G, (T *)Lam, mu, dmu, res, flags);
    return cudaGetLastError();
  }
};

// Prefetch maps of a fused launch (pf: whether they are in use).
struct TubePrefetch {
  bool pf = false;
  int RBG = 0, nbox = 0;
  TubeMaps tm;
};

template <typename T, int NK, int VEC>
struct FusedLauncher {
  static cudaError_t run(const TubeLaunch &g, const TransformDesc &td, const void *mats,
                         const void *Gbar, double mu_prev, const double *dmu_prev,
                         const void *M, const uint8_t *mask, void *L, void *E, void *Y, void *G,
                         void *Lam, void *Abar, const TubeScalars &sc,
                         unsigned long long *res_prev, unsigned long long *res, int *flags,
                         const TubePrefetch &pf, cudaStream_t s) {
    auto k = tube_fused_kernel<T, NK, VEC, false>;
    if constexpr (sizeof(T) == 4 && VEC == 4)
      if (pf.pf) k = tube_fused_kernel<T, NK, VEC, true>;
    cudaError_t e = prep(k, g.smem);
    if (e != cudaSuccess) return e;
    return launch_pdl(k, dim3(g.grid), dim3(kTubeThreads), g.smem, s, g.P, g.n, g.tp, td,
                      (const T *)mats, (const T *)Gbar, mu_prev, dmu_prev, (const T *)M, mask,
                      (T *)L, (T *)E, (T *)Y, (T *)G, (T *)Lam, (T *)Abar, sc, res_prev, res,
                      flags, pf.tm, pf.RBG, pf.nbox);
  }
};

template <typename T, int NK, int VEC>
struct XfLauncher {
  static cudaError_t run(const TubeLaunch &g, const TransformDesc &td, const void *mats,
                         const void *src, void *dst, bool inverse, cudaStream_t s) {
    auto k = transform_kernel<T, NK, VEC>;
    cudaError_t e = prep(k, g.smem);
    if (e != cudaSuccess) return e;
    k<<<g.grid, kTubeThreads, g.smem, s>>>(g.P, g.n, g.tp, td, (const T *)mats, (const T *)src,
                                          (T *)dst, inverse ? 1 : 0);
    return cudaGetLastError();
  }
};

template <typename T>
cudaError_t fwd_t(int64_t P, int n, const TransformDesc &td, const void *mats, const void *M,
                  const uint8_t *mask, void *L, void *E, void *Y, const void *G, const void *Lam,
                  void *Abar, const TubeScalars &sc, unsigned long long *res, int *flags,
                  cudaStream_t s) {
  TubeLaunch g;
  if (!tube_geometry<T>(P, n, td, g)) return cudaErrorInvalidValue;
  const int vec = pick_vec<T>(P, g.tp, {M, L, E, Y, G, Lam, Abar}, mask);
  return dispatch<T, FwdLauncher>(td.nkpad, vec, g, td, mats, M, mask, L, E, Y, G, Lam, Abar, sc,
                                  res, flags, s);
}

template <typename T>
cudaError_t inv_t(int64_t P, int n, const TransformDesc &td, const void *mats, const void *Gbar,
                  const void *L, void *G, void *Lam, double mu, const double *dmu,
                  unsigned long long *res, int *flags, cudaStream_t s) {
  TubeLaunch g;
  if (!tube_geometry<T>(P, n, td, g)) return cudaErrorInvalidValue;
  const int vec = pick_vec<T>(P, g.tp, {Gbar, L, G, Lam}, nullptr);
  return dispatch<T, InvLauncher>(td.nkpad, vec, g, td, mats, Gbar, L, G, Lam, mu, dmu, res,
                                  flags, s);
}

// Prefetch maps for an FP32 fused launch with 16-byte packs, P and the tile
// a multiple of 16 (mask rows and tensor-copy x coordinates on 16-byte
// boundaries).  False: the launch runs without prefetch.
bool fused_prefetch_maps(const TubeLaunch &g, const void *Gbar, const void *M, const uint8_t *mask,
                         const void *L, const void *E, const void *Y, const void *G,
                         const void *Lam, TubePrefetch &pf) {
  if (g.P % 16 != 0 || g.tp % 16 != 0 || g.P > INT32_MAX) return false;
  const void *ptrs[8] = {Gbar, M, L, E, Y, G, Lam, mask};
  for (const void *p : ptrs)
    if ((uintptr_t)p % 16 != 0) return false;
  pf.nbox = (g.n + 255) / 256;
  pf.RBG = (g.n + pf.nbox - 1) / pf.nbox;
  const int rows = kTubeThreads * kUnroll / (g.tp / 4);
  if (rows < 1 || rows > 256) return false;
  pf.pf = encode_tensor_2d(&pf.tm.gbar, Gbar, false, g.P, g.n, g.P, g.tp, pf.RBG) &&
          encode_tensor_2d(&pf.tm.m, M, false, g.P, g.n, g.P, g.tp, rows) &&
          encode_tensor_2d(&pf.tm.l, L, false, g.P, g.n, g.P, g.tp, rows) &&
          encode_tensor_2d(&pf.tm.e, E, false, g.P, g.n, g.P, g.tp, rows) &&
          encode_tensor_2d(&pf.tm.y, Y, false, g.P, g.n, g.P, g.tp, rows) &&
          encode_tensor_2d(&pf.tm.g, G, false, g.P, g.n, g.P, g.tp, rows) &&
          encode_tensor_2d(&pf.tm.lam, Lam, false, g.P, g.n, g.P, g.tp, rows) &&
          encode_tensor_2d(&pf.tm.mask, mask, true, g.P, g.n, g.P, g.tp, rows);
  return pf.pf;
}

template <typename T>
cudaError_t fused_t(int64_t P, int n, const TransformDesc &td, const void *mats, const void *Gbar,
                    double mu_prev, const double *dmu_prev, const void *M, const uint8_t *mask,
                    void *L, void *E, void *Y, void *G, void *Lam, void *Abar,
                    const TubeScalars &sc, unsigned long long *res_prev, unsigned long long *res,
                    int *flags, cudaStream_t s) {
  TubeLaunch g;
  if (!tube_geometry<T>(P, n, td, g)) return cudaErrorInvalidValue;
  const int vec = pick_vec<T>(P, g.tp, {Gbar, M, L, E, Y, G, Lam, Abar}, mask);
  TubePrefetch pf;
  if (sizeof(T) == 4 && vec == 4) fused_prefetch_maps(g, Gbar, M, mask, L, E, Y, G, Lam, pf);
  return dispatch<T, FusedLauncher>(td.nkpad, vec, g, td, mats, Gbar, mu_prev, dmu_prev, M, mask,
                                    L, E, Y, G, Lam, Abar, sc, res_prev, res, flags, pf, s);
}

template <typename T>
cudaError_t xf_t(int64_t P, int n, const TransformDesc &td, const void *mats, const void *src,
                 void *dst, bool inverse, cudaStream_t s) {
  TubeLaunch g;
  if (!tube_geometry<T>(P, n, td, g)) return cudaErrorInvalidValue;
  const int vec = pick_vec<T>(P, g.tp, {src, dst}, nullptr);
  return dispatch<T, XfLauncher>(td.nkpad, vec, g, td, mats, src, dst, inverse, s);
}

}  // namespace

cudaError_t launch_tube_forward(tr_dtype dt, int64_t P, int n, const TransformDesc &td,
                                const void *mats, const void *M, const uint8_t *mask, void *L,
                                void *E, void *Y, const void *G, const void *Lam, void *Abar,
                                const TubeScalars &sc, unsigned long long *res, int *flags,
                                cudaStream_t s) {
  if (dt == TR_F64)
    return fwd_t<double>(P, n, td, mats, M, mask, L, E, Y, G, Lam, Abar, sc, res, flags, s);
  return fwd_t<float>(P, n, td, mats, M, mask, L, E, Y, G, Lam, Abar, sc, res, flags, s);
}

cudaError_t launch_tube_inverse(tr_dtype dt, int64_t P, int n, const TransformDesc &td,
                                const void *mats, const void *Gbar, const void *L, void *G,
                                void *Lam, double mu, const double *dmu, unsigned long long *res,
                                int *flags, cudaStream_t s) {
  if (dt == TR_F64) return inv_t<double>(P, n, td, mats, Gbar, L, G, Lam, mu, dmu, res, flags, s);
  return inv_t<float>(P, n, td, mats, Gbar, L, G, Lam, mu, dmu, res, flags, s);
}

cudaError_t launch_tube_fused(tr_dtype dt, int64_t P, int n, const TransformDesc &td,
                              const void *mats, const void *Gbar, double mu_prev,
                              const double *dmu_prev, const void *M, const uint8_t *mask, void *L,
                              void *E, void *Y, void *G, void *Lam, void *Abar,
                              const TubeScalars &sc, unsigned long long *res_prev,
                              unsigned long long *res, int *flags, cudaStream_t s) {
  if (dt == TR_F64)
    return fused_t<double>(P, n, td, mats, Gbar, mu_prev, dmu_prev, M, mask, L, E, Y, G, Lam,
                           Abar, sc, res_prev, res, flags, s);
  return fused_t<float>(P, n, td, mats, Gbar, mu_prev, dmu_prev, M, mask, L, E, Y, G, Lam, Abar,
                        sc, res_prev, res, flags, s);
}

__global__ void schedule_kernel(DevSched *d, double growth, double mu_max) {
  pdl_wait();
  const double next = growth * d->mu;
  d->mu_prev = d->mu;
  d->mu = next < mu_max ? next : mu_max;
  d->t += 1;
  pdl_trigger();
}

cudaError_t launch_schedule(DevSched *d, double growth, double mu_max, cudaStream_t s) {
  return launch_pdl(schedule_kernel, dim3(1), dim3(1), 0, s, d, growth, mu_max);
}

cudaError_t launch_transform(tr_dtype dt, int64_t P, int n, const TransformDesc &td,
                             const void *mats, const void *src, void *dst, bool inverse,
                             cudaStream_t s) {
  if (dt == TR_F64) return xf_t<double>(P, n, td, mats, src, dst, inverse, s);
  return xf_t<float>(P, n, td, mats, src, dst, inverse, s);
}

// Tile widths (tubes per block) that fit, for the autotuner.  The tile only
// partitions the tubes among blocks: every tube's arithmetic is the same.
int tube_tile_candidates(tr_dtype dt, int n, const TransformDesc &td, int *tps, int cap) {
  int k = 0;
  for (int tp = kMaxTP; tp >= 4 && k < cap; tp >>= 1) {
    const size_t b = dt == TR_F64 ? tube_smem_for<double>(n, td, tp) : tube_smem_for<float>(n, td, tp);
    if (b <= kSmemBudget) tps[k++] = tp;
  }
  return k;
}

size_t tube_smem_bytes(tr_dtype dt, int n, const TransformDesc &td, int *tp_out) {
  int tp = dt == TR_F64 ? pick_tp<double>(n, td) : pick_tp<float>(n, td);
  if (tp_out) *tp_out = tp;
  if (!tp) return 0;
  return dt == TR_F64 ? tube_smem_for<double>(n, td, tp) : tube_smem_for<float>(n, td, tp);
}

// Elements of the matrix buffer for the transformed modes: per mode the
// forward rows (dim x nkpad) and the folded inverse rows (ceil(dim/2) x 2 HK).
int transform_mats_layout(TransformDesc &td) {
  const int hk = ((td.nkpad / 2 + 3) / 4) * 4;
  int off = 0;
  for (int k = 0; k < td.nt; ++k) {
    td.off_fwd[k] = off;
    off += td.dim[k] * td.nkpad;
    td.off_inv[k] = off;
    off += ((td.dim[k] + 1) / 2) * 2 * hk;
  }
  td.mats_len = off < 4 ? 4 : ((off + 3) / 4) * 4;
  return hk;
}
