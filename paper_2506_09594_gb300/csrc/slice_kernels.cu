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
#include "tr_rng.cuh"
#include "umma_gemm.cuh"
#include "umma_tma.cuh"

namespace {

template <typename T>
__global__ void sketch_kernel(int64_t per_slice, T *__restrict__ Om, uint32_t k0, uint32_t k1,
                              uint32_t t_host, const int *dt, uint32_t stream, SliceSel sel) {
  pdl_wait();
  const uint32_t t = dt ? (uint32_t)*dt : t_host;
  const int b = blockIdx.y;
  if (sel.count && b >= *sel.count) return;
  const int j = sel.ids ? sel.ids[b] : b;
  const int64_t ngroups = (per_slice + 3) / 4;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ngroups;
       g += (int64_t)gridDim.x * blockDim.x) {
    uint32_t c[4] = {(uint32_t)g, (uint32_t)j, t, stream};
    trrng::philox4x32_10(c, k0, k1);
    T z[4];
    trrng::box_muller(c[0], c[1], z[0], z[1]);
    trrng::box_muller(c[2], c[3], z[2], z[3]);
    T *dst = Om + (int64_t)b * per_slice;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int64_t m = 4 * g + i;
      if (m < per_slice) dst[m] = z[i];
    }
  }
  pdl_trigger();
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
  // optional batch indirection (see SliceSel): A and/or C of entry b come
  // from batch sel.ids[b]; B always from entry b
  SliceSel sel{};
  int a_by_id = 0, c_by_id = 0;
};

template <typename T, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
bgemm_kernel(GemmArgs g) {
  pdl_wait();
  constexpr int NT = (BM / TM) * (BN / TN);
  __shared__ __align__(16) T As[BK][BM + 4];
  __shared__ __align__(16) T Bs[BK][BN + 4];
  const int tid = threadIdx.x;
  const int tx = tid % (BN / TN), ty = tid / (BN / TN);
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int64_t b = blockIdx.z;
  if (g.sel.count && b >= *g.sel.count) return;
  const int64_t jb = g.sel.ids ? g.sel.ids[b] : b;
  const T *A = (const T *)g.A + (g.a_by_id ? jb : b) * g.sAb;
  const T *B = (const T *)g.B + b * g.sBb;
  T *C = (T *)g.C + (g.c_by_id ? jb : b) * g.sCb;
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
  pdl_trigger();
}

template <typename T>
cudaError_t bgemm(const GemmArgs &g, int batch, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0 || batch <= 0) return cudaSuccess;
  if (g.N <= 32) {
    dim3 grid((g.M + 63) / 64, (g.N + 31) / 32, batch);
    cudaError_t e = launch_pdl(bgemm_kernel<T, 64, 32, 32, 4, 2>, grid, dim3(256), 0, s, g);
    if (e != cudaSuccess) return e;
  } else {
    dim3 grid((g.M + 63) / 64, (g.N + 63) / 64, batch);
    cudaError_t e = launch_pdl(bgemm_kernel<T, 64, 64, 16, 4, 4>, grid, dim3(256), 0, s, g);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

// Rank-l rebuild Gbar^<j> = Z Qb^T (n1 x n2, row-major) from the column-major
// panels Z (n1 x l) and Qb (n2 x l).  A CTA owns a BT x BT output tile (a
// whole slice for slices up to BT x BT) and stages the tile's rows of Z and
// of Qb k-major in shared memory (Zk[k][i], Qk[k][j]: copies of contiguous
// panel columns).  Each thread forms 8 x 4 outputs: per k two 16-byte reads
// of eight rows of Zk (the same address across most of a warp: a broadcast)
// and one of four columns of Qk (consecutive lanes, consecutive 16 bytes),
// 32 FMAs, and it writes its rows as 16-byte segments, consecutive lanes
// covering consecutive columns (scalar stores when n2 is not a multiple of
// 4).  Large tiles make few, long-lived CTAs whose stores stream back to
// back; the earlier 64 x 64 tiles spent most of their time loading.
template <typename T>
__device__ __forceinline__ void ld4s(const T *p, T (&v)[4]) {
  if constexpr (sizeof(T) == 4) {
    const float4 x = *reinterpret_cast<const float4 *>(p);
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
  } else {
    const double2 x = *reinterpret_cast<const double2 *>(p);
    const double2 y = *reinterpret_cast<const double2 *>(p + 2);
    v[0] = x.x; v[1] = x.y; v[2] = y.x; v[3] = y.y;
  }
}

template <typename T>
__global__ void __launch_bounds__(256)
rank_update_kernel(int n1, int n2, int l, int BT, const T *__restrict__ Z, int64_t sZ,
                   const T *__restrict__ Qb, int64_t sQ, T *__restrict__ C, int64_t sC,
                   int vec_ok, SliceSel sel) {
  pdl_wait();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *Zk = reinterpret_cast<T *>(smem_raw);          // [l][BT]
  T *Qk = Zk + (size_t)l * BT;                      // [l][BT]
  const int r0 = blockIdx.x * BT, c0 = blockIdx.y * BT;
  const int64_t b = blockIdx.z;
  if (sel.count && b >= *sel.count) return;
  const int64_t jb = sel.ids ? sel.ids[b] : b;
  const T *Zb = Z + b * sZ;
  const T *Qbb = Qb + b * sQ;
  const int tr = n1 - r0 < BT ? n1 - r0 : BT, tc = n2 - c0 < BT ? n2 - c0 : BT;
  // eight element pairs per thread in flight (BT is a power of two)
  const int lgbt = 31 - __clz(BT);
  constexpr int UL = 8;
  for (int e0 = threadIdx.x; e0 < l * BT; e0 += 256 * UL) {
    T za[UL], qa[UL];
#pragma unroll
    for (int u = 0; u < UL; ++u) {
      const int e = e0 + u * 256, k = e >> lgbt, i = e & (BT - 1);
      const bool in = e < l * BT;
      za[u] = in && i < tr ? Zb[(int64_t)k * n1 + r0 + i] : T(0);
      qa[u] = in && i < tc ? Qbb[(int64_t)k * n2 + c0 + i] : T(0);
    }
#pragma unroll
    for (int u = 0; u < UL; ++u) {
      const int e = e0 + u * 256;
      if (e < l * BT) {
        Zk[e] = za[u];
        Qk[e] = qa[u];
      }
    }
  }
  __syncthreads();
  T *Cb = C + jb * sC;
  // tasks of 8 rows x 4 columns; consecutive threads take consecutive column groups
  const int RG = (tr + 7) / 8, CG = (tc + 3) / 4;
  int rg = threadIdx.x / CG, cg = threadIdx.x % CG;
  const int step_r = 256 / CG, step_c = 256 % CG;
  for (int t = threadIdx.x; t < RG * CG; t += 256) {
    T acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) acc[i][jj] = T(0);
    const T *za = Zk + rg * 8, *qa = Qk + cg * 4;
    for (int k = 0; k < l; ++k) {
      T a[8], q[4];
      ld4s(za + (size_t)k * BT, *reinterpret_cast<T(*)[4]>(a));
      ld4s(za + (size_t)k * BT + 4, *reinterpret_cast<T(*)[4]>(a + 4));
      ld4s(qa + (size_t)k * BT, q);
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) acc[i][jj] = fma(a[i], q[jj], acc[i][jj]);
    }
    const int col = c0 + cg * 4;
    const bool vec = sizeof(T) == 4 && vec_ok && col + 4 <= n2;
    T *dst = Cb + (int64_t)(r0 + rg * 8) * n2 + col;
#pragma unroll
    for (int i = 0; i < 8; ++i, dst += n2) {
      if (rg * 8 + i >= tr) break;
      if (vec) {
        *reinterpret_cast<float4 *>(dst) =
            make_float4((float)acc[i][0], (float)acc[i][1], (float)acc[i][2], (float)acc[i][3]);
      } else {
#pragma unroll
        for (int jj = 0; jj < 4; ++jj)
          if (col + jj < c0 + tc) dst[jj] = acc[i][jj];
      }
    }
    // next task: t + 256 = (rg + step_r) CG + cg + step_c
    rg += step_r;
    cg += step_c;
    if (cg >= CG) {
      cg -= CG;
      ++rg;
    }
  }
  pdl_trigger();
}

template <typename T>
cudaError_t rank_update(int n, int n1, int n2, int l, const T *Z, const T *Qb, T *C,
                        cudaStream_t s, SliceSel sel = SliceSel{}) {
  // the largest tile (256, 128 or 64) whose staged panels take at most 96 KB,
  // so that two CTAs share an SM
  int BT = 256;
  while (BT > 64 && 2 * (size_t)l * BT * sizeof(T) > 96 * 1024) BT >>= 1;
  const size_t smem = 2 * (size_t)l * BT * sizeof(T);
  cudaError_t e = cudaFuncSetAttribute(rank_update_kernel<T>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const dim3 grid((n1 + BT - 1) / BT, (n2 + BT - 1) / BT, n);
  // 16-byte row stores need n2 % 4 == 0 and a 16-byte aligned base
  const int vec_ok = (n2 % 4 == 0) && ((uintptr_t)C % 16 == 0);
  return launch_pdl(rank_update_kernel<T>, grid, dim3(256), smem, s, n1, n2, l, BT, Z,
                    (int64_t)n1 * l, Qb, (int64_t)n2 * l, C, (int64_t)n1 * n2, vec_ok, sel);
}

// Skinny product on the tensor cores (FP32 in/out, column tiles of up to
// 128): split = 1 is
// BF16 operands, split = 3 the hi/lo split (FP32-level accuracy).
cudaError_t umma_gemm(const GemmArgs &g, int batch, int split, int *err, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0 || batch <= 0) return cudaSuccess;
  umma::Args a{g.M, g.N, g.K, (const float *)g.A, g.sAb, g.sAi, g.sAk, (const float *)g.B,
               g.sBb, g.sBk, g.sBn, (float *)g.C, g.sCb, g.sCi, g.sCn,
               g.sel.ids, g.sel.count, g.a_by_id, g.c_by_id};
  // the operand A (Abar) is streamed from HBM; its next K chunk is prefetched
  // into L2 when A is a plain slice-major array
  if (g.sAk == 1 && g.sAb == (int64_t)g.M * g.sAi)
    a.a_pf = encode_tensor_2d(&a.amap, g.A, false, g.K, (int64_t)batch * g.M, g.sAi, umma::kKC,
                              umma::kBM);
  else if (g.sAi == 1 && g.sAb == (int64_t)g.K * g.sAk)
    a.a_pf = encode_tensor_2d(&a.amap, g.A, false, g.M, (int64_t)batch * g.K, g.sAk, umma::kBM,
                              umma::kKC);
  const unsigned ntiles = g.N <= 128 ? 1u : (unsigned)((g.N + 127) / 128);
  const dim3 grid((g.M + umma::kBM - 1) / umma::kBM, ntiles, batch);
#define TR_UMMA(NP, SP)                                                                        \
  {                                                                                            \
    auto k = umma::gemm_kernel<NP, SP>;                                                        \
    const int smem = umma::Layout<NP, SP>::total;                                              \
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem); \
    if (e != cudaSuccess) return e;                                                            \
    return launch_pdl(k, grid, dim3(umma::kThreads), smem, s, a, err);                        \
  }
  if (g.N <= 32) {
    if (split > 1) TR_UMMA(32, 3) else TR_UMMA(32, 1)
  }
  if (g.N <= 64) {
    if (split > 1) TR_UMMA(64, 3) else TR_UMMA(64, 1)
  }
  if (split > 1) TR_UMMA(128, 3) else TR_UMMA(128, 1)
#undef TR_UMMA
}

// The same product with TMA-fed operands (tmag::gemm_kernel) when the views
// allow 3D tensor copies: N <= 64, B with k contiguous, A with k or m
// contiguous, 16-byte strides.  *used is false (and nothing is launched)
// otherwise.  nA: slices in A's array when A is addressed by slice id.
cudaError_t tma_gemm(const GemmArgs &g, int batch, int nA, int split, int *err, cudaStream_t s,
                     bool *used) {
  *used = false;
  if (g.M <= 0 || g.N <= 0 || g.K <= 0 || batch <= 0 || g.N > 64 || g.sBk != 1) return cudaSuccess;
  tmag::Args a{};
  const int64_t za = g.a_by_id ? (int64_t)nA : (int64_t)batch;
  bool ok;
  if (g.sAk == 1) {
    a.a_kcontig = 1;
    ok = encode_tensor_3d_f32(&a.amap, g.A, g.K, g.M, za, g.sAi, g.sAb, tmag::kKC, tmag::kBM, true);
  } else if (g.sAi == 1) {
    a.a_kcontig = 0;
    ok = encode_tensor_3d_f32(&a.amap, g.A, g.M, g.K, za, g.sAk, g.sAb, tmag::kBM, tmag::kKC, false);
  } else {
    return cudaSuccess;
  }
  const int np = g.N <= 32 ? 32 : 64;
  ok = ok && encode_tensor_3d_f32(&a.bmap, g.B, g.K, g.N, batch, g.sBn,
                                  g.sBb > 0 ? g.sBb : (int64_t)g.N * g.sBn, tmag::kKC, np, true);
  if (!ok) return cudaSuccess;
  a.M = g.M;
  a.N = g.N;
  a.K = g.K;
  a.C = (float *)g.C;
  a.sCb = g.sCb;
  a.sCi = g.sCi;
  a.sCn = g.sCn;
  a.ids = g.sel.ids;
  a.count = g.sel.count;
  a.a_by_id = g.a_by_id;
  a.c_by_id = g.c_by_id;
  a.batch = batch;
  // persistent: two CTAs per SM (their shared memory allows two), or one per
  // tile when there are fewer tiles
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
      sms = 1;
  }
  const int64_t tiles = (int64_t)((g.M + tmag::kBM - 1) / tmag::kBM) * batch;
  const dim3 grid((unsigned)(tiles < 2 * sms ? tiles : 2 * sms), 1, 1);
  *used = true;
#define TR_TMAG(NP, ST, SP)                                                                    \
  {                                                                                            \
    auto k = tmag::gemm_kernel<NP, ST, SP>;                                                    \
    const int smem = tmag::Layout<NP, ST, SP>::total + 1024;                                   \
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem); \
    if (e != cudaSuccess) return e;                                                            \
    return launch_pdl(k, grid, dim3(tmag::kThreads), smem, s, a, err);                        \
  }
  if (np == 32) {
    if (split > 1) TR_TMAG(32, 3, 3) else TR_TMAG(32, 3, 1)
  }
  if (split > 1) TR_TMAG(64, 2, 3) else TR_TMAG(64, 2, 1)
#undef TR_TMAG
}

__global__ void split_planes_kernel(const float *__restrict__ x, __nv_bfloat16 *__restrict__ dst,
                                    int64_t count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float v = x[i];
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    dst[i] = hi;
    dst[count + i] = __float2bfloat16_rn(v - __bfloat162float(hi));
  }
}

cudaError_t split_planes(const float *x, void *dst, int64_t count, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  int64_t blocks = (count + 255) / 256;
  if (blocks > 8192) blocks = 8192;
  split_planes_kernel<<<(unsigned)blocks, 256, 0, s>>>(x, (__nv_bfloat16 *)dst, count);
  return cudaGetLastError();
}

// Whether the split planes of an n x n1 x n2 FP32 stack serve the TMA-fed
// products: rows of n2 BF16 and slices of n1 n2 BF16 at 16-byte multiples,
// FP32 panel columns of n1 and n2 at 16-byte multiples (the B operands), and
// panels of at most 64 columns.
bool planes_view_ok(int64_t n, int n1, int n2, int l) {
  return n >= 1 && n1 >= 1 && n2 >= 1 && l >= 1 && l <= 64 && n2 % 8 == 0 && n1 % 4 == 0;
}

// The product with A given as BF16 planes (A = hi + lo, tmag::planes_kernel).
// hi, lo: the planes of A's array, laid out as g.A's FP32 view would be
// (strides g.sAi, g.sAk, g.sAb in elements).  Fails (cudaErrorNotSupported)
// when the views do not allow it: the planes have no FP32 fallback.
cudaError_t tma_gemm_planes(const GemmArgs &g, int batch, int nA, int split, const void *hi,
                            const void *lo, int *err, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0 || g.K <= 0 || batch <= 0) return cudaSuccess;
  if (g.N > 64 || g.sBk != 1) return cudaErrorNotSupported;
  tmag::Args a{};
  const int64_t za = g.a_by_id ? (int64_t)nA : (int64_t)batch;
  bool ok;
  if (g.sAk == 1) {
    a.a_kcontig = 1;
    ok = encode_tensor_3d(&a.amap, hi, 2, g.K, g.M, za, g.sAi, g.sAb, tmag::kKP, tmag::kBM, true) &&
         (split == 1 ||
          encode_tensor_3d(&a.amap_lo, lo, 2, g.K, g.M, za, g.sAi, g.sAb, tmag::kKP, tmag::kBM, true));
  } else if (g.sAi == 1) {
    a.a_kcontig = 0;
    ok = encode_tensor_3d(&a.amap, hi, 2, g.M, g.K, za, g.sAk, g.sAb, 64, tmag::kKP, true) &&
         (split == 1 ||
          encode_tensor_3d(&a.amap_lo, lo, 2, g.M, g.K, za, g.sAk, g.sAb, 64, tmag::kKP, true));
  } else {
    return cudaErrorNotSupported;
  }
  const int np = g.N <= 32 ? 32 : 64;
  ok = ok && encode_tensor_3d_f32(&a.bmap, g.B, g.K, g.N, batch, g.sBn,
                                  g.sBb > 0 ? g.sBb : (int64_t)g.N * g.sBn, 32, np, true);
  if (!ok) return cudaErrorNotSupported;
  a.M = g.M;
  a.N = g.N;
  a.K = g.K;
  a.C = (float *)g.C;
  a.sCb = g.sCb;
  a.sCi = g.sCi;
  a.sCn = g.sCn;
  a.ids = g.sel.ids;
  a.count = g.sel.count;
  a.a_by_id = g.a_by_id;
  a.c_by_id = g.c_by_id;
  a.batch = batch;
  // persistent, one CTA per SM (its shared memory holds 4-5 stages)
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
      sms = 1;
  }
  const int64_t tiles = (int64_t)((g.M + tmag::kBM - 1) / tmag::kBM) * batch;
  const dim3 grid((unsigned)(tiles < sms ? tiles : sms), 1, 1);
#define TR_TMAP(NP, ST, SP)                                                                    \
  {                                                                                            \
    auto k = tmag::planes_kernel<NP, ST, SP>;                                                  \
    const int smem = tmag::PlanesLayout<NP, ST, SP>::total + 1024;                             \
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem); \
    if (e != cudaSuccess) return e;                                                            \
    return launch_pdl(k, grid, dim3(tmag::kPlanesThreads), smem, s, a, err);                  \
  }
  if (np == 32) {
    if (split > 1) TR_TMAP(32, 5, 3) else TR_TMAP(32, 5, 1)
  }
  if (split > 1) TR_TMAP(64, 4, 3) else TR_TMAP(64, 4, 1)
#undef TR_TMAP
}

// -------------------------------------------------- block Householder QR
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Register-resident Householder QR of an m x l column-major panel
// (l <= m <= 32*RPL).  Column c lives in the registers of warp c mod nw
// (slot q = c / nw < CPW); lane `lane` holds rows lane + 32 r, r < RPL.
// Reflector k (LAPACK geqr2 convention: H_k = I - tau_k v v^T, v = (1,
// x[k+1:]/(x_k - beta)), H_k x = beta e_k, beta = -sign(x_k) ||x[k:]||) is
// published in shared memory V (column k, rows > k) with tau[k].  The
// factorisation needs one barrier per column; forming Q = H_0...H_{l-1}[I;0]
// needs none, since every warp then updates only its own columns against
// the read-only reflectors.
template <typename T, int CPW, int RPL>
struct RegPanel {
  T x[CPW][RPL];

  __device__ __forceinline__ static int owner_slot(int c, int warp, int nw) {
    return (c % nw) == warp ? c / nw : -1;
  }

  __device__ __forceinline__ void load(const T *P, int ldp, int m, int l, int warp, int nw,
                                       int lane) {
#pragma unroll
    for (int q = 0; q < CPW; ++q) {
      const int c = warp + q * nw;
#pragma unroll
      for (int r = 0; r < RPL; ++r) {
        const int i = lane + 32 * r;
        x[q][r] = (c < l && i < m) ? P[(size_t)c * ldp + i] : T(0);
      }
    }
  }

  __device__ __forceinline__ void store(T *Q, int ldq, int m, int l, int warp, int nw, int lane) const {
#pragma unroll
    for (int q = 0; q < CPW; ++q) {
      const int c = warp + q * nw;
      if (c >= l) continue;
#pragma unroll
      for (int r = 0; r < RPL; ++r) {
        const int i = lane + 32 * r;
        if (i < m) Q[(size_t)c * ldq + i] = x[q][r];
      }
    }
  }

  // Householder reflector of slot qs's column (rows k..m-1); v -> V[k],
  // tau -> tau[k].  The slot is copied out through a static loop so that
  // the panel stays in registers.
  __device__ __forceinline__ void reflector(int qs, int k, int m, int lane, T *Vk, T *tau) {
    T col[RPL];
#pragma unroll
    for (int r = 0; r < RPL; ++r) {
      col[r] = x[0][r];
#pragma unroll
      for (int q = 1; q < CPW; ++q)
        if (q == qs) col[r] = x[q][r];
    }
    T ss = T(0), xk = T(0);
#pragma unroll
    for (int r = 0; r < RPL; ++r) {
      const int i = lane + 32 * r;
      if (i > k && i < m) ss = fma(col[r], col[r], ss);
      if (r == (k >> 5)) xk = col[r];
    }
    ss = warp_sum(ss);
    const T x0 = __shfl_sync(0xffffffffu, xk, k & 31);
    T beta = x0, tk = T(0), scale = T(0);
    if (ss > T(0)) {
      const T nrm = sqrt(fma(x0, x0, ss));
      beta = x0 >= T(0) ? -nrm : nrm;
      tk = (beta - x0) / beta;
      scale = T(1) / (x0 - beta);
    }
#pragma unroll
    for (int r = 0; r < RPL; ++r) {
      const int i = lane + 32 * r;
      if (i > k && i < m) {
        col[r] *= scale;
        Vk[i] = col[r];
      } else if (i == k) {
        col[r] = beta;
      }
    }
#pragma unroll
    for (int q = 0; q < CPW; ++q)
      if (q == qs)
#pragma unroll
        for (int r = 0; r < RPL; ++r) x[q][r] = col[r];
    if (lane == 0) tau[k] = tk;
  }

  // Apply H_k to the owned columns c >= c_lo (c < l).
  __device__ __forceinline__ void apply(const T *Vk, T tk, int k, int m, int l, int c_lo, int warp,
                                        int nw, int lane) {
    T v[RPL];
#pragma unroll
    for (int r = 0; r < RPL; ++r) {
      const int i = lane + 32 * r;
      v[r] = (i > k && i < m) ? Vk[i] : (i == k ? T(1) : T(0));
    }
#pragma unroll
    for (int q = 0; q < CPW; ++q) {
      const int c = warp + q * nw;
      if (c < c_lo || c >= l) continue;   // warp-uniform
      T s = T(0);
#pragma unroll
      for (int r = 0; r < RPL; ++r) s = fma(v[r], x[q][r], s);
      s = tk * warp_sum(s);
#pragma unroll
      for (int r = 0; r < RPL; ++r) x[q][r] = fma(-s, v[r], x[q][r]);
    }
  }
};

// QR of the panel P (global, column-major m x l, ld m): R (l x l, column-
// major, zero below the diagonal) to Rout when non-null, Q overwrites P.
// FORM_Q = false stops after R (P is left as it was).
template <typename T, int CPW, int RPL, bool FORM_Q = true>
__device__ void block_reg_qr(T *P, int m, int l, T *V, T *tau, T *Rout) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  RegPanel<T, CPW, RPL> pn;
  pn.load(P, m, m, l, warp, nw, lane);
  {
    const int q0 = RegPanel<T, CPW, RPL>::owner_slot(0, warp, nw);
    if (q0 >= 0) pn.reflector(q0, 0, m, lane, V, tau);
  }
  __syncthreads();
  for (int k = 0; k < l; ++k) {
    pn.apply(V + (size_t)k * m, tau[k], k, m, l, k + 1, warp, nw, lane);
    if (k + 1 < l) {
      const int q1 = RegPanel<T, CPW, RPL>::owner_slot(k + 1, warp, nw);
      if (q1 >= 0) pn.reflector(q1, k + 1, m, lane, V + (size_t)(k + 1) * m, tau);
    }
    __syncthreads();
  }
  if (Rout) {
#pragma unroll
    for (int q = 0; q < CPW; ++q) {
      const int c = warp + q * nw;
      if (c >= l) continue;
#pragma unroll
      for (int r = 0; r < RPL; ++r) {
        const int i = lane + 32 * r;
        if (i < l) Rout[(size_t)c * l + i] = i <= c ? pn.x[q][r] : T(0);
      }
    }
  }
  if (!FORM_Q) return;
  // form Q in registers: start from [I; 0] on the owned columns
#pragma unroll
  for (int q = 0; q < CPW; ++q) {
    const int c = warp + q * nw;
#pragma unroll
    for (int r = 0; r < RPL; ++r) pn.x[q][r] = (lane + 32 * r == c) ? T(1) : T(0);
  }
  for (int k = l - 1; k >= 0; --k) pn.apply(V + (size_t)k * m, tau[k], k, m, l, k, warp, nw, lane);
  pn.store(P, m, m, l, warp, nw, lane);
}

// Shared-memory Householder QR, for panels too large for the register file
// (same reflectors as block_reg_qr).  The panel S (column-major, ld m) holds
// v_k below the diagonal of column k and R on and above it.  Column c
// belongs to warp c mod nw; the owner of column k+1 builds reflector k+1 as
// soon as it has applied H_k, so the factorisation needs one barrier per
// column.  Q is then formed in place backwards (LAPACK org2r order), two
// barriers per column.
template <typename T>
__device__ void smem_reflector(T *col, int k, int m, int lane, T *tau) {
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
  __syncwarp();
}

template <typename T>
__device__ __forceinline__ void smem_apply(const T *v, T tk, T *col, int k, int m, int lane) {
  const T ck = col[k];
  T s = T(0);
  for (int i = k + 1 + lane; i < m; i += 32) s = fma(v[i], col[i], s);
  s = warp_sum(s) + ck;
  const T w = tk * s;
  for (int i = k + 1 + lane; i < m; i += 32) col[i] = fma(-w, v[i], col[i]);
  __syncwarp();
  if (lane == 0) col[k] = ck - w;
  __syncwarp();
}

// QR of P (global, column-major m x l, ld m) through the shared panel S
// (m * l) and tau (l): R to Rout when non-null, Q overwrites P.
template <typename T, bool FORM_Q = true>
__device__ void block_smem_qr(T *P, int m, int l, T *S, T *tau, T *Rout) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int e = threadIdx.x; e < m * l; e += blockDim.x) S[e] = P[e];
  __syncthreads();
  if (warp == 0) smem_reflector(S, 0, m, lane, tau);
  __syncthreads();
  for (int k = 0; k < l; ++k) {
    const T tk = tau[k];
    const T *v = S + (size_t)k * m;
    for (int c = warp; c < l; c += nw) {
      if (c <= k) continue;
      smem_apply(v, tk, S + (size_t)c * m, k, m, lane);
      if (c == k + 1) smem_reflector(S + (size_t)c * m, c, m, lane, tau);
    }
    __syncthreads();
  }
  if (Rout)
    for (int e = threadIdx.x; e < l * l; e += blockDim.x) {
      const int i = e % l, c = e / l;
      Rout[e] = i <= c ? S[(size_t)c * m + i] : T(0);
    }
  if (!FORM_Q) return;
  for (int k = l - 1; k >= 0; --k) {
    const T tk = tau[k];
    const T *v = S + (size_t)k * m;
    for (int c = warp; c < l; c += nw)
      if (c > k) smem_apply(v, tk, S + (size_t)c * m, k, m, lane);
    __syncthreads();
    T *colk = S + (size_t)k * m;
    for (int i = threadIdx.x; i < m; i += blockDim.x)
      colk[i] = i < k ? T(0) : (i == k ? T(1) - tk : -tk * colk[i]);
    __syncthreads();
  }
  for (int e = threadIdx.x; e < m * l; e += blockDim.x) P[e] = S[e];
}

template <typename T>
__global__ void qr_smem_kernel(int m, int l, T *__restrict__ P, int64_t sP, SliceSel sel) {
  pdl_wait();
  if (sel.count && (int)blockIdx.x >= *sel.count) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *S = reinterpret_cast<T *>(smem_raw);
  block_smem_qr<T>(P + (int64_t)blockIdx.x * sP, m, l, S, S + (size_t)m * l, nullptr);
  pdl_trigger();
}

template <typename T, int CPW, int RPL>
__global__ void qr_kernel(int m, int l, T *__restrict__ P, int64_t sP, SliceSel sel) {
  pdl_wait();
  if (sel.count && (int)blockIdx.x >= *sel.count) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *V = reinterpret_cast<T *>(smem_raw);
  T *tau = V + (size_t)m * l;
  block_reg_qr<T, CPW, RPL>(P + (int64_t)blockIdx.x * sP, m, l, V, tau, nullptr);
  pdl_trigger();
}

// ------------------------------------- Gram-Schmidt QR for narrow panels
// Classical Gram-Schmidt with reorthogonalisation ("twice is enough") for
// panels of at most 32 columns: thread t holds rows t + r*blockDim (r < RPT)
// of every column in registers, so a column's projection coefficients
// against all previous columns (and its squared norm) come from one block
// reduction per pass, and Q needs no separate formation.  A column is
// accepted after a pass that kept more than half of its squared norm, or
// after a second or later pass that kept a quarter (it is then orthogonal to
// the previous columns to working precision); the final norm follows from
// the last pass by Pythagoras.  A column that stays numerically dependent
// after four passes restarts from the next unit vector e_u (its R entries
// are the coefficients found so far, R_jj = 0): Q is always orthonormal and
// Q R reproduces the panel.  Same span and R up to column signs as the
// Householder QR, which the parity tests compare through the slice prox.
constexpr int kCgsCols = 32;

// Sum of V values over the block: `p` per thread in, every thread reads the
// totals from coef[0..V).  Within a warp a reduce-scatter butterfly: at the
// level of lane bit b every lane keeps half of its values (the upper half
// when its bit b is set) and adds its partner's copy of that half, so VP
// values (V padded to a power of two) cost VP - 1 shuffles plus one per
// remaining level, and lane L ends with the sum of value idx(L) (the lane's
// high log2(VP) bits).  red holds nw x 33 partials.
template <typename T, int V>
__device__ __forceinline__ void block_sum_vec(T (&p)[kCgsCols + 1], T *red, T *coef) {
  constexpr int VP = V <= 1 ? 1 : V <= 2 ? 2 : V <= 4 ? 4 : V <= 8 ? 8 : V <= 16 ? 16 : 32;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
#pragma unroll
  for (int v = V; v < VP; ++v) p[v] = T(0);
  int idx = 0;
#pragma unroll
  for (int h = VP / 2, o = 16; h >= 1; h >>= 1, o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int k = 0; k < h; ++k) {
      const T give = up ? p[k] : p[k + h];
      const T keep = up ? p[k + h] : p[k];
      p[k] = keep + __shfl_xor_sync(0xffffffffu, give, o);
    }
    idx += up ? h : 0;
  }
  constexpr int LOW = 32 / VP;   // lanes still holding partial sums of one value
#pragma unroll
  for (int o = LOW / 2; o > 0; o >>= 1) p[0] += __shfl_xor_sync(0xffffffffu, p[0], o);
  if ((lane & (LOW - 1)) == 0 && idx < V) red[warp * (kCgsCols + 1) + idx] = p[0];
  __syncthreads();
  if (warp == 0 && lane < V) {
    T t = T(0);
    for (int w = 0; w < nw; ++w) t += red[w * (kCgsCols + 1) + lane];
    coef[lane] = t;
  }
  __syncthreads();
}

template <typename T, int RPT, int J>
__device__ __forceinline__ void cgs_column(T (&x)[RPT][kCgsCols], int m, int l, T *Rout, T *red,
                                           T *coef) {
  const int tid = threadIdx.x, nthr = blockDim.x;
  const T tiny = sizeof(T) == 4 ? T(FLT_MIN) : T(DBL_MIN);
  int pass = 0, unit = -1, restarts = 0;
  T after = T(0);
  while (true) {
    T p[kCgsCols + 1];
#pragma unroll
    for (int i = 0; i <= J; ++i) p[i] = T(0);
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
#pragma unroll
      for (int i = 0; i < J; ++i) p[i] = fma(x[r][i], x[r][J], p[i]);
      p[J] = fma(x[r][J], x[r][J], p[J]);
    }
    block_sum_vec<T, J + 1>(p, red, coef);
    T c[kCgsCols];
    T csq = T(0);
#pragma unroll
    for (int i = 0; i < J; ++i) {
      c[i] = coef[i];
      csq = fma(c[i], c[i], csq);
    }
    const T s = coef[J];
#pragma unroll
    for (int r = 0; r < RPT; ++r)
#pragma unroll
      for (int i = 0; i < J; ++i) x[r][J] = fma(-c[i], x[r][i], x[r][J]);
    if (Rout && unit < 0 && tid < J) {
#pragma unroll
      for (int i = 0; i < J; ++i)
        if (i == tid) Rout[(size_t)J * l + i] += c[i];
    }
    after = s - csq;
    ++pass;
    // accept: a pass that kept more than half the squared norm leaves the
    // column orthogonal to working precision; after a second pass, a
    // quarter suffices
    if (after > tiny && (after > T(0.5) * s || (pass >= 2 && after > T(0.25) * s))) break;
    if (pass >= 4) {   // numerically dependent: continue from a unit vector
      if (++restarts > m) break;
      unit = unit < 0 ? J % m : (unit + 1) % m;
#pragma unroll
      for (int r = 0; r < RPT; ++r) x[r][J] = (tid + r * nthr == unit) ? T(1) : T(0);
      pass = 0;
    }
  }
  const T nrm = sqrt(after > T(0) ? after : T(0));
  const T inv = nrm > T(0) ? T(1) / nrm : T(0);
#pragma unroll
  for (int r = 0; r < RPT; ++r) x[r][J] *= inv;
  if (Rout && tid == 0) Rout[(size_t)J * l + J] = unit < 0 ? nrm : T(0);
}

template <typename T, int RPT, int J>
__device__ __forceinline__ void cgs_columns(T (&x)[RPT][kCgsCols], int m, int l, T *Rout, T *red,
                                            T *coef) {
  if constexpr (J < kCgsCols) {
    if (J >= l) return;
    cgs_column<T, RPT, J>(x, m, l, Rout, red, coef);
    cgs_columns<T, RPT, J + 1>(x, m, l, Rout, red, coef);
  }
}

// QR of P (global, column-major m x l, ld m, l <= 32, m <= RPT * blockDim):
// Q overwrites P, R (l x l, column-major, zero below the diagonal) goes to
// Rout (shared memory) when non-null.  red: (blockDim/32) x 33, coef: 33
// elements of shared memory.
template <typename T, int RPT>
__device__ void block_cgs_qr(T *P, int m, int l, T *Rout, T *red, T *coef) {
  const int tid = threadIdx.x, nthr = blockDim.x;
  T x[RPT][kCgsCols];
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    const int row = tid + r * nthr;
#pragma unroll
    for (int c = 0; c < kCgsCols; ++c) x[r][c] = (c < l && row < m) ? P[(size_t)c * m + row] : T(0);
  }
  if (Rout)
    for (int e = tid; e < l * l; e += nthr) Rout[e] = T(0);
  __syncthreads();
  cgs_columns<T, RPT, 0>(x, m, l, Rout, red, coef);
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    const int row = tid + r * nthr;
    if (row < m)
#pragma unroll
      for (int c = 0; c < kCgsCols; ++c)
        if (c < l) P[(size_t)c * m + row] = x[r][c];
  }
}

template <typename T, int RPT>
__global__ void __launch_bounds__(256) cgs_qr_kernel(int m, int l, T *__restrict__ P, int64_t sP,
                                                     SliceSel sel) {
  pdl_wait();
  if (sel.count && (int)blockIdx.x >= *sel.count) return;
  __shared__ T red[8 * (kCgsCols + 1)];
  __shared__ T coef[kCgsCols + 1];
  block_cgs_qr<T, RPT>(P + (int64_t)blockIdx.x * sP, m, l, nullptr, red, coef);
  pdl_trigger();
}

// ------------------------------------------- Gram-Schmidt, panel in smem
// Classical Gram-Schmidt with reorthogonalisation for panels the register
// form cannot hold (more than 32 columns or 512 rows; here l <= 64, m <=
// 1024 and the m x l panel in shared memory).  The acceptance and restart
// rules are those of cgs_column: a column is kept after a pass that retains
// more than half of its squared norm (a quarter after the second pass); a
// column still dependent after four passes restarts from a unit vector.
// Per pass the j + 1 inner products of column j (with Q_0 .. Q_{j-1} and
// itself) are taken eight at a time: each warp reduce-scatters eight
// partial sums in nine shuffles, lane 4k ends with value k, and the
// warps' results meet in shared memory.
constexpr int kCgsSmemThreads = 512;

template <typename T>
__global__ void __launch_bounds__(kCgsSmemThreads)
cgs_smem_qr_kernel(int m, int l, T *__restrict__ P, int64_t sP, SliceSel sel) {
  pdl_wait();
  if (sel.count && (int)blockIdx.x >= *sel.count) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *S = reinterpret_cast<T *>(smem_raw);             // m x l, column-major
  T *red = S + (size_t)m * l;                         // 16 warps x 72
  T *coef = red + 16 * 72;                            // 72
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = kCgsSmemThreads / 32;
  constexpr int RPT = 1024 / kCgsSmemThreads;          // rows per thread
  T *Pj = P + (int64_t)blockIdx.x * sP;
  for (int e = tid; e < m * l; e += kCgsSmemThreads) S[e] = Pj[e];
  __syncthreads();
  const T tiny = sizeof(T) == 4 ? T(FLT_MIN) : T(DBL_MIN);
  for (int j = 0; j < l; ++j) {
    T *xj = S + (size_t)j * m;
    int pass = 0, unit = -1, restarts = 0;
    T after = T(0);
    while (true) {
      // inner products with columns 0 .. j (column j: the squared norm)
      for (int c0 = 0; c0 <= j; c0 += 8) {
        T p[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) p[k] = T(0);
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
          const int row = tid + r * kCgsSmemThreads;
          if (row < m) {
            const T xr = xj[row];
#pragma unroll
            for (int k = 0; k < 8; ++k)
              if (c0 + k <= j) p[k] = fma(S[(size_t)(c0 + k) * m + row], xr, p[k]);
          }
        }
        // reduce-scatter: after the levels 16, 8, 4 lane L holds value
        // ((L>>4)&1)*4 + ((L>>3)&1)*2 + ((L>>2)&1) summed over 8 lanes
        int idx = 0;
#pragma unroll
        for (int h = 4, o = 16; h >= 1; h >>= 1, o >>= 1) {
          const bool up = (lane & o) != 0;
#pragma unroll
          for (int k = 0; k < h; ++k) {
            const T give = up ? p[k] : p[k + h];
            const T keep = up ? p[k + h] : p[k];
            p[k] = keep + __shfl_xor_sync(0xffffffffu, give, o);
          }
          idx += up ? h : 0;
        }
        p[0] += __shfl_xor_sync(0xffffffffu, p[0], 2);
        p[0] += __shfl_xor_sync(0xffffffffu, p[0], 1);
        if ((lane & 3) == 0 && c0 + idx <= j) red[warp * 72 + c0 + idx] = p[0];
      }
      __syncthreads();
      for (int i = tid; i <= j; i += kCgsSmemThreads) {
        T t = T(0);
        for (int w = 0; w < NW; ++w) t += red[w * 72 + i];
        coef[i] = t;
      }
      __syncthreads();
      const T sq = coef[j];
      T csq = T(0);
      for (int i = 0; i < j; ++i) csq = fma(coef[i], coef[i], csq);
#pragma unroll
      for (int r = 0; r < RPT; ++r) {
        const int row = tid + r * kCgsSmemThreads;
        if (row < m) {
          T v = xj[row];
          for (int i = 0; i < j; ++i) v = fma(-coef[i], S[(size_t)i * m + row], v);
          xj[row] = v;
        }
      }
      after = sq - csq;
      ++pass;
      __syncthreads();
      if (after > tiny && (after > T(0.5) * sq || (pass >= 2 && after > T(0.25) * sq))) break;
      if (pass >= 4) {   // numerically dependent: continue from a unit vector
        if (++restarts > m) break;
        unit = unit < 0 ? j % m : (unit + 1) % m;
        for (int row = tid; row < m; row += kCgsSmemThreads) xj[row] = row == unit ? T(1) : T(0);
        pass = 0;
        __syncthreads();
      }
    }
    const T nrm = sqrt(after > T(0) ? after : T(0));
    const T inv = nrm > T(0) ? T(1) / nrm : T(0);
    for (int row = tid; row < m; row += kCgsSmemThreads) xj[row] *= inv;
    __syncthreads();
  }
  for (int e = tid; e < m * l; e += kCgsSmemThreads) Pj[e] = S[e];
  pdl_trigger();
}

inline size_t cgs_smem_bytes(size_t esz, int m, int l) {
  return esz * ((size_t)m * l + 16 * 72 + 72);
}

// ------------------------------------------------------ one-sided Jacobi
// Hestenes one-sided Jacobi on the l x l matrix W (column-major): rotate
// column pairs until all are mutually orthogonal, accumulating the
// rotations in J (W_in J = W_out) when J is given.  Pairs follow the round-robin (circle)
// ordering, l/2 disjoint pairs per round; each pair is handled by a group
// of G lanes that split the rows, so its inner products need log2(G)
// shuffle levels.
// A pair is rotated while its cosine |gamma| / sqrt(alpha beta) exceeds tol.
// Cyclic Jacobi converges quadratically (Wilkinson 1962; van Kempen 1966):
// after a sweep whose cosines all stayed below sqrt(tol), the next sweep's
// are of order tol, so the loop stops there instead of running a sweep that
// would only confirm convergence.
// The rotation that zeroes gamma: with d = beta - alpha, t = tan(theta) =
// sign(d) 2 gamma / (|d| + h), h = sqrt(d^2 + 4 gamma^2) (the smaller root of
// t^2 + (d / gamma) t - 1 = 0), and since 1 + t^2 = 2 h / (h + |d|),
//   c = q / sqrt(2 h q),  s = sign(d) 2 gamma / sqrt(2 h q),  q = h + |d|.
// The FP32 form takes its square roots from the special function unit
// (rsqrtf): two in sequence, where the ratio form zeta = d / (2 gamma) needs
// five (rsqrt, reciprocal, rsqrt, reciprocal, rsqrt) on the latency chain of
// every round.  d and 2 gamma are first scaled by an exact power of two that
// brings the larger near 1, so the squares neither overflow nor underflow.
// A rotation only has to be accurate to a few units in the last place (the
// sweeps correct the angle, and c, s come from one r, so c^2 + s^2 = 1 to
// rounding).  The caller forms (c, s) alongside the acceptance test and uses
// them only when a pair is rotated.

template <typename T>
__device__ __forceinline__ bool jacobi_wants(T al, T be, T ga, T tol) {
  if constexpr (sizeof(T) == 4) return ga != T(0) && fabsf(ga) * rsqrtf(al) * rsqrtf(be) > tol;
  else return ga != T(0) && fabs(ga) > tol * sqrt(al * be);
}

template <typename T>
__device__ __forceinline__ void jacobi_rotation(T al, T be, T ga, T &c, T &s) {
  if constexpr (sizeof(T) == 4) {
    const T d = be - al, g2 = T(2) * ga;
    const T m = fmaxf(fabsf(d), fabsf(g2));
    const int e = (__float_as_int(m) >> 23) & 0xff;        // biased exponent of m
    const T sc = __int_as_float((254 - (e < 254 ? e : 253)) << 23);   // 2^(127 - e)
    const T dn = d * sc, gn = g2 * sc;
    const T hh = fmaf(dn, dn, gn * gn);
    const T h = hh * rsqrtf(hh);
    const T q = h + fabsf(dn);
    const T r = rsqrtf(T(2) * h * q);
    c = q * r;
    s = (d >= T(0) ? gn : -gn) * r;
  } else {
    const T zeta = (be - al) / (T(2) * ga);
    const T az = fabs(zeta);
    const T t = T(1) / (az + hypot(T(1), az));
    const T ts = zeta >= T(0) ? t : -t;
    c = T(1) / sqrt(fma(ts, ts, T(1)));
    s = c * ts;
  }
}

// Only the first `nthr` threads (a multiple of 32) take part; they
// synchronise among themselves with named barrier 1, so the other warps of
// the block wait at the caller's next __syncthreads.
__device__ __forceinline__ void named_sync(int nthr) {
  asm volatile("bar.sync 1, %0;" ::"r"(nthr) : "memory");
}

// A lane holds its rows of the pair's two columns of W and J in registers
// between the inner products and the rotation (JR >= ceil(l / G) rows), so
// the J loads overlap the reductions and the update needs no reloads.
template <typename T, int G, int JR>
__device__ void block_jacobi(T *W, T *J, int l, int *flag, T tol, int max_sweeps, int nthr) {
  // J == nullptr: the rotations are not accumulated
  const int lp = l + (l & 1);
  if (lp < 2 || (int)threadIdx.x >= nthr) return;
  const int npairs = lp / 2;
  const int gid = threadIdx.x / G, gl = threadIdx.x % G, ngroups = nthr / G;
  const T stop = sqrt(tol);   // a cosine above this asks for another sweep
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) *flag = 0;
    named_sync(nthr);
    for (int r = 0; r < lp - 1; ++r) {
      for (int base = 0; base < npairs; base += ngroups) {
        const int pi = base + gid;
        int p = 0, q = 0;
        if (pi < npairs) {
          int a, b;
          if (pi == 0) { a = lp - 1; b = r; }
          else {
            a = r + pi; if (a >= lp - 1) a -= lp - 1;
            b = r - pi; if (b < 0) b += lp - 1;
          }
          p = a < b ? a : b;
          q = a < b ? b : a;
        }
        const bool valid = pi < npairs && q < l;
        T *wp = W + (size_t)p * l, *wq = W + (size_t)q * l;
        T *jp = J + (size_t)p * l, *jq = J + (size_t)q * l;
        T x[JR], y[JR], u[JR], v[JR];
        T al = T(0), be = T(0), ga = T(0);
#pragma unroll
        for (int t = 0; t < JR; ++t) {
          const int i = gl + G * t;
          const bool in = valid && i < l;
          x[t] = in ? wp[i] : T(0);
          y[t] = in ? wq[i] : T(0);
          u[t] = in && J ? jp[i] : T(0);
          v[t] = in && J ? jq[i] : T(0);
          al = fma(x[t], x[t], al);
          be = fma(y[t], y[t], be);
          ga = fma(x[t], y[t], ga);
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          ga += __shfl_xor_sync(0xffffffffu, ga, o);
        }
        T c, s;
        jacobi_rotation(al, be, ga, c, s);
        if (valid && jacobi_wants(al, be, ga, tol)) {
#pragma unroll
          for (int t = 0; t < JR; ++t) {
            const int i = gl + G * t;
            if (i < l) {
              wp[i] = c * x[t] - s * y[t];
              wq[i] = s * x[t] + c * y[t];
              if (J) {
                jp[i] = c * u[t] - s * v[t];
                jq[i] = s * u[t] + c * v[t];
              }
            }
          }
          if (gl == 0 && jacobi_wants(al, be, ga, stop)) *flag = 1;
        }
      }
      named_sync(nthr);
    }
    const int any = *flag;
    named_sync(nthr);
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

// The core's shared memory (svd_smem) rounded up to 16 bytes: where the
// fused rebuild keeps Z
template <typename T>
__host__ __device__ size_t svd_base_bytes(int n1, int n2, int l) {
  const int mx = n1 > n2 ? n1 : n2;
  const size_t b = sizeof(T) * ((size_t)mx * l + 3 * (size_t)l * l + 2 * (size_t)l) + 16;
  return (b + 15) & ~(size_t)15;
}

// Per slice: R of B^T = Qb R (P2 holds B^T = Abar^T Q), one-sided Jacobi of
// R^T (R^T J = W with orthogonal columns, J orthogonal: B = R^T Qb^T = W (Qb
// J)^T, so B's left singular vectors are W's normalised columns and sigma
// their norms; J is not needed and not accumulated), the shrink, the core
// C = U diag(shrunk sigma / sigma) U^T, and P1 <- P1 C (= Q C).  Since
// U diag(sigma~) V_B^T = U diag(sigma~/sigma) U^T B, the rebuild is
// Gbar = (Q C) B = P1 P2^T with P2 left as B^T: Qb is never formed.  A
// singular value shrunk to zero drops out (ratio 0).
template <typename T, int CPW, int RPL, int G, int JR, bool REG>
__global__ void svd_core_kernel(int n1, int n2, int l, T *__restrict__ P1, int64_t sP1,
                                T *__restrict__ P2, int64_t sP2, ShrinkScalars sh,
                                T *__restrict__ sig_out, int ldsig,
                                int *__restrict__ rank_out, int *__restrict__ width_out,
                                SliceSel sel, T *__restrict__ Gout) {
  pdl_wait();
  if (sel.count && (int)blockIdx.x >= *sel.count) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int mx = n1 > n2 ? n1 : n2;
  T *panel = reinterpret_cast<T *>(smem_raw);
  T *W = panel + (size_t)mx * l;
  T *J = W + l * l;
  T *C = J + l * l;
  T *tau = C + l * l;
  T *ratio = tau + l;
  int *flag = reinterpret_cast<int *>(ratio + l);
  ShrinkScalars shr = sh;
  if (sh.dmu) shr.tau = 1.0 / *sh.dmu;
  const int bb = blockIdx.x;                       // panel entry
  const int j = sel.ids ? sel.ids[bb] : bb;        // slice id (statistics)
  T *P1j = P1 + (int64_t)bb * sP1;
  T *P2j = P2 + (int64_t)bb * sP2;

  // B^T = Qb R: R lands in W, P2 keeps B^T
  if constexpr (REG) block_reg_qr<T, CPW, RPL, false>(P2j, n2, l, panel, tau, W);
  else block_smem_qr<T, false>(P2j, n2, l, panel, tau, W);
  __syncthreads();
  // R^T into U = J (column c of R^T = row c of R)
  T *U = J;
  const int ldu = l;
  for (int e = threadIdx.x; e < l * l; e += blockDim.x) U[e] = W[(size_t)(e % l) * l + e / l];
  // Rotate only while a pair's cosine exceeds max(l, 8) * eps: below that the
  // computed inner product is rounding noise (an l-term dot product).
  const T eps = sizeof(T) == 4 ? T(FLT_EPSILON) : T(DBL_EPSILON);
  const T tol = T(l > 8 ? l : 8) * eps;
  const int max_sweeps = sizeof(T) == 4 ? 16 : 30;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  {
    const int lp = l + (l & 1);
    int nthr = ((lp / 2) * G + 31) / 32 * 32;
    if (nthr > (int)blockDim.x) nthr = blockDim.x;
    __syncthreads();
    block_jacobi<T, G, JR>(U, nullptr, l, flag, tol, max_sweeps, nthr);
  }
  __syncthreads();

  // sigma_i = ||W_i||; U_i = W_i / sigma_i in place
  for (int i = warp; i < l; i += nw) {
    T ss = T(0);
    for (int r = lane; r < l; r += 32) ss = fma(U[(size_t)i * ldu + r], U[(size_t)i * ldu + r], ss);
    ss = warp_sum(ss);
    const T sg = sqrt(ss);
    const T inv = sg > T(0) ? T(1) / sg : T(0);
    for (int r = lane; r < l; r += 32) U[(size_t)i * ldu + r] *= inv;
    if (lane == 0) {
      const T sp = prox_sv(sg, shr);
      ratio[i] = sg > T(0) ? sp / sg : T(0);
      sig_out[(int64_t)j * ldsig + i] = sg;
      tau[i] = sp;   // reuse tau[] for the shrunk values
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int k = 0;
    for (int i = 0; i < l; ++i) k += tau[i] > T(0);
    rank_out[j] = k;
    if (width_out) width_out[j] = l;
  }
  for (int i = l + threadIdx.x; i < ldsig; i += blockDim.x) sig_out[(int64_t)j * ldsig + i] = T(0);
  // C[a][b] = sum_i U[a][i] ratio_i U[b][i], stored row-major (C[a * l + b])
  for (int e = threadIdx.x; e < l * l; e += blockDim.x) {
    const int a = e % l, b = e / l;
    T acc = T(0);
    for (int i = 0; i < l; ++i)
      acc = fma(U[(size_t)i * ldu + a] * ratio[i], U[(size_t)i * ldu + b], acc);
    C[(size_t)a * l + b] = acc;
  }
  for (int e = threadIdx.x; e < n1 * l; e += blockDim.x) panel[e] = P1j[e];
  __syncthreads();
  // Z = Q C, four output columns per work item: to P1, or (Gout) to shared
  // memory (Zs, column-major n1 x l past the small buffers)
  T *Zs = Gout ? reinterpret_cast<T *>(smem_raw + svd_base_bytes<T>(n1, n2, l)) : nullptr;
  T *Zd = Gout ? Zs : P1j;
  // 4 rows x 4 columns of Z per work item (16-byte shared loads of Q's rows
  // and of C's row a where n1, l are multiples of 4); consecutive threads
  // take consecutive row groups
  const int nr4 = (n1 + 3) / 4, nb4 = (l + 3) / 4;
  const bool vq = n1 % 4 == 0, vc = l % 4 == 0;
  for (int e = threadIdx.x; e < nr4 * nb4; e += blockDim.x) {
    const int r0 = (e % nr4) * 4, b0 = (e / nr4) * 4;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[i][u] = T(0);
    for (int a = 0; a < l; ++a) {
      T x[4], c[4];
      if (vq) {
        ld4s(panel + (size_t)a * n1 + r0, x);
      } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) x[i] = r0 + i < n1 ? panel[(size_t)a * n1 + r0 + i] : T(0);
      }
      if (vc) {
        ld4s(C + (size_t)a * l + b0, c);
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) c[u] = b0 + u < l ? C[(size_t)a * l + b0 + u] : T(0);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[i][u] = fma(x[i], c[u], acc[i][u]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (b0 + u < l && r0 + i < n1) Zd[(size_t)(b0 + u) * n1 + r0 + i] = acc[i][u];
  }
  if (Gout) {
    // the rank-l rebuild of this slice, Gbar = Z B = Z P2^T (row-major n1 x
    // n2; n1, n2 multiples of 4): B^T staged over the panel, 4 x 4 outputs
    // per task, rows written as 16-byte segments
    __syncthreads();
    for (int e = threadIdx.x; e < n2 * l; e += blockDim.x) panel[e] = P2j[e];
    __syncthreads();
    T *Gj = Gout + (int64_t)j * n1 * n2;
    const int RG = n1 / 4, CG = n2 / 4;
    for (int t = threadIdx.x; t < RG * CG; t += blockDim.x) {
      const int rg = t / CG, cg = t % CG;
      T acc[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) acc[i][jj] = T(0);
      for (int k = 0; k < l; ++k) {
        T a[4], q[4];
        ld4s(Zs + (size_t)k * n1 + rg * 4, a);
        ld4s(panel + (size_t)k * n2 + cg * 4, q);
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) acc[i][jj] = fma(a[i], q[jj], acc[i][jj]);
      }
      T *dst = Gj + (int64_t)(rg * 4) * n2 + cg * 4;
#pragma unroll
      for (int i = 0; i < 4; ++i, dst += n2) {
        if constexpr (sizeof(T) == 4) {
          *reinterpret_cast<float4 *>(dst) = make_float4((float)acc[i][0], (float)acc[i][1],
                                                         (float)acc[i][2], (float)acc[i][3]);
        } else {
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) dst[jj] = acc[i][jj];
        }
      }
    }
  }
  pdl_trigger();
}

// Threads for the panel kernels: each warp owns at most CPW columns.
inline int panel_warps(int l, int cpw) {
  int nw = (l + cpw - 1) / cpw;
  if (nw < 1) nw = 1;
  if (nw > 32) nw = 32;
  return nw;
}

inline int pick_cpw(int l) { return l <= 64 ? 2 : 4; }

// rows per lane of the register panel: m <= 32 * RPL
inline int pick_rpl(int m) {
  const int r = (m + 31) / 32;
  return r <= 1 ? 1 : r <= 2 ? 2 : r <= 4 ? 4 : r <= 8 ? 8 : r <= 16 ? 16 : 32;
}

template <typename T>
size_t qr_smem(int m, int l) {
  return sizeof(T) * ((size_t)m * l + ((l + 3) & ~3));
}

template <typename T>
size_t svd_smem(int n1, int n2, int l) {
  const int mx = n1 > n2 ? n1 : n2;
  return sizeof(T) * ((size_t)mx * l + 3 * (size_t)l * l + 2 * (size_t)l) + 16;
}

// Whether svd_core can write Gbar itself (the rank-l rebuild fused): n1, n2
// multiples of 4 (16-byte rows and panel columns), slices of at most 512 x
// 512, and Z (n1 x l) fitting beside the core's buffers.
template <typename T>
bool svd_fused_ok(int n1, int n2, int l, const void *G) {
  return G && (uintptr_t)G % 16 == 0 && n1 % 4 == 0 && n2 % 4 == 0 && n1 <= 512 && n2 <= 512 &&
         svd_base_bytes<T>(n1, n2, l) + sizeof(T) * (size_t)n1 * l <= 100 * 1024;
}

constexpr size_t kSliceSmemMax = 227 * 1024;

// Whether one block of `threads` threads of kernel k fits on an SM (the
// register-resident panels of large slices need more registers than an SM
// has; those take the shared-memory variant).
template <typename K>
cudaError_t fits_one_block(K k, int threads, size_t smem, bool &fits) {
  int nb = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, threads, smem);
  fits = nb >= 1;
  return e;
}

constexpr int kSmemPanelWarps = 16;

template <typename T, int CPW, int RPL>
cudaError_t run_qr_t(int m, int l, T *P, int n, cudaStream_t s, SliceSel sel) {
  const size_t smem = qr_smem<T>(m, l);
  auto k = qr_kernel<T, CPW, RPL>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int threads = 32 * panel_warps(l, CPW);
  bool fits = false;
  if ((e = fits_one_block(k, threads, smem, fits)) != cudaSuccess) return e;
  if (fits) {
    e = launch_pdl(k, dim3(n), dim3(threads), smem, s, m, l, P, (int64_t)m * l, sel);
    if (e != cudaSuccess) return e;
  } else {
    auto k2 = qr_smem_kernel<T>;
    if ((e = cudaFuncSetAttribute(k2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
        cudaSuccess)
      return e;
    e = launch_pdl(k2, dim3(n), dim3(32 * kSmemPanelWarps), smem, s, m, l, P, (int64_t)m * l, sel);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

template <typename T, int CPW, int RPL, int G, int JR>
cudaError_t run_svd_t(int n1, int n2, int l, T *P1, T *P2, int n, const ShrinkScalars &sh, T *sig,
                      int ldsig, int *rank, int *width, cudaStream_t s, SliceSel sel, T *Gout) {
  const size_t smem = Gout ? svd_base_bytes<T>(n1, n2, l) + sizeof(T) * (size_t)n1 * l
                           : svd_smem<T>(n1, n2, l);
  auto k = svd_core_kernel<T, CPW, RPL, G, JR, true>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int lp = l + (l & 1);
  int nw = panel_warps(l, CPW);
  const int jw = (lp / 2 * G + 31) / 32;   // warps giving every Jacobi pair a lane group
  if (jw > nw) nw = jw > 32 ? 32 : jw;
  if (nw < 4) nw = 4;
  bool fits = false;
  if ((e = fits_one_block(k, 32 * nw, smem, fits)) != cudaSuccess) return e;
  if (!fits) {
    auto k2 = svd_core_kernel<T, 4, 1, G, JR, false>;
    if ((e = cudaFuncSetAttribute(k2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
        cudaSuccess)
      return e;
    nw = jw > kSmemPanelWarps ? (jw > 32 ? 32 : jw) : kSmemPanelWarps;
    return launch_pdl(k2, dim3(n), dim3(32 * nw), smem, s, n1, n2, l, P1, (int64_t)n1 * l, P2,
                      (int64_t)n2 * l, sh, sig, ldsig > l ? ldsig : l, rank, width, sel, Gout);
  }
  return launch_pdl(k, dim3(n), dim3(32 * nw), smem, s, n1, n2, l, P1, (int64_t)n1 * l, P2,
                    (int64_t)n2 * l, sh, sig, ldsig > l ? ldsig : l, rank, width, sel, Gout);
}

#define TR_RPL_DISPATCH(RPLV, CALL) \
  switch (RPLV) {                   \
    case 1: { constexpr int RPL = 1; return CALL; } \
    case 2: { constexpr int RPL = 2; return CALL; } \
    case 4: { constexpr int RPL = 4; return CALL; } \
    case 8: { constexpr int RPL = 8; return CALL; } \
    case 16: { constexpr int RPL = 16; return CALL; } \
    default: { constexpr int RPL = 32; return CALL; } \
  }

// Gram-Schmidt QR for panels of at most 32 columns and 512 rows.
inline bool cgs_panel_ok(int m, int l) { return l <= kCgsCols && m <= 512; }

template <typename T>
cudaError_t run_cgs_qr(int m, int l, T *P, int n, cudaStream_t s, SliceSel sel) {
  // two rows per thread: at most 128 registers x 256 threads per block
  const int threads = ((m + 1) / 2 + 31) / 32 * 32;
  return launch_pdl(cgs_qr_kernel<T, 2>, dim3(n), dim3(threads), 0, s, m, l, P, (int64_t)m * l,
                    sel);
}

// The shared-memory Gram-Schmidt form: up to 64 columns and 1024 rows within
// the shared-memory budget.
inline bool cgs_smem_ok(size_t esz, int m, int l) {
  return l <= 64 && m <= 1024 && cgs_smem_bytes(esz, m, l) <= kSliceSmemMax;
}

template <typename T>
cudaError_t run_qr(int m, int l, T *P, int n, cudaStream_t s, SliceSel sel = SliceSel{}) {
  if (cgs_panel_ok(m, l)) return run_cgs_qr<T>(m, l, P, n, s, sel);
  if (cgs_smem_ok(sizeof(T), m, l)) {
    const size_t smem = cgs_smem_bytes(sizeof(T), m, l);
    cudaError_t e = cudaFuncSetAttribute(cgs_smem_qr_kernel<T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return launch_pdl(cgs_smem_qr_kernel<T>, dim3(n), dim3(kCgsSmemThreads), smem, s, m, l, P,
                      (int64_t)m * l, sel);
  }
  if (pick_cpw(l) == 2) { TR_RPL_DISPATCH(pick_rpl(m), (run_qr_t<T, 2, RPL>(m, l, P, n, s, sel))) }
  TR_RPL_DISPATCH(pick_rpl(m), (run_qr_t<T, 4, RPL>(m, l, P, n, s, sel)))
}

template <typename T>
cudaError_t run_svd_core(int n1, int n2, int l, T *P1, T *P2, int n, const ShrinkScalars &sh,
                         T *sig, int *rank, cudaStream_t s, SliceSel sel = SliceSel{},
                         int ldsig = 0, int *width = nullptr, T *Gout = nullptr) {
#define TR_SVD_ARGS n1, n2, l, P1, P2, n, sh, sig, ldsig, rank, width, s, sel, Gout
  // eight lanes per Jacobi pair; JR = rows of a pair's columns per lane
  if (pick_cpw(l) == 2) {
    if (l <= 32) { TR_RPL_DISPATCH(pick_rpl(n2), (run_svd_t<T, 2, RPL, 8, 4>(TR_SVD_ARGS))) }
    TR_RPL_DISPATCH(pick_rpl(n2), (run_svd_t<T, 2, RPL, 8, 8>(TR_SVD_ARGS)))
  }
  TR_RPL_DISPATCH(pick_rpl(n2), (run_svd_t<T, 4, RPL, 8, 16>(TR_SVD_ARGS)))
#undef TR_SVD_ARGS
}

// ------------------------------- shared Tucker factors (Alg. 1 + Alg. 4)
// The paper's own randomized GNHTSVT on the transformed stack: factors F1
// (n1 x r1) and F2 (n2 x r2) shared by all slices from the block Krylov
// spaces of the mode-1 and mode-2 unfoldings (R-STHOSVD-BKI, processing
// order (1, 2)), then the prox of every slice restricted to them.  The
// unfolding products are batched per-slice products with a shared operand
// followed by a sum over the slices.

// out[i] = sum_j in[j * count + i]
template <typename T>
__global__ void reduce_slices_kernel(T *__restrict__ out, const T *__restrict__ in, int64_t count,
                                     int n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    T acc = T(0);
    for (int j = 0; j < n; ++j) acc += in[(int64_t)j * count + i];
    out[i] = acc;
  }
}

// dst[j * count + i] = src[i]
template <typename T>
__global__ void bcast_slices_kernel(T *__restrict__ dst, const T *__restrict__ src, int64_t count,
                                    int n) {
  const int64_t total = count * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = src[e % count];
}

// The r top singular vectors of the symmetric positive semi-definite L x L
// matrix M (column-major), L <= 32, as the columns of Ur (L x r): one-sided
// Jacobi M J = W (block_jacobi), sigma_i = ||W_i||, the columns of J sorted
// by sigma.  One block of 128 threads.
template <typename T>
__global__ void __launch_bounds__(128) eig_top_kernel(int L, const T *__restrict__ M, int r,
                                                     T *__restrict__ Ur) {
  __shared__ T W[32 * 32], J[32 * 32], sg[32];
  __shared__ int order[32];
  __shared__ int flag;
  for (int e = threadIdx.x; e < L * L; e += blockDim.x) {
    W[e] = M[e];
    J[e] = (e % L == e / L) ? T(1) : T(0);
  }
  __syncthreads();
  const T eps = sizeof(T) == 4 ? T(FLT_EPSILON) : T(DBL_EPSILON);
  const int lp = L + (L & 1);
  int nthr = ((lp / 2) * 8 + 31) / 32 * 32;
  if (nthr > (int)blockDim.x) nthr = blockDim.x;
  block_jacobi<T, 8, 4>(W, J, L, &flag, T(L > 8 ? L : 8) * eps, sizeof(T) == 4 ? 16 : 30, nthr);
  __syncthreads();
  if (threadIdx.x < L) {
    T ss = T(0);
    for (int i = 0; i < L; ++i) ss = fma(W[threadIdx.x * L + i], W[threadIdx.x * L + i], ss);
    sg[threadIdx.x] = ss;
  }
  __syncthreads();
  if (threadIdx.x == 0) {   // selection by decreasing sigma (stable for ties)
    bool used[32] = {};
    for (int c = 0; c < L; ++c) {
      int best = -1;
      for (int i = 0; i < L; ++i)
        if (!used[i] && (best < 0 || sg[i] > sg[best])) best = i;
      used[best] = true;
      order[c] = best;
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < L * r; e += blockDim.x) {
    const int i = e % L, c = e / L;
    Ur[e] = J[order[c] * L + i];
  }
}

// Columns of F (m x r, column-major) scaled by +-1 so that each column's
// entry of largest magnitude (the first one on ties) is positive: the sign
// convention of the factors (the mode-2 sketch depends on F1's signs).  One
// warp per column; the signed winner travels with the reduction.
template <typename T>
__global__ void canon_sign_kernel(T *__restrict__ F, int m, int r) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int c = warp; c < r; c += nw) {
    T *col = F + (size_t)c * m;
    T best = T(-1), val = T(0);
    int bi = m;
    for (int i = lane; i < m; i += 32) {
      const T a = fabs(col[i]);
      if (a > best) {   // i increases within a lane: first index on ties
        best = a;
        val = col[i];
        bi = i;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const T ob = __shfl_xor_sync(0xffffffffu, best, o);
      const T ov = __shfl_xor_sync(0xffffffffu, val, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) {
        best = ob;
        val = ov;
        bi = oi;
      }
    }
    const T sgn = val < T(0) ? T(-1) : T(1);
    for (int i = lane; i < m; i += 32) col[i] *= sgn;
  }
}

struct TuckerDims {
  int n, n1, n2, r1, r2, b1, b2, q1, q2;
  int L1() const { return (q1 + 1) * b1; }
  int L2() const { return (q2 + 1) * b2; }
};

template <typename T>
size_t tucker_ws_elems(const TuckerDims &d) {
  const size_t L1 = d.L1(), L2 = d.L2();
  size_t pm = (size_t)d.n1 * L1;
  pm = pm > (size_t)d.n2 * L2 ? pm : (size_t)d.n2 * L2;
  pm = pm > L1 * L1 ? pm : L1 * L1;
  pm = pm > L2 * L2 ? pm : L2 * L2;
  size_t wm = (size_t)d.n2 * L1;
  wm = wm > (size_t)d.r1 * L2 ? wm : (size_t)d.r1 * L2;
  return (size_t)d.n * (pm + wm) + (size_t)d.n1 * L1 + (size_t)d.n2 * L2 + 2 * 32 * 32 +
         (size_t)d.n1 * d.r1 + (size_t)d.n2 * d.r2 +
         (size_t)d.n * ((size_t)d.n2 * d.r1 + (size_t)d.r2 * d.r1 + (size_t)d.n1 * d.r1 +
                        (size_t)d.n2 * d.r1 + d.r1) +
         (size_t)d.n + 64;   // the ranks (n ints) after the singular values
}

template <typename T>
cudaError_t reduce_slices(T *out, const T *in, int64_t count, int n, cudaStream_t s) {
  const int threads = 256;
  const int blocks = (int)((count + threads - 1) / threads);
  reduce_slices_kernel<T><<<blocks < 1 ? 1 : blocks, threads, 0, s>>>(out, in, count, n);
  return cudaGetLastError();
}

// Block Krylov factor of one unfolding A = [A_0 ... A_{n-1}] (A_j: m x k,
// the slice blocks of the unfolding, given by their element strides sAi,
// sAk and slice stride sAb): K = [A G, (A A^T) A G, ..., (A A^T)^q A G],
// Z = qr(K), M = Z^T A A^T Z, F = Z U_r (Alg. 1 loop body).  The block of G
// that multiplies A_j starts at j * sGb, columns sGn apart.
template <typename T>
cudaError_t tucker_factor(int n, int m, int k, const T *A, int64_t sAb, int64_t sAi, int64_t sAk,
                          const T *G, int64_t sGb, int64_t sGn, int b, int q, int r, T *K, T *part,
                          T *W, T *Mm, T *Ur, T *F, cudaStream_t s) {
  const int L = (q + 1) * b;
  cudaError_t e;
  // K block 0 = sum_j A_j G_j (G_j: k x b, slice stride sGb, column stride sGn)
  GemmArgs g0{m, b, k, A, sAb, sAi, sAk, G, sGb, 1, sGn, part, (int64_t)m * b, 1, m};
  if ((e = bgemm<T>(g0, n, s)) != cudaSuccess) return e;
  if ((e = reduce_slices<T>(K, part, (int64_t)m * b, n, s)) != cudaSuccess) return e;
  for (int i = 1; i <= q; ++i) {
    const T *X = K + (size_t)(i - 1) * b * m;
    GemmArgs gw{k, b, m, A, sAb, sAk, sAi, X, 0, 1, m, W, (int64_t)k * b, 1, k};   // W_j = A_j^T X
    if ((e = bgemm<T>(gw, n, s)) != cudaSuccess) return e;
    GemmArgs gp{m, b, k, A, sAb, sAi, sAk, W, (int64_t)k * b, 1, k, part, (int64_t)m * b, 1, m};
    if ((e = bgemm<T>(gp, n, s)) != cudaSuccess) return e;
    if ((e = reduce_slices<T>(K + (size_t)i * b * m, part, (int64_t)m * b, n, s)) != cudaSuccess)
      return e;
  }
  if ((e = run_qr<T>(m, L, K, 1, s)) != cudaSuccess) return e;                   // Z
  GemmArgs gz{k, L, m, A, sAb, sAk, sAi, K, 0, 1, m, W, (int64_t)k * L, 1, k};      // W_j = A_j^T Z
  if ((e = bgemm<T>(gz, n, s)) != cudaSuccess) return e;
  GemmArgs gm{L, L, k, W, (int64_t)k * L, k, 1, W, (int64_t)k * L, 1, k, part, (int64_t)L * L, 1, L};
  if ((e = bgemm<T>(gm, n, s)) != cudaSuccess) return e;                         // W_j^T W_j
  if ((e = reduce_slices<T>(Mm, part, (int64_t)L * L, n, s)) != cudaSuccess) return e;
  eig_top_kernel<T><<<1, 128, 0, s>>>(L, Mm, r, Ur);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  GemmArgs gf{m, r, L, K, 0, 1, m, Ur, 0, 1, L, F, 0, 1, m};                        // F = Z U_r
  if ((e = bgemm<T>(gf, 1, s)) != cudaSuccess) return e;
  canon_sign_kernel<T><<<1, 256, 0, s>>>(F, m, r);
  return cudaGetLastError();
}

// G1, G2: one column-major matrix each (rows j k + i for slice j), or, with
// g_blocks, one column-major k x b block per slice (the sketch layout).
// sig_out/rank_out (optional): per-slice singular values (row stride r1)
// and kept ranks.
template <typename T>
cudaError_t run_tucker(const TuckerDims &d, const T *Abar, T *Gbar, const T *G1, const T *G2,
                       T *ws, const ShrinkScalars &sh, T *F1_out, T *F2_out, cudaStream_t s,
                       bool g_blocks = false, T *sig_out = nullptr, int *rank_out = nullptr) {
  const int n = d.n, n1 = d.n1, n2 = d.n2, r1 = d.r1, r2 = d.r2;
  const int L1 = d.L1(), L2 = d.L2();
  size_t pm = (size_t)n1 * L1;
  pm = pm > (size_t)n2 * L2 ? pm : (size_t)n2 * L2;
  pm = pm > (size_t)L1 * L1 ? pm : (size_t)L1 * L1;
  pm = pm > (size_t)L2 * L2 ? pm : (size_t)L2 * L2;
  size_t wm = (size_t)n2 * L1;
  wm = wm > (size_t)r1 * L2 ? wm : (size_t)r1 * L2;
  T *part = ws;
  T *W = part + (size_t)n * pm;
  T *K1 = W + (size_t)n * wm;
  T *K2 = K1 + (size_t)n1 * L1;
  T *Mm = K2 + (size_t)n2 * L2;
  T *Ur = Mm + 32 * 32;
  T *F1 = Ur + 32 * 32;
  T *F2 = F1 + (size_t)n1 * r1;
  T *Tt = F2 + (size_t)n2 * r2;       // T_j = Abar_j^T F1       (n2 x r1)
  T *U = Tt + (size_t)n * n2 * r1;    // U_j = F2^T T_j          (r2 x r1)
  T *P1 = U + (size_t)n * r2 * r1;    // copies of F1            (n1 x r1)
  T *P2 = P1 + (size_t)n * n1 * r1;   // F2 F2^T Abar_j^T F1     (n2 x r1)
  T *sig = sig_out ? sig_out : P2 + (size_t)n * n2 * r1;
  int *rank = rank_out ? rank_out
                       : reinterpret_cast<int *>(P2 + (size_t)n * n2 * r1 + (size_t)n * r1 + 1);
  const int64_t sA = (int64_t)n1 * n2;
  cudaError_t e;
  // mode 1: the slice blocks of the unfolding are Abar_j (n1 x n2)
  const int64_t g1b = g_blocks ? (int64_t)n2 * d.b1 : n2, g1n = g_blocks ? n2 : (int64_t)n * n2;
  const int64_t g2b = g_blocks ? (int64_t)r1 * d.b2 : r1, g2n = g_blocks ? r1 : (int64_t)n * r1;
  if ((e = tucker_factor<T>(n, n1, n2, Abar, sA, n2, 1, G1, g1b, g1n, d.b1, d.q1, r1, K1, part, W,
                            Mm, Ur, F1, s)) != cudaSuccess)
    return e;
  // mode 2 of C = Abar x_1 F1^T: its slice blocks are T_j = Abar_j^T F1 (n2 x r1)
  GemmArgs gt{n2, r1, n1, Abar, sA, 1, n2, F1, 0, 1, n1, Tt, (int64_t)n2 * r1, 1, n2};
  if ((e = bgemm<T>(gt, n, s)) != cudaSuccess) return e;
  if ((e = tucker_factor<T>(n, n2, r1, Tt, (int64_t)n2 * r1, 1, n2, G2, g2b, g2n, d.b2, d.q2, r2, K2,
                            part, W, Mm, Ur, F2, s)) != cudaSuccess)
    return e;
  // per slice: B_j^T = F2 F2^T T_j, basis F1; the slice prox of Abar_j
  // restricted to the factors is F1 SVT(F1^T Abar_j F2) F2^T
  GemmArgs gu{r2, r1, n2, F2, 0, n2, 1, Tt, (int64_t)n2 * r1, 1, n2, U, (int64_t)r2 * r1, 1, r2};
  if ((e = bgemm<T>(gu, n, s)) != cudaSuccess) return e;
  GemmArgs gp{n2, r1, r2, F2, 0, 1, n2, U, (int64_t)r2 * r1, 1, r2, P2, (int64_t)n2 * r1, 1, n2};
  if ((e = bgemm<T>(gp, n, s)) != cudaSuccess) return e;
  {
    const int64_t cnt = (int64_t)n1 * r1;
    const int64_t tot = cnt * n;
    const int blocks = (int)((tot + 255) / 256);
    bcast_slices_kernel<T><<<blocks < 1 ? 1 : blocks, 256, 0, s>>>(P1, F1, cnt, n);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if ((e = run_svd_core<T>(n1, n2, r1, P1, P2, n, sh, sig, rank, s)) != cudaSuccess) return e;
  if ((e = rank_update<T>(n, n1, n2, r1, P1, P2, Gbar, s)) != cudaSuccess) return e;
  if (F1_out && (e = cudaMemcpyAsync(F1_out, F1, sizeof(T) * n1 * r1, cudaMemcpyDeviceToDevice,
                                     s)) != cudaSuccess)
    return e;
  if (F2_out && (e = cudaMemcpyAsync(F2_out, F2, sizeof(T) * n2 * r2, cudaMemcpyDeviceToDevice,
                                     s)) != cudaSuccess)
    return e;
  return cudaSuccess;
}

#include "adapt_kernels.cuh"

template <typename T>
cudaError_t run_rsvd(const SliceWork &w, const T *Abar, T *Gbar, const ShrinkScalars &sh, int t,
                     cudaStream_t s) {
  const int n = w.n, n1 = w.n1, n2 = w.n2, l = w.l;
  const int64_t sA = (int64_t)n1 * n2;
  T *Om = (T *)w.Om, *P1 = (T *)w.P1, *P2 = (T *)w.P2;
  cudaError_t e;
  auto mark = [&](const char *nm) {
    if (w.prof) w.prof->mark(s, nm);
  };
  // Omega for every slice
  {
    const int64_t per = (int64_t)n2 * l;
    const int64_t groups = (per + 3) / 4;
    dim3 grid((unsigned)((groups + 255) / 256), n);
    e = launch_pdl(sketch_kernel<T>, grid, dim3(256), 0, s, per, Om,
                   (uint32_t)(w.seed & 0xffffffffu), (uint32_t)(w.seed >> 32), (uint32_t)t, w.dt,
                   0u, w.sel);
    if (e != cudaSuccess) return e;
    mark("sketch");
  }
  // Precision of each skinny product: 0 = SIMT FP32, 1 = BF16, 3 = split
  // BF16.  The BF16 form keeps the sketch and the early power products in
  // BF16 and computes the last power product and B^T = Abar^T Q in split
  // BF16, so the final basis and B are refined at FP32-level accuracy.
  const bool tc = sizeof(T) == 4 && w.l <= 128 &&
                  (w.prec == TR_PREC_BF16 || w.prec == TR_PREC_BF16X3);
  const int early = !tc ? 0 : (w.prec == TR_PREC_BF16 ? 1 : 3);
  const int late = !tc ? 0 : 3;
  // Abar as BF16 planes (hi: the first nA n1 n2 BF16, lo: the next) when
  // the pass is given them: the products of Abar read the planes
  const int nA = w.nA > 0 ? w.nA : n;
  const bool planes = w.asplit && tc;
  if (w.asplit && !planes) return cudaErrorNotSupported;
  const void *a_hi = Abar;
  const void *a_lo = reinterpret_cast<const uint16_t *>(Abar) + (int64_t)nA * sA;
  auto run_gemm = [&](const GemmArgs &g, int mode) {
    if (mode == 0) return bgemm<T>(g, n, s);
    if (planes && g.A == Abar) return tma_gemm_planes(g, n, nA, mode, a_hi, a_lo, w.err, s);
    bool used = false;
    cudaError_t e2 = tma_gemm(g, n, w.nA > 0 ? w.nA : n, mode, w.err, s, &used);
    if (e2 != cudaSuccess || used) return e2;
    return umma_gemm(g, n, mode, w.err, s);
  };
  // Abar is indexed by slice id, the panels by batch entry
  auto AX = [&](const T *X, T *Y, int mode) {
    GemmArgs g{n1, l, n2, Abar, sA, n2, 1, X, (int64_t)n2 * l, 1, n2, Y, (int64_t)n1 * l, 1, n1,
               w.sel, 1, 0};
    return run_gemm(g, mode);
  };
  auto AtX = [&](const T *X, T *Wt, int mode) {
    GemmArgs g{n2, l, n1, Abar, sA, 1, n2, X, (int64_t)n1 * l, 1, n1, Wt, (int64_t)n2 * l, 1, n2,
               w.sel, 1, 0};
    return run_gemm(g, mode);
  };
  static const char *kAX0[4] = {"product A*X fp32 simt", "product A*X bf16 tcgen05", "",
                                "product A*X split-bf16 tcgen05"};
  static const char *kAtX0[4] = {"product A^T*Q fp32 simt", "product A^T*Q bf16 tcgen05", "",
                                 "product A^T*Q split-bf16 tcgen05"};
  static const char *kAXp[4] = {"", "product A*X bf16 planes tcgen05", "",
                                "product A*X split-bf16 planes tcgen05"};
  static const char *kAtXp[4] = {"", "product A^T*Q bf16 planes tcgen05", "",
                                 "product A^T*Q split-bf16 planes tcgen05"};
  const char *const *kAX = planes ? kAXp : kAX0;
  const char *const *kAtX = planes ? kAtXp : kAtX0;
  const int m0 = w.q > 0 ? early : late;
  if ((e = AX(Om, P1, m0)) != cudaSuccess) return e;
  mark(kAX[m0]);
  for (int it = 0; it < w.q; ++it) {
    const bool last = it == w.q - 1;
    if ((e = run_qr<T>(n1, l, P1, n, s, w.sel)) != cudaSuccess) return e;
    mark("qr");
    if ((e = AtX(P1, P2, early)) != cudaSuccess) return e;
    mark(kAtX[early]);
    if ((e = run_qr<T>(n2, l, P2, n, s, w.sel)) != cudaSuccess) return e;
    mark("qr");
    if ((e = AX(P2, P1, last ? late : early)) != cudaSuccess) return e;
    mark(kAX[last ? late : early]);
  }
  if ((e = run_qr<T>(n1, l, P1, n, s, w.sel)) != cudaSuccess) return e;
  mark("qr");
  if ((e = AtX(P1, P2, late)) != cudaSuccess) return e;
  mark(kAtX[late]);
  // small slices: the core writes Gbar itself (the rank-l rebuild fused)
  const bool fused = svd_fused_ok<T>(n1, n2, l, Gbar);
  if ((e = run_svd_core<T>(n1, n2, l, P1, P2, n, sh, (T *)w.sig, w.rank, s, w.sel, w.ldsig,
                           w.width, fused ? Gbar : nullptr)) != cudaSuccess)
    return e;
  mark(fused ? "svd_core + rank_update" : "svd_core");
  if (fused) return cudaSuccess;
  // Gbar = Z Qb^T : (n1 x l) (l x n2), row-major output.  It stays on FP32
  // FMA in every form: with K = l the product is short, both operands are
  // k-strided panels and the output is row-major, and the tcgen05 kernel
  // measured 109 us against 38 us here on 400 slices of 200 x 200, l = 20.
  if ((e = rank_update<T>(n, n1, n2, l, P1, P2, Gbar, s, w.sel)) != cudaSuccess) return e;
  mark("rank_update");
  return cudaSuccess;
}

template <typename T>
cudaError_t run_adaptive(const SliceWork &sw, const AdaptWork &aw, const T *Abar, T *Gbar,
                         const ShrinkScalars &sh, int t, cudaStream_t s) {
  const int n = sw.n, n1 = sw.n1, n2 = sw.n2, b = aw.b, kcap = aw.kcap;
  const int64_t sA = (int64_t)n1 * n2;
  const int64_t xs = (int64_t)(n1 > n2 ? n1 : n2) * b;
  AdaptPtrs<T> w{(T *)aw.Ucat, (T *)aw.Vcat, (T *)aw.X, (T *)aw.Lm, (T *)aw.Rm,
                 aw.E, aw.nrm2, aw.active, aw.kept, aw.draws};
  const uint32_t k0 = (uint32_t)(sw.seed & 0xffffffffu), k1 = (uint32_t)(sw.seed >> 32);
  cudaError_t e;
  if ((e = cudaMemsetAsync(aw.Ucat, 0, (size_t)n * n1 * kcap * sizeof(T), s)) != cudaSuccess) return e;
  const size_t sm1 = adapt_smem<T>(n1, b, kcap), sm2 = adapt_smem<T>(n2, b, kcap);
  const size_t smx = sm1 > sm2 ? sm1 : sm2;
  if ((e = cudaFuncSetAttribute(adapt_init_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smx)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(adapt_u_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smx)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(adapt_v_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smx)) != cudaSuccess) return e;
  const SliceSel sel = sw.sel;
  adapt_init_kernel<T><<<n, 256, sm2, s>>>(n1, n2, b, kcap, Abar, w, k0, k1, (uint32_t)t, sw.dt,
                                          sel);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int nblk = kcap / b;
  for (int i = 0; i < nblk; ++i) {
    // X = Abar V_i
    GemmArgs g1{n1, b, n2, Abar, sA, n2, 1, w.Vcat + (int64_t)i * b * n2,
                (int64_t)n2 * (kcap + b), 1, n2, w.X, xs, 1, n1, sel, 1, 0};
    if ((e = bgemm<T>(g1, n, s)) != cudaSuccess) return e;
    adapt_u_kernel<T><<<n, 256, sm1, s>>>(i, n1, b, kcap, xs, w, aw.delta_rel, sel);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (i + 1 == nblk) break;
    // X = Abar^T U_i
    GemmArgs g2{n2, b, n1, Abar, sA, 1, n2, w.Ucat + (int64_t)i * b * n1, (int64_t)n1 * kcap, 1,
                n1, w.X, xs, 1, n2, sel, 1, 0};
    if ((e = bgemm<T>(g2, n, s)) != cudaSuccess) return e;
    adapt_v_kernel<T><<<n, 256, sm2, s>>>(i, n2, b, kcap, xs, w, aw.delta_rel, aw.eps, k0, k1,
                                         (uint32_t)t, sw.dt, sel);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  // B^T = Abar^T U (U zero-padded to kcap columns), SVD core, rebuild
  T *P2 = (T *)sw.P2;
  GemmArgs g3{n2, kcap, n1, Abar, sA, 1, n2, w.Ucat, (int64_t)n1 * kcap, 1, n1, P2,
              (int64_t)n2 * kcap, 1, n2, sel, 1, 0};
  if ((e = bgemm<T>(g3, n, s)) != cudaSuccess) return e;
  if ((e = run_svd_core<T>(n1, n2, kcap, w.Ucat, P2, n, sh, (T *)sw.sig, sw.rank, s, sel,
                           sw.ldsig)) != cudaSuccess)
    return e;
  if ((e = rank_update<T>(n, n1, n2, kcap, w.Ucat, P2, Gbar, s, sel)) != cudaSuccess) return e;
  if (sel.ids && sw.width) {
    adapt_width_kernel<<<(n + 255) / 256, 256, 0, s>>>(sel.ids, sel.count, aw.kept, sw.width, n);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace

bool planes_ok(int64_t n, int n1, int n2, int l) { return planes_view_ok(n, n1, n2, l); }

cudaError_t launch_split_planes(const float *x, void *dst, int64_t count, cudaStream_t s) {
  return split_planes(x, dst, count, s);
}

cudaError_t launch_slice_adaptive(tr_dtype dt, const SliceWork &w, const AdaptWork &aw,
                                  const void *Abar, void *Gbar, const ShrinkScalars &sh, int t,
                                  cudaStream_t s) {
  if (dt == TR_F64)
    return run_adaptive<double>(w, aw, (const double *)Abar, (double *)Gbar, sh, t, s);
  return run_adaptive<float>(w, aw, (const float *)Abar, (float *)Gbar, sh, t, s);
}

size_t adapt_smem_bytes(tr_dtype dt, int n1, int n2, int b, int kcap) {
  const int mx = n1 > n2 ? n1 : n2;
  return dt == TR_F64 ? adapt_smem<double>(mx, b, kcap) : adapt_smem<float>(mx, b, kcap);
}

cudaError_t launch_slice_rsvd(tr_dtype dt, const SliceWork &w, const void *Abar, void *Gbar,
                              const ShrinkScalars &sh, int t, cudaStream_t s) {
  if (dt == TR_F64) return run_rsvd<double>(w, (const double *)Abar, (double *)Gbar, sh, t, s);
  return run_rsvd<float>(w, (const float *)Abar, (float *)Gbar, sh, t, s);
}

size_t slice_smem_limit_ok(tr_dtype dt, int n1, int n2, int l) {
  const int mx = n1 > n2 ? n1 : n2;
  const size_t a = dt == TR_F64 ? svd_smem<double>(n1, n2, l) : svd_smem<float>(n1, n2, l);
  const size_t b = dt == TR_F64 ? qr_smem<double>(mx, l) : qr_smem<float>(mx, l);
  return (a <= kSliceSmemMax && b <= kSliceSmemMax && mx <= 1024 && l <= 128) ? 1 : 0;
}

size_t tucker_ws_bytes(tr_dtype dt, int n, int n1, int n2, int r1, int r2, int b1, int b2, int q1,
                       int q2) {
  const TuckerDims d{n, n1, n2, r1, r2, b1, b2, q1, q2};
  return dt == TR_F64 ? sizeof(double) * tucker_ws_elems<double>(d)
                      : sizeof(float) * tucker_ws_elems<float>(d);
}

cudaError_t launch_slice_tucker(tr_dtype dt, int n, int n1, int n2, int r1, int r2, int b1, int b2,
                                int q1, int q2, const void *Abar, void *Gbar, const void *G1,
                                const void *G2, void *ws, const ShrinkScalars &sh, void *F1_out,
                                void *F2_out, cudaStream_t s, bool g_blocks, void *sig,
                                int *rank) {
  const TuckerDims d{n, n1, n2, r1, r2, b1, b2, q1, q2};
  if (dt == TR_F64)
    return run_tucker<double>(d, (const double *)Abar, (double *)Gbar, (const double *)G1,
                              (const double *)G2, (double *)ws, sh, (double *)F1_out,
                              (double *)F2_out, s, g_blocks, (double *)sig, rank);
  return run_tucker<float>(d, (const float *)Abar, (float *)Gbar, (const float *)G1,
                           (const float *)G2, (float *)ws, sh, (float *)F1_out, (float *)F2_out, s,
                           g_blocks, (float *)sig, rank);
}

cudaError_t launch_canon_signs(tr_dtype dt, void *F, int m, int r, cudaStream_t s) {
  if (m < 1 || r < 1) return cudaSuccess;
  if (dt == TR_F64)
    canon_sign_kernel<double><<<1, 256, 0, s>>>((double *)F, m, r);
  else
    canon_sign_kernel<float><<<1, 256, 0, s>>>((float *)F, m, r);
  return cudaGetLastError();
}

cudaError_t launch_gaussian_blocks(tr_dtype dt, int n, int64_t per_slice, void *out, uint64_t seed,
                                   int t, const int *dt_dev, uint32_t stream, cudaStream_t s) {
  const int64_t groups = (per_slice + 3) / 4;
  const dim3 grid((unsigned)((groups + 255) / 256), n);
  if (dt == TR_F64)
    return launch_pdl(sketch_kernel<double>, grid, dim3(256), 0, s, per_slice, (double *)out,
                      (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32), (uint32_t)t, dt_dev,
                      stream, SliceSel{});
  return launch_pdl(sketch_kernel<float>, grid, dim3(256), 0, s, per_slice, (float *)out,
                    (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32), (uint32_t)t, dt_dev,
                    stream, SliceSel{});
}
