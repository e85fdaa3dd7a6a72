// Small elementwise kernels shared by the model steps built from the public
// building blocks (one-bit completion, gradient-domain prior).
#pragma once

#include <stdint.h>

namespace ew {

inline int grid(int64_t N) {
  const int64_t blocks = (N + 255) / 256;
  return (int)(blocks < 152 * 32 ? (blocks < 1 ? 1 : blocks) : 152 * 32);
}

// out = a X + b Y (out may be X or Y).
template <typename T>
__global__ void axpby_kernel(T *out, T a, const T *X, T b, const T *Y, int64_t N) {
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < N; f += step)
    out[f] = a * X[f] + b * Y[f];
}

// Lam += mu (A - B).
template <typename T>
__global__ void multiplier_kernel(T *Lam, T mu, const T *__restrict__ A, const T *__restrict__ B,
                                  int64_t N) {
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < N; f += step)
    Lam[f] += mu * (A[f] - B[f]);
}

// Block maximum of a non-negative value, folded into *slot (the bits of a
// non-negative double order like the value).
__device__ inline void block_max_to(double v, unsigned long long *slot) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __shared__ double s[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) s[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, s[w]);
    atomicMax(slot, (unsigned long long)__double_as_longlong(m));
  }
}

}  // namespace ew

namespace ew {

// Periodic neighbours along a mode of flat stride S and size nk (the
// face-slice layout of the gradient operators): forward i_k + 1, backward
// i_k - 1, both mod nk.
__device__ inline int64_t fwd_neighbour(int64_t f, int64_t S, int64_t nk) {
  return ((f / S) % nk == nk - 1) ? f - (nk - 1) * S : f + S;
}
__device__ inline int64_t bwd_neighbour(int64_t f, int64_t S, int64_t nk) {
  return ((f / S) % nk == 0) ? f + (nk - 1) * S : f - S;
}

// R += nabla^T (G - Lam/mu) along the mode: with W = G - inv_mu Lam,
// (nabla^T W)[f] = W[f - e_k] - W[f].
template <typename T>
__global__ void adj_grad_accum_kernel(T *R, const T *__restrict__ G, const T *__restrict__ Lam,
                                      T inv_mu, int64_t N, int64_t S, int64_t nk) {
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < N; f += step) {
    const int64_t g = bwd_neighbour(f, S, nk);
    R[f] += (G[g] - inv_mu * Lam[g]) - (G[f] - inv_mu * Lam[f]);
  }
}

// R = nabla X + Lam/mu along the mode: (X[f + e_k] - X[f]) + inv_mu Lam[f].
template <typename T>
__global__ void grad_plus_kernel(T *R, const T *__restrict__ X, const T *__restrict__ Lam, T inv_mu,
                                 int64_t N, int64_t S, int64_t nk) {
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < N; f += step)
    R[f] = (X[fwd_neighbour(f, S, nk)] - X[f]) + inv_mu * Lam[f];
}

}  // namespace ew

namespace ew {

// Lam += mu (nabla X - G) along the mode, nabla X computed on the fly.
template <typename T>
__global__ void grad_multiplier_kernel(T *Lam, T mu, const T *__restrict__ X, const T *__restrict__ G,
                                       int64_t N, int64_t S, int64_t nk) {
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < N; f += step)
    Lam[f] += mu * ((X[fwd_neighbour(f, S, nk)] - X[f]) - G[f]);
}

// Flat stride of mode k (1-based) in the face-slice layout: n2 for mode 1,
// 1 for mode 2, n1 n2 n3 ... n_{k-1} for k >= 3.
inline int64_t mode_stride(const int64_t *dims, int k) {
  if (k == 1) return dims[1];
  if (k == 2) return 1;
  int64_t s = dims[0] * dims[1];
  for (int m = 3; m < k; ++m) s *= dims[m - 1];
  return s;
}

}  // namespace ew
