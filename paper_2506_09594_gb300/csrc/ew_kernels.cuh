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
