// Strided batched SIMT GEMM shared by the gradient-domain solve and the
// fixed-accuracy Tucker loop: C[o][x][y] = sum_b A[o][x][b] B[o][b][y] for
// o < batch, with every operand addressed by element strides, so row- and
// column-major operands, transposes and per-slice blocks are all expressed
// by the strides alone.
#pragma once

#include <stdint.h>

namespace sg {

// C[o][x][y] = sum_b A[o][x][b] B[o][b][y] with element strides; 64 x 64
// output tile per block, 16-deep K chunks through shared memory, 256 threads
// with a 4 x 4 register tile each (rows ty + 16 i, columns tx + 16 j).
struct GemmArgs {
  const void *A, *B;
  void *C;
  int64_t ao, ax, ab, bo, bb, by, co, cx, cy;
  int64_t X, Y, K;
};

constexpr int kBX = 64, kBY = 64, kBK = 16, kGemmThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kGemmThreads) strided_gemm_kernel(GemmArgs g) {
  __shared__ T As[kBK][kBX + 1];
  __shared__ T Bs[kBK][kBY + 1];
  const T *A = (const T *)g.A;
  const T *B = (const T *)g.B;
  T *C = (T *)g.C;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int64_t o = blockIdx.z;
  const int64_t x0 = (int64_t)blockIdx.y * kBX, y0 = (int64_t)blockIdx.x * kBY;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
  for (int64_t k0 = 0; k0 < g.K; k0 += kBK) {
#pragma unroll
    for (int q = 0; q < (kBX * kBK) / kGemmThreads; ++q) {
      const int e = tid + q * kGemmThreads;
      const int xi = e / kBK, bi = e % kBK;
      const int64_t x = x0 + xi, b = k0 + bi;
      As[bi][xi] = (x < g.X && b < g.K) ? A[o * g.ao + x * g.ax + b * g.ab] : T(0);
    }
#pragma unroll
    for (int q = 0; q < (kBY * kBK) / kGemmThreads; ++q) {
      const int e = tid + q * kGemmThreads;
      const int bi = e / kBY, yi = e % kBY;
      const int64_t y = y0 + yi, b = k0 + bi;
      Bs[bi][yi] = (y < g.Y && b < g.K) ? B[o * g.bo + b * g.bb + y * g.by] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int bi = 0; bi < kBK; ++bi) {
      T a[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[bi][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Bs[bi][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t x = x0 + ty + 16 * i;
    if (x >= g.X) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t y = y0 + tx + 16 * j;
      if (y < g.Y) C[o * g.co + x * g.cx + y * g.cy] = acc[i][j];
    }
  }
}


// Launch C = A B over `batch` entries (grid y <= 65535 tiles of X, z = batch).
template <typename T>
inline cudaError_t gemm(const GemmArgs &g, int64_t batch, cudaStream_t st) {
  if (g.X < 1 || g.Y < 1 || batch < 1) return cudaSuccess;
  const dim3 grid((unsigned)((g.Y + kBY - 1) / kBY), (unsigned)((g.X + kBX - 1) / kBX),
                  (unsigned)batch);
  strided_gemm_kernel<T><<<grid, kGemmThreads, 0, st>>>(g);
  return cudaGetLastError();
}

}  // namespace sg
