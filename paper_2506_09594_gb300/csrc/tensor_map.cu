// Tensor maps (TMA descriptors) for 2D and 3D views of device arrays, encoded through
// the driver entry point cuTensorMapEncodeTiled and cached by view.
#include <cudaTypedefs.h>

#include <stdint.h>

#include <mutex>

#include "tr_internal.cuh"

namespace {

PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

struct MapEntry {
  const void *base;
  int64_t cols, rows, stride;
  int bx, by, u8;
  CUtensorMap map;
};

constexpr int kCacheSize = 128;

}  // namespace

bool encode_tensor_2d(CUtensorMap *out, const void *base, bool u8, int64_t cols, int64_t rows,
                      int64_t row_stride, int box_cols, int box_rows) {
  static std::mutex mu;
  static MapEntry cache[kCacheSize];
  static int used = 0, next = 0;
  const int esz = u8 ? 1 : 4;
  if (!base || (uintptr_t)base % 16 != 0 || (row_stride * esz) % 16 != 0 || cols < 1 ||
      rows < 1 || box_cols < 1 || box_cols > 256 || box_rows < 1 || box_rows > 256 ||
      (box_cols * esz) % 16 != 0)
    return false;
  std::lock_guard<std::mutex> lock(mu);
  for (int i = 0; i < used; ++i) {
    const MapEntry &c = cache[i];
    if (c.base == base && c.cols == cols && c.rows == rows && c.stride == row_stride &&
        c.bx == box_cols && c.by == box_rows && c.u8 == (int)u8) {
      *out = c.map;
      return true;
    }
  }
  auto fn = tmap_encoder();
  if (!fn) return false;
  const cuuint64_t dim[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t stride[1] = {(cuuint64_t)(row_stride * esz)};
  const cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  const cuuint32_t es[2] = {1, 1};
  CUtensorMap m;
  if (fn(&m, u8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
         const_cast<void *>(base), dim, stride, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
         CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return false;
  cache[next] = MapEntry{base, cols, rows, row_stride, box_cols, box_rows, (int)u8, m};
  next = (next + 1) % kCacheSize;
  if (used < kCacheSize) ++used;
  *out = m;
  return true;
}

namespace {
struct Map3Entry {
  const void *base;
  int64_t d0, d1, d2, s1, s2;
  int b0, b1, swz, esz;
  CUtensorMap map;
};
}  // namespace

bool encode_tensor_3d(CUtensorMap *out, const void *base, int esz, int64_t d0, int64_t d1,
                      int64_t d2, int64_t s1, int64_t s2, int box0, int box1, bool swizzle128) {
  static std::mutex mu;
  static Map3Entry cache[kCacheSize];
  static int used = 0, next = 0;
  if (!base || (esz != 2 && esz != 4) || (uintptr_t)base % 16 != 0 || d0 < 1 || d1 < 1 ||
      d2 < 1 || (s1 * esz) % 16 != 0 || (s2 * esz) % 16 != 0 || box0 < 1 || box0 > 256 ||
      box1 < 1 || box1 > 256 || (box0 * esz) % 16 != 0 || (swizzle128 && box0 * esz != 128) ||
      d0 > INT32_MAX || d1 > INT32_MAX || d2 > INT32_MAX)
    return false;
  std::lock_guard<std::mutex> lock(mu);
  for (int i = 0; i < used; ++i) {
    const Map3Entry &c = cache[i];
    if (c.base == base && c.d0 == d0 && c.d1 == d1 && c.d2 == d2 && c.s1 == s1 && c.s2 == s2 &&
        c.b0 == box0 && c.b1 == box1 && c.swz == (int)swizzle128 && c.esz == esz) {
      *out = c.map;
      return true;
    }
  }
  auto fn = tmap_encoder();
  if (!fn) return false;
  const cuuint64_t dim[3] = {(cuuint64_t)d0, (cuuint64_t)d1, (cuuint64_t)d2};
  const cuuint64_t stride[2] = {(cuuint64_t)(s1 * esz), (cuuint64_t)(s2 * esz)};
  const cuuint32_t box[3] = {(cuuint32_t)box0, (cuuint32_t)box1, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  CUtensorMap m;
  if (fn(&m, esz == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3,
         const_cast<void *>(base), dim, stride, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
         swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return false;
  cache[next] = Map3Entry{base, d0, d1, d2, s1, s2, box0, box1, (int)swizzle128, esz, m};
  next = (next + 1) % kCacheSize;
  if (used < kCacheSize) ++used;
  *out = m;
  return true;
}

bool encode_tensor_3d_f32(CUtensorMap *out, const void *base, int64_t d0, int64_t d1, int64_t d2,
                          int64_t s1, int64_t s2, int box0, int box1, bool swizzle128) {
  return encode_tensor_3d(out, base, 4, d0, d1, d2, s1, s2, box0, box1, swizzle128);
}
