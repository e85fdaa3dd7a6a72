// Batched skinny GEMM on the tcgen05 tensor cores with operands fed by tensor
// copies (TMA), for the products of the slice pass with the transformed
// slices (Y = Abar X, W = Abar^T Q; Alg. 1's sketch and power steps).  Two
// forms: gemm_kernel (A given in FP32 and converted in shared memory,
// described here) and planes_kernel (A given as BF16 hi/lo planes; its own
// description below).
//
// C[b] (M x N) = A[b] (M x K) * B[b] (K x N), FP32 in and out, N <= 64.  The
// work is a list of 128-row tiles (batch entry, row block); a persistent CTA
// (8 warps, two per SM) takes every gridDim-th tile and streams their K
// chunks of 32 as one sequence: one thread keeps STAGES chunks of both
// operands in flight as 3D tensor copies (cp.async.bulk.tensor.3d,
// completion counted on an mbarrier) into FP32 staging tiles, so the HBM
// latency of a chunk -- the next tile's first ones included -- overlaps the
// work on the chunks before it.  Seven warps convert a landed chunk
// to BF16 (x = hi + lo, both BF16, for the split form) in the canonical
// K-major core-matrix layout without swizzle (8-row x 16-byte core
// matrices, leading byte offset 128, stride byte offset 512), and one
// elected thread issues tcgen05.mma (kind::f16, BF16 x BF16 -> FP32) into
// a TMEM accumulator of 128 lanes x NP columns, committing to an mbarrier
// per conversion buffer (two buffers).  The epilogue reads TMEM with
// tcgen05.ld and writes C with element strides.
//
// Staging layouts.  A with k contiguous (A = Abar): box {32 k, 128 m, 1},
// 128-byte rows with the 128-byte swizzle (16-byte chunk c of row r sits at
// chunk c ^ (r mod 8)), so that threads taking consecutive rows read
// distinct banks.  A with m contiguous (A = Abar^T): box {128 m, 32 k, 1},
// rows of 128 m without swizzle (a thread reads one column).  B (k
// contiguous): box {32 k, NP n, 1} with the 128-byte swizzle.  Every box
// is a 3D view (inner, middle, batch), so rows past M, columns past N and
// k past K read as zeros.
//
// Warps 1-7 convert chunk c + 1 while thread 0 issues the copies and MMAs of
// chunk c (one block barrier per chunk); the tcgen05.ld epilogue runs in warps
// 0-3, whose lane quarters cover the accumulator's 128 lanes.
//
// SPLIT = 3: A_hi B_hi + A_hi B_lo + A_lo B_hi (products carry about 16
// significant bits, FP32-form accuracy); SPLIT = 1: the plain BF16 form.
//
// Every mbarrier wait is bounded; on time-out the CTA records the failure
// in *err, stops issuing work, waits (bounded) for its own copies and MMAs
// and frees its TMEM before returning.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "umma_gemm.cuh"

namespace tmag {

constexpr int kThreads = 256;   // warp 0 issues, warps 1-7 convert, warps 0-3 read TMEM
constexpr int kBM = 128;
constexpr int kKC = 32;   // K elements per chunk: two MMAs of K = 16

struct Args {
  CUtensorMap amap;   // FP32 3D view of A: {K, M, nA} (k contiguous) or {M, K, nA};
                      // planes_kernel: BF16 view of A's hi plane
  CUtensorMap amap_lo;  // planes_kernel: BF16 view of A's lo plane (SPLIT = 3)
  CUtensorMap bmap;   // FP32 3D view of B: {K, N, batch}
  int M, N, K;
  int a_kcontig;      // 1: A's k is contiguous (A = Abar), 0: A's m is (A = Abar^T)
  float *C;
  int64_t sCb, sCi, sCn;
  const int *ids = nullptr;    // optional batch indirection (as umma::Args)
  const int *count = nullptr;
  int a_by_id = 0, c_by_id = 0;
  int batch = 0;               // batch entries (the launch's upper bound on *count)
};

template <int NP, int STAGES, int SPLIT>
struct Layout {
  static constexpr int a_stage = kBM * kKC * 4;           // FP32 staging of A
  static constexpr int b_stage = NP * kKC * 4;            // FP32 staging of B
  static constexpr int stage = a_stage + b_stage;         // a multiple of 1024
  static constexpr int a_conv = kBM * kKC * 2;            // one BF16 copy of A
  static constexpr int b_conv = NP * kKC * 2;
  static constexpr int conv = (a_conv + b_conv) * (SPLIT > 1 ? 2 : 1);
  static constexpr int total = STAGES * stage + 2 * conv;
  static_assert(stage % 1024 == 0, "swizzled staging tiles need 1024-byte alignment");
};

// Bounded wait for the mbarrier phase with parity `parity`: try_wait lets the
// hardware suspend the thread for a while instead of spinning; at most
// kSpinLimit tries, false on timeout.
__device__ __forceinline__ bool wait_phase(uint64_t *bar, uint32_t parity) {
  const uint32_t addr = umma::smem_u32(bar);
  for (uint32_t it = 0; it < umma::kSpinLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                   umma::smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z,
                                            uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(umma::smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(umma::smem_u32(bar))
      : "memory");
}

// Eight FP32 values -> one 16-byte BF16 core-matrix row (hi) and its
// remainder (lo).
template <int SPLIT>
__device__ __forceinline__ void put8(const float (&x)[8], uint8_t *hi, uint8_t *lo, int off) {
  // pairs rounded to BF16 at once; lo = x - hi exactly in FP32, then rounded
  __nv_bfloat162 h[4], l[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    h[e] = __floats2bfloat162_rn(x[2 * e], x[2 * e + 1]);
    if (SPLIT > 1) {
      const float2 f = __bfloat1622float2(h[e]);
      l[e] = __floats2bfloat162_rn(x[2 * e] - f.x, x[2 * e + 1] - f.y);
    }
  }
  *reinterpret_cast<uint4 *>(hi + off) = *reinterpret_cast<const uint4 *>(h);
  if (SPLIT > 1) *reinterpret_cast<uint4 *>(lo + off) = *reinterpret_cast<const uint4 *>(l);
}

// Byte offset of row r, k-core c in a K-major core-matrix tile with kKC = 32
// (four k-cores per 8-row group).
__device__ __forceinline__ int core_off(int r, int c) { return ((r >> 3) * 4 + c) * 128 + (r & 7) * 16; }

// Eight consecutive k (k-core c) of row r of a 128-byte-swizzled staging
// tile (rows of 32 FP32).
__device__ __forceinline__ void get8_swz(const uint8_t *tile, int r, int c, float (&x)[8]) {
  const uint8_t *row = tile + r * 128;
  const float4 v0 = *reinterpret_cast<const float4 *>(row + (((2 * c) ^ (r & 7)) << 4));
  const float4 v1 = *reinterpret_cast<const float4 *>(row + (((2 * c + 1) ^ (r & 7)) << 4));
  x[0] = v0.x; x[1] = v0.y; x[2] = v0.z; x[3] = v0.w;
  x[4] = v1.x; x[5] = v1.y; x[6] = v1.z; x[7] = v1.w;
}

template <int NP, int STAGES, int SPLIT>
__global__ void __launch_bounds__(kThreads)
    gemm_kernel(const __grid_constant__ Args g, int *err) {
  pdl_wait();
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full[STAGES];
  __shared__ __align__(8) uint64_t mdone[2];
  __shared__ uint32_t tmem_base_s;
  constexpr int kMaxTiles = 64;          // slice ids of this CTA's tiles, read once
  __shared__ int tile_jb[kMaxTiles];
  using Lay = Layout<NP, STAGES, SPLIT>;
  constexpr int TMEM_COLS = NP < 32 ? 32 : NP;
  // the dynamic window is aligned up to 1024 bytes (the launch reserves it)
  uint8_t *smem = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // Tiles (batch entry b, 128-row block mt) in order t = b * mtiles + mt; this
  // CTA takes t = blockIdx.x, blockIdx.x + gridDim.x, ... below the entry
  // count, and streams their K chunks as one sequence, so the copies of the
  // next tile's first chunks are in flight while this tile finishes.
  const int mtiles = (g.M + kBM - 1) / kBM;
  int entries = g.count ? *g.count : g.batch;
  if (entries > g.batch) entries = g.batch;
  const int ntiles = entries * mtiles;
  const int my_tiles = blockIdx.x < ntiles ? (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  if (my_tiles == 0) return;   // block-uniform, before any TMEM use
  const int nk = (g.K + kKC - 1) / kKC;
  const int total = my_tiles * nk;   // chunks this CTA streams

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     umma::smem_u32(&tmem_base_s)),
                 "r"((uint32_t)TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  for (int lt = tid; lt < my_tiles && lt < kMaxTiles; lt += kThreads) {
    const int b = (blockIdx.x + lt * gridDim.x) / mtiles;
    tile_jb[lt] = g.ids ? g.ids[b] : b;
  }
  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) umma::mbar_init(&full[s], 1);
    umma::mbar_init(&mdone[0], 1);
    umma::mbar_init(&mdone[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  umma::fence_before();
  __syncthreads();
  umma::fence_after();
  const uint32_t tmem = tmem_base_s;

  struct Tile {
    int m0, b, za;
    float *C;
  };
  auto tile_of = [&](int lt) {   // this CTA's lt-th tile
    const int t = blockIdx.x + lt * gridDim.x;
    Tile r;
    r.b = t / mtiles;
    r.m0 = (t % mtiles) * kBM;
    const int jb = lt < kMaxTiles ? tile_jb[lt] : (g.ids ? g.ids[r.b] : r.b);
    r.za = g.a_by_id ? jb : r.b;
    r.C = g.C + (int64_t)(g.c_by_id ? jb : r.b) * g.sCb;
    return r;
  };
  auto issue = [&](int gc) {   // one thread: chunk gc into staging stage gc % STAGES
    const int s = gc % STAGES, kc = gc % nk;
    const Tile tl = tile_of(gc / nk);
    uint8_t *st = smem + s * Lay::stage;
    expect_tx(&full[s], (uint32_t)Lay::stage);
    if (g.a_kcontig) tma_load_3d(st, &g.amap, kc * kKC, tl.m0, tl.za, &full[s]);
    else tma_load_3d(st, &g.amap, tl.m0, kc * kKC, tl.za, &full[s]);
    tma_load_3d(st + Lay::a_stage, &g.bmap, kc * kKC, 0, tl.b, &full[s]);
  };
  if (tid == 0)
    for (int c = 0; c < STAGES && c < total; ++c) issue(c);
  int issued = STAGES < total ? STAGES : total;   // meaningful in thread 0 only

  constexpr uint32_t idesc = umma::idesc_bf16(kBM, NP);
  constexpr uint32_t LBO = 128, SBO = (kKC / 8) * 128;
  bool ok = true;
  int done_chunks = 0;   // chunks whose MMAs were committed
  Tile cur = tile_of(0);
#pragma unroll 1
  for (int gc = 0; gc < total; ++gc) {
    const int s = gc % STAGES, h = gc & 1, kc = gc % nk;
    if (kc == 0 && gc > 0) cur = tile_of(gc / nk);
    // warps 1-7 convert chunk gc while thread 0 still issues chunk gc - 1
    bool okc = true;
    if (warp != 0) {
      okc = wait_phase(&full[s], (uint32_t)((gc / STAGES) & 1));
      // the MMAs that read conversion buffer h two chunks ago must be done
      if (okc && gc >= 2) okc = wait_phase(&mdone[h], (uint32_t)(((gc - 2) >> 1) & 1));
      if (okc) {
        const uint8_t *sa = smem + s * Lay::stage;
        const uint8_t *sb = sa + Lay::a_stage;
        uint8_t *cv = smem + STAGES * Lay::stage + h * Lay::conv;
        uint8_t *a_hi = cv, *b_hi = cv + Lay::a_conv;
        uint8_t *a_lo = cv + Lay::a_conv + Lay::b_conv, *b_lo = a_lo + Lay::a_conv;
        constexpr int UA = kBM * 4, UT = UA + NP * 4;   // A units, all units
        for (int u = tid - 32; u < UT; u += kThreads - 32) {
          float x[8];
          if (u < UA) {   // A: row u % 128, k-core u / 128
            const int r = u & (kBM - 1), kq = u / kBM;
            if (g.a_kcontig) {
              get8_swz(sa, r, kq, x);
            } else {
              const float *col = reinterpret_cast<const float *>(sa) + r;
#pragma unroll
              for (int e = 0; e < 8; ++e) x[e] = col[(kq * 8 + e) * kBM];
            }
            put8<SPLIT>(x, a_hi, a_lo, core_off(r, kq));
          } else {        // B: row (u - UA) % NP, k-core (u - UA) / NP
            const int r = (u - UA) % NP, kq = (u - UA) / NP;
            get8_swz(sb, r, kq, x);
            put8<SPLIT>(x, b_hi, b_lo, core_off(r, kq));
          }
        }
      }
      umma::fence_async_smem();
    }
    if (!__syncthreads_and(okc)) { ok = false; break; }
    if (tid == 0) {
      // staging stage s has been read by every converter: refill it
      if (issued < total) {
        issue(issued);
        ++issued;
      }
      uint8_t *cv = smem + STAGES * Lay::stage + h * Lay::conv;
      uint8_t *a_hi = cv, *b_hi = cv + Lay::a_conv;
      uint8_t *a_lo = cv + Lay::a_conv + Lay::b_conv, *b_lo = a_lo + Lay::a_conv;
      umma::fence_after();
#pragma unroll
      for (int ks = 0; ks < kKC / 16; ++ks) {
        const uint32_t off = ks * 2 * 128;   // two k-cores per MMA (K = 16)
        const uint64_t dah = umma::smem_desc(umma::smem_u32(a_hi) + off, LBO, SBO);
        const uint64_t dbh = umma::smem_desc(umma::smem_u32(b_hi) + off, LBO, SBO);
        umma::mma_bf16(tmem, dah, dbh, idesc, (kc > 0 || ks > 0) ? 1u : 0u);
        if (SPLIT > 1) {
          const uint64_t dal = umma::smem_desc(umma::smem_u32(a_lo) + off, LBO, SBO);
          const uint64_t dbl = umma::smem_desc(umma::smem_u32(b_lo) + off, LBO, SBO);
          umma::mma_bf16(tmem, dah, dbl, idesc, 1u);
          umma::mma_bf16(tmem, dal, dbh, idesc, 1u);
        }
      }
      umma::mma_commit(&mdone[h]);
    }
    done_chunks = gc + 1;
    if (kc == nk - 1) {
      // last chunk of the tile: its MMAs done, the accumulator goes out; the
      // next tile's first MMA (accumulate 0) is issued only after this
      const bool wd = wait_phase(&mdone[h], (uint32_t)((gc >> 1) & 1));
      if (!__syncthreads_and(wd)) { ok = false; break; }
      if (warp < 4) {   // TMEM lanes 32w .. 32w + 31 belong to warp w mod 4
        umma::fence_after();
        const int row = cur.m0 + warp * 32 + lane;
#pragma unroll
        for (int c0 = 0; c0 < NP; c0 += 32) {
          float v[32];
          umma::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
          if (row < g.M) {
#pragma unroll
            for (int c = 0; c < 32; ++c)
              if (c0 + c < g.N) cur.C[(int64_t)row * g.sCi + (int64_t)(c0 + c) * g.sCn] = v[c];
          }
        }
      }
      umma::fence_before();
      __syncthreads();
    }
  }
  if (!ok) {
    // wait (bounded) for the MMAs committed on each conversion buffer and
    // for the copies issued but never consumed, then give up
    for (int h = 0; h < 2; ++h) {
      const int used = done_chunks > h ? (done_chunks - 1 - h) / 2 + 1 : 0;
      if (used > 0) wait_phase(&mdone[h], (uint32_t)((used - 1) & 1));
    }
    if (tid == 0) {
      atomicExch(err, 1);
      for (int c = done_chunks; c < issued; ++c)
        wait_phase(&full[c % STAGES], (uint32_t)((c / STAGES) & 1));
    }
  }
  pdl_trigger();
  umma::fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)TMEM_COLS));
}

// ---------------------------------------------------------------------------
// The same products with A already split: the tube pass writes Abar as two
// BF16 planes (x = hi + lo), so A's tiles go from HBM straight into the
// operand layout and only B (the FP32 panel, N <= 64 columns) is converted.
// K chunks of 64.  A tiles use the 128-byte swizzle: with k contiguous
// (Y = Abar X) a box {64 k, 128 m} is the K-major operand (rows of 128
// bytes, 8-row groups 1024 bytes apart); with m contiguous (W = Abar^T Q)
// two boxes {64 m, 64 k} are the MN-major operand (rows are k; the second
// 64-row block of m 8192 bytes on).  B is staged as two FP32 boxes {32 k,
// NP n} (128-byte swizzle) and converted into a K-major BF16 tile with the
// same swizzle, B_hi's NP rows followed by B_lo's.  K steps past K are not
// issued.  An M = 128 MMA costs about the same for any N up to 64, so the
// split form takes two MMAs per K step instead of three: A_hi [B_hi; B_lo]
// (N = 2 NP, columns NP.. of the accumulator take A_hi B_lo) and A_lo B_hi
// (N = NP, accumulated onto A_hi B_hi); the epilogue adds the two column
// halves.
//
// One persistent CTA per SM; its warps take fixed roles and hand chunks to
// one another through mbarriers, so that no role waits on another's latency
// chain:
//   warp 0 (one thread)  copies chunk c into stage c % STAGES once the MMAs
//                        of chunk c - STAGES have released it (empty);
//   warp 1 (one thread)  issues chunk c's MMAs once it has landed (full)
//                        and its B is converted (cfull); commits release
//                        the stage (empty) and the conversion buffer
//                        (cempty); a tile's last chunk commits its
//                        accumulator (afull).  Two TMEM accumulators
//                        alternate; a tile's first MMA waits until the
//                        epilogue has drained its accumulator (aempty);
//   warps 2-7            convert B of chunk c into conversion buffer c % 2
//                        (two warps took ~850 cycles a chunk, longer than the
//                        chunk's MMAs);
//   warps 8-11           epilogue: accumulator -> C (warp w reads TMEM
//                        lanes 32 (w - 8) ..).
// Every wait is bounded and also gives up once another role has (abort);
// the CTA then records the failure in *err, waits (bounded) for its copies
// and MMAs in flight, and frees its TMEM.
constexpr int kKP = 64;   // K elements per chunk: four MMAs of K = 16
constexpr int kPlanesThreads = 384;   // copies, MMAs, 6 converting warps, 4 epilogue warps
constexpr int kCvtWarps = 6;

template <int NP, int STAGES, int SPLIT>
struct PlanesLayout {
  static constexpr int a_plane = kBM * kKP * 2;                  // one BF16 plane tile
  static constexpr int a_stage = a_plane * (SPLIT > 1 ? 2 : 1);
  static constexpr int b_half = NP * 128;                        // FP32 box {32 k, NP n}
  static constexpr int b_stage = 2 * b_half;
  static constexpr int stage = a_stage + b_stage;
  static constexpr int b_conv = NP * kKP * 2;                    // one BF16 copy of B
  static constexpr int conv = b_conv * (SPLIT > 1 ? 2 : 1);
  static constexpr int total = STAGES * stage + 2 * conv;
  static_assert(stage % 1024 == 0 && b_conv % 1024 == 0 && a_plane % 1024 == 0,
                "swizzled tiles need 1024-byte alignment");
};

// wait_phase that also returns false once *abort is set
__device__ __forceinline__ bool wait_or_abort(uint64_t *bar, uint32_t parity,
                                              const volatile int *abort) {
  const uint32_t addr = umma::smem_u32(bar);
  for (uint32_t it = 0; it < umma::kSpinLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 63) == 63 && *abort) return false;
  }
  return false;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(umma::smem_u32(bar)) : "memory");
}

template <int NP, int STAGES, int SPLIT>
__global__ void __launch_bounds__(kPlanesThreads)
    planes_kernel(const __grid_constant__ Args g, int *err) {
  pdl_wait();
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES];
  __shared__ __align__(8) uint64_t cfull[2], cempty[2], afull[2], aempty[2], drain;
  __shared__ uint32_t tmem_base_s;
  __shared__ int abort_s, issued_s, consumed_s;
  constexpr int kMaxTiles = 64;
  __shared__ int tile_jb[kMaxTiles];
  using Lay = PlanesLayout<NP, STAGES, SPLIT>;
  constexpr int ACC = SPLIT > 1 ? 2 * NP : NP;   // accumulator columns
  constexpr int TMEM_COLS = 2 * ACC;              // two accumulators
  uint8_t *smem = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int mtiles = (g.M + kBM - 1) / kBM;
  int entries = g.count ? *g.count : g.batch;
  if (entries > g.batch) entries = g.batch;
  const int ntiles = entries * mtiles;
  const int my_tiles = blockIdx.x < ntiles ? (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  if (my_tiles == 0) return;   // block-uniform, before any TMEM use
  const int nk = (g.K + kKP - 1) / kKP;
  const int total = my_tiles * nk;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     umma::smem_u32(&tmem_base_s)),
                 "r"((uint32_t)TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  for (int lt = tid; lt < my_tiles && lt < kMaxTiles; lt += kPlanesThreads) {
    const int b = (blockIdx.x + lt * gridDim.x) / mtiles;
    tile_jb[lt] = g.ids ? g.ids[b] : b;
  }
  if (tid == 0) {
    // the copies' descriptors into the descriptor cache once, not per copy
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&g.amap)) : "memory");
    if (SPLIT > 1)
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&g.amap_lo)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&g.bmap)) : "memory");
    for (int s = 0; s < STAGES; ++s) {
      umma::mbar_init(&full[s], 1);
      umma::mbar_init(&empty[s], 1);
    }
    for (int h = 0; h < 2; ++h) {
      umma::mbar_init(&cfull[h], kCvtWarps);   // one arrival per converter warp
      umma::mbar_init(&cempty[h], 1);
      umma::mbar_init(&afull[h], 1);
      umma::mbar_init(&aempty[h], 4);   // one arrival per epilogue warp
    }
    umma::mbar_init(&drain, 1);
    abort_s = 0;
    issued_s = 0;
    consumed_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  umma::fence_before();
  __syncthreads();
  umma::fence_after();
  const uint32_t tmem = tmem_base_s;
  volatile int *abort = &abort_s;

  struct Tile {
    int m0, b, za;
    float *C;
  };
  auto tile_of = [&](int lt) {
    const int t = blockIdx.x + lt * gridDim.x;
    Tile r;
    r.b = t / mtiles;
    r.m0 = (t % mtiles) * kBM;
    const int jb = lt < kMaxTiles ? tile_jb[lt] : (g.ids ? g.ids[r.b] : r.b);
    r.za = g.a_by_id ? jb : r.b;
    r.C = g.C + (int64_t)(g.c_by_id ? jb : r.b) * g.sCb;
    return r;
  };

  if (warp == 0) {
    // ---- copies
    if (lane == 0) {
      int c = 0, s = 0, round = 0, kc = 0;   // chunk, its stage, the stage's use, its k chunk
      Tile tl = tile_of(0);
      for (; c < total; ++c) {
        if (c >= STAGES && !wait_or_abort(&empty[s], (uint32_t)((round - 1) & 1), abort)) {
          *abort = 1;
          break;
        }
        uint8_t *st = smem + s * Lay::stage;
        expect_tx(&full[s], (uint32_t)Lay::stage);
        if (g.a_kcontig) {
          tma_load_3d(st, &g.amap, kc * kKP, tl.m0, tl.za, &full[s]);
          if (SPLIT > 1)
            tma_load_3d(st + Lay::a_plane, &g.amap_lo, kc * kKP, tl.m0, tl.za, &full[s]);
        } else {
          tma_load_3d(st, &g.amap, tl.m0, kc * kKP, tl.za, &full[s]);
          tma_load_3d(st + Lay::a_plane / 2, &g.amap, tl.m0 + 64, kc * kKP, tl.za, &full[s]);
          if (SPLIT > 1) {
            tma_load_3d(st + Lay::a_plane, &g.amap_lo, tl.m0, kc * kKP, tl.za, &full[s]);
            tma_load_3d(st + Lay::a_plane + Lay::a_plane / 2, &g.amap_lo, tl.m0 + 64, kc * kKP,
                        tl.za, &full[s]);
          }
        }
        uint8_t *sb = st + Lay::a_stage;
        tma_load_3d(sb, &g.bmap, kc * kKP, 0, tl.b, &full[s]);
        tma_load_3d(sb + Lay::b_half, &g.bmap, kc * kKP + 32, 0, tl.b, &full[s]);
        if (++s == STAGES) {
          s = 0;
          ++round;
        }
        if (++kc == nk && c + 1 < total) {
          kc = 0;
          tl = tile_of((c + 1) / nk);
        }
      }
      issued_s = c;
    }
  } else if (warp == 1) {
    // ---- MMAs
    if (lane == 0) {
      const uint32_t amaj = g.a_kcontig ? 0u : umma::kIdescAMajorMN;
      const uint32_t idesc = umma::idesc_bf16(kBM, NP) | amaj;
      const uint32_t idesc2 = umma::idesc_bf16(kBM, 2 * NP) | amaj;
      // K-major A: 32 bytes per K = 16 inside the swizzled rows; MN-major A:
      // two 8-row k groups per K = 16, 64-row m blocks half a plane apart
      const uint32_t a_step = g.a_kcontig ? 32u : 2048u;
      const uint32_t a_lbo = g.a_kcontig ? 16u : (uint32_t)(Lay::a_plane / 2);
      int c = 0;
      bool okm = true;
      for (int lt = 0; lt < my_tiles && okm; ++lt) {
        const int a = lt & 1;
        if (lt >= 2 && !wait_or_abort(&aempty[a], (uint32_t)(((lt >> 1) - 1) & 1), abort)) {
          okm = false;
          break;
        }
        umma::fence_after();
        const uint32_t acc = tmem + (uint32_t)(a * ACC);
        for (int kc = 0; kc < nk; ++kc) {
          const int s = c % STAGES, h = c & 1;
          if (!wait_or_abort(&full[s], (uint32_t)((c / STAGES) & 1), abort) ||
              !wait_or_abort(&cfull[h], (uint32_t)((c >> 1) & 1), abort)) {
            okm = false;
            break;
          }
          umma::fence_after();
          const uint32_t a_hi = umma::smem_u32(smem + s * Lay::stage), a_lo = a_hi + Lay::a_plane;
          // B_hi's rows, then B_lo's: one K-major tile of 2 NP rows
          const uint32_t bh = umma::smem_u32(smem + STAGES * Lay::stage + h * Lay::conv);
#pragma unroll
          for (int ks = 0; ks < kKP / 16; ++ks) {
            if (kc * kKP + ks * 16 >= g.K) break;
            const uint32_t first = (kc > 0 || ks > 0) ? 1u : 0u;
            const uint64_t dah = umma::smem_desc_sw128(a_hi + ks * a_step, a_lbo, 1024);
            const uint64_t dbh = umma::smem_desc_sw128(bh + ks * 32, 16, 1024);
            if (SPLIT > 1) {
              const uint64_t dal = umma::smem_desc_sw128(a_lo + ks * a_step, a_lbo, 1024);
              umma::mma_bf16(acc, dah, dbh, idesc2, first);   // A_hi [B_hi; B_lo]
              umma::mma_bf16(acc, dal, dbh, idesc, 1u);       // + A_lo B_hi
            } else {
              umma::mma_bf16(acc, dah, dbh, idesc, first);
            }
          }
          umma::mma_commit(&empty[s]);
          umma::mma_commit(&cempty[h]);
          ++c;
        }
        if (okm) umma::mma_commit(&afull[a]);
      }
      if (!okm) *abort = 1;
      consumed_s = c;
      // every MMA issued completes before the CTA tears down
      umma::mma_commit(&drain);
      wait_phase(&drain, 0u);
    }
  } else if (warp < 2 + kCvtWarps) {
    // ---- B conversion (kCvtWarps warps)
    const int ct = tid - 64;
    for (int c = 0; c < total; ++c) {
      const int s = c % STAGES, h = c & 1;
      bool okc = wait_or_abort(&full[s], (uint32_t)((c / STAGES) & 1), abort);
      if (okc && c >= 2) okc = wait_or_abort(&cempty[h], (uint32_t)(((c >> 1) - 1) & 1), abort);
      if (!__all_sync(0xffffffffu, okc)) {
        if (lane == 0) *abort = 1;
        break;
      }
      const uint8_t *sb = smem + s * Lay::stage + Lay::a_stage;
      uint8_t *b_hi = smem + STAGES * Lay::stage + h * Lay::conv;
      uint8_t *b_lo = b_hi + Lay::b_conv;
      for (int u = ct; u < NP * (kKP / 8); u += 32 * kCvtWarps) {
        const int r = u % NP, kq = u / NP;   // row r, k-core kq (8 k)
        float x[8];
        get8_swz(sb + (kq >> 2) * Lay::b_half, r, kq & 3, x);
        put8<SPLIT>(x, b_hi, b_lo, r * 128 + ((kq ^ (r & 7)) << 4));
      }
      umma::fence_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&cfull[h]);
    }
  } else {
    // ---- epilogue (warps 8-11)
    const int q = warp & 3;
    for (int lt = 0; lt < my_tiles; ++lt) {
      const int a = lt & 1;
      const bool oke = wait_or_abort(&afull[a], (uint32_t)((lt >> 1) & 1), abort);
      if (!__all_sync(0xffffffffu, oke)) {
        if (lane == 0) *abort = 1;
        break;
      }
      umma::fence_after();
      const Tile tl = tile_of(lt);
      const int row = tl.m0 + q * 32 + lane;
      const uint32_t lanes = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(a * ACC);
#pragma unroll
      for (int c0 = 0; c0 < NP; c0 += 32) {
        float v[32];
        umma::tmem_ld32(lanes + (uint32_t)c0, v);
        if (SPLIT > 1) {   // + the A_hi B_lo half
          float w[32];
          umma::tmem_ld32(lanes + (uint32_t)(NP + c0), w);
#pragma unroll
          for (int c = 0; c < 32; ++c) v[c] += w[c];
        }
        if (row < g.M) {
#pragma unroll
          for (int c = 0; c < 32; ++c)
            if (c0 + c < g.N) tl.C[(int64_t)row * g.sCi + (int64_t)(c0 + c) * g.sCn] = v[c];
        }
      }
      umma::fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&aempty[a]);
    }
  }
  __syncthreads();
  if (abort_s && tid == 0) {
    atomicExch(err, 1);
    // copies issued but never consumed by an MMA land before the CTA exits
    for (int c = consumed_s; c < issued_s; ++c)
      wait_phase(&full[c % STAGES], (uint32_t)((c / STAGES) & 1));
  }
  pdl_trigger();
  umma::fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)TMEM_COLS));
}

}  // namespace tmag
