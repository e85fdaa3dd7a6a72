// Batched skinny GEMM on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// C[b] (M x N) = A[b] (M x K) * B[b] (K x N), FP32 in and out.  One CTA
// (4 warps) owns a 128-row x NP-column tile of one batch entry (NP in {32,
// 64, 128}; N above 128 takes several column tiles).  K is consumed
// in chunks of 64: the 128 threads load the FP32 operands from global
// memory, round them to BF16 (optionally split x = hi + lo, both BF16) and
// store them in shared memory in the canonical K-major layout without
// swizzle -- 8-row x 16-byte core matrices, core (g, c) at byte
// (g * KC/8 + c) * 128, i.e. leading-dimension (K) byte offset 128 and
// stride-dimension (M/N) byte offset KC/8 * 128.  One elected thread issues
// tcgen05.mma (kind::f16, BF16 x BF16 -> FP32) into a TMEM accumulator of
// 128 lanes x NP columns and commits each chunk to an mbarrier, so the next
// chunk is staged while the tensor core works on this one (two stages).
// The epilogue reads TMEM with tcgen05.ld (32x32b: warp w owns lanes
// 32w..32w+31 = rows) and writes C with element strides.
//
// SPLIT = 3 adds A_hi*B_lo + A_lo*B_hi (A_lo*B_lo dropped): products carry
// ~16 significant bits, enough for FP32-form accuracy (1e-4); SPLIT = 1 is
// the plain BF16 form.
//
// Every mbarrier wait is bounded; on timeout the CTA records the failure in
// *err, stops issuing work, waits (bounded) for its own MMAs and frees its
// TMEM before returning.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace umma {

constexpr int kThreads = 128;
constexpr int kBM = 128;
constexpr int kKC = 64;                  // K elements per chunk (4 MMAs of K = 16)
constexpr uint32_t kSpinLimit = 1u << 24;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

// Bounded wait for the mbarrier phase with parity `parity`; false on timeout.
// test_wait never blocks, so kSpinLimit polls bound the wait (~1 s).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  const uint32_t addr = smem_u32(bar);
  for (uint32_t it = 0; it < kSpinLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Shared-memory matrix descriptor: start, leading (K) and stride (M/N) byte
// offsets >> 4, descriptor version 1 (bits 46-47), no swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// The same with the 128-byte swizzle (layout type 2 in bits 61-63): tiles of
// 8 rows x 128 bytes whose 16-byte chunk c of row r sits at chunk c ^ (r mod
// 8), 1024-byte aligned.  K-major: rows are M/N, sbo = 8-row group stride
// (lbo unused).  MN-major: rows are k, 128 bytes = 64 BF16 along M/N; lbo =
// stride between 64-wide M/N blocks, sbo = stride between 8-row k groups.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return smem_desc(saddr, lbo, sbo) | ((uint64_t)2 << 61);
}

// Instruction descriptor, kind::f16: D = F32 (bits 4-5 = 1), A = B = BF16
// (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 in bits
// 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

// Bit 15 of the instruction descriptor: A is MN-major (transposed).
constexpr uint32_t kIdescAMajorMN = 1u << 15;

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 32 lanes x 32 columns of FP32 from TMEM into 32 registers per thread.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

struct Args {
  int M, N, K;
  const float *A;
  int64_t sAb, sAi, sAk;
  const float *B;
  int64_t sBb, sBk, sBn;
  float *C;
  int64_t sCb, sCi, sCn;
  // optional batch indirection: entry b uses A/C of batch ids[b] when
  // a_by_id/c_by_id; entries b >= *count exit (null: identity, all)
  const int *ids = nullptr;
  const int *count = nullptr;
  int a_by_id = 0, c_by_id = 0;
  // optional L2 prefetch of A's next K chunk (a_pf != 0) through a tensor map
  // of A as a 2D view: slices x M rows of K elements (box 64 x 128) when k is
  // contiguous (sAk == 1), slices x K rows of M elements (box 128 x 64) when
  // m is (sAi == 1)
  int a_pf = 0;
  CUtensorMap amap;
};

__device__ __forceinline__ void l2_prefetch_2d(const CUtensorMap *map, int x, int y) {
  asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(x), "r"(y)
               : "memory");
}

// Round x to BF16 (hi) and, for the split form, its remainder (lo).
__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16 &hi, __nv_bfloat16 &lo) {
  hi = __float2bfloat16_rn(x);
  lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// Staging of a (ROWS x KC) chunk of an operand whose element (r, k) is
// P[r * s_r + k * s_k] into the core-matrix layout (hi and, if SPLIT, lo).
// A unit is (row r, k-core c): 8 consecutive k of one row, one 16-byte
// shared store.  Each thread owns ROWS*KC/8/kThreads units.  `load` issues
// all of a chunk's global loads into registers (16-byte vectors when k is
// the contiguous, aligned dimension); `store` converts and writes them.
// Out-of-range elements are 0.
template <int ROWS>
struct Stager {
  static constexpr int KCORES = kKC / 8;
  static constexpr int U = ROWS * KCORES / kThreads;
  static_assert(U * kThreads == ROWS * KCORES, "ROWS must be a multiple of 16");
  float x[U][8];

  __device__ __forceinline__ static void unit(int u, bool k_contig, int &r, int &c) {
    // eight consecutive threads take eight consecutive rows of one core
    // matrix, so their 16-byte shared stores are conflict-free
    if (k_contig) {
      const int rest = u >> 3;
      c = rest % KCORES;
      r = (rest / KCORES) * 8 + (u & 7);
    } else {
      r = u % ROWS;
      c = u / ROWS;
    }
  }

  __device__ __forceinline__ void load(const float *P, int64_t s_r, int64_t s_k, int rows_total,
                                       int row0, int k0, int K, bool vec_ok) {
    const bool k_contig = s_k == 1;
#pragma unroll
    for (int j = 0; j < U; ++j) {
      int r, c;
      unit(threadIdx.x + j * kThreads, k_contig, r, c);
      const int gr = row0 + r, gk = k0 + c * 8;
      if (k_contig && vec_ok && gr < rows_total && gk + 8 <= K) {
        const float4 *q = reinterpret_cast<const float4 *>(P + (int64_t)gr * s_r + gk);
        const float4 v0 = q[0], v1 = q[1];
        x[j][0] = v0.x; x[j][1] = v0.y; x[j][2] = v0.z; x[j][3] = v0.w;
        x[j][4] = v1.x; x[j][5] = v1.y; x[j][6] = v1.z; x[j][7] = v1.w;
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e)
          x[j][e] = (gr < rows_total && gk + e < K)
                        ? P[(int64_t)gr * s_r + (int64_t)(gk + e) * s_k]
                        : 0.f;
      }
    }
  }

  template <int SPLIT>
  __device__ __forceinline__ void store(uint8_t *hi_base, uint8_t *lo_base, bool k_contig) const {
#pragma unroll
    for (int j = 0; j < U; ++j) {
      int r, c;
      unit(threadIdx.x + j * kThreads, k_contig, r, c);
      const int off = ((r >> 3) * KCORES + c) * 128 + (r & 7) * 16;
      __align__(16) __nv_bfloat16 h[8];
      __align__(16) __nv_bfloat16 l[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) split_bf16(x[j][e], h[e], l[e]);
      *reinterpret_cast<uint4 *>(hi_base + off) = *reinterpret_cast<const uint4 *>(h);
      if (SPLIT > 1) *reinterpret_cast<uint4 *>(lo_base + off) = *reinterpret_cast<const uint4 *>(l);
    }
  }
};

// Shared memory of one stage: A hi/lo (kBM x KC), B hi/lo (NP x KC), BF16.
template <int NP, int SPLIT>
struct Layout {
  static constexpr int a_bytes = kBM * kKC * 2;
  static constexpr int b_bytes = NP * kKC * 2;
  static constexpr int stage_bytes = (a_bytes + b_bytes) * (SPLIT > 1 ? 2 : 1);
  static constexpr int total = 2 * stage_bytes;
};

// Resident CTAs per SM the register budget is sized for: the single-pass
// BF16 kernels with N <= 64 stage 41 KB of shared memory, so five fit; a
// limit of four CTAs (<= 128 registers) keeps more loads in flight than the
// unconstrained three.
template <int NP, int SPLIT>
constexpr int min_blocks() { return (SPLIT == 1 && NP <= 64) ? 4 : 1; }

template <int NP, int SPLIT>
__global__ void __launch_bounds__(kThreads, min_blocks<NP, SPLIT>())
    gemm_kernel(const __grid_constant__ Args g, int *err) {
  pdl_wait();
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ uint32_t tmem_base_s;
  using Lay = Layout<NP, SPLIT>;
  constexpr int TMEM_COLS = NP < 32 ? 32 : NP;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * kBM;
  const int n0 = blockIdx.y * NP;          // N tile (N > NP takes several)
  const int64_t b = blockIdx.z;
  if (g.count && b >= *g.count) return;   // block-uniform, before any TMEM use
  const int64_t jb = g.ids ? g.ids[b] : b;
  const float *A = g.A + (g.a_by_id ? jb : b) * g.sAb;
  const float *B = g.B + b * g.sBb;
  float *C = g.C + (g.c_by_id ? jb : b) * g.sCb;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base_s)),
                 "r"((uint32_t)TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_base_s;

  const int nchunks = (g.K + kKC - 1) / kKC;
  // 16-byte loads along k need 16-byte aligned rows
  const bool a_vec = g.sAk == 1 && (g.sAi % 4) == 0 && ((uintptr_t)A % 16) == 0;
  const bool b_vec = g.sBk == 1 && (g.sBn % 4) == 0 && ((uintptr_t)B % 16) == 0;
  constexpr uint32_t idesc = idesc_bf16(kBM, NP);
  constexpr uint32_t LBO = 128, SBO = (kKC / 8) * 128;
  bool ok = true;
  uint32_t issued[2] = {0, 0};
  Stager<kBM> sa;
  Stager<NP> sb;
  const int64_t aslice = g.a_by_id ? jb : b;
#pragma unroll 1
  for (int ci = 0; ci < nchunks; ++ci) {
    const int h = ci & 1;
    if (g.a_pf && threadIdx.x == 0 && ci + 1 < nchunks) {   // warm L2 for the next chunk
      if (g.sAk == 1) l2_prefetch_2d(&g.amap, (ci + 1) * kKC, (int)(aslice * g.M + m0));
      else l2_prefetch_2d(&g.amap, m0, (int)(aslice * g.K + (ci + 1) * kKC));
    }
    sa.load(A, g.sAi, g.sAk, g.M, m0, ci * kKC, g.K, a_vec);
    sb.load(B, g.sBn, g.sBk, g.N, n0, ci * kKC, g.K, b_vec);
    uint8_t *st = smem + h * Lay::stage_bytes;
    uint8_t *a_hi = st, *b_hi = st + Lay::a_bytes;
    uint8_t *a_lo = st + Lay::a_bytes + Lay::b_bytes, *b_lo = a_lo + Lay::a_bytes;
    // the MMAs that read this stage two chunks ago must be done; the wait's
    // outcome is made block-uniform so that no thread skips a barrier
    const bool w = ci >= 2 ? mbar_wait(&bar[h], (issued[h] - 1) & 1) : true;
    if (!__syncthreads_and(w)) { ok = false; break; }
    sa.template store<SPLIT>(a_hi, a_lo, g.sAk == 1);
    sb.template store<SPLIT>(b_hi, b_lo, g.sBk == 1);
    fence_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
      fence_after();
#pragma unroll
      for (int ks = 0; ks < kKC / 16; ++ks) {
        const uint32_t off = ks * 2 * 128;   // two k-cores per MMA (K = 16)
        const uint64_t dah = smem_desc(smem_u32(a_hi) + off, LBO, SBO);
        const uint64_t dbh = smem_desc(smem_u32(b_hi) + off, LBO, SBO);
        mma_bf16(tmem, dah, dbh, idesc, (ci > 0 || ks > 0) ? 1u : 0u);
        if (SPLIT > 1) {
          const uint64_t dal = smem_desc(smem_u32(a_lo) + off, LBO, SBO);
          const uint64_t dbl = smem_desc(smem_u32(b_lo) + off, LBO, SBO);
          mma_bf16(tmem, dah, dbl, idesc, 1u);
          mma_bf16(tmem, dal, dbh, idesc, 1u);
        }
      }
      mma_commit(&bar[h]);
    }
    issued[h] += 1;
  }
  // wait for the last commit of each stage that was used
  bool done = true;
  for (int s = 0; s < 2; ++s)
    if (issued[s] && !mbar_wait(&bar[s], (issued[s] - 1) & 1)) done = false;
  done = __syncthreads_and(done);
  if (!ok || !done) {
    if (threadIdx.x == 0) atomicExch(err, 1);
  } else {
    fence_after();
    const int row = m0 + warp * 32 + lane;
#pragma unroll
    for (int c0 = 0; c0 < NP; c0 += 32) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (row < g.M) {
#pragma unroll
        for (int c = 0; c < 32; ++c)
          if (n0 + c0 + c < g.N) C[(int64_t)row * g.sCi + (int64_t)(n0 + c0 + c) * g.sCn] = v[c];
      }
    }
  }
  pdl_trigger();
  fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)TMEM_COLS));
}

}  // namespace umma
