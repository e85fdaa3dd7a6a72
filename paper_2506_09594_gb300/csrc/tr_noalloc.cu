// tr_slice_prox_noalloc: the slice pass (per-slice randomized prox of a
// transformed tensor) for callers that must not allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is off limits -- a host
// thread on a latency-critical loop (cudaMalloc/cudaFree synchronise the
// device and stall every stream), a plugin living inside another
// framework's memory pool (that framework owns all device memory and
// forbids private allocations), or a caller that builds its work once and
// must not touch the allocator afterwards.  Such callers can still hand in
// their input and output buffers; the scratch the slice pass needs (the
// Gaussian sketches, two panels, singular values and ranks) comes from a
// fixed array compiled into this library instead.
//
// The array is a file-scope __device__ buffer of kNoAllocScratchBytes: every
// GPU that loads this library keeps it until the process exits.  All calls
// share it and it keeps whatever the previous call left; nothing in it has
// to start at zero, because every entry is written before it is read.  Two
// calls whose work overlaps on the GPU (different streams, or different
// host threads without ordering) race on it.

#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include "tr_internal.cuh"

namespace {

constexpr size_t kNoAllocScratchBytes = 16u << 20;   // 16 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Copy a message into the caller's buffer (if any) and return `st`.
tr_status report(char *buf, size_t len, tr_status st, const char *fmt, ...) {
  if (buf && len) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, len, fmt, ap);
    va_end(ap);
  }
  return st;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

// Device address of the static scratch array on the current device.  It is
// looked up on every call (cheap next to the slice pass): after a device
// reset the module is loaded again and the array may sit elsewhere.  The
// first call on a device also loads the module there, so that call should
// come before any stream capture.
static tr_status noalloc_scratch(void **out, char *err, size_t err_len) {
  void *p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p)
    return report(err, err_len, TR_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
  *out = p;
  return TR_OK;
}

extern "C" tr_status tr_slice_prox_noalloc(tr_dtype dtype, int n, int n1, int n2,
                                           const void *Abar, void *Gbar, int l, int q,
                                           tr_penalty phi, double theta, double gamma,
                                           double tau, uint64_t seed, int t,
                                           void *cuda_stream, char *err, size_t err_len) {
  if (err && err_len) err[0] = 0;
  if (dtype != TR_F32 && dtype != TR_F64) return report(err, err_len, TR_EINVAL, "bad dtype");
  if (n < 1 || n1 < 1 || n2 < 1 || l < 1 || q < 0 || t < 0 || !(tau >= 0))
    return report(err, err_len, TR_EINVAL, "need n, n1, n2, l >= 1, q, t >= 0, tau >= 0");
  if (!Abar || !Gbar || Abar == Gbar)
    return report(err, err_len, TR_EINVAL, "Abar and Gbar must be distinct device pointers");
  if (phi != TR_PEN_L1 && phi != TR_PEN_MCP) return report(err, err_len, TR_EINVAL, "bad penalty");
  if (n > 65535) return report(err, err_len, TR_EUNSUPPORTED, "at most 65535 slices per call");
  if (l > n1) l = n1;
  if (l > n2) l = n2;
  if (l > TR_MAX_L || !slice_smem_limit_ok(dtype, n1, n2, l))
    return report(err, err_len, TR_EUNSUPPORTED, "slice panels exceed shared memory");
  const size_t esz = dtype == TR_F64 ? 8 : 4;
  const size_t b_om = align256((size_t)n * n2 * l * esz);
  const size_t b_p1 = align256((size_t)n * n1 * l * esz);
  const size_t b_p2 = align256((size_t)n * n2 * l * esz);
  const size_t b_sig = align256((size_t)n * l * esz);
  const size_t b_rank = align256((size_t)n * sizeof(int));
  const size_t need = b_om + b_p1 + b_p2 + b_sig + b_rank;
  if (need > kNoAllocScratchBytes)
    return report(err, err_len, TR_EUNSUPPORTED,
                  "scratch for %d slices of %dx%d with sketch width %d is %zu bytes; the fixed "
                  "array holds %zu",
                  n, n1, n2, l, need, kNoAllocScratchBytes);
  void *base = nullptr;
  const tr_status st = noalloc_scratch(&base, err, err_len);
  if (st != TR_OK) return st;
  unsigned char *p = static_cast<unsigned char *>(base);
  SliceWork w{};
  w.n = n;
  w.n1 = n1;
  w.n2 = n2;
  w.l = l;
  w.q = q;
  w.seed = seed;
  w.Om = p;
  w.P1 = p + b_om;
  w.P2 = p + b_om + b_p1;
  w.sig = p + b_om + b_p1 + b_p2;
  w.rank = reinterpret_cast<int *>(p + b_om + b_p1 + b_p2 + b_sig);
  ShrinkScalars sh{tau, (int)phi, theta, gamma};
  const cudaError_t e =
      launch_slice_rsvd(dtype, w, Abar, Gbar, sh, t, static_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess)
    return report(err, err_len, TR_ECUDA, "slice pass launch: %s", cudaGetErrorString(e));
  return TR_OK;
}
