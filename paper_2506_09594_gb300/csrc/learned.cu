// Learned sketch widths (engine TR_LR_LEARNED) and the rank-predictor MLP.
//
// The paper sizes every randomized product with one fixed rank (Alg. 1) or
// grows the basis until the error indicator falls below a tolerance (Alg. 3);
// it names sketches driven by a learned model only as future work (Sec. 7).
// This engine gives every transformed slice its own sketch width l_j:
//
//   1. features of slice j from the previous slice pass: its kept rank, the
//      width it used, order statistics of its singular values and their
//      position relative to the previous and the current shrink thresholds;
//   2. a ReLU MLP (16 -> 128 -> 128 -> 128 -> 1; FP16 weights, FP32 biases
//      and accumulation) predicts y_j ~ log(1 + rank_j);
//   3. l_j = round_up(round(exp(y_j) - 1) + p, 8), clipped to [8, l_max];
//      slices are grouped by width on the device (a stable counting sort;
//      classes of fewer than a few slices join the next wider one), and
//      every width class runs the randomized slice prox at its width on a
//      side stream, launched for all n slices and sized on the device
//      (blocks past the class count exit), so a pass needs no host
//      synchronisation and can be captured in a graph;
//   4. judge and fallback: a sketch is kept when it meets Alg. 3's stop
//      test (the energy its basis misses, E_j = ||Abar_j||^2 -
//      ||Q_j^T Abar_j||^2, below eps^2 ||Abar_j||^2), or when it saw p
//      directions beyond every singular value the prox keeps (kept rank <=
//      l_j - p), or when it is as wide as the adaptive basis cap; the
//      other slices are recomputed by the plain adaptive method (Alg. 3 per
//      slice).  The first pass of a handle has no history and is the
//      adaptive method on every slice.
//
// Training uses the same MLP kernels: forward with stored activations,
// backward deltas per 32-row tile, weight gradients by a deterministic
// per-parameter reduction over the batch, and an Adam step (Kingma & Ba,
// 2015) on FP32 master parameters.

#include <math.h>
#include <stdint.h>

#include <cuda_fp16.h>

#include "tr_internal.cuh"
#include "tr_rng.cuh"

namespace {

constexpr int kIn = TR_MLP_IN, kH = TR_MLP_HIDDEN, kLayers = TR_MLP_LAYERS;
constexpr int kRows = 32;   // rows per MLP tile
constexpr int kMaxClasses = (TR_MAX_L + 7) / 8;

// Parameter offsets: layer 0 maps kIn -> kH, layers 1..kLayers-1 map kH -> kH,
// the output layer maps kH -> 1; each layer stores W (out x in, row-major)
// then b (out).
__host__ __device__ constexpr int64_t layer_in(int i) { return i == 0 ? kIn : kH; }
__host__ __device__ constexpr int64_t layer_out(int i) { return i == kLayers ? 1 : kH; }
__host__ __device__ constexpr int64_t layer_off(int i) {
  int64_t o = 0;
  for (int k = 0; k < i; ++k) o += layer_out(k) * layer_in(k) + layer_out(k);
  return o;
}
constexpr int64_t kParams = layer_off(kLayers + 1);
static_assert(kParams == 16 * 128 + 128 + 2 * (128 * 128 + 128) + 128 + 1, "parameter count");

// shared memory of the MLP tile kernels: one layer's weights as FP16
// (kH x kH) and two activation tiles
constexpr size_t kMlpSmem = (size_t)kH * kH * sizeof(__half) + 2 * (size_t)kRows * kH * sizeof(float);

// Stage layer i's weights as FP16.  TRANS: Ws[k * out + o] = W[o][k]
// (threads index o); otherwise Ws[o * in + k] (threads index k).
template <bool TRANS>
__device__ void stage_weights(const float *__restrict__ prm, int i, __half *Ws) {
  const float *W = prm + layer_off(i);
  const int in = (int)layer_in(i), out = (int)layer_out(i);
  for (int e = threadIdx.x; e < in * out; e += blockDim.x) {
    const int o = e / in, k = e % in;
    Ws[TRANS ? k * out + o : e] = __float2half_rn(W[e]);
  }
}

// The hidden layers' weights as FP16 in stage_weights<true>'s layout, layer i
// at w16 + i kH kH: converted once per model (tr_set_model), so that the
// inference passes copy them instead of converting them on every call.
__global__ void mlp_pack_kernel(const float *__restrict__ prm, __half *__restrict__ w16) {
  for (int li = 0; li < kLayers; ++li) {
    const float *W = prm + layer_off(li);
    const int in = (int)layer_in(li), out = (int)layer_out(li);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < in * out; e += gridDim.x * blockDim.x) {
      const int o = e / in, k = e % in;
      w16[(int64_t)li * kH * kH + k * out + o] = __float2half_rn(W[e]);
    }
  }
}

// Forward pass of kRows rows.  128 threads: thread o owns hidden unit o.
// STORE keeps the post-ReLU activations H[l] (B x kH) for the backward pass.
// w16 (optional): the packed FP16 hidden weights of prm.
template <bool STORE>
__global__ void __launch_bounds__(kH) mlp_forward_kernel(const float *__restrict__ prm,
                                                         const float *__restrict__ X, int B,
                                                         float *__restrict__ H,
                                                         float *__restrict__ yhat,
                                                         const __half *__restrict__ w16) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __half *Ws = reinterpret_cast<__half *>(smem_raw);
  float *act = reinterpret_cast<float *>(smem_raw + (size_t)kH * kH * sizeof(__half));
  float *nxt = act + kRows * kH;
  const int r0 = blockIdx.x * kRows;
  const int o = threadIdx.x;
  for (int e = threadIdx.x; e < kRows * kIn; e += blockDim.x) {
    const int r = e / kIn;
    act[e] = r0 + r < B ? X[(int64_t)(r0 + r) * kIn + e % kIn] : 0.f;
  }
  for (int li = 0; li < kLayers; ++li) {
    const int in = (int)layer_in(li);
    __syncthreads();
    if (w16) {   // in * kH halves, 16 bytes at a time
      const uint4 *src = reinterpret_cast<const uint4 *>(w16 + (int64_t)li * kH * kH);
      uint4 *dst = reinterpret_cast<uint4 *>(Ws);
      for (int e = threadIdx.x; e < in * kH / 8; e += blockDim.x) dst[e] = src[e];
    } else {
      stage_weights<true>(prm, li, Ws);
    }
    __syncthreads();
    const float bo = prm[layer_off(li) + (int64_t)kH * in + o];
    float acc[kRows];
#pragma unroll
    for (int r = 0; r < kRows; ++r) acc[r] = bo;
    for (int k = 0; k < in; ++k) {
      const float w = __half2float(Ws[k * kH + o]);
#pragma unroll
      for (int r = 0; r < kRows; ++r) acc[r] = fmaf(w, act[r * in + k], acc[r]);
    }
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
      const float v = acc[r] > 0.f ? acc[r] : 0.f;
      nxt[r * kH + o] = v;
      if (STORE && r0 + r < B) H[((int64_t)li * B + r0 + r) * kH + o] = v;
    }
    float *tmp = act;
    act = nxt;
    nxt = tmp;
  }
  __syncthreads();
  // output unit: warp w reduces rows w, w + 4, ...
  const float *Wo = prm + layer_off(kLayers);
  const float wk[4] = {__half2float(__float2half_rn(Wo[threadIdx.x % 32])),
                       __half2float(__float2half_rn(Wo[32 + threadIdx.x % 32])),
                       __half2float(__float2half_rn(Wo[64 + threadIdx.x % 32])),
                       __half2float(__float2half_rn(Wo[96 + threadIdx.x % 32]))};
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  for (int r = warp; r < kRows; r += kH / 32) {
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) s = fmaf(wk[q], act[r * kH + q * 32 + lane], s);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0 && r0 + r < B) yhat[r0 + r] = s + Wo[kH];
  }
}

// Backward deltas of kRows rows.  Loss (1/B) sum_r w_r (yhat_r - y_r)^2 with
// w_r = 1 + under * [yhat_r < y_r].  Writes DY (B), DZ[l] (B x kH) = dLoss /
// d(pre-activation of hidden layer l), and the per-row loss terms.
__global__ void __launch_bounds__(kH) mlp_backward_kernel(const float *__restrict__ prm,
                                                          const float *__restrict__ H,
                                                          const float *__restrict__ yhat,
                                                          const float *__restrict__ y, int B,
                                                          float under, float *__restrict__ DY,
                                                          float *__restrict__ DZ,
                                                          float *__restrict__ loss_rows) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __half *Ws = reinterpret_cast<__half *>(smem_raw);
  float *dz = reinterpret_cast<float *>(smem_raw + (size_t)kH * kH * sizeof(__half));
  float *dzn = dz + kRows * kH;
  __shared__ float dy[kRows];
  const int r0 = blockIdx.x * kRows;
  const int o = threadIdx.x;
  if (threadIdx.x < kRows) {
    const int r = r0 + threadIdx.x;
    float g = 0.f, lr = 0.f;
    if (r < B) {
      const float d = yhat[r] - y[r];
      const float w = 1.f + (yhat[r] < y[r] ? under : 0.f);
      g = 2.f * w * d / (float)B;
      lr = w * d * d / (float)B;
      DY[r] = g;
      loss_rows[r] = lr;
    }
    dy[threadIdx.x] = g;
  }
  __syncthreads();
  {
    const float wo = __half2float(__float2half_rn(prm[layer_off(kLayers) + o]));
    const int li = kLayers - 1;
#pragma unroll 4
    for (int r = 0; r < kRows; ++r) {
      const bool in_b = r0 + r < B;
      const float h = in_b ? H[((int64_t)li * B + r0 + r) * kH + o] : 0.f;
      const float v = h > 0.f ? dy[r] * wo : 0.f;
      dz[r * kH + o] = v;
      if (in_b) DZ[((int64_t)li * B + r0 + r) * kH + o] = v;
    }
  }
  // dz_{l-1}[r][k] = (sum_o dz_l[r][o] W_l[o][k]) * [H_{l-1}[r][k] > 0]; thread = k
  for (int li = kLayers - 1; li >= 1; --li) {
    __syncthreads();
    stage_weights<false>(prm, li, Ws);
    __syncthreads();
    float acc[kRows];
#pragma unroll
    for (int r = 0; r < kRows; ++r) acc[r] = 0.f;
    for (int oo = 0; oo < kH; ++oo) {
      const float w = __half2float(Ws[oo * kH + o]);
#pragma unroll
      for (int r = 0; r < kRows; ++r) acc[r] = fmaf(dz[r * kH + oo], w, acc[r]);
    }
#pragma unroll 4
    for (int r = 0; r < kRows; ++r) {
      const bool in_b = r0 + r < B;
      const float h = in_b ? H[((int64_t)(li - 1) * B + r0 + r) * kH + o] : 0.f;
      const float v = h > 0.f ? acc[r] : 0.f;
      dzn[r * kH + o] = v;
      if (in_b) DZ[((int64_t)(li - 1) * B + r0 + r) * kH + o] = v;
    }
    float *tmp = dz;
    dz = dzn;
    dzn = tmp;
  }
}

// Weight gradients: thread p owns parameter p and sums over the batch in row
// order (deterministic).  Layer l's input is X (l = 0) or H[l-1]; its delta
// is DZ[l] (hidden) or DY (output).
__global__ void mlp_wgrad_kernel(const float *__restrict__ X, const float *__restrict__ H,
                                 const float *__restrict__ DZ, const float *__restrict__ DY,
                                 int B, float *__restrict__ grad) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kParams) return;
  int li = 0;
  while (li < kLayers && p >= layer_off(li + 1)) ++li;
  const int64_t q = p - layer_off(li);
  const int64_t in = layer_in(li), out = layer_out(li);
  const float *dl = li == kLayers ? DY : DZ + (int64_t)li * B * kH;
  const int64_t lds = li == kLayers ? 1 : kH;
  float acc = 0.f;
  if (q < out * in) {
    const int64_t o = q / in, k = q % in;
    const float *src = li == 0 ? X : H + (int64_t)(li - 1) * B * kH;
    const int64_t ldx = li == 0 ? kIn : kH;
    for (int r = 0; r < B; ++r) acc = fmaf(dl[(int64_t)r * lds + o], src[(int64_t)r * ldx + k], acc);
  } else {
    const int64_t o = q - out * in;
    for (int r = 0; r < B; ++r) acc += dl[(int64_t)r * lds + o];
  }
  grad[p] = acc;
}

__global__ void sum_kernel(const float *__restrict__ v, int n, float *__restrict__ out) {
  __shared__ float part[256];
  float s = 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += v[i];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = part[0];
}

// Adam on FP32 master parameters; c1 = 1 / (1 - beta1^t), c2 = 1 / (1 - beta2^t).
__global__ void adam_kernel(float *__restrict__ prm, const float *__restrict__ g,
                            float *__restrict__ m, float *__restrict__ v, int64_t n, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  prm[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
}

// He-uniform weights U(-a, a), a = sqrt(6 / fan_in), zero biases; uniforms
// from Philox4x32-10 with counter (p, 0, 0, 0x4d4c50) and the seed as key.
__global__ void mlp_init_kernel(float *__restrict__ prm, uint32_t k0, uint32_t k1) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kParams) return;
  int li = 0;
  while (li < kLayers && p >= layer_off(li + 1)) ++li;
  const int64_t q = p - layer_off(li);
  if (q >= layer_out(li) * layer_in(li)) {
    prm[p] = 0.f;
    return;
  }
  uint32_t c[4] = {(uint32_t)p, 0u, 0u, 0x4d4c50u};
  trrng::philox4x32_10(c, k0, k1);
  const float u = ((float)(c[0] >> 8) + 0.5f) * (1.0f / 16777216.0f);   // (0, 1)
  const float a = sqrtf(6.0f / (float)layer_in(li));
  prm[p] = (2.f * u - 1.f) * a;
}

// Minibatch: row i of step s is sample philox((i, s, 0, 0x42), seed) mod n.
__global__ void gather_kernel(const float *__restrict__ X, const float *__restrict__ y, int n,
                              int B, uint32_t step, uint32_t k0, uint32_t k1,
                              float *__restrict__ Xb, float *__restrict__ yb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B) return;
  uint32_t c[4] = {(uint32_t)i, step, 0u, 0x42u};
  trrng::philox4x32_10(c, k0, k1);
  const int src = (int)(((uint64_t)c[0] * (uint64_t)n) >> 32);
  for (int k = 0; k < kIn; ++k) Xb[(int64_t)i * kIn + k] = X[(int64_t)src * kIn + k];
  yb[i] = y[src];
}

// ---------------------------------------------------------------- features
// One warp per slice.  With w = width[j] values s_0..s_{w-1} (unsorted) in
// row j of sig, s1 = max s, thresholds thr (current pass) and thr0 (the pass
// that produced s), and c(x) = #{s_i > x}:
//   f0 = log(1 + rank_j) / log(129)       f1 = log(w) / log(129)
//   f2 = clip(log(s1 / thr), -8, 8) / 8   f3 = clip(log(s1 / thr0), -8, 8) / 8
//   f4..f9 = s_(i) / s1 for i in {2, 4, 8, 16, 32, 64} (i-th largest; 0 if i > w)
//   f10, f11, f12 = log(1 + c(thr)), log(1 + c(thr / 2)), log(1 + c(2 thr)), / log(129)
//   f13 = (w - c(thr)) / w                f14 = clip(log(thr / thr0), -1, 1)
//   f15 = clip(t / T, 0, 1)
// A zero s1 gives f2 = f3 = -1 and f4..f9 = 0; a zero threshold counts as
// +infinity in the logarithms' ratios (f2/f3 = 1, f14 = 0).
// Smallest singular value the shrink keeps nonzero (the threshold of the
// features): tau theta for l1 and for MCP with gamma > tau, theta sqrt(gamma
// tau) otherwise.
__device__ __forceinline__ double shrink_threshold_dev(int phi, double theta, double gamma,
                                                       double tau) {
  if (phi == TR_PEN_L1 || gamma > tau) return tau * theta;
  return theta * sqrt(gamma * tau);
}

template <typename T>
__global__ void features_kernel(int n, const T *__restrict__ sig, int ldsig,
                                const int *__restrict__ rank, const int *__restrict__ width,
                                float thr, float thr0, float tfrac, FeatSched fs,
                                float *__restrict__ F) {
  if (fs.d) {   // thresholds and run fraction from the device schedule
    thr = (float)shrink_threshold_dev(fs.phi, fs.theta, fs.gamma, 1.0 / fs.d->mu);
    thr0 = (float)shrink_threshold_dev(fs.phi, fs.theta, fs.gamma, 1.0 / fs.d->mu_prev);
    tfrac = fs.T > 0 ? (float)((double)fs.d->t / (double)fs.T) : 0.f;
  }
  __shared__ float sv[4][TR_MAX_L];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int j = blockIdx.x * 4 + warp;
  if (j >= n) return;
  int w = width[j];
  w = w < 1 ? 1 : (w > TR_MAX_L ? TR_MAX_L : w);
  float *s = sv[warp];
  float mx = 0.f;
  int c_now = 0, c_half = 0, c_two = 0;
  for (int i = lane; i < w; i += 32) {
    float x = (float)sig[(int64_t)j * ldsig + i];
    x = x > 0.f ? x : 0.f;   // also maps NaN to 0
    s[i] = x;
    mx = fmaxf(mx, x);
    c_now += x > thr;
    c_half += x > 0.5f * thr;
    c_two += x > 2.f * thr;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    c_now += __shfl_xor_sync(0xffffffffu, c_now, off);
    c_half += __shfl_xor_sync(0xffffffffu, c_half, off);
    c_two += __shfl_xor_sync(0xffffffffu, c_two, off);
  }
  __syncwarp();
  float *f = F + (int64_t)j * kIn;
  // order statistics by rank counting (ties broken by index)
  for (int i = lane; i < w; i += 32) {
    const float x = s[i];
    int r = 0;
    for (int e = 0; e < w; ++e) r += (s[e] > x) || (s[e] == x && e < i);
    const int pos = r + 1;   // 1-based position in descending order
    if (pos == 2 || pos == 4 || pos == 8 || pos == 16 || pos == 32 || pos == 64) {
      const int slot = 4 + (31 - __clz(pos)) - 1;   // 2 -> 4, 4 -> 5, ..., 64 -> 9
      f[slot] = mx > 0.f ? x / mx : 0.f;
    }
  }
  if (lane == 0) {
    const float L129 = logf(129.f);
    f[0] = log1pf((float)(rank[j] > 0 ? rank[j] : 0)) / L129;
    f[1] = logf((float)w) / L129;
    auto lratio = [&](float a, float b) {
      if (!(a > 0.f)) return -1.f;
      if (!(b > 0.f)) return 1.f;
      return fminf(fmaxf(logf(a / b), -8.f), 8.f) / 8.f;
    };
    f[2] = lratio(mx, thr);
    f[3] = lratio(mx, thr0);
    for (int q = 0; q < 6; ++q)
      if ((2 << q) > w) f[4 + q] = 0.f;
    f[10] = log1pf((float)c_now) / L129;
    f[11] = log1pf((float)c_half) / L129;
    f[12] = log1pf((float)c_two) / L129;
    f[13] = (float)(w - c_now) / (float)w;
    f[14] = (thr > 0.f && thr0 > 0.f) ? fminf(fmaxf(logf(thr / thr0), -1.f), 1.f) : 0.f;
    f[15] = fminf(fmaxf(tfrac, 0.f), 1.f);
  }
}

// ------------------------------------------------------------------- plan
// Width of a prediction: r = round(exp(y) - 1) clipped to [0, lmax],
// l = round_up(r + p, 8) clipped to [min(8, lmax), lmax]; class (l - 1) / 8.
__device__ __forceinline__ int width_of(float y, int p, int lmax) {
  float r;
  if (!(y == y)) r = (float)lmax;
  else r = floorf(expm1f(fminf(fmaxf(y, -20.f), 20.f)) + 0.5f);
  r = fminf(fmaxf(r, 0.f), (float)lmax);
  int l = (((int)r + p + 7) / 8) * 8;
  if (l > lmax) l = lmax;
  const int lo = lmax < 8 ? lmax : 8;
  return l < lo ? lo : l;
}

// One block of 1024 threads: width classes, counts, slice ids stably
// sorted by class (pass 1 counts, pass 2 scatters chunk by chunk with
// per-warp ballots).
__global__ void __launch_bounds__(1024) plan_kernel(int n, const float *__restrict__ yhat, int p,
                                                    int lmax, int *__restrict__ width,
                                                    int *__restrict__ ids,
                                                    int *__restrict__ counts) {
  __shared__ int cnt[kMaxClasses], start[kMaxClasses], wcnt[kMaxClasses][32];
  const int C = (lmax + 7) / 8;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if ((int)threadIdx.x < kMaxClasses) cnt[threadIdx.x] = 0;
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const int l = width_of(yhat[j], p, lmax);
    width[j] = l;
    atomicAdd(&cnt[(l - 1) / 8], 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int c = 0; c < C; ++c) {
      start[c] = acc;
      acc += cnt[c];
      counts[c] = cnt[c];
    }
  }
  __syncthreads();
  for (int base = 0; base < n; base += blockDim.x) {
    const int j = base + threadIdx.x;
    const int c = j < n ? (width[j] - 1) / 8 : -1;
    unsigned mine = 0;
    for (int q = 0; q < C; ++q) {
      const unsigned m = __ballot_sync(0xffffffffu, c == q);
      if (c == q) mine = m;
      if (lane == 0) wcnt[q][warp] = __popc(m);
    }
    __syncthreads();
    if (c >= 0) {
      int off = start[c];
      for (int w2 = 0; w2 < warp; ++w2) off += wcnt[c][w2];
      ids[off + __popc(mine & ((1u << lane) - 1u))] = j;
    }
    __syncthreads();
    if ((int)threadIdx.x < C) {
      int s = 0;
      for (int w2 = 0; w2 < 32; ++w2) s += wcnt[threadIdx.x][w2];
      start[threadIdx.x] += s;
    }
    __syncthreads();
  }
}

// Width groups on the device: walking the classes from narrow to wide, a
// class with fewer than merge_min slices (while a wider non-empty class
// follows) joins the next one.  Group g is launched at the width of its
// widest class c: its slice ids go to gids[c * n ...], its size to
// gcount[c]; classes merged away get gcount 0.  One block.
__global__ void group_kernel(int n, int C, int merge_min, const int *__restrict__ counts,
                             const int *__restrict__ ids, int *__restrict__ gids,
                             int *__restrict__ gcount) {
  __shared__ int src[kMaxClasses], cnt[kMaxClasses];
  if (threadIdx.x == 0) {
    int start = 0, pend = 0, pstart = 0;
    for (int c = 0; c < C; ++c) {
      src[c] = 0;
      cnt[c] = 0;
      const int k = counts[c];
      if (k == 0) continue;
      if (pend == 0) pstart = start;
      pend += k;
      start += k;
      bool later = false;
      for (int c2 = c + 1; c2 < C; ++c2) later = later || counts[c2] > 0;
      if (pend < merge_min && later) continue;
      src[c] = pstart;
      cnt[c] = pend;
      pend = 0;
    }
    for (int c = 0; c < C; ++c) gcount[c] = cnt[c];
  }
  __syncthreads();
  for (int c = 0; c < C; ++c)
    for (int i = threadIdx.x; i < cnt[c]; i += blockDim.x) gids[(int64_t)c * n + i] = ids[src[c] + i];
}

// ||Abar_j||_F^2 per slice: one block per slice, four FP32 partial sums per
// thread (at most a few thousand terms each), folded and reduced in double.
template <typename T>
__global__ void slice_norm2_kernel(int64_t per, const T *__restrict__ A,
                                   double *__restrict__ out) {
  const T *a = A + (int64_t)blockIdx.x * per;
  double acc = 0.0;
  for (int64_t base = 0; base < per; base += (int64_t)blockDim.x * 1024) {
    T p[4] = {T(0), T(0), T(0), T(0)};
    const int64_t end = base + (int64_t)blockDim.x * 1024 < per ? base + (int64_t)blockDim.x * 1024
                                                                  : per;
    int u = 0;
    for (int64_t e = base + threadIdx.x; e < end; e += blockDim.x, u = (u + 1) & 3)
      p[u] = fma(a[e], a[e], p[u]);
    acc += ((double)p[0] + (double)p[1]) + ((double)p[2] + (double)p[3]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ double red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
    out[blockIdx.x] = tot;
  }
}

// The judge of a learned width.  Slice j's sketch (width l_j, kept rank k_j
// after the shrink) is kept when
//   (a) it meets Alg. 3's stop test: the energy its basis misses,
//       E_j = ||Abar_j||^2 - ||B_j||^2 (B_j = Q_j^T Abar_j, whose squared
//       singular values are row j of sig), is below eps^2 ||Abar_j||^2; or
//   (b) it saw p directions beyond every singular value the prox keeps
//       (k_j <= l_j - p, the oversampling of the plain width); or
//   (c) it is at least as wide as the adaptive engine's basis cap;
// otherwise it is listed for the adaptive engine (Alg. 3 per slice).
template <typename T>
__global__ void judge_kernel(int n, const T *__restrict__ sig, int ldsig,
                             const double *__restrict__ anorm2, double eps2,
                             const int *__restrict__ rank, const int *__restrict__ width, int p,
                             int kcap, int *__restrict__ fb_ids, int *__restrict__ fb_count) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const T *s = sig + (int64_t)j * ldsig;
  double cap = 0.0;
  for (int i = 0; i < ldsig; ++i) cap += (double)s[i] * (double)s[i];
  const double a2 = anorm2[j];
  const bool alg3 = !(a2 > 0.0) || a2 - cap < eps2 * a2;
  const bool margin = rank[j] <= width[j] - p;
  const bool wide = width[j] >= kcap;
  if (!(alg3 || margin || wide)) fb_ids[atomicAdd(fb_count, 1)] = j;
}

}  // namespace

int64_t mlp_param_count() { return kParams; }

size_t mlp_workspace_floats(int B) { return (size_t)B * (2 * kLayers * kH + 2); }

cudaError_t launch_mlp_init(float *prm, uint64_t seed, cudaStream_t s) {
  mlp_init_kernel<<<(unsigned)((kParams + 255) / 256), 256, 0, s>>>(
      prm, (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32));
  return cudaGetLastError();
}

size_t mlp_pack_halves() { return (size_t)kLayers * kH * kH; }

cudaError_t launch_mlp_pack(const float *prm, void *w16, cudaStream_t s) {
  mlp_pack_kernel<<<64, 256, 0, s>>>(prm, (__half *)w16);
  return cudaGetLastError();
}

cudaError_t launch_mlp_forward(const float *prm, const float *X, int B, float *yhat, float *H,
                               cudaStream_t s, const void *w16) {
  if (B <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)((B + kRows - 1) / kRows);
  cudaError_t e;
  if (H) {
    if ((e = cudaFuncSetAttribute(mlp_forward_kernel<true>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMlpSmem)) != cudaSuccess)
      return e;
    mlp_forward_kernel<true><<<grid, kH, kMlpSmem, s>>>(prm, X, B, H, yhat,
                                                     (const __half *)w16);
  } else {
    if ((e = cudaFuncSetAttribute(mlp_forward_kernel<false>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMlpSmem)) != cudaSuccess)
      return e;
    mlp_forward_kernel<false><<<grid, kH, kMlpSmem, s>>>(prm, X, B, nullptr, yhat,
                                                      (const __half *)w16);
  }
  return cudaGetLastError();
}

// work: H (kLayers B kH) | DZ (kLayers B kH) | DY (B) | loss rows (B)
cudaError_t launch_mlp_loss_grad(const float *prm, const float *X, const float *y, int B,
                                 float under, float *work, float *yhat, float *grad, float *loss,
                                 cudaStream_t s) {
  if (B <= 0) return cudaErrorInvalidValue;
  float *H = work, *DZ = H + (size_t)kLayers * B * kH, *DY = DZ + (size_t)kLayers * B * kH;
  float *rows = DY + B;
  cudaError_t e;
  if ((e = launch_mlp_forward(prm, X, B, yhat, H, s)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(mlp_backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kMlpSmem)) != cudaSuccess)
    return e;
  mlp_backward_kernel<<<(B + kRows - 1) / kRows, kH, kMlpSmem, s>>>(prm, H, yhat, y, B, under, DY,
                                                                   DZ, rows);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  mlp_wgrad_kernel<<<(unsigned)((kParams + 127) / 128), 128, 0, s>>>(X, H, DZ, DY, B, grad);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (loss) {
    sum_kernel<<<1, 256, 0, s>>>(rows, B, loss);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_mlp_adam(float *prm, const float *g, float *m, float *v, int64_t n, double lr,
                            double b1, double b2, double eps, int step, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const double c1 = 1.0 / (1.0 - pow(b1, step)), c2 = 1.0 / (1.0 - pow(b2, step));
  adam_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(prm, g, m, v, n, (float)lr, (float)b1,
                                                         (float)b2, (float)eps, (float)c1,
                                                         (float)c2);
  return cudaGetLastError();
}

cudaError_t launch_mlp_gather(const float *X, const float *y, int n, int B, int step,
                              uint64_t seed, float *Xb, float *yb, cudaStream_t s) {
  gather_kernel<<<(B + 127) / 128, 128, 0, s>>>(X, y, n, B, (uint32_t)step,
                                               (uint32_t)(seed & 0xffffffffu),
                                               (uint32_t)(seed >> 32), Xb, yb);
  return cudaGetLastError();
}

cudaError_t launch_features(tr_dtype dt, int n, const void *sig, int ldsig, const int *rank,
                            const int *width, double thr, double thr0, double tfrac, float *F,
                            cudaStream_t s, FeatSched fs) {
  if (n <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)((n + 3) / 4);
  if (dt == TR_F64)
    features_kernel<double><<<grid, 128, 0, s>>>(n, (const double *)sig, ldsig, rank, width,
                                                 (float)thr, (float)thr0, (float)tfrac, fs, F);
  else
    features_kernel<float><<<grid, 128, 0, s>>>(n, (const float *)sig, ldsig, rank, width,
                                                (float)thr, (float)thr0, (float)tfrac, fs, F);
  return cudaGetLastError();
}

int plan_classes(int lmax) { return (lmax + 7) / 8; }

cudaError_t launch_plan(int n, const float *yhat, int p, int lmax, int *width, int *ids,
                        int *counts, cudaStream_t s) {
  if (lmax < 1 || lmax > TR_MAX_L) return cudaErrorInvalidValue;
  plan_kernel<<<1, 1024, 0, s>>>(n, yhat, p, lmax, width, ids, counts);
  return cudaGetLastError();
}

// Panel columns the device-planned pass reserves: every width class owns a
// region able to hold all n slices at its width.
int learned_panel_cols(int lmax) {
  int cols = 0;
  for (int c = 0; c < plan_classes(lmax); ++c) cols += 8 * (c + 1) < lmax ? 8 * (c + 1) : lmax;
  return cols;
}

cudaError_t launch_slice_learned(tr_dtype dt, const SliceWork &w, LearnedWork &lw,
                                 const void *Abar, void *Gbar, const ShrinkScalars &sh,
                                 double thr, int t, int T, FeatSched fs, cudaStream_t s,
                                 uint64_t *launches) {
  const int n = w.n, lmax = lw.lmax, p = lw.p;
  const size_t esz = dt == TR_F64 ? 8 : 4;
  SliceWork base = w;
  base.l = lmax;
  base.ldsig = lmax;
  base.width = lw.width;
  base.sel = SliceSel{};
  cudaError_t e;
  const uint64_t adapt_launches = 4 * (uint64_t)(lw.aw.kcap / lw.aw.b) + 3;
  if (!lw.have_hist) {
    // no previous pass: the plain adaptive method on every slice
    if ((e = cudaMemsetAsync(lw.fb_count, 0, sizeof(int), s)) != cudaSuccess) return e;
    SliceWork aw0 = base;
    aw0.sel.ids = lw.iota;
    if ((e = launch_slice_adaptive(dt, aw0, lw.aw, Abar, Gbar, sh, t, s)) != cudaSuccess) return e;
    *launches += adapt_launches;
    lw.have_hist = true;
    lw.thr_prev = thr;
    return cudaSuccess;
  }
  // 1-3: features of the previous pass, predicted log-ranks, width plan and
  // groups, all on the device (no host synchronisation: the pass can be
  // captured in a graph)
  const double tfrac = T > 0 ? (double)t / (double)T : 0.0;
  if ((e = launch_features(dt, n, w.sig, lmax, w.rank, lw.width, thr, lw.thr_prev, tfrac, lw.feat,
                           s, fs)) != cudaSuccess)
    return e;
  if ((e = launch_mlp_forward(lw.params, lw.feat, n, lw.pred, nullptr, s, lw.w16)) != cudaSuccess)
    return e;
  if ((e = launch_plan(n, lw.pred, p, lmax, lw.width, lw.ids, lw.counts, s)) != cudaSuccess) return e;
  const int C = plan_classes(lmax);
  group_kernel<<<1, 256, 0, s>>>(n, C, lw.merge_min, lw.counts, lw.ids, lw.gids, lw.gcount);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // ||Abar_j||^2 for the judge
  if (dt == TR_F64)
    slice_norm2_kernel<double><<<n, 256, 0, s>>>((int64_t)w.n1 * w.n2, (const double *)Abar,
                                                 lw.anorm2);
  else
    slice_norm2_kernel<float><<<n, 256, 0, s>>>((int64_t)w.n1 * w.n2, (const float *)Abar,
                                                lw.anorm2);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  *launches += 5;
  // every class on a side stream, sized on the device (blocks past the
  // class count exit at once), panels in the class's own region
  if ((e = cudaEventRecord(lw.fork, s)) != cudaSuccess) return e;
  const int nstreams = C < TR_LEARNED_STREAMS ? C : TR_LEARNED_STREAMS;
  for (int i = 0; i < nstreams; ++i)
    if ((e = cudaStreamWaitEvent(lw.aux[i], lw.fork, 0)) != cudaSuccess) return e;
  size_t o_om = 0, o_p1 = 0, o_p2 = 0;
  for (int c = 0; c < C; ++c) {
    SliceWork gw = base;
    gw.l = 8 * (c + 1) < lmax ? 8 * (c + 1) : lmax;
    gw.sel.ids = lw.gids + (size_t)c * n;
    gw.sel.count = lw.gcount + c;
    gw.Om = (char *)w.Om + o_om * esz;
    gw.P1 = (char *)w.P1 + o_p1 * esz;
    gw.P2 = (char *)w.P2 + o_p2 * esz;
    o_om += (size_t)n * w.n2 * gw.l;
    o_p1 += (size_t)n * w.n1 * gw.l;
    o_p2 += (size_t)n * w.n2 * gw.l;
    if ((e = launch_slice_rsvd(dt, gw, Abar, Gbar, sh, t, lw.aux[c % TR_LEARNED_STREAMS])) !=
        cudaSuccess)
      return e;
    *launches += 7 + 4 * (uint64_t)w.q;
  }
  for (int i = 0; i < nstreams; ++i) {
    if ((e = cudaEventRecord(lw.join[i], lw.aux[i])) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(s, lw.join[i], 0)) != cudaSuccess) return e;
  }
  // 4: Alg. 3's judge, and the adaptive engine on the slices it rejects
  // (sized on the device)
  if ((e = cudaMemsetAsync(lw.fb_count, 0, sizeof(int), s)) != cudaSuccess) return e;
  const double eps2 = lw.aw.eps * lw.aw.eps;
  if (dt == TR_F64)
    judge_kernel<double><<<(n + 255) / 256, 256, 0, s>>>(n, (const double *)w.sig, lmax,
                                                        lw.anorm2, eps2, w.rank, lw.width, p,
                                                        lw.aw.kcap, lw.fb_ids, lw.fb_count);
  else
    judge_kernel<float><<<(n + 255) / 256, 256, 0, s>>>(n, (const float *)w.sig, lmax, lw.anorm2,
                                                       eps2, w.rank, lw.width, p, lw.aw.kcap,
                                                       lw.fb_ids, lw.fb_count);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  SliceWork fw = base;
  fw.sel.ids = lw.fb_ids;
  fw.sel.count = lw.fb_count;
  if ((e = launch_slice_adaptive(dt, fw, lw.aw, Abar, Gbar, sh, t, s)) != cudaSuccess) return e;
  *launches += 1 + adapt_launches;
  lw.thr_prev = thr;
  return cudaSuccess;
}
