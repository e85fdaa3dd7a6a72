// Fixed-accuracy engine: Alg. 3 (block Lanczos bidiagonalisation with
// one-sided reorthogonalisation, defl-QR of Alg. 2 and Gaussian refill)
// restated for one transformed face slice, batched over all slices.
// Included inside the slice-pass translation unit's anonymous namespace.
//
// Per slice j (A = Abar^<j>, n1 x n2), block size b, cap kcap (a multiple of
// b), starting from V_1 = qr(G), G Gaussian (Philox stream 1 + 2 * draw):
//   [U_i, R_i]        = defl-QR(A V_i - U_{i-1} L_i, delta)      E -= ||R_i||^2
//   V'                = A^T U_i - V_i R_i^T
//   V'               -= Vcat Vcat^T V'         (one-sided reorthogonalisation)
//   [V_{i+1}, L^T, s] = defl-QR(V', delta)                        E -= ||L||^2
//   if s < b: refill with qr(G' - Vcat Vcat^T G'), G' Gaussian (n2 x (b - s))
//   stop when E < eps^2 ||A||_F^2, the cap is reached or nothing is left.
// Blocks have a fixed width b in the workspace (deflated columns are zero),
// so every slice's products have the same shape and run as one batched
// GEMM; a slice that has stopped skips its per-slice kernels.  With a slice
// selection (SliceSel) batch entry e works on slice ids[e]: the transformed
// slice, the Philox counters and the slice statistics are the slice's, the
// panels and the loop state (E, norms, flags, counts) the entry's.
//
// defl-QR: Householder QR with column pivoting (largest remaining column
// norm first); s = number of pivots whose norm is at least delta; R = Rt(1:s,
// :) P^T; Q = first s columns (the rest zero).

template <typename T>
struct AdaptPtrs {
  T *Ucat;        // n x (n1 x kcap), column-major blocks of width b
  T *Vcat;        // n x (n2 x (kcap + b))
  T *X;           // n x (max(n1, n2) x b): GEMM output scratch
  T *Lm, *Rm;     // n x (b x b), column-major
  double *E, *nrm2;
  int *active, *kept, *draws;
};

// Householder QR with column pivoting of the m x bb panel P (shared memory,
// column-major, leading dim ld) by the whole block; stops at the first pivot
// whose remaining column norm is below delta.  Returns s (block-uniform);
// reflectors below the diagonal, tau[k], perm[k] = original column of pivot k.
template <typename T>
__device__ int block_pivoted_qr(T *P, int m, int bb, int ld, T *tau, int *perm, T *cn,
                                int *pick, T delta) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
  for (int c = tid; c < bb; c += blockDim.x) perm[c] = c;
  __syncthreads();
  int s = 0;
  const int kmax = bb < m ? bb : m;
  for (int k = 0; k < kmax; ++k) {
    for (int c = k + warp; c < bb; c += nw) {
      T ss = T(0);
      for (int i = k + lane; i < m; i += 32) ss = fma(P[(size_t)c * ld + i], P[(size_t)c * ld + i], ss);
      ss = warp_sum(ss);
      if (lane == 0) cn[c] = ss;
    }
    __syncthreads();
    if (tid == 0) {
      int p = k;
      T best = cn[k];
      for (int c = k + 1; c < bb; ++c)
        if (cn[c] > best) { best = cn[c]; p = c; }
      *pick = (best < delta * delta || !(best > T(0))) ? -1 : p;
    }
    __syncthreads();
    const int p = *pick;
    if (p < 0) break;
    if (p != k) {
      for (int i = tid; i < m; i += blockDim.x) {
        const T a = P[(size_t)k * ld + i];
        P[(size_t)k * ld + i] = P[(size_t)p * ld + i];
        P[(size_t)p * ld + i] = a;
      }
      if (tid == 0) {
        const int t0 = perm[k];
        perm[k] = perm[p];
        perm[p] = t0;
      }
    }
    __syncthreads();
    if (warp == 0) {
      T *col = P + (size_t)k * ld;
      T ss = T(0);
      for (int i = k + 1 + lane; i < m; i += 32) ss = fma(col[i], col[i], ss);
      const T x0 = col[k];
      ss = warp_sum(ss);
      T beta = x0, tk = T(0), scale = T(0);
      if (ss > T(0)) {
        const T nrm = sqrt(fma(x0, x0, ss));
        beta = x0 >= T(0) ? -nrm : nrm;
        tk = (beta - x0) / beta;
        scale = T(1) / (x0 - beta);
      }
      for (int i = k + 1 + lane; i < m; i += 32) col[i] *= scale;
      if (lane == 0) {
        col[k] = beta;
        tau[k] = tk;
      }
    }
    __syncthreads();
    const T tk = tau[k];
    const T *v = P + (size_t)k * ld;
    for (int c = k + 1 + warp; c < bb; c += nw) {
      T *col = P + (size_t)c * ld;
      const T ck = col[k];
      T sum = T(0);
      for (int i = k + 1 + lane; i < m; i += 32) sum = fma(v[i], col[i], sum);
      sum = warp_sum(sum) + ck;
      const T w = tk * sum;
      for (int i = k + 1 + lane; i < m; i += 32) col[i] = fma(-w, v[i], col[i]);
      if (lane == 0) col[k] = ck - w;
    }
    __syncthreads();
    s = k + 1;
  }
  return s;
}

// Q = H_0 ... H_{s-1} [I_s; 0] into Qo (m x bb, column-major, ld m); columns
// s..bb-1 of Qo are zero.  Reflectors are read from P (not modified).
template <typename T>
__device__ void block_form_q_cols(const T *P, int m, int bb, int ld, const T *tau, int s, T *Qo) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
  for (int e = tid; e < m * bb; e += blockDim.x) {
    const int i = e % m, c = e / m;
    Qo[(size_t)c * m + i] = (c < s && i == c) ? T(1) : T(0);
  }
  __syncthreads();
  for (int k = s - 1; k >= 0; --k) {
    const T tk = tau[k];
    const T *v = P + (size_t)k * ld;
    for (int c = k + warp; c < s; c += nw) {
      T *col = Qo + (size_t)c * m;
      const T ck = col[k];
      T sum = T(0);
      for (int i = k + 1 + lane; i < m; i += 32) sum = fma(v[i], col[i], sum);
      sum = warp_sum(sum) + ck;
      const T w = tk * sum;
      for (int i = k + 1 + lane; i < m; i += 32) col[i] = fma(-w, v[i], col[i]);
      if (lane == 0) col[k] = ck - w;
    }
    __syncthreads();
  }
}

// Gaussian block G (rows x cols, column-major) of draw `draw` for slice j
// at iteration t: Philox counter (m/4, j, t, 1 + 2 draw), element m = c*rows + r.
template <typename T>
__device__ void gaussian_block_smem(T *G, int rows, int cols, uint32_t k0, uint32_t k1, uint32_t j,
                                    uint32_t t, uint32_t draw) {
  const int total = rows * cols;
  for (int g = threadIdx.x; g * 4 < total; g += blockDim.x) {
    uint32_t c[4] = {(uint32_t)g, j, t, 1u + 2u * draw};
    trrng::philox4x32_10(c, k0, k1);
    T z[4];
    trrng::box_muller(c[0], c[1], z[0], z[1]);
    trrng::box_muller(c[2], c[3], z[2], z[3]);
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (4 * g + i < total) G[4 * g + i] = z[i];
  }
}

// Subtract from the panel P (m x cols, ld m) its projection onto the columns
// of the blocks V[0 .. nblk) (global, m x b each) and the first `extra` columns
// of Xs (shared, m x ?, ld m): P -= W W^T P with all coefficients computed
// from the unmodified P (classical Gram-Schmidt, as Vcat Vcat^T V').
template <typename T>
__device__ void block_project_out(T *P, int m, int cols, const T *V, int nblk, int b,
                                  const T *Xs, int extra, T *coef) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
  const int nv = nblk * b + extra;
  for (int e = warp; e < nv * cols; e += nw) {
    const int q = e % nv, c = e / nv;
    const T *w = q < nblk * b ? V + (size_t)q * m : Xs + (size_t)(q - nblk * b) * m;
    T sum = T(0);
    for (int i = lane; i < m; i += 32) sum = fma(w[i], P[(size_t)c * m + i], sum);
    sum = warp_sum(sum);
    if (lane == 0) coef[q + (size_t)c * nv] = sum;
  }
  __syncthreads();
  for (int e = tid; e < m * cols; e += blockDim.x) {
    const int i = e % m, c = e / m;
    T acc = P[(size_t)c * m + i];
    for (int q = 0; q < nv; ++q) {
      const T *w = q < nblk * b ? V + (size_t)q * m : Xs + (size_t)(q - nblk * b) * m;
      acc = fma(-w[i], coef[q + (size_t)c * nv], acc);
    }
    P[(size_t)c * m + i] = acc;
  }
  __syncthreads();
}

template <typename T>
__device__ T block_sum(T v, T *red) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  T tot = T(0);
  for (int w = 0; w < nw; ++w) tot += red[w];
  __syncthreads();
  return tot;
}

// Shared memory of the per-slice adaptive kernels: two m x b panels, the
// projection coefficients ((kcap + b) x b) and small vectors.
template <typename T>
size_t adapt_smem(int m, int b, int kcap) {
  return sizeof(T) * (2 * (size_t)m * b + (size_t)(kcap + 2 * b) * b + 4 * (size_t)b + 64) +
         sizeof(int) * (size_t)(b + 4);
}

// Start: ||A||^2, E, flags, V_1 = qr(G) into Vcat block 0.
template <typename T>
__global__ void adapt_init_kernel(int n1, int n2, int b, int kcap, const T *__restrict__ Abar,
                                  AdaptPtrs<T> w, uint32_t k0, uint32_t k1, uint32_t t_host,
                                  const int *dt, SliceSel sel) {
  const uint32_t t = dt ? (uint32_t)*dt : t_host;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *P = reinterpret_cast<T *>(smem_raw);
  T *Q = P + (size_t)n2 * b;
  T *tau = Q + (size_t)n2 * b;
  T *cn = tau + b;
  T *red = cn + b;
  int *perm = reinterpret_cast<int *>(red + 64);
  int *pick = perm + b;
  const int e0 = blockIdx.x;   // batch entry
  if (sel.count && e0 >= *sel.count) return;
  const int j = sel.ids ? sel.ids[e0] : e0;   // slice id
  const T *A = Abar + (int64_t)j * n1 * n2;
  double part = 0.0;
  for (int64_t e = threadIdx.x; e < (int64_t)n1 * n2; e += blockDim.x) part += (double)A[e] * A[e];
  // block reduction in double through the T scratch is lossy for float: use
  // a dedicated double reduction
  __shared__ double dred[32];
  {
    double v = part;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) dred[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double tot = 0.0;
      for (int q = 0; q < (int)(blockDim.x >> 5); ++q) tot += dred[q];
      w.nrm2[e0] = tot;
      w.E[e0] = tot;
      w.active[e0] = tot > 0.0;
      w.kept[e0] = 0;
      w.draws[e0] = 1;
    }
  }
  gaussian_block_smem(P, n2, b, k0, k1, (uint32_t)j, t, 0u);
  __syncthreads();
  const int s = block_pivoted_qr(P, n2, b, n2, tau, perm, cn, pick, T(0));
  block_form_q_cols(P, n2, b, n2, tau, s, Q);
  T *V0 = w.Vcat + (int64_t)e0 * n2 * (kcap + b);
  for (int e = threadIdx.x; e < n2 * b; e += blockDim.x) V0[e] = Q[e];
  (void)red;
}

// U side of iteration i: X = A V_i (already in w.X) minus U_{i-1} L_i,
// defl-QR, U_i into Ucat block i, R_i (original column order) into Rm.
template <typename T>
__global__ void adapt_u_kernel(int i, int n1, int b, int kcap, int64_t xs, AdaptPtrs<T> w,
                               double delta_rel, SliceSel sel) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int j = blockIdx.x;   // batch entry (the slice itself is not read here)
  if (sel.count && j >= *sel.count) return;
  if (!w.active[j]) return;
  T *P = reinterpret_cast<T *>(smem_raw);
  T *Q = P + (size_t)n1 * b;
  T *coef = Q + (size_t)n1 * b;
  T *tau = coef + (size_t)(kcap + 2 * b) * b;
  T *cn = tau + b;
  T *red = cn + b;
  int *perm = reinterpret_cast<int *>(red + 64);
  int *pick = perm + b;
  const T *Xj = w.X + (int64_t)j * xs;   // A V_i, n1 x b, leading dim n1
  for (int e = threadIdx.x; e < n1 * b; e += blockDim.x) P[e] = Xj[e];
  T *Uc = w.Ucat + (int64_t)j * n1 * kcap;
  T *L = w.Lm + (int64_t)j * b * b;
  __syncthreads();
  if (i > 0) {
    const T *Up = Uc + (size_t)(i - 1) * b * n1;
    for (int e = threadIdx.x; e < n1 * b; e += blockDim.x) {
      const int r = e % n1, c = e / n1;
      T acc = P[e];
      for (int k = 0; k < b; ++k) acc = fma(-Up[(size_t)k * n1 + r], L[k + (size_t)c * b], acc);
      P[e] = acc;
    }
    __syncthreads();
  }
  const T delta = T(delta_rel * sqrt(w.nrm2[j]));
  const int s = block_pivoted_qr(P, n1, b, n1, tau, perm, cn, pick, delta);
  // R = Rt(1:s, :) P^T, energy removed from E
  T *R = w.Rm + (int64_t)j * b * b;
  T part = T(0);
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    const int r = e % b, c = e / b;                 // Rt(r, c)
    const T v = (r < s && r <= c) ? P[(size_t)c * n1 + r] : T(0);
    R[r + (size_t)perm[c] * b] = v;
    part = fma(v, v, part);
  }
  const T tot = block_sum(part, red);
  block_form_q_cols(P, n1, b, n1, tau, s, Q);
  T *Ui = Uc + (size_t)i * b * n1;
  for (int e = threadIdx.x; e < n1 * b; e += blockDim.x) Ui[e] = Q[e];
  if (threadIdx.x == 0) {
    w.E[j] -= (double)tot;
    w.kept[j] += s;
  }
}

// V side of iteration i: V' = A^T U_i (in w.X) - V_i R_i^T, reorthogonalised
// against Vcat, defl-QR -> V_{i+1}, L_{i+1}; refill; stopping test.
template <typename T>
__global__ void adapt_v_kernel(int i, int n2, int b, int kcap, int64_t xs, AdaptPtrs<T> w,
                               double delta_rel, double eps, uint32_t k0, uint32_t k1,
                               uint32_t t_host, const int *dt, SliceSel sel) {
  const uint32_t t = dt ? (uint32_t)*dt : t_host;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int j = blockIdx.x;   // batch entry; the Philox draws use the slice id
  if (sel.count && j >= *sel.count) return;
  const uint32_t slice = sel.ids ? (uint32_t)sel.ids[j] : (uint32_t)j;
  if (!w.active[j]) return;
  T *P = reinterpret_cast<T *>(smem_raw);
  T *Q = P + (size_t)n2 * b;
  T *coef = Q + (size_t)n2 * b;
  T *tau = coef + (size_t)(kcap + 2 * b) * b;
  T *cn = tau + b;
  T *red = cn + b;
  int *perm = reinterpret_cast<int *>(red + 64);
  int *pick = perm + b;
  const T *Xj = w.X + (int64_t)j * xs;   // A^T U_i, n2 x b, leading dim n2
  T *Vc = w.Vcat + (int64_t)j * n2 * (kcap + b);
  const T *Vi = Vc + (size_t)i * b * n2;
  const T *R = w.Rm + (int64_t)j * b * b;
  for (int e = threadIdx.x; e < n2 * b; e += blockDim.x) {
    const int r = e % n2, c = e / n2;
    T acc = Xj[e];
    for (int k = 0; k < b; ++k) acc = fma(-Vi[(size_t)k * n2 + r], R[c + (size_t)k * b], acc);
    P[e] = acc;
  }
  __syncthreads();
  block_project_out(P, n2, b, Vc, i + 1, b, (const T *)nullptr, 0, coef);
  const T delta = T(delta_rel * sqrt(w.nrm2[j]));
  const int s = block_pivoted_qr(P, n2, b, n2, tau, perm, cn, pick, delta);
  // L^T = Rt(1:s, :) P^T  (s x b);  L = (L^T)^T is b x s, stored b x b
  T *L = w.Lm + (int64_t)j * b * b;
  T part = T(0);
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    const int r = e % b, c = e / b;                 // Rt(r, c)
    const T v = (r < s && r <= c) ? P[(size_t)c * n2 + r] : T(0);
    L[perm[c] + (size_t)r * b] = v;                 // L(perm[c], r) = Lt(r, perm[c])
    part = fma(v, v, part);
  }
  const T tot = block_sum(part, red);
  block_form_q_cols(P, n2, b, n2, tau, s, Q);
  // refill the deflated columns with orthogonalised Gaussian vectors
  const int have = (i + 1) * b + s;                 // columns of Vcat after V_{i+1}'s kept part
  int nref = b - s;
  if (nref > n2 - have) nref = n2 - have;
  if (nref < 0) nref = 0;
  if (nref > 0) {
    T *G = P;                                        // the factored panel is no longer needed
    gaussian_block_smem(G, n2, nref, k0, k1, slice, t, (uint32_t)w.draws[j]);
    __syncthreads();
    block_project_out(G, n2, nref, Vc, i + 1, b, Q, s, coef);
    const int s2 = block_pivoted_qr(G, n2, nref, n2, tau, perm, cn, pick, T(0));
    // append the orthonormal refill after the kept columns of Q
    T *Qr = Q + (size_t)s * n2;
    block_form_q_cols(G, n2, s2, n2, tau, s2, Qr);
    __syncthreads();
  }
  T *Vn = Vc + (size_t)(i + 1) * b * n2;
  for (int e = threadIdx.x; e < n2 * b; e += blockDim.x) Vn[e] = Q[e];
  if (threadIdx.x == 0) {
    if (nref > 0) w.draws[j] += 1;
    const double E = w.E[j] - (double)tot;
    w.E[j] = E;
    const bool done = E < eps * eps * w.nrm2[j] || w.kept[j] >= kcap || (i + 2) * b > kcap ||
                      (s + nref) == 0;
    if (done) w.active[j] = 0;
  }
}

// Width of a selected slice after an adaptive pass: its basis size.
__global__ void adapt_width_kernel(const int *__restrict__ ids, const int *__restrict__ count,
                                   const int *__restrict__ kept, int *__restrict__ width, int n) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n || (count && e >= *count)) return;
  width[ids[e]] = kept[e];
}
