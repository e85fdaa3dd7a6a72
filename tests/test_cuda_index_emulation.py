"""CPU emulation of the index arithmetic and launch sequences of the
gradient-domain and one-bit CUDA code (csrc/grad_kernels.cu, csrc/ctv.cu,
csrc/onebit.cu, csrc/ew_kernels.cuh), checked against the FP64 oracle.

Each kernel is restated as one numpy operation on flat buffers, with the
kernels' own formulas:
* flat stride of mode k: S_1 = n2, S_2 = 1, S_k = n1 n2 n3 ... n_{k-1};
* periodic neighbours f +- S_k with the wrap at i_k = (f / S_k) mod n_k;
* the strided batched GEMM C[o][x][y] = sum_b A[o][x][b] B[o][b][y] with the
  operand strides the host code passes for each mode (left product for
  k != 2, right product for the contiguous mode 2);
* the ping-pong of the Hartley solve between the scratch and the output;
* the fused stencils and their order in the two ADMM steps.
* for the fixed-accuracy Tucker loop still to be built on the GPU: A V and
  A^T U on a mode unfolding as per-slice strided GEMMs (plus a sum over
  slices for A V), without forming the unfolding.
Numpy's fancy indexing raises on any out-of-range index, so these runs also
show every access stays inside its buffer.  This checks the arithmetic the
kernels encode, not the compiled kernels: their parity tests against the
oracle are tests/test_gpu_grad.py, test_gpu_ctv.py and test_gpu_onebit.py.
"""

import numpy as np
import pytest

from oracle import admm, ctv, onebit, prox, svt, transform
from paper_2506_09594_gb300 import synth


def mode_stride(dims, k):
    if k == 1:
        return dims[1]
    if k == 2:
        return 1
    s = dims[0] * dims[1]
    for m in range(3, k):
        s *= dims[m - 1]
    return s


def fwd(N, S, nk):
    f = np.arange(N)
    return np.where((f // S) % nk == nk - 1, f - (nk - 1) * S, f + S)


def bwd(N, S, nk):
    f = np.arange(N)
    return np.where((f // S) % nk == 0, f + (nk - 1) * S, f - S)


def gemm(A, ao, ax, ab, B, bo, bb, by, C, co, cx, cy, X, Y, K, batch):
    o = np.arange(batch)[:, None, None, None]
    x = np.arange(X)[None, :, None, None]
    y = np.arange(Y)[None, None, :, None]
    b = np.arange(K)[None, None, None, :]
    vals = (A[o * ao + x * ax + b * ab] * B[o * bo + b * bb + y * by]).sum(-1)
    oo, xx, yy = np.meshgrid(np.arange(batch), np.arange(X), np.arange(Y), indexing="ij")
    C[oo * co + xx * cx + yy * cy] = vals


def hartley(n):
    a = 2 * np.pi * (np.outer(np.arange(n), np.arange(n)) % n) / n
    return (np.cos(a) + np.sin(a)) / np.sqrt(n)


def mode_product(src, dst, dims, k):
    N, m, S = src.size, dims[k - 1], mode_stride(dims, k)
    H = hartley(m).ravel()
    if k == 2:
        gemm(src, 0, m, 1, H, 0, m, 1, dst, 0, m, 1, N // m, m, m, 1)
    else:
        gemm(H, 0, m, 1, src, m * S, S, 1, dst, m * S, S, 1, m, S, m, N // (m * S))


def gradient_solve(rhs, dims, modes):
    N = rhs.size
    bufs = [np.zeros(N), np.zeros(N)]          # [scratch, out]: product p writes bufs[p % 2]
    cur, p = rhs.ravel(), 0
    for k in modes:
        mode_product(cur, bufs[p % 2], dims, k)
        cur, p = bufs[p % 2], p + 1
    f = np.arange(N)
    den = np.ones(N)
    for k in modes:
        nk = dims[k - 1]
        den += 2 - 2 * np.cos(2 * np.pi * ((f // mode_stride(dims, k)) % nk) / nk)
    cur /= den
    for k in modes:
        mode_product(cur, bufs[p % 2], dims, k)
        cur, p = bufs[p % 2], p + 1
    assert cur is bufs[1]                      # the last product lands in `out`
    return cur


@pytest.mark.parametrize("dims,modes", [((7, 5, 4, 3), (1, 2, 3, 4)), ((6, 9, 5), (1, 3)),
                                        ((8, 8), (1, 2)), ((4, 6, 1, 3), (3, 4)),
                                        ((37, 29, 5, 3), (2, 4))])
def test_gradient_kernels_and_solve(dims, modes):
    tdims = tuple(dims[2:])
    n = int(np.prod(tdims)) if tdims else 1
    rng = np.random.default_rng(sum(dims))
    X = rng.standard_normal((n, dims[0], dims[1]))
    N = X.size
    for k in range(1, len(dims) + 1):
        S, nk = mode_stride(dims, k), dims[k - 1]
        got = (X.ravel()[fwd(N, S, nk)] - X.ravel()).reshape(X.shape)
        assert np.abs(got - ctv.grad(X, tdims, k)).max() < 1e-14
        got = (X.ravel()[bwd(N, S, nk)] - X.ravel()).reshape(X.shape)
        assert np.abs(got - ctv.grad_t(X, tdims, k)).max() < 1e-14
    got = gradient_solve(X, dims, modes).reshape(X.shape)
    want = ctv.l_update(X, {k: np.zeros_like(X) for k in modes}, tdims, modes)
    assert np.abs(got - want).max() < 1e-13


def prox_through_handle(Rin, tau, t, p, tdims):
    Ab = transform.forward(Rin, tdims)
    Gb, _ = svt.transformed_prox(Ab, tau, p.phi, p.phi_theta, p.phi_gamma, engine="rsvd", l=p.l,
                                 q=p.q, seed=p.seed, t=t)
    return transform.inverse(Gb, tdims).ravel()


@pytest.mark.parametrize("dims,modes,noise", [((12, 10, 5, 4), (1, 2), admm.NOISE_L1),
                                              ((12, 10, 5, 4), (1, 2, 4), admm.NOISE_NONE),
                                              ((9, 7, 6), (1, 3), admm.NOISE_L1)])
def test_gradient_step_sequence(dims, modes, noise):
    tdims = tuple(dims[2:])
    shape = (int(np.prod(tdims)), dims[0], dims[1])
    N = int(np.prod(shape))
    rng = np.random.default_rng(5)
    draw = lambda s: s * rng.standard_normal(shape)
    mask = (rng.random(shape) < 0.6).astype(np.uint8)
    M = np.where(mask == 1, draw(1.0), 0.0)
    st = ctv.State(L=draw(0.5), E=draw(0.1), Y=draw(0.05), G={k: draw(0.3) for k in modes},
                   Lam={k: draw(0.05) for k in modes}, mu=0.4, t=2)
    p = ctv.Params(modes=modes, transform="dct", engine="rsvd", l=6, q=1, seed=8, phi=prox.MCP,
                   phi_gamma=30.0, psi=prox.MCP, psi_gamma=30.0, noise=noise, lam=0.2)
    ref, res_ref = ctv.step(st, M, mask, tdims, p)
    # the launch sequence of ctv_step
    mu = st.mu
    L, E, Y, Mf = st.L.ravel().copy(), st.E.ravel().copy(), st.Y.ravel().copy(), M.ravel()
    G = {k: st.G[k].ravel().copy() for k in modes}
    Lam = {k: st.Lam[k].ravel().copy() for k in modes}
    res = np.zeros(5)
    R = Mf - E + Y * (1 / mu)                                     # ctv_rhs_kernel
    for k in modes:                                               # adj_grad_accum_kernel
        b = bwd(N, mode_stride(dims, k), dims[k - 1])
        W = G[k] - (1 / mu) * Lam[k]
        R = R + (W[b] - W)
    W = gradient_solve(R.reshape(shape), dims, modes)            # tr_gradient_solve
    res[0] = np.abs(W - L).max()                                  # ctv_commit_l_kernel
    L = W.copy()
    tau = 1.0 / (len(modes) * mu)
    for k in modes:
        fw = fwd(N, mode_stride(dims, k), dims[k - 1])
        R = (L[fw] - L) + (1 / mu) * Lam[k]                       # grad_plus_kernel
        Gn = prox_through_handle(R.reshape(shape), tau, st.t, p, tdims)
        d = L[fw] - L                                             # ctv_commit_g_kernel
        res[3] = max(res[3], np.abs(Gn - G[k]).max())
        res[2] = max(res[2], np.abs(d - Gn).max())
        G[k], Lam[k] = Gn, Lam[k] + mu * (d - Gn)
    H = Mf - L + Y / mu                                           # ctv_e_kernel
    on = np.zeros(N) if noise == admm.NOISE_NONE else prox.prox_scalar(H, p.lam / mu, p.psi,
                                                                        p.psi_theta, p.psi_gamma)
    e = np.where(mask.ravel() == 1, on, H)
    res[1] = np.abs(e - E).max()
    r = Mf - L - e
    res[4] = np.abs(r).max()
    Y = Y + mu * r
    assert np.abs(L.reshape(shape) - ref.L).max() < 1e-13
    assert np.abs(Y.reshape(shape) - ref.Y).max() < 1e-13
    for k in modes:
        assert np.abs(G[k].reshape(shape) - ref.G[k]).max() < 1e-13
        assert np.abs(Lam[k].reshape(shape) - ref.Lam[k]).max() < 1e-13
    assert np.abs(res - res_ref).max() < 1e-13


@pytest.mark.parametrize("dims,modes", [((12, 10, 6), (1, 2)), ((12, 10, 6), (1, 2, 3)),
                                        ((8, 9, 3, 2), (2, 4))])
def test_onebit_step_sequence(dims, modes):
    tdims = tuple(dims[2:])
    shape = (int(np.prod(tdims)), dims[0], dims[1])
    N = int(np.prod(shape))
    rng = np.random.default_rng(6)
    S = 0.3 * rng.standard_normal(shape)
    s, q = synth.one_bit_observations(S, 3 * S.size, 1.2, 0.05, rng)
    p = onebit.Params(modes=modes, engine="rsvd", l=6, q=1, seed=7, mu0=0.05, lam=2e-3, theta=1.2,
                      alpha=0.9, phi=prox.MCP, phi_gamma=50.0)
    m = len(s)
    # J1, J2 from integer counts (onebit_count_kernel, onebit_j_kernel)
    pos = np.bincount(s[q > 0], minlength=N)
    neg = np.bincount(s[q <= 0], minlength=N)
    J1, J2 = (p.theta * (pos - neg)).reshape(shape), (pos + neg).reshape(shape).astype(float)
    J1o, J2o = onebit.sample_tensors(shape, s, q, p.theta)
    assert np.abs(J1 - J1o).max() < 1e-12 and np.array_equal(J2, J2o)
    st = onebit.State(L=0.3 * rng.standard_normal(shape), Z=0.3 * rng.standard_normal(shape),
                      Y=0.01 * rng.standard_normal(shape),
                      G={i: 0.1 * rng.standard_normal(shape) for i in modes},
                      Lam={i: 0.01 * rng.standard_normal(shape) for i in modes}, mu=0.05, t=4)
    ref, rel_ref = onebit.step(st, J1o, J2o, m, tdims, p)
    mu = st.mu
    L = np.clip((m * mu * st.Z + J1 - m * st.Y) / (m * mu + J2), -p.alpha, p.alpha).ravel()
    rel = np.sqrt(np.sum((L - st.L.ravel()) ** 2) / np.sum(st.L ** 2))   # onebit_l_kernel sums
    Y = st.Y.ravel().copy()
    G = {k: st.G[k].ravel().copy() for k in modes}
    Lam = {k: st.Lam[k].ravel().copy() for k in modes}
    R = L + (1 / mu) * Y                                          # axpby_kernel
    for k in modes:                                               # adj_grad_accum_kernel
        b = bwd(N, mode_stride(dims, k), dims[k - 1])
        W = G[k] - (1 / mu) * Lam[k]
        R = R + (W[b] - W)
    Z = gradient_solve(R.reshape(shape), dims, modes)
    tau = p.lam / (len(modes) * mu)
    for k in modes:
        fw = fwd(N, mode_stride(dims, k), dims[k - 1])
        R = (Z[fw] - Z) + (1 / mu) * Lam[k]                       # grad_plus_kernel
        G[k] = prox_through_handle(R.reshape(shape), tau, st.t, p, tdims)
        Lam[k] = Lam[k] + mu * ((Z[fw] - Z) - G[k])               # grad_multiplier_kernel
    Y = Y + mu * (L - Z)                                          # multiplier_kernel
    for name, got in (("L", L), ("Z", Z), ("Y", Y)):
        assert np.abs(got.reshape(shape) - getattr(ref, name)).max() < 1e-13, name
    for k in modes:
        assert np.abs(G[k].reshape(shape) - ref.G[k]).max() < 1e-13
        assert np.abs(Lam[k].reshape(shape) - ref.Lam[k]).max() < 1e-13
    assert abs(rel - rel_ref) < 1e-13


def unfold_times(C, mode, V):
    """A V for the mode unfolding A of the slice stack C (n, p1, p2), with V
    column-major (n p_other) x k (rows j p_other + i): one strided GEMM per
    slice into a (n, rows, k) buffer, then the sum over slices."""
    n, p1, p2 = C.shape
    k = V.shape[1]
    Cf, Vf = C.ravel(), V.ravel(order="F")
    ldv = V.shape[0]
    out = np.zeros(n * (p1 if mode == 1 else p2) * k)
    if mode == 1:   # sum_j C_j V_j, V_j = rows j p2 ..: x = i1, b = i2
        gemm(Cf, p1 * p2, p2, 1, Vf, p2, 1, ldv, out, p1 * k, k, 1, p1, k, p2, n)
        return out.reshape(n, p1, k).sum(axis=0)
    # mode 2: sum_j C_j^T V_j, V_j = rows j p1 ..: x = i2, b = i1
    gemm(Cf, p1 * p2, 1, p2, Vf, p1, 1, ldv, out, p2 * k, k, 1, p2, k, p1, n)
    return out.reshape(n, p2, k).sum(axis=0)


def unfold_t_times(C, mode, U):
    """A^T U for the mode unfolding, U column-major rows x k: one strided GEMM
    per slice writing rows j p_other + i of a column-major result."""
    n, p1, p2 = C.shape
    k = U.shape[1]
    Cf, Uf = C.ravel(), U.ravel(order="F")
    other = p2 if mode == 1 else p1
    ldo = n * other
    out = np.zeros(ldo * k)
    if mode == 1:   # (C_j^T U)[i2][c]: x = i2, b = i1
        gemm(Cf, p1 * p2, 1, p2, Uf, 0, 1, p1, out, p2, 1, ldo, p2, k, p1, n)
    else:           # (C_j U)[i1][c]: x = i1, b = i2
        gemm(Cf, p1 * p2, p2, 1, Uf, 0, 1, p2, out, p1, 1, ldo, p1, k, p2, n)
    return out.reshape(k, ldo).T


@pytest.mark.parametrize("n,p1,p2,k", [(1, 5, 7, 3), (6, 12, 9, 4), (4, 20, 31, 1), (3, 1, 6, 2)])
def test_unfolding_products_without_forming_the_unfolding(n, p1, p2, k):
    # the planned GPU form of the fixed-accuracy Tucker loop's products
    from oracle import tucker
    rng = np.random.default_rng(n + p1 + p2 + k)
    C = rng.standard_normal((n, p1, p2))
    for mode, rows, cols in ((1, p1, n * p2), (2, p2, n * p1)):
        A = tucker.unfold(C, mode)
        V = rng.standard_normal((cols, k))
        U = rng.standard_normal((rows, k))
        assert np.abs(unfold_times(C, mode, V) - A @ V).max() < 1e-12
        assert np.abs(unfold_t_times(C, mode, U) - A.T @ U).max() < 1e-12


# ---------------------------------------------------------------------------
# tr_slice_prox_ad_tucker (csrc/ad_tucker.cu): its host loop restated with
# numpy in place of each launch, on flat column-major buffers with the same
# column offsets, capacities and draw counters.

def cgs2_defl_qr(W, rows, k, delta, pivot=True):
    """defl_qr of csrc/ad_tucker.cu: pivot = largest residual norm, stop once
    it is below delta (pivot=False, orth(): columns in order); second pass
    against the columns kept; R = Q^T W0."""
    W0 = W.copy()
    used = [False] * k
    Q = []
    for step in range(k):
        j = step
        if pivot:
            norms = [np.dot(W[:, c], W[:, c]) if not used[c] else -1.0 for c in range(k)]
            j = int(np.argmax(norms))
            if used[j] or not np.sqrt(max(norms[j], 0.0)) >= delta:
                break
        used[j] = True
        q = W[:, j].copy()
        if Q:
            Qm = np.stack(Q, axis=1)
            q -= Qm @ (Qm.T @ q)
        nq = np.linalg.norm(q)
        if not nq > 0:
            break
        q /= nq
        W -= np.outer(q, q @ W)
        Q.append(q)
    Qm = np.stack(Q, axis=1) if Q else np.zeros((rows, 0))
    return Qm, Qm.T @ W0


def gauss_panel(seed, t, n, per, k, stream):
    from oracle import philox
    return np.concatenate([philox.gaussian_block(seed, t, j, per, k, stream) for j in range(n)],
                          axis=0)


def blbp_mode_emul(Cst, mode, eps, b, delta_rel, cap, capV, seed, t):
    from oracle import tucker
    A = tucker.unfold(Cst, mode)
    rows, cols = A.shape
    n = Cst.shape[0]
    normA2 = float(np.sum(A * A))
    delta = delta_rel * np.sqrt(normA2)
    E = normA2
    if normA2 == 0.0:
        return np.zeros((rows, 0)), 0.0
    base = 0x10000 if mode == 1 else 0x20000
    draw = [0]

    def gauss(k):
        G = gauss_panel(seed, t, n, cols // n, k, base + 2 * draw[0])
        draw[0] += 1
        return G

    b0 = min(b, cols)
    Vq, _ = cgs2_defl_qr(gauss(b0), cols, b0, 0.0, pivot=False)
    Vcat = Vq.copy()
    vstart, kv = 0, Vq.shape[1]
    Ucat = np.zeros((rows, 0))
    sprev, lcols, L = 0, 0, np.zeros((0, 0))
    while True:
        V = Vcat[:, vstart:vstart + kv]
        P = A @ V
        if sprev > 0 and lcols > 0:
            P[:, :lcols] -= Ucat[:, -sprev:] @ L[:, :lcols]
        U, R = cgs2_defl_qr(P.copy(), rows, kv, delta)
        su = U.shape[1]
        E -= float(np.sum(R * R))
        sv = 0
        new_vstart = Vcat.shape[1]
        Vn = np.zeros((cols, 0))
        if su > 0:
            Vn = A.T @ U - V @ R.T
            Vn = Vn - Vcat @ (Vcat.T @ Vn)
            assert Vcat.shape[1] + su <= capV
            Vn, Lt = cgs2_defl_qr(Vn, cols, su, delta)
            sv = Vn.shape[1]
            E -= float(np.sum(Lt * Lt))
            Vcat = np.concatenate([Vcat, Vn], axis=1)
            L = Lt.T
        knext = sv
        if sv < b and Vcat.shape[1] < cols:
            want = b - sv
            G = gauss(want)
            G = G - Vcat @ (Vcat.T @ G)
            keep = max(0, min(want, cols - Vcat.shape[1]))
            assert Vcat.shape[1] + want <= capV
            Vr, _ = cgs2_defl_qr(G, cols, want, 0.0, pivot=False)
            Vr = Vr[:, :min(Vr.shape[1], keep)]
            Vcat = np.concatenate([Vcat, Vr], axis=1)
            knext += Vr.shape[1]
        Ucat = np.concatenate([Ucat, U], axis=1)
        sprev, lcols, vstart, kv = su, sv, new_vstart, knext
        if E < eps * eps * normA2 or Ucat.shape[1] >= cap or kv == 0:
            break
    return Ucat[:, :cap], E


@pytest.mark.parametrize("n,n1,n2,s1,s2,b", [(6, 30, 22, 5, 3, 2), (4, 12, 19, 10, 13, 1),
                                             (3, 16, 16, 4, 4, 4), (1, 9, 7, 3, 2, 2)])
def test_ad_tucker_host_loop_emulation(n, n1, n2, s1, s2, b):
    # on stacks with shared spaces the restated loop finds the unfoldings'
    # ranks and the result is the full-SVD prox of every slice, as the oracle's
    from oracle import tucker
    rng = np.random.default_rng(n * 100 + n1 + n2)
    P, _ = np.linalg.qr(rng.standard_normal((n1, s1)))
    Q, _ = np.linalg.qr(rng.standard_normal((n2, s2)))
    Ab = np.einsum("ia,jab,kb->jik", P, 3.0 * rng.standard_normal((n, s1, s2)), Q)
    r1w = min(s1, n * s2)
    cap1 = min(n1, n * n2)
    capV = min(n * max(n1, n2), b * (max(n1, n2) + 4)) + b
    F1, _ = blbp_mode_emul(Ab, 1, 1e-6, b, 1e-10, cap1, capV, 5, 2)
    assert F1.shape[1] == r1w
    F1 = tucker.canonical_signs(F1)
    C1 = tucker.mode_product_t(Ab, F1, 1)
    F2, _ = blbp_mode_emul(C1, 2, 1e-6, b, 1e-10, min(n2, n * r1w), capV, 5, 2)
    F2 = tucker.canonical_signs(F2)
    assert F2.shape[1] == min(s2, n * r1w)
    C2 = tucker.mode_product_t(C1, F2, 2)
    Ct, _ = svt.transformed_prox(C2, 0.4, prox.MCP, gamma=30.0)
    got = tucker.mode_product(tucker.mode_product(Ct, F1, 1), F2, 2)
    want, _ = svt.transformed_prox(Ab, 0.4, prox.MCP, gamma=30.0, engine="ad_tucker", eps=1e-6,
                                   b=b, delta_rel=1e-10, seed=5, t=2)
    full, _ = svt.transformed_prox(Ab, 0.4, prox.MCP, gamma=30.0)
    assert np.abs(got - full).max() <= 1e-9 * max(1.0, np.abs(full).max())
    assert np.abs(want - full).max() <= 1e-9 * max(1.0, np.abs(full).max())


# ---------------------------------------------------------------------------
# tr_slice_prox_ad_tucker on the flat buffers of csrc/ad_tucker.cu: every
# strided GEMM with the element strides the host code passes (not a plain
# matrix product), every panel at the element count the host code allocates,
# every panel pointer at the host code's offset.  Numpy raises on an index
# past a panel's end, so a run also shows the capacities hold.

def sgemm(A, B, C, X, Y, K, batch=1, ao=0, ax=0, ab=0, bo=0, bb=0, by=0, co=0, cx=0, cy=0):
    if X < 1 or Y < 1 or batch < 1:       # sg::gemm launches nothing
        return
    gemm(A, ao, ax, ab, B, bo, bb, by, C, co, cx, cy, X, Y, K, batch)


def col(rows, c, ld):
    return np.arange(rows) + c * ld


def canon_signs_flat(F, m, r):
    # canon_sign_kernel: each column's first entry of largest magnitude positive
    for c in range(r):
        v = F[col(m, c, m)]
        if v[int(np.argmax(np.abs(v)))] < 0:
            F[col(m, c, m)] = -v


def defl_qr_flat(W, Worig, rows, k, delta, pivot, Q, Rout):
    used = [False] * k
    s = 0
    for step in range(k):
        j = step
        if pivot:
            norms = [float(np.sum(W[col(rows, c, rows)] ** 2)) for c in range(k)]   # col_dots_kernel
            j, best = -1, -1.0
            for c in range(k):
                if not used[c] and norms[c] > best:
                    j, best = c, norms[c]
            if j < 0 or not np.sqrt(max(best, 0.0)) >= delta:
                break
        used[j] = True
        qi = col(rows, s, rows)
        Q[qi] = W[col(rows, j, rows)]
        if s > 0:                        # col_dot_vec_kernel, gemv_sub_kernel
            coef = np.array([np.dot(Q[col(rows, i, rows)], Q[qi]) for i in range(s)])
            Q[qi] = Q[qi] - sum(Q[col(rows, i, rows)] * coef[i] for i in range(s))
        nq = np.sqrt(np.sum(Q[qi] ** 2))
        if not nq > 0:
            break
        Q[qi] = Q[qi] * (1.0 / nq)       # scale_kernel
        coef = [np.dot(W[col(rows, c, rows)], Q[qi]) for c in range(k)]
        for c in range(k):               # rank1_kernel
            W[col(rows, c, rows)] -= Q[qi] * coef[c]
        s += 1
    if s > 0:                            # R = Q^T Worig, s x k, ld s
        sgemm(Q, Worig, Rout, s, k, rows, ax=rows, ab=1, bb=1, by=rows, cx=1, cy=s)
    return s


def blbp_mode_flat(C, mode, n, p1, p2, eps, b, delta_rel, cap, capV, seed, t, pn):
    from oracle import philox
    rows, cols = (p1, n * p2) if mode == 1 else (p2, n * p1)
    Ucat, Vcat, P, P0, Vn, Vn0 = pn["Ucat"], pn["Vcat"], pn["P"], pn["P0"], pn["Vn"], pn["Vn0"]
    tmp, X, R, Lt, L, G, Gs = pn["tmp"], pn["X"], pn["R"], pn["Lt"], pn["L"], pn["G"], pn["Gs"]
    normA2 = float(np.sum(C[np.arange(n * p1 * p2)] ** 2))
    delta = delta_rel * np.sqrt(normA2)
    E = normA2
    if normA2 == 0.0:
        return 0, 0.0
    base = 0x10000 if mode == 1 else 0x20000
    per = cols // n
    draw = [0]

    def gauss(k, dst):                   # launch_gaussian_blocks + gather_slices_kernel
        blocks = [philox.gaussian_block(seed, t, j, per, k, base + 2 * draw[0]).ravel(order="F")
                  for j in range(n)]
        draw[0] += 1
        Gs[np.arange(n * per * k)] = np.concatenate(blocks)
        e = np.arange(n * per * k)
        i, c, j = e % per, (e // per) % k, e // (per * k)
        dst[(j * per + i) + c * cols] = Gs[e]

    def unfold_times(V, ldv, k):         # P = A V: per-slice GEMMs into tmp, then batch_sum_kernel
        if mode == 1:
            sgemm(C, V, tmp, p1, k, p2, n, ao=p1 * p2, ax=p2, ab=1, bo=p2, bb=1, by=ldv,
                  co=p1 * k, cx=1, cy=p1)
        else:
            sgemm(C, V, tmp, p2, k, p1, n, ao=p1 * p2, ax=1, ab=p2, bo=p1, bb=1, by=ldv,
                  co=p2 * k, cx=1, cy=p2)
        M = rows * k
        P[np.arange(M)] = sum(tmp[o * M + np.arange(M)] for o in range(n))

    def unfold_t_times(U, k):            # Vn = A^T U
        if mode == 1:
            sgemm(C, U, Vn, p2, k, p1, n, ao=p1 * p2, ax=1, ab=p2, bb=1, by=rows, co=p2, cx=1,
                  cy=cols)
        else:
            sgemm(C, U, Vn, p1, k, p2, n, ao=p1 * p2, ax=p2, ab=1, bb=1, by=rows, co=p1, cx=1,
                  cy=cols)

    def matmul(A, la, B, lb, Cm, lc, M, N_, K, transA):
        if transA:
            sgemm(A, B, Cm, M, N_, K, ax=la, ab=1, bb=1, by=lb, cx=1, cy=lc)
        else:
            sgemm(A, B, Cm, M, N_, K, ax=1, ab=la, bb=1, by=lb, cx=1, cy=lc)

    def sub(Xd, Ys, r, k, ldx, ldy):     # sub_kernel
        for c in range(k):
            Xd[col(r, c, ldx)] -= Ys[col(r, c, ldy)]

    def copy(dst, src, count):           # cudaMemcpyAsync device to device
        dst[np.arange(count)] = src[np.arange(count)]

    b0 = min(b, cols)
    gauss(b0, G)
    copy(Vn0, G, cols * b0)
    kv = defl_qr_flat(G, Vn0, cols, b0, 0.0, False, Vcat, R)
    vcols, vstart, ucols, ustart, sprev, lcols = kv, 0, 0, 0, 0, 0
    while True:
        unfold_times(Vcat[vstart * cols:], cols, kv)
        if sprev > 0 and lcols > 0:
            matmul(Ucat[ustart * rows:], rows, L, sprev, X, rows, rows, lcols, sprev, False)
            sub(P, X, rows, lcols, rows, rows)
        copy(P0, P, rows * kv)
        su = defl_qr_flat(P, P0, rows, kv, delta, True, Ucat[ucols * rows:], R)
        E -= float(np.sum(R[np.arange(su * kv)] ** 2))
        sv = 0
        if su > 0:
            unfold_t_times(Ucat[ucols * rows:], su)
            sgemm(Vcat[vstart * cols:], R, X, cols, su, kv, ax=1, ab=cols, bb=su, by=1, cx=1,
                  cy=cols)                                     # X = V R^T
            sub(Vn, X, cols, su, cols, cols)
            matmul(Vcat, cols, Vn, cols, Lt, vcols, vcols, su, cols, True)
            matmul(Vcat, cols, Lt, vcols, X, cols, cols, su, vcols, False)
            sub(Vn, X, cols, su, cols, cols)
            copy(Vn0, Vn, cols * su)
            assert vcols + su <= capV
            sv = defl_qr_flat(Vn, Vn0, cols, su, delta, True, Vcat[vcols * cols:], Lt)
            E -= float(np.sum(Lt[np.arange(sv * su)] ** 2))
        new_vstart = vcols
        vcols += sv
        if sv > 0:                       # L = Lt^T (su x sv, ld su), through the host
            h = Lt[np.arange(sv * su)].copy()
            i, c = np.meshgrid(np.arange(sv), np.arange(su), indexing="ij")
            L[(c + i * su).ravel()] = h[(i + c * sv).ravel()]
        knext = sv
        if sv < b and vcols < cols:
            want = b - sv
            gauss(want, G)
            matmul(Vcat, cols, G, cols, X, vcols, vcols, want, cols, True)
            matmul(Vcat, cols, X, vcols, Vn, cols, cols, want, vcols, False)
            sub(G, Vn, cols, want, cols, cols)
            copy(Vn0, G, cols * want)
            keep = max(0, min(want, cols - vcols))
            assert vcols + want <= capV
            sr = min(defl_qr_flat(G, Vn0, cols, want, 0.0, False, Vcat[vcols * cols:], X), keep)
            vcols += sr
            knext += sr
        ucols += su
        ustart, sprev, lcols, vstart, kv = ucols - su, su, sv, new_vstart, knext
        if E < eps * eps * normA2 or ucols >= cap or kv == 0:
            break
    return min(ucols, cap), E


def ad_tucker_flat(Ab, tau, kind, gamma, eps, b, delta_rel, max_rank, seed, t):
    n, n1, n2 = Ab.shape
    N = n * n1 * n2
    rows_max, cols_max = max(n1, n2), n * max(n1, n2)
    cap_max = min(rows_max, max_rank if max_rank > 0 else rows_max)
    capV = min(cols_max, b * (cap_max + 4)) + b
    sizes = dict(Ucat=rows_max * (cap_max + b), Vcat=cols_max * capV, P=rows_max * b,
                 P0=rows_max * b, Vn=cols_max * b, Vn0=cols_max * b, tmp=n * rows_max * b,
                 X=max(cols_max, rows_max) * max(b, capV), R=b * b, Lt=max(b * b, capV * b),
                 L=b * b, G=cols_max * b, Gs=cols_max * b)
    pn = {k: np.full(max(v, 2), np.nan) for k, v in sizes.items()}   # unwritten reads show as NaN
    F1, C1, C2, Ct, Tb = (np.full(v, np.nan) for v in (n1 * cap_max, N, N, N, N))
    A = Ab.ravel().copy()
    Gbar = np.full(N, np.nan)
    cap1 = min(n1, n * n2, max_rank if max_rank > 0 else n1)
    r1, _ = blbp_mode_flat(A, 1, n, n1, n2, eps, b, delta_rel, cap1, capV, seed, t, pn)
    if r1 == 0:
        return np.zeros(Ab.shape), (0, 0)
    F1[np.arange(n1 * r1)] = pn["Ucat"][np.arange(n1 * r1)]
    canon_signs_flat(F1, n1, r1)
    # truncate_core, mode 1: C1_j = F1^T A_j (r1 x n2)
    sgemm(F1, A, C1, r1, n2, n1, n, ax=n1, ab=1, bo=n1 * n2, bb=n2, by=1, co=r1 * n2, cx=n2, cy=1)
    cap2 = min(n2, n * r1, max_rank if max_rank > 0 else n2)
    r2, _ = blbp_mode_flat(C1, 2, n, r1, n2, eps, b, delta_rel, cap2, capV, seed, t, pn)
    if r2 == 0:
        return np.zeros(Ab.shape), (r1, 0)
    F2 = pn["Ucat"]
    canon_signs_flat(F2, n2, r2)
    # truncate_core, mode 2: C2_j = C1_j F2 (r1 x r2)
    sgemm(C1, F2, C2, r1, r2, n2, n, ao=r1 * n2, ax=n2, ab=1, bb=1, by=n2, co=r1 * r2, cx=r2, cy=1)
    # the core's prox at full width is exact: the full-SVD prox of each slice
    core = C2[np.arange(n * r1 * r2)].reshape(n, r1, r2)
    Ct[np.arange(n * r1 * r2)] = svt.transformed_prox(core, tau, kind, gamma=gamma)[0].ravel()
    # T_j = Ct_j F2^T (r1 x n2), then Gbar_j = F1 T_j
    sgemm(Ct, F2, Tb, r1, n2, r2, n, ao=r1 * r2, ax=r2, ab=1, bb=n2, by=1, co=r1 * n2, cx=n2, cy=1)
    sgemm(F1, Tb, Gbar, n1, n2, r1, n, ax=1, ab=n1, bo=r1 * n2, bb=n2, by=1, co=n1 * n2, cx=n2,
          cy=1)
    return Gbar.reshape(Ab.shape), (r1, r2)


@pytest.mark.parametrize("n,n1,n2,s1,s2,b,max_rank",
                         [(6, 30, 22, 5, 3, 2, 0), (4, 12, 19, 10, 13, 1, 0),
                          (3, 16, 16, 4, 4, 4, 0), (1, 9, 7, 3, 2, 2, 0),
                          (5, 14, 11, 6, 5, 3, 4), (1, 3, 2, 3, 2, 4, 0),
                          (2, 8, 20, 3, 6, 32, 0)])
def test_ad_tucker_flat_buffers_and_strides(n, n1, n2, s1, s2, b, max_rank):
    # the launch sequence with the host code's strides, offsets and panel
    # sizes gives the oracle's fixed-accuracy Tucker prox and its ranks
    rng = np.random.default_rng(7 * n + n1 + 3 * n2 + b)
    P, _ = np.linalg.qr(rng.standard_normal((n1, s1)))
    Q, _ = np.linalg.qr(rng.standard_normal((n2, s2)))
    Ab = np.einsum("ia,jab,kb->jik", P, 3.0 * rng.standard_normal((n, s1, s2)), Q)
    got, ranks = ad_tucker_flat(Ab, 0.4, prox.MCP, 30.0, 1e-6, b, 1e-10, max_rank, 5, 2)
    want, info = svt.transformed_prox(Ab, 0.4, prox.MCP, gamma=30.0, engine="ad_tucker", eps=1e-6,
                                      b=b, delta_rel=1e-10, seed=5, t=2,
                                      max_rank=max_rank if max_rank > 0 else None)
    assert ranks == tuple(info["tucker_ranks"])
    assert np.isfinite(got).all()
    # the two loops round differently (the oracle's Householder QR, Gram-Schmidt
    # here) and keep U orthogonal only between adjacent blocks, so the gap
    # grows with the number of blocks: ten one-column blocks reach ~1e-10
    scale = max(1.0, np.abs(want).max())
    assert np.abs(got - want).max() <= 1e-9 * scale
    if max_rank == 0:   # uncapped on exact low-rank stacks: the full-SVD prox
        full, _ = svt.transformed_prox(Ab, 0.4, prox.MCP, gamma=30.0)
        assert np.abs(got - full).max() <= 1e-9 * scale


def test_ad_tucker_flat_zero_stack():
    got, ranks = ad_tucker_flat(np.zeros((3, 5, 4)), 0.4, prox.L1, 4.0, 1e-6, 2, 1e-10, 0, 1, 0)
    assert ranks == (0, 0) and not got.any()
