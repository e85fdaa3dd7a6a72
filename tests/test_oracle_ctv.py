"""Pins of the gradient-domain (GNHTCTV) oracle and of GNHTSVT under the DFT
transform.

The pins use what the definitions and the mathematics fix:

* nabla_k against a shift written with numpy.roll, its adjoint identity,
  constants in its kernel, telescoping sums, and the circulant's symbol
  |F(D_k)|^2 = 2 - 2 cos(2 pi f / n_k);
* the FFT solve of Eq. coef-tensor against the linear system applied with
  numpy.roll and against a dense solve on a tiny tensor;
* Gamma = {identity} reproduces the pure-L step (oracle.admm, pinned on its
  own by KKT and exact recovery);
* two identities every ADMM step satisfies exactly, derived from the
  L-system and the multiplier updates (dual residual; Y = 0 off Omega);
* the G-step threshold tau = 1/(gamma mu) seen in the multiplier spectrum;
* the DFT transform against numpy.fft, a real result, the closed form on
  slice-constant tensors (threshold tau/n), and optimality against random
  perturbations of the objective with the 1/rho factor;
* exact recovery of a smooth low-rank tensor from half of its entries
  (empirical).
"""

import numpy as np
import pytest

from oracle import admm, ctv, prox, svt, transform
from shifts import roll_grad, roll_grad_t


# ------------------------------------------------------------ gradient

@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_gradient_is_a_forward_difference(k):
    rng = np.random.default_rng(1)
    tdims = (4, 3)
    X = rng.standard_normal((12, 7, 5))
    assert np.array_equal(ctv.grad(X, tdims, k), roll_grad(X, tdims, k))
    Y = rng.standard_normal(X.shape)
    # adjoint: <nabla X, Y> = <X, nabla^T Y>
    lhs = np.sum(ctv.grad(X, tdims, k) * Y)
    rhs = np.sum(X * ctv.grad_t(Y, tdims, k))
    assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(lhs))
    assert np.allclose(ctv.grad_t(Y, tdims, k), roll_grad_t(Y, tdims, k), atol=1e-15)
    # constants are in the kernel; sums along the mode telescope to zero
    assert np.abs(ctv.grad(np.full(X.shape, 2.5), tdims, k)).max() == 0.0
    n, n1, n2 = X.shape
    V = ctv.grad(X, tdims, k).reshape(tuple(reversed(tdims)) + (n1, n2))
    ax = {1: 2, 2: 3, 3: 1, 4: 0}[k]
    assert np.abs(V.sum(axis=ax)).max() < 1e-12


def test_difference_matrix_is_the_stated_circulant():
    D = ctv.difference_matrix(5)
    assert np.array_equal(D[0], [-1.0, 1.0, 0.0, 0.0, 0.0])
    for i in range(5):
        assert np.array_equal(D[i], np.roll(D[0], i))
    assert np.array_equal(ctv.difference_matrix(1), [[0.0]])


def test_difference_tensor_symbol():
    # nabla_k is a circular convolution with D_k; its DFT symbol has
    # |F(D_k)|^2 = 2 - 2 cos(2 pi f_k / n_k), constant along the other modes
    tdims = (4, 3)
    shape = (12, 6, 5)
    for k, nk, ax in ((1, 6, 2), (2, 5, 3), (3, 4, 1), (4, 3, 0)):
        FD = np.fft.fftn(ctv.difference_tensor(shape, tdims, k))
        f = np.arange(nk)
        want = 2.0 - 2.0 * np.cos(2.0 * np.pi * f / nk)
        bshape = [1] * 4
        bshape[ax] = nk
        assert np.allclose(np.abs(FD) ** 2, np.broadcast_to(want.reshape(bshape), FD.shape),
                           atol=1e-13)
        # convolution by brute force on a random tensor equals the gradient
        rng = np.random.default_rng(k)
        X = rng.standard_normal(shape)
        conv = np.fft.ifftn(FD * np.fft.fftn(X.reshape(3, 4, 6, 5))).real.reshape(shape)
        assert np.allclose(conv, roll_grad(X, tdims, k), atol=1e-13)


# ------------------------------------------------------------ L-update

@pytest.mark.parametrize("modes", [(1, 2), (1, 2, 3), (1, 2, 4), (3,), (0, 1)])
def test_l_update_solves_the_linear_system(modes):
    rng = np.random.default_rng(2)
    tdims = (4, 3)
    shape = (12, 7, 5)
    R0 = rng.standard_normal(shape)
    Rk = {k: rng.standard_normal(shape) for k in modes}
    L = ctv.l_update(R0, Rk, tdims, modes)

    def g(S, k):
        return S if k == 0 else roll_grad(S, tdims, k)

    def gt(S, k):
        return S if k == 0 else roll_grad_t(S, tdims, k)

    lhs = L + sum(gt(g(L, k), k) for k in modes)
    rhs = R0 + sum(gt(Rk[k], k) for k in modes)
    assert np.abs(lhs - rhs).max() < 1e-12 * np.abs(rhs).max()


def test_l_update_matches_a_dense_solve():
    rng = np.random.default_rng(3)
    tdims = (3,)
    shape = (3, 4, 2)
    N = int(np.prod(shape))
    modes = (1, 2, 3)
    # the operator I + sum nabla^T nabla as an explicit N x N matrix
    A = np.eye(N)
    for k in modes:
        Dk = np.stack([roll_grad(e.reshape(shape), tdims, k).ravel() for e in np.eye(N)], axis=1)
        A += Dk.T @ Dk
    R0 = rng.standard_normal(shape)
    Rk = {k: rng.standard_normal(shape) for k in modes}
    b = R0.ravel() + sum(roll_grad_t(Rk[k], tdims, k).ravel() for k in modes)
    want = np.linalg.solve(A, b).reshape(shape)
    got = ctv.l_update(R0, Rk, tdims, modes)
    assert np.abs(got - want).max() < 1e-12


# ------------------------------------------------------------ ADMM step

def problem(shape, rng, sr=0.6):
    X = rng.standard_normal(shape)
    mask = rng.random(shape) < sr
    return np.where(mask, X, 0.0), mask


@pytest.mark.parametrize("noise", [admm.NOISE_L1, admm.NOISE_NONE])
def test_identity_direction_reproduces_the_pure_l_step(noise):
    rng = np.random.default_rng(4)
    tdims = (4, 3)
    M, mask = problem((12, 7, 5), rng)
    kw = dict(engine="full", lam=0.3, mu0=0.5, noise=noise, phi=prox.MCP, phi_gamma=20.0)
    st = ctv.init_state(M.shape, 0.5, (ctv.IDENTITY,))
    sa = admm.init_state(M.shape, 0.5)
    for _ in range(5):
        st, r = ctv.step(st, M, mask, tdims, ctv.Params(modes=(ctv.IDENTITY,), **kw))
        sa, ra = admm.step(sa, M, mask, tdims, admm.Params(**kw))
        for a, b in ((st.L, sa.L), (st.E, sa.E), (st.Y, sa.Y), (st.G[0], sa.G), (st.Lam[0], sa.Lam)):
            assert np.abs(a - b).max() < 1e-12
        assert np.abs(r - ra).max() < 1e-12 and st.mu == sa.mu


@pytest.mark.parametrize("tk,tdims,modes", [("dct", (4, 3), (1, 2)), ("fft", (4, 3), (1, 2, 4)),
                                            ("fft", (6,), (1, 2, 3))])
@pytest.mark.parametrize("noise", [admm.NOISE_L1, admm.NOISE_NONE])
def test_every_step_satisfies_the_dual_identities(tk, tdims, modes, noise):
    # From the L-system and the multiplier updates:
    #   Y' - sum nabla^T Lambda' = mu (E - E') + mu sum nabla^T (G' - G)
    # and, since E = H off Omega, Y' = 0 off Omega.
    rng = np.random.default_rng(5)
    n = int(np.prod(tdims))
    M, mask = problem((n, 8, 6), rng)
    p = ctv.Params(modes=modes, transform=tk, engine="full", lam=0.2, mu0=0.3, noise=noise,
                   phi=prox.L1)
    st = ctv.init_state(M.shape, p.mu0, modes)
    for _ in range(4):
        new, _ = ctv.step(st, M, mask, tdims, p)
        mu = st.mu
        lhs = new.Y - sum(roll_grad_t(new.Lam[k], tdims, k) for k in modes)
        rhs = mu * (st.E - new.E) + mu * sum(roll_grad_t(new.G[k] - st.G[k], tdims, k)
                                             for k in modes)
        assert np.abs(lhs - rhs).max() < 1e-10 * max(1.0, np.abs(new.Y).max())
        assert np.abs(new.Y[~mask]).max() < 1e-12 * max(1.0, np.abs(new.Y).max())
        st = new


@pytest.mark.parametrize("tk", ["dct", "fft"])
def test_g_step_threshold_is_one_over_gamma_mu(tk):
    # l1: Lambda'/mu = A - D_tau(A) with A = nabla L + Lambda/mu, so every
    # transformed slice of Lambda'/mu has spectral norm <= tau, equal to tau
    # where a singular value of A exceeded it; tau = 1/(gamma mu)
    rng = np.random.default_rng(6)
    tdims, modes = (4, 3), (1, 2, 3)
    M, mask = problem((12, 9, 7), rng, sr=0.8)
    p = ctv.Params(modes=modes, transform=tk, engine="full", lam=0.2, mu0=2.0, phi=prox.L1)
    st = ctv.init_state(M.shape, p.mu0, modes)
    new, _ = ctv.step(st, M, mask, tdims, p)
    tau = 1.0 / (len(modes) * p.mu0)
    for k in modes:
        Wb = transform.forward(new.Lam[k] / p.mu0, tdims, tk)
        norms = np.array([np.linalg.norm(Wb[j], 2) for j in range(Wb.shape[0])])
        assert norms.max() <= tau * (1 + 1e-10)
        assert abs(norms.max() - tau) < 1e-10 * tau


@pytest.mark.parametrize("tk,modes", [("fft", (1, 2)), ("dct", (1, 2, 3))])
def test_recovers_a_smooth_low_rank_tensor(tk, modes):
    # CP rank 3 with smooth periodic factors, half of the entries observed,
    # l1 prior, noise-free: relative error below 1e-5 (measured ~4e-7)
    rng = np.random.default_rng(0)
    n1, n2, n3 = 32, 32, 8
    i1, i2, i3 = np.arange(n1) / n1, np.arange(n2) / n2, np.arange(n3) / n3
    X = np.zeros((n1, n2, n3))
    for r in range(3):
        X += np.einsum("i,j,k->ijk", np.cos(2 * np.pi * (r + 1) * i1 + rng.random() * 6),
                       np.sin(2 * np.pi * (r + 1) * i2 + rng.random() * 6),
                       np.cos(2 * np.pi * r * i3 + rng.random() * 6))
    S = np.ascontiguousarray(np.moveaxis(X, 2, 0))
    mask = rng.random(S.shape) < 0.5
    p = ctv.Params(modes=modes, transform=tk, engine="full", phi=prox.L1, noise=admm.NOISE_NONE,
                   mu0=1e-2, growth=1.1, tol=1e-6, max_iter=300)
    st, hist = ctv.run(np.where(mask, S, 0.0), mask, (n3,), p)
    assert hist[-1].max() <= 1e-6
    assert np.linalg.norm(st.L - S) <= 1e-5 * np.linalg.norm(S)


# ------------------------------------------------------------ DFT GNHTSVT

def test_dft_transform_is_numpy_fft():
    rng = np.random.default_rng(7)
    tdims = (4, 3)
    X = rng.standard_normal((12, 5, 6))
    got = transform.forward(X, tdims, "fft").reshape(3, 4, 5, 6)
    assert np.abs(got - np.fft.fftn(X.reshape(3, 4, 5, 6), axes=(0, 1))).max() < 1e-12
    back = transform.inverse(transform.forward(X, tdims, "fft"), tdims, "fft")
    assert np.abs(back - X).max() < 1e-13
    F = transform.dft_matrix(6)
    assert np.allclose(F @ F.conj().T, 6 * np.eye(6), atol=1e-12)
    assert transform.rho(tdims, "fft") == 12.0 and transform.rho(tdims) == 1.0


@pytest.mark.parametrize("kind", [prox.L1, prox.MCP])
def test_dft_gnhtsvt_is_real_and_optimal(kind):
    rng = np.random.default_rng(8)
    tdims = (5, 2)
    A = rng.standard_normal((10, 6, 4))
    tau = 1.5
    G, _ = svt.gnhtsvt(A, tdims, tau, kind, gamma=6.0, transform_kind="fft")
    Gbar, _ = svt.transformed_prox(transform.forward(A, tdims, "fft"), tau, kind, gamma=6.0)
    assert np.abs(transform.inverse(Gbar, tdims, "fft").imag).max() < 1e-12

    def objective(Z):
        # tau (1/rho) sum Phi(sigma) over the DFT slices + ||Z - A||^2 / 2
        Zb = np.fft.fftn(Z.reshape(2, 5, 6, 4), axes=(0, 1)).reshape(10, 6, 4)
        s = np.concatenate([np.linalg.svd(Zb[j], compute_uv=False) for j in range(10)])
        return tau * np.sum(prox.penalty(s, kind, 1.0, 6.0)) / 10.0 + 0.5 * np.sum((Z - A) ** 2)

    f0 = objective(G)
    for scale in (1e-1, 1e-2, 1e-3):
        for _ in range(100):
            assert objective(G + scale * rng.standard_normal(G.shape)) >= f0 - 1e-12


@pytest.mark.parametrize("tk,scale", [("fft", 12.0), ("dct", np.sqrt(12.0))])
def test_slice_constant_tensor_closed_form(tk, scale):
    # every slice equal to A0: only the zero-frequency transformed slice is
    # nonzero, equal to c A0 (c = n for the DFT, sqrt(n) for the DCT), so the
    # l1 result is the matrix SVT of A0 with threshold tau / c in every slice
    rng = np.random.default_rng(9)
    tdims = (4, 3)
    A0 = rng.standard_normal((7, 5))
    A = np.broadcast_to(A0, (12, 7, 5)).copy()
    tau = 2.0
    G, _ = svt.gnhtsvt(A, tdims, tau, prox.L1, transform_kind=tk)
    U, s, Vt = np.linalg.svd(A0, full_matrices=False)
    want = (U * np.maximum(s - tau / scale, 0.0)) @ Vt
    assert np.abs(G - want[None]).max() < 1e-12


def test_dft_transform_needs_the_full_engine():
    with pytest.raises(ValueError):
        svt.gnhtsvt(np.zeros((4, 3, 3)), (4,), 1.0, prox.L1, engine="rsvd", transform_kind="fft",
                    l=2)


def test_hartley_basis_diagonalises_the_difference_operators():
    # the real Hartley matrix H[k, m] = cas(2 pi k m / n)/sqrt(n) is symmetric,
    # orthogonal and its own inverse, and diagonalises every symmetric
    # circulant, D^T D among them (eigenvalues 2 - 2 cos(2 pi k / n)); so the
    # FFT solve of Eq. gnrhtc-L equals real mode products with H
    for n in (5, 8, 20):
        a = 2 * np.pi * np.outer(np.arange(n), np.arange(n)) / n
        H = (np.cos(a) + np.sin(a)) / np.sqrt(n)
        D = ctv.difference_matrix(n)
        lam = 2 - 2 * np.cos(2 * np.pi * np.arange(n) / n)
        assert np.abs(H @ H - np.eye(n)).max() < 1e-13
        assert np.abs(H @ D.T @ D @ H - np.diag(lam)).max() < 1e-12
    rng = np.random.default_rng(10)
    tdims, shape, modes = (6,), (6, 8, 10), (1, 2, 3)
    R0 = rng.standard_normal(shape)
    Rk = {k: rng.standard_normal(shape) for k in modes}
    rhs = R0 + sum(roll_grad_t(Rk[k], tdims, k) for k in modes)

    def hartley(n):
        a = 2 * np.pi * np.outer(np.arange(n), np.arange(n)) / n
        return (np.cos(a) + np.sin(a)) / np.sqrt(n)

    def apply(W):
        W = np.einsum("ab,bij->aij", hartley(6), W)
        W = np.einsum("ia,jab->jib", hartley(8), W)
        return np.einsum("jib,cb->jic", W, hartley(10))

    lam = [2 - 2 * np.cos(2 * np.pi * np.arange(n) / n) for n in (6, 8, 10)]
    den = 1 + lam[0][:, None, None] + lam[1][None, :, None] + lam[2][None, None, :]
    got = apply(apply(rhs) / den)
    assert np.abs(got - ctv.l_update(R0, Rk, tdims, modes)).max() < 1e-12


def test_multipliers_are_subgradients_and_the_loop_reaches_feasibility():
    # convex case (l1 Phi and psi): after every step
    #   Y = 0 off Omega; |Y| <= lambda on Omega, Y = lambda sign(E) where E != 0
    #     (Y' = mu (H - E') with E' the l1 prox of H);
    #   every transformed slice of gamma Lambda_k has spectral norm <= 1 and
    #   <gamma Lambda_k, G_k> equals the transformed nuclear norm of G_k
    #     (Lambda_k' = mu (A - G_k') with G_k' the prox of A, tau = 1/(gamma mu));
    # and the loop ends at a point with nabla_k L = G_k and L + E = M
    rng = np.random.default_rng(3)
    tdims, shape, modes, lam = (6,), (6, 10, 8), (1, 2), 0.3
    X = rng.standard_normal(shape)
    mask = rng.random(shape) < 0.7
    M = np.where(mask, X, 0.0)
    p = ctv.Params(modes=modes, transform="dct", engine="full", phi=prox.L1, psi=prox.L1,
                   noise=admm.NOISE_L1, lam=lam, mu0=0.05, growth=1.1, mu_max=1e6, tol=1e-10,
                   max_iter=600)
    gam = len(modes)
    checked = []

    def check(st, res):
        Y = st.Y
        assert np.abs(Y[~mask]).max() == 0.0
        # Y is formed as Y + mu (M - L - E) with mu up to 1e6, so it carries
        # rounding of order eps * mu: the bounds are 1e-8 relative
        assert np.abs(Y[mask]).max() <= lam * (1 + 1e-8)
        nz = mask & (np.abs(st.E) > 1e-8)
        if nz.any():
            assert np.abs(Y[nz] - lam * np.sign(st.E[nz])).max() <= 1e-8 * lam
        for k in modes:
            W = transform.forward(gam * st.Lam[k], tdims)
            Gb = transform.forward(st.G[k], tdims)
            assert max(np.linalg.norm(W[j], 2) for j in range(W.shape[0])) <= 1 + 1e-8
            inner = sum(np.sum(W[j] * Gb[j]) for j in range(W.shape[0]))
            nuc = sum(np.linalg.svd(Gb[j], compute_uv=False).sum() for j in range(W.shape[0]))
            assert abs(inner - nuc) <= 1e-8 * max(1.0, nuc)
        checked.append(st.t)

    st, hist = ctv.run(M, mask, tdims, p, callback=check)
    assert len(checked) == len(hist) and hist[-1].max() <= 1e-8
    for k in modes:
        assert np.abs(ctv.grad(st.L, tdims, k) - st.G[k]).max() <= 1e-8
    assert np.abs(M - st.L - st.E).max() <= 1e-8


def test_gradient_solve_property_over_random_shapes():
    # any order 2..5, sizes 1..7 (size-1 modes included), any subset of modes:
    # nabla_k is the roll difference, nabla_k^T its adjoint, and the FFT solve
    # satisfies its linear system
    hyp = pytest.importorskip("hypothesis")
    st = hyp.strategies

    @hyp.settings(max_examples=60, deadline=None, derandomize=True)
    @hyp.given(st.lists(st.integers(1, 7), min_size=2, max_size=5), st.data())
    def check(dims, data):
        tdims = tuple(dims[2:])
        n = int(np.prod(tdims)) if tdims else 1
        shape = (n, dims[0], dims[1])
        modes = tuple(sorted(data.draw(st.sets(st.integers(1, len(dims)), min_size=1))))
        rng = np.random.default_rng(len(dims) * 100 + sum(dims))
        X = rng.standard_normal(shape)
        Y = rng.standard_normal(shape)
        for k in range(1, len(dims) + 1):
            assert np.array_equal(ctv.grad(X, tdims, k), roll_grad(X, tdims, k))
            assert abs(np.sum(ctv.grad(X, tdims, k) * Y) - np.sum(X * ctv.grad_t(Y, tdims, k))) \
                < 1e-12 * (1 + np.abs(X).sum() * np.abs(Y).max())
        R0 = rng.standard_normal(shape)
        Rk = {k: rng.standard_normal(shape) for k in modes}
        L = ctv.l_update(R0, Rk, tdims, modes)
        lhs = L + sum(roll_grad_t(roll_grad(L, tdims, k), tdims, k) for k in modes)
        rhs = R0 + sum(roll_grad_t(Rk[k], tdims, k) for k in modes)
        assert np.abs(lhs - rhs).max() < 1e-11 * (1 + np.abs(rhs).max())

    check()


def test_transforms_and_l1_prox_property_over_random_shapes():
    # random slice sizes and transformed modes, DCT and DFT: the inverse undoes
    # the transform, the DFT is numpy's FFT, and the l1 GNHTSVT output G of A
    # satisfies the per-slice optimality of the nuclear-norm prox: every
    # transformed slice of (A - G)/tau has spectral norm <= 1 and is aligned
    # with G's (inner product = nuclear norm)
    hyp = pytest.importorskip("hypothesis")
    st = hyp.strategies

    @hyp.settings(max_examples=40, deadline=None, derandomize=True)
    @hyp.given(st.integers(1, 6), st.integers(1, 6),
               st.lists(st.integers(1, 5), min_size=1, max_size=3),
               st.sampled_from(["dct", "fft"]), st.floats(0.05, 3.0))
    def check(n1, n2, tdims, kind, tau):
        tdims = tuple(tdims)
        n = int(np.prod(tdims))
        rng = np.random.default_rng(n1 * 7 + n2 * 11 + n)
        A = rng.standard_normal((n, n1, n2))
        Ab = transform.forward(A, tdims, kind)
        assert np.abs(transform.inverse(Ab, tdims, kind) - A).max() < 1e-12
        if kind == "fft":
            V = A.reshape(tuple(reversed(tdims)) + (n1, n2))
            ref = np.fft.fftn(V, axes=tuple(range(len(tdims)))).reshape(n, n1, n2)
            assert np.abs(Ab - ref).max() < 1e-11
        G, _ = svt.gnhtsvt(A, tdims, tau, prox.L1, transform_kind=kind)
        Gb = transform.forward(G, tdims, kind)
        Wb = (Ab - Gb) / tau
        for j in range(n):
            assert np.linalg.norm(Wb[j], 2) <= 1 + 1e-9
            nuc = np.linalg.svd(Gb[j], compute_uv=False).sum()
            assert abs(np.vdot(Wb[j], Gb[j]).real - nuc) <= 1e-9 * max(1.0, nuc)

    check()
