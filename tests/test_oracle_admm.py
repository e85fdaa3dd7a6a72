"""Pins for the oracle's ADMM iteration (Alg. 5, pure-L form)."""

import numpy as np
import pytest

from oracle import admm, prox, svt, transform
from paper_2506_09594_gb300 import synth


def test_exact_recovery_small_tubal_rank():
    # empirical invariant: noise-free completion of a tubal-rank-5 64x64x16
    # tensor from 50% of its entries, run to varpi = 1e-8, recovers X*.
    w = synth.WORKLOADS["tubal64_r5"]
    X, M, mask, _ = synth.make_problem(w)
    p = admm.Params(phi=prox.MCP, psi=prox.MCP, noise=admm.NOISE_NONE, engine="rsvd",
                    l=w.l, q=w.q, seed=7, tol=1e-8, max_iter=400)
    st, hist = admm.run(M, mask, w.tdims, p)
    assert np.max(hist[-1]) <= 1e-8
    assert np.linalg.norm(st.L - X) / np.linalg.norm(X) <= 1e-6


def _convex_problem(seed=0, full=False):
    rng = np.random.default_rng(seed)
    dims = (12, 10, 3, 2)
    n = 6
    X = synth.lowrank_tensor(dims, 2, rng)[0]
    S = np.zeros_like(X)
    idx = rng.permutation(X.size)[: X.size // 20]
    S.flat[idx] = rng.uniform(-3, 3, size=idx.size)
    mask = np.ones(X.size, np.uint8) if full else synth.exact_count_mask(X.size, 0.8, rng)
    mask = mask.reshape(X.shape)
    M = np.where(mask == 1, X + S, 0.0)
    return dims, M, mask


@pytest.mark.parametrize("full,xi", [(True, 3.0), (False, 2.0)])
def test_l1_fixed_point_satisfies_kkt(full, xi):
    # With Phi = psi = l1 the model is convex (T-CTV-TRPCA when Omega is full).
    # At an ADMM fixed point: Lambda = Y; Y in lambda * d||E_Omega||_1 and Y = 0
    # off Omega; Lambda in d||G||_{*,L} (per transformed slice: U1^T Lbar V1 = I,
    # ||Lbar - U1 V1^T||_2 <= 1 with the remainder orthogonal to U1, V1).
    # mu is held fixed (vartheta = 1): then the L-update gives
    # Y - Lambda = mu * O(residual), so the dual conditions become sharp.
    dims, M, mask, = _convex_problem(full=full)
    lam = xi / np.sqrt(max(dims[0], dims[1]) * 6)     # a fixed lambda: KKT holds for any
    p = admm.Params(phi=prox.L1, psi=prox.L1, noise=admm.NOISE_L1, lam=lam,
                    engine="full", tol=1e-10, max_iter=5000, mu0=1.0, growth=1.0)
    st, hist = admm.run(M, mask, dims[2:], p)
    assert np.max(hist[-1]) <= 1e-10
    om = mask.astype(bool)
    tol = 1e-6
    assert np.max(np.abs(st.Lam - st.Y)) < tol
    if (~om).any():
        assert np.max(np.abs(st.Y[~om])) < tol
    Yo, Eo = st.Y[om], st.E[om]
    assert np.max(np.abs(Yo)) <= lam * (1 + 1e-6)
    big = np.abs(Eo) > 1e-6
    assert np.max(np.abs(Yo[big] - lam * np.sign(Eo[big]))) < tol * 10
    Gb = transform.forward(st.G, dims[2:])
    Lb = transform.forward(st.Lam, dims[2:])
    for j in range(Gb.shape[0]):
        U, s, Vt = np.linalg.svd(Gb[j])
        k = int(np.sum(s > 1e-8))
        assert k == 2                     # the planted transform-domain rank
        U1, V1 = U[:, :k], Vt[:k].T
        assert np.max(np.abs(U1.T @ Lb[j] @ V1 - np.eye(k))) < 1e-5
        W = Lb[j] - U1 @ V1.T
        assert np.linalg.norm(W, 2) <= 1 + 1e-5
    # and the constraint holds
    assert np.max(np.abs(M - st.L - st.E)) < 1e-9


def test_residuals_decay_and_multiplier_support():
    w = synth.WORKLOADS["tubal64_r5"]
    X, M, mask, _ = synth.make_problem(w)
    p = admm.Params(phi=prox.L1, psi=prox.L1, noise=admm.NOISE_NONE, engine="rsvd",
                    l=15, q=1, seed=3, tol=0.0, max_iter=120)
    st, hist = admm.run(M, mask, w.tdims, p)
    mx = hist.max(axis=1)
    assert mx[-1] < 1e-3 * mx[:10].max()
    om = mask.astype(bool)
    assert np.max(np.abs(st.Y[~om])) == 0.0          # E absorbs Omega-perp exactly
    assert np.max(np.abs(st.E[om])) == 0.0           # noise-free: E = 0 on Omega


def test_mu_schedule():
    st = admm.init_state((1, 2, 2), 1e-3)
    p = admm.Params(engine="full", mu_max=2e-3, growth=1.5)
    M = np.zeros((1, 2, 2)); mask = np.ones((1, 2, 2), np.uint8)
    mus = []
    for _ in range(4):
        st, _ = admm.step(st, M, mask, (), p)
        mus.append(st.mu)
    assert np.allclose(mus, [1.5e-3, 2e-3, 2e-3, 2e-3])


def test_default_lambda_keeps_the_papers_balance_under_the_orthonormal_transform():
    # Sec. 6: lambda_FFT = xi / sqrt(max(n1,n2) n) with rho = n; with the
    # orthonormal transform (rho = 1) the TNN of a tensor is sqrt(n) times its
    # FFT-convention TNN, so the equivalent lambda is sqrt(n) * lambda_FFT.
    n1, n2, tdims = 200, 100, (20, 20)
    n = 400
    lam_fft = 2.0 / np.sqrt(max(n1, n2) * n)
    assert abs(admm.default_lambda(n1, n2, tdims, 2.0) - np.sqrt(n) * lam_fft) < 1e-15
    # the TNN scaling itself: for a real tensor, the unnormalised DFT along the
    # slice modes scales every transformed slice's Frobenius norm by sqrt(n) on
    # average, while the orthonormal DCT preserves it
    rng = np.random.default_rng(0)
    S = rng.standard_normal((n, 6, 5))
    F = np.fft.fft(np.fft.fft(S.reshape(20, 20, 6, 5), axis=0), axis=1).reshape(n, 6, 5)
    D = transform.forward(S, tdims)
    assert abs(np.linalg.norm(F) / np.linalg.norm(D) - np.sqrt(n)) < 1e-9


def test_first_step_from_zero_state_closed_form():
    # from the zero state: L^1 = M/2, G^1 = D_{1/mu}(M/2), H = M/2,
    # E^1 = Prox_{lam/mu}(M/2) on Omega and 0 off it (M = 0 there)
    w = synth.WORKLOADS["tubal64_r5"]
    _, M, mask, _ = synth.make_problem(w)
    p = admm.Params(phi=prox.L1, psi=prox.L1, noise=admm.NOISE_L1, lam=0.3,
                    engine="full", mu0=0.5)
    st, _ = admm.step(admm.init_state(M.shape, 0.5), M, mask, w.tdims, p)
    assert np.array_equal(st.L, M / 2)
    G, _ = svt.gnhtsvt(M / 2, w.tdims, 2.0, prox.L1)
    assert np.max(np.abs(st.G - G)) < 1e-12
    E = np.where(mask == 1, np.sign(M / 2) * np.maximum(np.abs(M / 2) - 0.6, 0), 0)
    assert np.max(np.abs(st.E - E)) < 1e-15
    assert np.max(np.abs(st.Y - 0.5 * (M - M / 2 - E))) < 1e-15


def test_every_step_satisfies_the_dual_identities_property():
    # Alg. 5 with nabla = I on random shapes, both engines, both noise models:
    # from the L-update 2L = (M - E + Y/mu) + (G - Lam/mu) and the multiplier
    # updates, every step gives Y' - Lam' = mu (E - E') + mu (G' - G), and
    # Y' = 0 off Omega (E = H there)
    hyp = pytest.importorskip("hypothesis")
    st = hyp.strategies

    @hyp.settings(max_examples=30, deadline=None, derandomize=True)
    @hyp.given(st.integers(2, 9), st.integers(2, 9), st.lists(st.integers(1, 4), min_size=1,
                                                                max_size=2), st.data())
    def check(n1, n2, tdims, data):
        tdims = tuple(tdims)
        n = int(np.prod(tdims))
        engine = data.draw(st.sampled_from(["full", "rsvd"]))
        noise = data.draw(st.sampled_from([admm.NOISE_L1, admm.NOISE_NONE]))
        rng = np.random.default_rng(n1 * 31 + n2 * 7 + n)
        X = rng.standard_normal((n, n1, n2))
        mask = rng.random(X.shape) < 0.6
        M = np.where(mask, X, 0.0)
        p = admm.Params(engine=engine, l=3, q=1, seed=4, noise=noise, lam=0.3, mu0=0.2,
                        phi=prox.MCP, phi_gamma=20.0, psi=prox.MCP, psi_gamma=20.0)
        s = admm.init_state(M.shape, p.mu0)
        for _ in range(4):
            new, _ = admm.step(s, M, mask, tdims, p)
            lhs = new.Y - new.Lam
            rhs = s.mu * (s.E - new.E) + s.mu * (new.G - s.G)
            assert np.abs(lhs - rhs).max() <= 1e-10 * max(1.0, np.abs(new.Y).max())
            assert np.abs(new.Y[~mask]).max() <= 1e-12 * max(1.0, np.abs(new.Y).max())
            s = new

    check()
