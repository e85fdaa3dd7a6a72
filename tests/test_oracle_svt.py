"""Pins for the oracle's GNHTSVT and its low-rank engines."""

import itertools

import numpy as np
import pytest

from oracle import philox, prox, svt, transform
from paper_2506_09594_gb300 import synth


def _stack(seed, n, n1, n2):
    return np.random.default_rng(seed).standard_normal((n, n1, n2))


# ------------------------------------------------------------------ l1
def test_l1_gnhtsvt_satisfies_subgradient_optimality():
    # D_tau(A) for l1 is the unique minimiser of a strongly convex problem
    # (Theorem theorem_wtsvt); its optimality condition per transformed slice:
    # (Abar - Gbar)/tau = U1 V1^T + W, ||W||_2 <= 1, U1^T W = 0, W V1 = 0.
    tdims = (3, 2)
    A = _stack(0, 6, 9, 7) * 3
    tau = 6.0
    G, _ = svt.gnhtsvt(A, tdims, tau, prox.L1)
    Ab, Gb = transform.forward(A, tdims), transform.forward(G, tdims)
    for j in range(6):
        U, s, Vt = np.linalg.svd(Gb[j])
        k = int(np.sum(s > 1e-9))
        assert 0 < k < 7
        U1, V1 = U[:, :k], Vt[:k].T
        R = (Ab[j] - Gb[j]) / tau
        W = R - U1 @ V1.T
        assert np.max(np.abs(U1.T @ W)) < 1e-10
        assert np.max(np.abs(W @ V1)) < 1e-10
        assert np.linalg.norm(W, 2) <= 1 + 1e-10


def test_l1_order2_is_matrix_svt_via_eigh():
    # order 2 (no transformed mode): D_tau(A) = A f(A^T A),
    # f(lambda) = max(1 - tau/sqrt(lambda), 0), computed with eigh instead of svd
    rng = np.random.default_rng(4)
    A = rng.standard_normal((1, 8, 5)) * 2
    tau = 1.3
    G, _ = svt.gnhtsvt(A, (), tau, prox.L1)
    lam, V = np.linalg.eigh(A[0].T @ A[0])
    f = np.where(lam > 0, np.maximum(1 - tau / np.sqrt(np.maximum(lam, 1e-300)), 0), 0)
    ref = A[0] @ (V * f) @ V.T
    assert np.max(np.abs(G[0] - ref)) < 1e-12


@pytest.mark.parametrize("kind", [prox.L1, prox.MCP])
def test_gnhtsvt_beats_perturbations(kind):
    # Theorem theorem_wtsvt: D_{Phi,tau}(A) minimises tau||G||_{Phi,L} + ||G-A||^2/2
    rng = np.random.default_rng(7)
    for dims in [(4, 3, 2), (5, 5, 3)]:
        n = int(np.prod(dims[2:]))
        A = rng.standard_normal((n, dims[0], dims[1])) * 2
        tau, theta, gamma = 0.8, 1.0, 2.5
        G, _ = svt.gnhtsvt(A, dims[2:], tau, kind, theta, gamma)
        f0 = svt.objective(G, A, dims[2:], tau, kind, theta, gamma)
        for _ in range(300):
            P = G + rng.standard_normal(G.shape) * rng.choice([1e-3, 1e-2, 1e-1, 1.0])
            assert f0 <= svt.objective(P, A, dims[2:], tau, kind, theta, gamma) + 1e-10


def test_mcp_gnhtsvt_beats_keep_k_truncations():
    rng = np.random.default_rng(8)
    dims = (5, 5, 3)
    A = rng.standard_normal((3, 5, 5)) * 2
    tau, theta, gamma = 1.0, 1.0, 1.5          # gamma > tau: firm regime
    G, _ = svt.gnhtsvt(A, dims[2:], tau, prox.MCP, theta, gamma)
    f0 = svt.objective(G, A, dims[2:], tau, prox.MCP, theta, gamma)
    Ab = transform.forward(A, dims[2:])
    svds = [np.linalg.svd(Ab[j]) for j in range(3)]
    for ks in itertools.product(range(6), repeat=3):   # keep top-k per slice
        Tb = np.stack([(u[:, :k] * s[:k]) @ vt[:k] for (u, s, vt), k in zip(svds, ks)])
        T = transform.inverse(Tb, dims[2:])
        assert f0 <= svt.objective(T, A, dims[2:], tau, prox.MCP, theta, gamma) + 1e-10


# ------------------------------------------------------------ randomized
@pytest.mark.parametrize("kind", [prox.L1, prox.MCP])
def test_randomized_equals_exact_on_low_rank_slices(kind):
    # rank(Abar^<j>) <= l: Q Q^T Abar = Abar almost surely, so the randomized
    # prox equals the deterministic one
    n, n1, n2, r, l = 16, 64, 64, 5, 15
    Ab = synth.lowrank_plus_noise_stack(n, n1, n2, r, 0.0, seed=3)
    tau = 0.7
    Gf, _ = svt.transformed_prox(Ab, tau, kind, 1.0, 40.0, engine="full")
    Gr, _ = svt.transformed_prox(Ab, tau, kind, 1.0, 40.0, engine="rsvd", l=l, q=1,
                                 seed=5, t=2)
    assert np.linalg.norm(Gr - Gf) / np.linalg.norm(Gf) < 1e-12
    Gk = np.stack([svt.slice_prox_krylov(Ab[j], philox.gaussian_block(5, 2, j, n2, 4),
                                         1, 8, tau, kind, 1.0, 40.0)[0] for j in range(n)])
    assert np.linalg.norm(Gk - Gf) / np.linalg.norm(Gf) < 1e-12


def test_randomized_l1_within_nonexpansive_certificate():
    # ||D(Abar) - D(QQ^T Abar)|| <= ||Abar - QQ^T Abar|| = sqrt(||Abar||^2 - ||B||^2)
    n, n1, n2 = 12, 60, 50
    Ab = synth.lowrank_plus_noise_stack(n, n1, n2, np.arange(n) + 3, 0.3, seed=9)
    for q in [0, 1, 2]:
        Gf, _ = svt.transformed_prox(Ab, 2.0, prox.L1, engine="full")
        Gr, info = svt.transformed_prox(Ab, 2.0, prox.L1, engine="rsvd", l=12, q=q,
                                        seed=1, t=0)
        for j in range(n):
            resid = np.sqrt(max(np.sum(Ab[j] ** 2) - np.sum(info["sigma"][j] ** 2), 0.0))
            assert np.linalg.norm(Gf[j] - Gr[j]) <= resid + 1e-9


def test_power_iterations_improve_basis():
    n1, n2 = 120, 100
    Ab = synth.lowrank_plus_noise_stack(1, n1, n2, 10, 0.5, seed=2)[0]
    errs = []
    for q in [0, 1, 2]:
        Om = philox.gaussian_block(3, 0, 0, n2, 14)
        _, s, _ = svt.slice_prox_randomized(Ab, Om, q, 0.0, prox.L1)
        errs.append(np.sum(Ab ** 2) - np.sum(s ** 2))
    assert errs[0] > errs[1] > errs[2] > 0


def test_randomized_sketch_wider_than_slice_is_exact():
    n1, n2 = 9, 6
    Ab = np.random.default_rng(1).standard_normal((2, n1, n2))
    Gf, _ = svt.transformed_prox(Ab, 0.5, prox.L1, engine="full")
    Gr, _ = svt.transformed_prox(Ab, 0.5, prox.L1, engine="rsvd", l=50, q=1, seed=0)
    assert np.max(np.abs(Gf - Gr)) < 1e-12


# -------------------------------------------------------------- adaptive
def test_defl_qr_reconstructs_and_deflates():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((20, 3)) @ rng.standard_normal((3, 6))   # rank 3
    Q, R, s = svt.defl_qr(A, 1e-10)
    assert s == 3
    assert np.max(np.abs(Q @ R - A)) < 1e-12
    assert np.max(np.abs(Q.T @ Q - np.eye(3))) < 1e-13


def test_adaptive_error_indicator_is_true_residual():
    # Theorem on Alg. 3: E equals ||A - U U^T A||_F^2 while orthogonality holds
    Ab = synth.lowrank_plus_noise_stack(1, 80, 70, 12, 0.05, seed=4)[0]
    for eps in [0.3, 0.1, 0.01]:
        U, E, hist = svt.adaptive_basis(Ab, eps, 4, 1e-12, seed=1, t=0, j=0)
        true = np.sum((Ab - U @ (U.T @ Ab)) ** 2)
        assert abs(E - true) <= 1e-9 * np.sum(Ab ** 2)
        assert np.max(np.abs(U.T @ U - np.eye(U.shape[1]))) < 1e-10
        assert true < eps ** 2 * np.sum(Ab ** 2) or U.shape[1] == 70
        # never better than the optimal rank-k error (brute-force SVD truncation)
        s = np.linalg.svd(Ab, compute_uv=False)
        assert true >= np.sum(s[U.shape[1]:] ** 2) - 1e-9


def test_adaptive_exact_rank_is_found_and_prox_exact():
    Ab = synth.lowrank_plus_noise_stack(4, 50, 40, [3, 7, 1, 11], 0.0, seed=6)
    Gf, _ = svt.transformed_prox(Ab, 0.5, prox.MCP, 1.0, 5.0, engine="full")
    Ga, info = svt.transformed_prox(Ab, 0.5, prox.MCP, 1.0, 5.0, engine="adaptive",
                                    eps=1e-6, b=4, seed=2, t=0)
    assert np.linalg.norm(Ga - Gf) / np.linalg.norm(Gf) < 1e-10


def test_adaptive_deflation_refills_block():
    # a rank-2 slice with block size 5: defl-QR keeps 2 columns, refill keeps b
    Ab = synth.lowrank_plus_noise_stack(1, 30, 25, 2, 0.0, seed=7)[0]
    U, E, hist = svt.adaptive_basis(Ab, 1e-8, 5, 1e-12, seed=1, t=0, j=0)
    assert U.shape[1] >= 2
    assert np.sum((Ab - U @ (U.T @ Ab)) ** 2) < 1e-20 * max(1.0, np.sum(Ab ** 2)) + 1e-18


def test_randomized_prox_is_exact_when_the_sketch_covers_the_rank_property():
    # any slice shape, slice ranks from 0 (a zero slice) to the sketch width,
    # widths above min(n1, n2) (clamped), q = 0..2, l1 and MCP: the randomized
    # prox equals the full-SVD prox, slice by slice
    hyp = pytest.importorskip("hypothesis")
    st = hyp.strategies

    @hyp.settings(max_examples=50, deadline=None, derandomize=True)
    @hyp.given(st.integers(1, 4), st.integers(1, 12), st.integers(1, 12), st.data())
    def check(n, n1, n2, data):
        l = data.draw(st.integers(1, 14))
        q = data.draw(st.integers(0, 2))
        kind = data.draw(st.sampled_from([prox.L1, prox.MCP]))
        ll = min(l, n1, n2)
        rng = np.random.default_rng(n * 400 + n1 * 20 + n2 + l)
        Ab = np.zeros((n, n1, n2))
        for j in range(n):
            r = int(rng.integers(0, ll + 1))
            Ab[j] = rng.standard_normal((n1, r)) @ rng.standard_normal((r, n2))
        got, _ = svt.transformed_prox(Ab, 0.7, kind, gamma=20.0, engine="rsvd", l=l, q=q, seed=3,
                                      t=1)
        want, _ = svt.transformed_prox(Ab, 0.7, kind, gamma=20.0)
        assert np.abs(got - want).max() <= 1e-9 * max(1.0, np.abs(want).max())

    check()


def test_adaptive_basis_finds_the_rank_property():
    # Alg. 3 per slice on any shape, rank (0 included) and block size: with
    # eps = 1e-6 the basis has exactly the slice's rank, captures the slice,
    # and the prox through it is the full-SVD prox
    hyp = pytest.importorskip("hypothesis")
    st = hyp.strategies

    @hyp.settings(max_examples=40, deadline=None, derandomize=True)
    @hyp.given(st.integers(2, 30), st.integers(2, 30), st.data())
    def check(n1, n2, data):
        r = data.draw(st.integers(0, min(n1, n2) - 1))
        b = data.draw(st.integers(1, 8))
        rng = np.random.default_rng(n1 * 40 + n2 + 1000 * r + b)
        A = rng.standard_normal((n1, r)) @ rng.standard_normal((r, n2))
        U, E, _ = svt.adaptive_basis(A, 1e-6, b, 1e-12, seed=5, t=1, j=0)
        assert U.shape[1] == r
        if r:
            assert np.linalg.norm(A - U @ (U.T @ A)) <= 1e-9 * np.linalg.norm(A)
        G, _, _, _, _ = svt.slice_prox_adaptive(A, 1e-6, b, 1e-12, 5, 1, 0, 0.5, prox.L1)
        want, _, _ = svt.slice_prox_full(A, 0.5, prox.L1)
        assert np.abs(G - want).max() <= 1e-9 * max(1.0, np.abs(want).max())

    check()


@pytest.mark.parametrize("kind", [prox.L1, prox.MCP])
def test_learned_engine_exact_for_any_widths_on_low_rank_slices(kind):
    # Exactly low-rank slices: a sketch at least as wide as the rank captures
    # the slice (E = 0, kept by Alg. 3's test), a narrower one misses energy
    # and keeps its whole width (no oversampling margin, below the cap), so
    # it is rejected and the adaptive engine finds the exact rank.  Either
    # way each slice's prox is the deterministic one, and the rejected
    # slices are exactly those sketched below their rank.
    ranks = [3, 9, 5, 12, 1, 7]
    Ab = synth.lowrank_plus_noise_stack(6, 40, 32, ranks, 0.0, seed=31)
    widths = [8, 8, 16, 8, 8, 16]
    tau = 0.3
    full, _ = svt.transformed_prox(Ab, tau, kind, 1.0, 5.0, engine="full")
    got, info = svt.transformed_prox(Ab, tau, kind, 1.0, 5.0, engine="learned", widths=widths,
                                     q=1, seed=4, t=2, eps=1e-3, b=4, delta_rel=1e-11,
                                     max_rank=24, p=4)
    assert np.linalg.norm(got - full) <= 1e-10 * np.linalg.norm(full)
    assert info["fallback"].tolist() == [1, 3]
    # rejected slices take the adaptive basis (the rank), kept ones the sketch
    assert info["widths"].tolist() == [8, 9, 16, 12, 8, 16]
    # a cap at the narrowest width keeps every sketch
    _, info = svt.transformed_prox(Ab, tau, kind, 1.0, 5.0, engine="learned", widths=widths,
                                   q=1, seed=4, t=2, eps=1e-3, b=4, delta_rel=1e-11,
                                   max_rank=8, p=4)
    assert info["fallback"].tolist() == []
