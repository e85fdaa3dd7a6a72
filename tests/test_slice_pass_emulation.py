"""CPU emulation (numpy, FP64) of the slice pass as the CUDA path orders it.

The GPU slice pass does not form the SVD of B = Q^T Abar the way the paper
writes it (Alg. 4, randomized branch): it takes R of the QR of B^T = Qb R,
runs a one-sided Jacobi on R^T (R^T J = W, J never formed), reads sigma and
B's left singular vectors U off W's columns, forms the l x l core
C = U diag(Prox(sigma) / sigma) U^T, and rebuilds Gbar = (Q C) B, since
U diag(Prox(sigma)) V^T = U diag(Prox(sigma) / sigma) U^T B.  This file runs
those steps in that order (round-robin pairs, the closed-form rotation, the
sweep-stop rule) and checks them against the oracle's randomized prox on the
same sketch: the restructuring is exact up to rounding, for l1 and MCP, for
rank-deficient slices (sigma = 0 drops out) and for a shrink that removes
every singular value."""

import numpy as np
import pytest

from oracle import philox, prox, svt


def _householder_r(Bt):
    """R (l x l) of the QR of the tall Bt (m x l); Qb is not formed."""
    A = Bt.copy()
    m, l = A.shape
    for k in range(min(m, l)):
        x = A[k:, k]
        nx = np.linalg.norm(x)
        if nx == 0.0:
            continue
        v = x.copy()
        v[0] += np.copysign(nx, x[0])
        v /= np.linalg.norm(v)
        A[k:, k:] -= 2.0 * np.outer(v, v @ A[k:, k:])
    return np.triu(A[:l, :l])


def _jacobi_columns(W, tol, max_sweeps=30):
    """One-sided Jacobi on W's columns in the round-robin order; a pair turns
    while its cosine exceeds tol, and the sweeps stop after one whose cosines
    all stayed below sqrt(tol)."""
    W = W.copy()
    l = W.shape[1]
    lp = l + (l & 1)
    stop = np.sqrt(tol)
    for _ in range(max_sweeps):
        more = False
        for r in range(lp - 1):
            for pi in range(lp // 2):
                a, b = (lp - 1, r) if pi == 0 else ((r + pi) % (lp - 1), (r - pi) % (lp - 1))
                p, q = min(a, b), max(a, b)
                if q >= l:
                    continue
                x, y = W[:, p].copy(), W[:, q].copy()
                al, be, ga = x @ x, y @ y, x @ y
                if ga == 0.0 or abs(ga) <= tol * np.sqrt(al * be):
                    continue
                d = be - al
                h = np.hypot(d, 2.0 * ga)
                qq = h + abs(d)
                rr = 1.0 / np.sqrt(2.0 * h * qq)
                c, s = qq * rr, (2.0 * ga if d >= 0 else -2.0 * ga) * rr
                W[:, p], W[:, q] = c * x - s * y, s * x + c * y
                more |= abs(ga) > stop * np.sqrt(al * be)
        if not more:
            break
    return W


def _slice_pass_as_ordered_on_the_gpu(Ab, Omega, q, tau, kind, theta, gamma):
    Y = Ab @ Omega
    for _ in range(q):
        Q = np.linalg.qr(Y)[0]
        W = np.linalg.qr(Ab.T @ Q)[0]
        Y = Ab @ W
    Q = np.linalg.qr(Y)[0]
    Bt = Ab.T @ Q                                   # P2 holds B^T
    R = _householder_r(Bt)
    l = R.shape[0]
    W = _jacobi_columns(R.T, max(l, 8) * np.finfo(np.float64).eps)
    sigma = np.linalg.norm(W, axis=0)
    U = np.divide(W, sigma, out=np.zeros_like(W), where=sigma > 0)
    shrunk = prox.prox_scalar(sigma, tau, kind, theta, gamma)
    ratio = np.divide(shrunk, sigma, out=np.zeros_like(sigma), where=sigma > 0)
    C = (U * ratio) @ U.T
    Z = Q @ C                                       # P1 <- Q C
    return Z @ Bt.T, np.sort(sigma)[::-1]           # Gbar = Z B


@pytest.mark.parametrize("n1, n2, l, rank, q", [(60, 45, 12, 5, 1), (45, 60, 16, 16, 1),
                                                (50, 50, 20, 8, 0), (33, 70, 9, 3, 2)])
@pytest.mark.parametrize("kind", [prox.L1, prox.MCP])
def test_restructured_core_equals_the_randomized_prox(n1, n2, l, rank, q, kind):
    rng = np.random.default_rng(n1 * 1000 + n2 + l)
    Ab = rng.standard_normal((n1, rank)) @ rng.standard_normal((rank, n2))
    Ab += 1e-3 * rng.standard_normal((n1, n2))
    Omega = philox.gaussian_block(7, 3, 2, n2, l)
    s_top = np.linalg.svd(Ab, compute_uv=False)
    tau = 0.3 * s_top[min(rank, len(s_top)) - 1]
    G0, s0, _ = svt.slice_prox_randomized(Ab, Omega, q, tau, kind, 1.0, 4.0)
    G1, s1 = _slice_pass_as_ordered_on_the_gpu(Ab, Omega, q, tau, kind, 1.0, 4.0)
    assert np.abs(s1 - np.sort(s0)[::-1]).max() <= 1e-12 * s_top[0]
    assert np.linalg.norm(G1 - G0) <= 1e-12 * max(np.linalg.norm(G0), 1.0)


def test_rank_deficient_slice_and_full_shrink():
    rng = np.random.default_rng(5)
    n1, n2, l = 40, 36, 10
    Ab = rng.standard_normal((n1, 3)) @ rng.standard_normal((3, n2))   # rank 3 < l
    Omega = philox.gaussian_block(11, 1, 0, n2, l)
    for tau in (0.5, 1e6):                          # keeps the top three / removes all
        G0, _, _ = svt.slice_prox_randomized(Ab, Omega, 1, tau, prox.L1)
        G1, _ = _slice_pass_as_ordered_on_the_gpu(Ab, Omega, 1, tau, prox.L1, 1.0, 4.0)
        assert np.linalg.norm(G1 - G0) <= 1e-11 * max(np.linalg.norm(Ab), 1.0)
        if tau == 1e6:
            assert not G1.any()
