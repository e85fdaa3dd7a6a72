"""FP32 emulation (numpy) of the panel QR's Gram-Schmidt rules.

The GPU orthonormalises the sketch panels (Alg. 1's Q = qr(Y) and the power
steps' re-orthonormalisation) by classical Gram-Schmidt with
reorthogonalisation: per pass a column's coefficients against the accepted
columns and its squared norm come from one reduction; the column is kept
after a pass that retained more than half of its squared norm, or a quarter
on the second or a later pass; its norm is taken by Pythagoras from the last
pass; a column still dependent after four passes restarts from a unit vector
(e_{j mod m}, then the next ones).  This file runs those rules in FP32 on
panels shaped like the slice pass's (200 x 20 and 1024 x 48), from a plain
sketch to power-step panels whose columns span eight decades, and on
rank-deficient panels that take the restart path, and checks that Q is
orthonormal to FP32 working precision and, where no column restarts, that
Q R reproduces the panel."""

import numpy as np
import pytest

f32 = np.float32
TINY = np.finfo(np.float32).tiny


def cgs2(P):
    """Q (m x l) and R (l x l) of the FP32 panel P by the kernels' rules."""
    Q = P.astype(np.float32).copy()
    m, l = Q.shape
    R = np.zeros((l, l), np.float32)
    restarted = False
    for j in range(l):
        passes, unit, restarts = 0, -1, 0
        while True:
            coef = Q[:, :j].T @ Q[:, j] if j else np.zeros(0, np.float32)
            sq = f32(Q[:, j] @ Q[:, j])
            csq = f32(coef @ coef) if j else f32(0)
            if j:
                Q[:, j] = Q[:, j] - Q[:, :j] @ coef
            R[:j, j] += coef
            after = f32(sq - csq)
            passes += 1
            if after > TINY and (after > 0.5 * sq or (passes >= 2 and after > 0.25 * sq)):
                break
            if passes >= 4:
                restarts += 1
                if restarts > m:
                    break
                restarted = True
                unit = j % m if unit < 0 else (unit + 1) % m
                Q[:, j] = 0
                Q[unit, j] = 1
                R[:, j] = 0
                passes = 0
        nrm = f32(np.sqrt(max(after, f32(0))))
        R[j, j] = nrm
        Q[:, j] *= f32(1) / nrm if nrm > 0 else f32(0)
    return Q, R, restarted


def _panels(m, l, rng):
    n = m
    A = (rng.standard_normal((n, 10)) * np.logspace(0, -3, 10)) @ rng.standard_normal((10, n))
    A += 1e-4 * rng.standard_normal((n, n))
    Om = rng.standard_normal((n, l))
    Y = A @ Om                                         # sketch
    Y2 = A @ (A.T @ Y)                                 # a power step without re-orthonormalisation
    G = rng.standard_normal((m, l)) * np.logspace(0, -8, l)   # columns over eight decades
    return {"sketch": Y, "power": Y2, "graded": G}


@pytest.mark.parametrize("m, l", [(200, 20), (1024, 48)])
def test_gram_schmidt_twice_is_orthonormal(m, l):
    rng = np.random.default_rng(m + l)
    eps = np.finfo(np.float32).eps
    for name, P in _panels(m, l, rng).items():
        P32 = P.astype(np.float32)
        Q, R, restarted = cgs2(P32)
        orth = np.abs(Q.astype(np.float64).T @ Q - np.eye(l)).max()
        assert orth <= 8 * np.sqrt(m) * eps, (name, orth)
        if not restarted:
            res = np.linalg.norm(Q.astype(np.float64) @ R - P32) / np.linalg.norm(P32)
            assert res <= 8 * np.sqrt(m) * eps, (name, res)


def test_dependent_columns_restart_from_unit_vectors():
    rng = np.random.default_rng(3)
    m, l = 200, 20
    P = rng.standard_normal((m, l)).astype(np.float32)
    P[:, 5] = P[:, 2]                    # a repeated column
    P[:, 9] = 0                          # a zero column
    P[:, 12] = 2 * P[:, 0] - P[:, 1]     # a combination of earlier columns
    Q, R, restarted = cgs2(P)
    assert restarted
    eps = np.finfo(np.float32).eps
    assert np.abs(Q.astype(np.float64).T @ Q - np.eye(l)).max() <= 8 * np.sqrt(m) * eps
    # the independent columns' span is kept: P = Q R on the columns that did not restart
    keep = [c for c in range(l) if c not in (5, 9, 12)]
    span_res = P[:, keep] - Q @ (Q.T @ P[:, keep])
    assert np.linalg.norm(span_res) <= 8 * np.sqrt(m) * eps * np.linalg.norm(P)
