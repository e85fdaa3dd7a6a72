"""FP32 emulation (numpy, CPU) of the SVD core's closed-form Jacobi rotation.

With d = beta - alpha, h = sqrt(d^2 + 4 gamma^2), q = h + |d| and r = 1/sqrt(2 h q),
c = q r and s = sign(d) 2 gamma r, after d and 2 gamma are scaled by an exact
power of two that brings the larger near 1.  The rotation of the column pair
must zero the pair's inner product, keep c^2 + s^2 = 1, and agree with the
classical t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), zeta = d / (2 gamma),
computed in FP64, across magnitudes from 1e-30 to 1e30."""

import numpy as np

f32 = np.float32


def _scale_pow2(m):
    e = (np.array([m], np.float32).view(np.int32)[0] >> 23) & 0xFF
    e = e if e < 254 else 253
    return np.array([(254 - e) << 23], np.int32).view(np.float32)[0]


def closed_form(al, be, ga):
    d, g2 = f32(be - al), f32(f32(2) * ga)
    sc = _scale_pow2(max(abs(d), abs(g2)))
    dn, gn = f32(d * sc), f32(g2 * sc)
    hh = f32(dn * dn + gn * gn)
    h = f32(hh * f32(1.0 / np.sqrt(np.float64(hh))))
    q = f32(h + abs(dn))
    r = f32(1.0 / np.sqrt(np.float64(f32(f32(2) * h * q))))
    return f32(q * r), f32((gn if d >= 0 else -gn) * r)


def ratio_form(al, be, ga):
    z = (float(be) - float(al)) / (2.0 * float(ga))
    t = np.sign(z if z != 0 else 1.0) / (abs(z) + np.hypot(1.0, z))
    c = 1.0 / np.sqrt(1.0 + t * t)
    return c, c * t


def test_closed_form_rotation_zeroes_the_pair():
    rng = np.random.default_rng(3)
    for _ in range(20000):
        scale = 10.0 ** rng.uniform(-30, 30)
        al, be = (f32(abs(x) * scale) for x in rng.standard_normal(2))
        ga = f32(rng.uniform(-1, 1) * np.sqrt(float(al) * float(be)))
        if ga == 0 or al == 0 or be == 0:
            continue
        c, s = closed_form(al, be, ga)
        # gamma' = (c^2 - s^2) gamma + c s (alpha - beta), relative to sqrt(alpha beta)
        gp = (float(c) ** 2 - float(s) ** 2) * float(ga) + float(c) * float(s) * (float(al) - float(be))
        assert abs(gp) <= 1e-5 * np.sqrt(float(al) * float(be))
        assert abs(float(c) ** 2 + float(s) ** 2 - 1.0) <= 1e-6
        if be != al:
            c0, s0 = ratio_form(al, be, ga)
            assert abs(float(c) - c0) <= 1e-5 and abs(float(s) - s0) <= 1e-5


def test_equal_norms_rotate_by_a_quarter_turn():
    # d = 0: |t| = 1, any sign of gamma
    for ga in (f32(0.5), f32(-0.5), f32(1e-20), f32(-3e20)):
        c, s = closed_form(f32(1.0), f32(1.0), ga)
        assert abs(float(c) - np.sqrt(0.5)) < 1e-6 and abs(abs(float(s)) - np.sqrt(0.5)) < 1e-6


def _round_robin_jacobi(W, tol, stop):
    """FP32 one-sided Jacobi on the columns of W in the kernel's round-robin
    order: a pair rotates while its cosine exceeds tol; another sweep runs
    only while some cosine exceeded `stop`.  Returns (W, sweeps)."""
    W = W.copy()
    l = W.shape[1]
    lp = l + (l & 1)
    for sweep in range(1, 31):
        more = False
        for r in range(lp - 1):
            for pi in range(lp // 2):
                a, b = (lp - 1, r) if pi == 0 else ((r + pi) % (lp - 1), (r - pi) % (lp - 1))
                p, q = min(a, b), max(a, b)
                if q >= l:
                    continue
                x, y = W[:, p].copy(), W[:, q].copy()
                al, be, ga = f32(x @ x), f32(y @ y), f32(x @ y)
                if ga == 0:
                    continue
                cos = f32(abs(ga) / np.sqrt(al) / np.sqrt(be))
                if cos > tol:
                    c, s = closed_form(al, be, ga)
                    W[:, p], W[:, q] = c * x - s * y, s * x + c * y
                    more |= bool(cos > stop)
        if not more:
            return W, sweep
    return W, 30


def test_stopping_after_a_sweep_below_sqrt_tol_keeps_the_accuracy():
    """Cyclic Jacobi converges quadratically: stopping after a sweep whose
    cosines all stayed below sqrt(tol), instead of after a sweep with no
    rotation, drops the confirming sweep and keeps the columns as orthogonal
    (weighted by the singular values, as the rebuild uses them)."""
    rng = np.random.default_rng(11)
    tol = f32(20 * np.finfo(np.float32).eps)
    full_sweeps = early_sweeps = 0
    for trial in range(6):
        n, r, l = 120, 10, 20
        U = np.linalg.qr(rng.standard_normal((n, r)))[0]
        V = np.linalg.qr(rng.standard_normal((n, r)))[0]
        A = (U * np.linspace(10, 3, r)) @ V.T + [1e-3, 0.05, 0.5][trial % 3] * rng.standard_normal((n, n))
        Q = np.linalg.qr(A @ (A.T @ (A @ rng.standard_normal((n, l)))))[0]
        Rt = np.linalg.qr((Q.T @ A).T)[1].T.astype(np.float32)
        sv = np.linalg.svd(Rt.astype(np.float64), compute_uv=False)
        errs = []
        for stop in (tol, np.sqrt(tol)):
            W, sweeps = _round_robin_jacobi(Rt, tol, stop)
            G = W.astype(np.float64).T @ W.astype(np.float64)
            errs.append(np.abs(G - np.diag(np.diag(G))).max() / sv[0] ** 2)
            s = np.sort(np.sqrt(np.diag(G)))[::-1]
            assert np.abs(s - sv).max() <= 1e-5 * sv[0]
            if stop == tol:
                full_sweeps += sweeps
            else:
                early_sweeps += sweeps
        assert errs[1] <= max(4 * errs[0], 4 * float(tol))
    assert early_sweeps < full_sweeps
