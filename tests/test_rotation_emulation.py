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
