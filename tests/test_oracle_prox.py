"""Pins for the scalar proximal maps (Eq. equ_gst1) against brute force."""

import numpy as np
import pytest

from oracle import prox


def _brute(v, mu, kind, theta, gamma):
    # global minimiser of mu*psi(x) + (x-v)^2/2 on a fine grid + local polish
    span = abs(v) + 1.0
    xs = np.linspace(-span, span, 200001)
    f = mu * prox.penalty(xs, kind, theta, gamma) + 0.5 * (xs - v) ** 2
    i = int(np.argmin(f))
    lo, hi = xs[max(i - 1, 0)], xs[min(i + 1, xs.size - 1)]
    for _ in range(60):                     # golden-section on the bracket
        a = lo + 0.382 * (hi - lo)
        b = lo + 0.618 * (hi - lo)
        fa = mu * prox.penalty(a, kind, theta, gamma) + 0.5 * (a - v) ** 2
        fb = mu * prox.penalty(b, kind, theta, gamma) + 0.5 * (b - v) ** 2
        if fa < fb:
            hi = b
        else:
            lo = a
    x = 0.5 * (lo + hi)
    fx = mu * prox.penalty(x, kind, theta, gamma) + 0.5 * (x - v) ** 2
    return x, fx


def _obj(x, v, mu, kind, theta, gamma):
    return float(mu * prox.penalty(x, kind, theta, gamma) + 0.5 * (x - v) ** 2)


@pytest.mark.parametrize("kind", [prox.L1, prox.MCP])
def test_prox_matches_bruteforce(kind):
    rng = np.random.default_rng(11)
    for _ in range(300):
        v = rng.uniform(-6, 6)
        mu = rng.uniform(0.05, 3)
        theta = rng.uniform(0.3, 2)
        gamma = rng.uniform(0.2, 6)          # both gamma > mu and gamma <= mu
        got = float(prox.prox_scalar(v, mu, kind, theta, gamma))
        xb, fb = _brute(v, mu, kind, theta, gamma)
        fg = _obj(got, v, mu, kind, theta, gamma)
        # the closed form is a global minimiser: its objective is never worse
        assert fg <= fb + 1e-9
        # and it is the minimiser itself (away from exact ties)
        if fb < _obj(0.0, v, mu, kind, theta, gamma) - 1e-6 or abs(xb) < 1e-6:
            assert abs(got - xb) < 1e-5 * max(1.0, abs(xb))


def test_l1_closed_form_values():
    v = np.array([-3.0, -1.0, -0.5, 0.0, 0.5, 1.0, 3.0])
    assert np.allclose(prox.prox_scalar(v, 1.0, prox.L1), [-2, 0, 0, 0, 0, 0, 2])


def test_mcp_regimes():
    # gamma > mu: firm shrinkage, continuous at gamma*theta
    g, mu, th = 3.0, 1.0, 1.0
    assert prox.prox_scalar(0.9, mu, prox.MCP, th, g) == 0.0
    assert abs(prox.prox_scalar(2.0, mu, prox.MCP, th, g) - (2.0 - 1.0) / (1 - 1 / 3)) < 1e-15
    assert prox.prox_scalar(3.5, mu, prox.MCP, th, g) == 3.5
    assert abs(prox.prox_scalar(3.0, mu, prox.MCP, th, g) - 3.0) < 1e-12
    # gamma <= mu: hard threshold at theta*sqrt(gamma*mu)
    g, mu = 1.0, 4.0
    assert prox.prox_scalar(1.99, mu, prox.MCP, th, g) == 0.0
    assert prox.prox_scalar(2.01, mu, prox.MCP, th, g) == 2.01


def test_mcp_penalty_continuous_and_flat():
    th, g = 1.5, 2.0
    k = g * th
    a = prox.penalty(k - 1e-9, prox.MCP, th, g)
    b = prox.penalty(k + 1e-9, prox.MCP, th, g)
    assert abs(a - b) < 1e-8
    assert prox.penalty(100.0, prox.MCP, th, g) == g * th * th / 2


def test_gnhtt_entrywise_shape_and_odd_symmetry():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((3, 4, 5))
    E = prox.gnhtt_entrywise(A, 0.4, prox.MCP, 1.0, 2.0)
    assert E.shape == A.shape
    assert np.array_equal(prox.gnhtt_entrywise(-A, 0.4, prox.MCP, 1.0, 2.0), -E)
