"""Scalar proximal maps and GNHTT (Sec. 4.2.1), in float64.

Test infrastructure (see the package docstring).

Eq. equ_gst1 defines Prox_{psi,mu}(v) = argmin_x mu*psi(x) + (x - v)^2 / 2.
The paper lists its closed forms only in its (unavailable) supplement, so
they are derived here from the definition and pinned against brute-force
1-D minimisation in the tests:

* l1 (weight theta): psi(x) = theta |x|.  Prox = sign(v) max(|v| - mu theta, 0).
* MCP (Zhang 2010, cited in Sec. 4.1): psi(x) = theta|x| - x^2/(2 gamma) for
  |x| <= gamma theta, gamma theta^2 / 2 beyond.
  - gamma > mu ("firm" shrinkage): 0 for |v| <= mu theta;
    sign(v)(|v| - mu theta)/(1 - mu/gamma) for mu theta < |v| <= gamma theta;
    v for |v| > gamma theta.
  - gamma <= mu: the objective is concave on |x| <= gamma theta, so the
    minimiser is 0 or v; v wins iff v^2/2 > mu gamma theta^2/2, i.e. hard
    thresholding at theta sqrt(gamma mu).

GNHTT with h = l1 (Sec. 4.2.1) applies the scalar prox entrywise.
"""

import numpy as np

L1 = "l1"
MCP = "mcp"


def penalty(x, kind, theta=1.0, gamma=4.0):
    """psi(|x|) for the l1 or MCP penalty (elementwise)."""
    a = np.abs(np.asarray(x, dtype=np.float64))
    if kind == L1:
        return theta * a
    if kind == MCP:
        inner = theta * a - a * a / (2.0 * gamma)
        outer = np.full_like(a, gamma * theta * theta / 2.0)
        return np.where(a <= gamma * theta, inner, outer)
    raise ValueError(kind)


def prox_scalar(v, mu, kind, theta=1.0, gamma=4.0):
    """Prox_{psi,mu}(v) of Eq. equ_gst1, elementwise, for psi = l1 or MCP."""
    v = np.asarray(v, dtype=np.float64)
    a = np.abs(v)
    sgn = np.sign(v)
    if kind == L1:
        return sgn * np.maximum(a - mu * theta, 0.0)
    if kind == MCP:
        if gamma > mu:
            mid = sgn * (a - mu * theta) / (1.0 - mu / gamma)
            out = np.where(a <= mu * theta, 0.0, mid)
            return np.where(a > gamma * theta, v, out)
        thr = theta * np.sqrt(gamma * mu)
        return np.where(a > thr, v, 0.0)
    raise ValueError(kind)


def gnhtt_entrywise(A, lam, kind, theta=1.0, gamma=4.0):
    """GNHTT with h = l1: every entry goes through Prox_{psi,lam} (Sec. 4.2.1)."""
    return prox_scalar(A, lam, kind, theta, gamma)
