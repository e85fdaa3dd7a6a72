"""Periodic differences written as array shifts (numpy.roll), independent of
the oracle's mode-product form: the reference the gradient pins use."""

import numpy as np


def _axis(tdims, k):
    d = 2 + len(tdims)
    return {1: d - 2, 2: d - 1}.get(k, d - k)


def roll_grad(S, tdims, k):
    """(nabla_k S)[i] = S[i + e_k] - S[i] on a slice stack S (n, n1, n2)."""
    n, n1, n2 = S.shape
    V = S.reshape(tuple(reversed(tdims)) + (n1, n2))
    ax = _axis(tdims, k)
    return (np.roll(V, -1, axis=ax) - V).reshape(S.shape)


def roll_grad_t(S, tdims, k):
    """(nabla_k^T S)[i] = S[i - e_k] - S[i]."""
    n, n1, n2 = S.shape
    V = S.reshape(tuple(reversed(tdims)) + (n1, n2))
    ax = _axis(tdims, k)
    return (np.roll(V, 1, axis=ax) - V).reshape(S.shape)
