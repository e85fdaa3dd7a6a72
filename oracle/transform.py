"""The invertible transform L and face slices (Sec. 2), in float64.

Test infrastructure (see the package docstring).

Layout.  An order-d tensor X (n1 x n2 x n3 x ... x nd) is held as its stack
of face slices S with shape (n, n1, n2), n = n3*...*nd, where
S[j] = X^<j> = X(:, :, i3, ..., id) and (0-based)
j = i3 + n3*(i4 + n4*(i5 + ...))  -- i3 varies fastest (Sec. 2, definition
of the face slice).  Viewing S as an array of shape (nd, ..., n4, n3, n1, n2)
in C order exposes one axis per transformed mode.

Transform (Eq. trans): L(X) = X x_3 U_{n3} x_4 U_{n4} ... x_d U_{nd}, with
U U^H = U^H U = alpha I (Eq. orth).  Here U_n is the orthonormal DCT-II
matrix U[k, m] = s_k cos(pi (2m + 1) k / (2n)), s_0 = sqrt(1/n),
s_k = sqrt(2/n) for k > 0, so alpha = 1 and U^{-1} = U^T.  The inverse
applies U^{-1} mode by mode from d down to 3 (Sec. 2).

kind="fft" takes instead the DFT matrix F_n[k, m] = exp(-2 pi i k m / n), the
transform of the paper's experiments: F F^H = n I, so alpha = n,
rho = n3 ... nd and F^{-1} = F^H / n; transformed slices are complex.
"""

import numpy as np


def dct_matrix(n):
    """Orthonormal DCT-II matrix U_n (n x n): U[k, m] = s_k cos(pi(2m+1)k/(2n))."""
    k = np.arange(n, dtype=np.float64)[:, None]
    m = np.arange(n, dtype=np.float64)[None, :]
    s = np.full((n, 1), np.sqrt(2.0 / n))
    s[0, 0] = np.sqrt(1.0 / n)
    return s * np.cos(np.pi * (2.0 * m + 1.0) * k / (2.0 * n))


def dft_matrix(n):
    """DFT matrix F_n (n x n): F[k, m] = exp(-2 pi i k m / n), F F^H = n I."""
    k = np.arange(n, dtype=np.float64)[:, None]
    m = np.arange(n, dtype=np.float64)[None, :]
    return np.exp(-2j * np.pi * k * m / n)


def _matrix(kind, n):
    if kind == "dct":
        return dct_matrix(n)
    if kind == "fft":
        return dft_matrix(n)
    raise ValueError(kind)


def _inverse_matrix(kind, n):
    if kind == "dct":
        return dct_matrix(n).T
    if kind == "fft":
        return dft_matrix(n).conj().T / n
    raise ValueError(kind)


def rho(tdims, kind="dct"):
    """rho = alpha_3 ... alpha_d: 1 for the orthonormal DCT, n3 ... nd for the DFT."""
    return 1.0 if kind == "dct" else float(num_slices(tdims))


def _as_array(S):
    S = np.asarray(S)
    return S.astype(np.complex128 if np.iscomplexobj(S) else np.float64)


def num_slices(tdims):
    n = 1
    for v in tdims:
        n *= int(v)
    return n


def _mode_axis(tdims, mode):
    """Axis of transformed mode `mode` (3..d) in the (nd,...,n3,n1,n2) view."""
    d = 2 + len(tdims)
    return d - mode   # mode 3 -> axis d-3 (just before n1), mode d -> axis 0


def mode_product(Xv, U, axis):
    """Mode product along `axis`: out[.., a, ..] = sum_b U[a, b] X[.., b, ..]."""
    out = np.tensordot(U, Xv, axes=([1], [axis]))   # new axis first
    return np.moveaxis(out, 0, axis)


def forward(S, tdims, kind="dct"):
    """L(X) on a slice stack S (n, n1, n2): x_3 U_3, then x_4 U_4, ..., x_d U_d."""
    n, n1, n2 = S.shape
    assert n == num_slices(tdims)
    Xv = _as_array(S).reshape(tuple(reversed(tdims)) + (n1, n2))
    for mode in range(3, 3 + len(tdims)):
        U = _matrix(kind, tdims[mode - 3])
        Xv = mode_product(Xv, U, _mode_axis(tdims, mode))
    return Xv.reshape(n, n1, n2)


def inverse(S, tdims, kind="dct"):
    """L^{-1}(X) = X x_d U_d^{-1} ... x_3 U_3^{-1}; U^{-1} = U^T for the DCT,
    F^H / n for the DFT."""
    n, n1, n2 = S.shape
    assert n == num_slices(tdims)
    Xv = _as_array(S).reshape(tuple(reversed(tdims)) + (n1, n2))
    for mode in range(2 + len(tdims), 2, -1):
        Ui = _inverse_matrix(kind, tdims[mode - 3])
        Xv = mode_product(Xv, Ui, _mode_axis(tdims, mode))
    return Xv.reshape(n, n1, n2)


def slices_from_tensor(X):
    """Face-slice stack (n, n1, n2) of a tensor given in mode order (n1, ..., nd)."""
    n1, n2 = X.shape[0], X.shape[1]
    rest = X.reshape(n1, n2, -1, order="F")         # j = i3 + n3*i4 + ...
    return np.ascontiguousarray(np.moveaxis(rest, 2, 0))


def tensor_from_slices(S, tdims):
    """Inverse of slices_from_tensor."""
    n, n1, n2 = S.shape
    rest = np.moveaxis(S, 0, 2)                       # (n1, n2, n)
    return rest.reshape((n1, n2) + tuple(tdims), order="F")
