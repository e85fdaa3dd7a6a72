"""CPU emulation (numpy) of the tube kernels' transform on a tile.

The tube kernels stage a tile of TP positions x n slices (tile[j TP + p],
slice index j with mode 3 fastest) and apply the orthonormal DCT-II along
every transformed mode (Eq. trans) fibre by fibre, folding each fibre by the
cosine symmetry C[k][n-1-m] = (-1)^k C[k][m]:
  forward  y_k = sum_{m<h} C[k][m] (x_m + x_{n-1-m}) for even k, with the
           difference for odd k (the centre of an odd fibre enters once);
  inverse  x_m = E_m + O_m, x_{n-1-m} = E_m - O_m from the even-k and odd-k
           sums of C[k][m] y_k.
The matrix buffer follows the host's layout: per mode, the forward rows
(padded to nkpad entries) and then, for m < h, a row of 2 HK entries holding
C[0][m], C[2][m], ... and C[1][m], C[3][m], ...  This file rebuilds that
buffer, runs the fibre loop with the kernels' index arithmetic and compares
with the oracle's transform, for even and odd mode sizes, one to three
transformed modes, and tiles of one to eight positions."""

import numpy as np
import pytest

from oracle import transform


def _layout(dims):
    nkpad = ((max(dims) + 7) // 8) * 8
    hk = ((nkpad // 2 + 3) // 4) * 4
    off_fwd, off_inv, off = [], [], 0
    for d in dims:
        off_fwd.append(off)
        off += d * nkpad
        off_inv.append(off)
        off += ((d + 1) // 2) * 2 * hk
    mats = np.zeros(max(4, ((off + 3) // 4) * 4))
    for k, d in enumerate(dims):
        U = transform.dct_matrix(d)
        for i in range(d):
            for m in range(d):
                mats[off_fwd[k] + i * nkpad + m] = U[i, m]
                if 2 * m + 1 <= d:
                    mats[off_inv[k] + m * 2 * hk + (i & 1) * hk + i // 2] = U[i, m]
    return mats, nkpad, hk, off_fwd, off_inv


def _tile_transform(tile, dims, TP, inverse):
    mats, NK, HK, off_fwd, off_inv = _layout(dims)
    tile = tile.copy()
    n = int(np.prod(dims))
    strides = np.cumprod([1] + list(dims[:-1]))
    order = range(len(dims) - 1, -1, -1) if inverse else range(len(dims))
    for k in order:
        nk, stp, h = dims[k], int(strides[k]), (dims[k] + 1) // 2
        U0 = off_inv[k] if inverse else off_fwd[k]
        nfib = n // nk
        for w in range(nfib * TP):
            p, f = w % TP, w // TP
            base = ((f % stp) + (f // stp) * (stp * nk)) * TP + p
            step = stp * TP
            a, b = np.zeros(HK), np.zeros(HK)
            if not inverse:
                for m in range(min(h, HK)):
                    x0 = tile[base + m * step]
                    if 2 * m + 1 == nk:
                        a[m] = b[m] = x0
                    else:
                        x1 = tile[base + (nk - 1 - m) * step]
                        a[m], b[m] = x0 + x1, x0 - x1
                for i in range(0, nk, 2):
                    tile[base + i * step] = mats[U0 + i * NK: U0 + i * NK + HK] @ a
                    if i + 1 < nk:
                        tile[base + (i + 1) * step] = mats[U0 + (i + 1) * NK: U0 + (i + 1) * NK + HK] @ b
            else:
                for i in range(HK):
                    a[i] = tile[base + 2 * i * step] if 2 * i < nk else 0.0
                    b[i] = tile[base + (2 * i + 1) * step] if 2 * i + 1 < nk else 0.0
                for m in range(h):
                    row = U0 + m * 2 * HK
                    e, o = mats[row: row + HK] @ a, mats[row + HK: row + 2 * HK] @ b
                    tile[base + m * step] = e + o
                    if 2 * m + 1 != nk:
                        tile[base + (nk - 1 - m) * step] = e - o
    return tile


@pytest.mark.parametrize("dims, TP", [((20, 20), 4), ((5,), 8), ((7, 3), 2), ((4, 9, 2), 4),
                                      ((1,), 1), ((2, 3), 8), ((16,), 4), ((13, 6), 2)])
def test_folded_transform_matches_the_oracle(dims, TP):
    rng = np.random.default_rng(sum(dims) * 10 + TP)
    n = int(np.prod(dims))
    # TP positions of a 1 x TP spatial face: slice stack (n, 1, TP)
    S = rng.standard_normal((n, 1, TP))
    tile = S[:, 0, :].reshape(-1)                       # tile[j TP + p]
    fwd = _tile_transform(tile, dims, TP, inverse=False)
    want = transform.forward(S, dims)[:, 0, :].reshape(-1)
    assert np.abs(fwd - want).max() <= 1e-13 * np.abs(want).max()
    back = _tile_transform(fwd, dims, TP, inverse=True)
    assert np.abs(back - tile).max() <= 1e-13 * np.abs(tile).max()
    want_inv = transform.inverse(S, dims)[:, 0, :].reshape(-1)
    inv = _tile_transform(tile, dims, TP, inverse=True)
    assert np.abs(inv - want_inv).max() <= 1e-13 * np.abs(want_inv).max()
