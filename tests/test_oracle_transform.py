"""Pins for the oracle's transform L (orthonormal DCT-II along modes 3..d)."""

import numpy as np
import scipy.fft

from oracle import transform


def test_dct_matrix_orthonormal():
    for n in [1, 2, 3, 16, 20, 64]:
        U = transform.dct_matrix(n)
        assert np.max(np.abs(U @ U.T - np.eye(n))) < 1e-14
        assert np.max(np.abs(U.T @ U - np.eye(n))) < 1e-14


def test_dct_matrix_matches_scipy():
    # scipy's DCT-II with norm="ortho" applied to the identity's columns
    for n in [2, 5, 16, 20]:
        ref = scipy.fft.dct(np.eye(n), type=2, norm="ortho", axis=0)
        assert np.max(np.abs(transform.dct_matrix(n) - ref)) < 1e-14


def test_forward_matches_scipy_dct_along_modes():
    rng = np.random.default_rng(0)
    dims = (5, 7, 4, 3)
    X = rng.standard_normal(dims)
    S = transform.slices_from_tensor(X)
    Sb = transform.forward(S, dims[2:])
    ref = scipy.fft.dct(scipy.fft.dct(X, type=2, norm="ortho", axis=2),
                        type=2, norm="ortho", axis=3)
    assert np.max(np.abs(transform.tensor_from_slices(Sb, dims[2:]) - ref)) < 1e-13


def test_inverse_undoes_forward():
    rng = np.random.default_rng(1)
    for dims in [(3, 4, 6), (6, 5, 4, 3), (2, 3, 2, 3, 4)]:
        S = rng.standard_normal((int(np.prod(dims[2:])), dims[0], dims[1]))
        back = transform.inverse(transform.forward(S, dims[2:]), dims[2:])
        assert np.linalg.norm(back - S) / np.linalg.norm(S) < 1e-14


def test_face_slice_order_i3_fastest():
    rng = np.random.default_rng(2)
    dims = (3, 2, 4, 5)
    X = rng.standard_normal(dims)
    S = transform.slices_from_tensor(X)
    for i3 in range(4):
        for i4 in range(5):
            assert np.array_equal(S[i3 + 4 * i4], X[:, :, i3, i4])
    assert np.array_equal(transform.tensor_from_slices(S, dims[2:]), X)


def test_constant_tube_maps_to_dc_slice():
    # a tensor constant along modes 3,4 has only the (0,0) transformed slice,
    # equal to sqrt(n3*n4) times the value (closed form of the DCT-II DC row)
    n3, n4 = 6, 5
    base = np.arange(12.0).reshape(3, 4)
    S = np.broadcast_to(base, (n3 * n4, 3, 4)).copy()
    Sb = transform.forward(S, (n3, n4))
    assert np.allclose(Sb[0], np.sqrt(n3 * n4) * base, atol=1e-12)
    assert np.max(np.abs(Sb[1:])) < 1e-12


def test_transform_preserves_frobenius_norm():
    rng = np.random.default_rng(3)
    S = rng.standard_normal((24, 7, 3))
    assert abs(np.linalg.norm(transform.forward(S, (4, 6))) - np.linalg.norm(S)) < 1e-12


def test_dft_forward_matches_numpy_fft_along_modes():
    # kind="fft": x_3 F_{n3} x_4 F_{n4} is numpy's unnormalised FFT along
    # modes 3 and 4 (Eq. trans with the DFT); F F^H = n I (Eq. orth, alpha = n)
    rng = np.random.default_rng(4)
    dims = (4, 3, 5, 6)
    X = rng.standard_normal(dims)
    S = transform.slices_from_tensor(X)
    Sb = transform.forward(S, dims[2:], kind="fft")
    ref = np.fft.fftn(X, axes=(2, 3))
    assert np.max(np.abs(transform.tensor_from_slices(Sb, dims[2:]) - ref)) < 1e-12
    for n in [1, 3, 8]:
        F = transform.dft_matrix(n)
        assert np.max(np.abs(F @ F.conj().T - n * np.eye(n))) < 1e-12
    assert transform.rho(dims[2:], "fft") == 30.0 and transform.rho(dims[2:]) == 1.0


def test_dft_inverse_matches_numpy_ifft_and_undoes_forward():
    rng = np.random.default_rng(5)
    dims = (3, 4, 2, 5, 3)
    S = rng.standard_normal((30, 3, 4)) + 1j * rng.standard_normal((30, 3, 4))
    X = transform.tensor_from_slices(S, dims[2:])
    got = transform.tensor_from_slices(transform.inverse(S, dims[2:], kind="fft"), dims[2:])
    assert np.max(np.abs(got - np.fft.ifftn(X, axes=(2, 3, 4)))) < 1e-13
    back = transform.inverse(transform.forward(S, dims[2:], kind="fft"), dims[2:], kind="fft")
    assert np.linalg.norm(back - S) / np.linalg.norm(S) < 1e-14
