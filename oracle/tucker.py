"""Randomized GNHTSVT with shared Tucker factors, in float64.

Test infrastructure (see the package docstring).

Alg. 4, randomized branch: the tensor A is first compressed by a Tucker
decomposition A ~ [C; F_1, F_2] computed by Alg. 1 (R-STHOSVD-BKI), the
deterministic GNTSVT is applied to the core, and the result is mapped back
with the factors:

    D_{Phi,tau}(A, L) ~ D_{Phi,tau}(C, L) x_1 F_1 x_2 F_2.

Here the processing order of Alg. 1 is rho = (1, 2): the two spatial modes
of the face slices get shared factors, the transformed modes 3..d keep
their full size, so L acts on the core exactly as on A.  For one mode
(Alg. 1, loop body), with A the mode unfolding of the current core C:

    K = [A G, (A A^T) A G, ..., (A A^T)^q A G]      (block Krylov space)
    Z = orthonormal basis of K
    M = Z^T A A^T Z,  U_r = its r top singular vectors
    F = Z U_r,        C <- C x_mode F^T             (sequential truncation)

The Gaussian block G is an input (the caller draws it), with one row per
column of the unfolding.  Unfoldings of a slice stack X[j][i1][i2]:
mode 1 is the n1 x (n n2) matrix with column j*n2 + i2, mode 2 the
n2 x (n n1) matrix with column j*n1 + i1.

When the ranks are not known, Alg. "AD-RSTHOSVD-BLBP" takes Alg. 1's place
(ad_rsthosvd_blbp below): each mode's factor is the block Lanczos basis of
Alg. 3 grown on the unfolding until its error estimate meets a relative
tolerance.
"""

import numpy as np

from . import svt


def unfold(X, mode):
    """Mode-1 or mode-2 unfolding of a slice stack X (n, n1, n2)."""
    n, n1, n2 = X.shape
    if mode == 1:
        return np.transpose(X, (1, 0, 2)).reshape(n1, n * n2)
    if mode == 2:
        return np.transpose(X, (2, 0, 1)).reshape(n2, n * n1)
    raise ValueError(mode)


def mode_product_t(X, F, mode):
    """C = X x_mode F^T for a slice stack: F^T X_j (mode 1) or X_j F (mode 2)."""
    if mode == 1:
        return np.einsum("ia,jib->jab", F, X)
    if mode == 2:
        return np.einsum("jia,ab->jib", X, F)
    raise ValueError(mode)


def mode_product(C, F, mode):
    """X = C x_mode F: F C_j (mode 1) or C_j F^T (mode 2)."""
    if mode == 1:
        return np.einsum("ia,jab->jib", F, C)
    if mode == 2:
        return np.einsum("jia,ba->jib", C, F)
    raise ValueError(mode)


def krylov_basis(A, G, q):
    """Z: an orthonormal basis of K = [A G, (A A^T) A G, ..., (A A^T)^q A G]
    (Alg. 1, "build the Krylov subspace", "form an orthonormal basis")."""
    blocks = [A @ G]
    for _ in range(q):
        blocks.append(A @ (A.T @ blocks[-1]))
    Z, _ = np.linalg.qr(np.concatenate(blocks, axis=1))
    return Z


def canonical_signs(F):
    """Columns scaled by +-1 so that each column's entry of largest magnitude
    (the first one on ties) is positive.  Singular vectors are defined up to
    sign; with processing order (1, 2) the mode-2 sketch is drawn on
    C x_1 F1^T, which depends on the signs of F1's columns, so the factor
    carries this fixed sign convention."""
    idx = np.argmax(np.abs(F), axis=0)
    sgn = np.where(F[idx, np.arange(F.shape[1])] < 0, -1.0, 1.0)
    return F * sgn


def bki_factor(A, G, q, r):
    """F = Z U_r for one mode (Alg. 1 loop body), with M = Z^T A A^T Z, the
    columns of U_r in decreasing order of singular value, signs canonical."""
    Z = krylov_basis(A, G, q)
    W = A.T @ Z
    M = W.T @ W
    U, _, _ = np.linalg.svd(M)
    return canonical_signs(Z @ U[:, :r]), Z


def rsthosvd_bki(X, ranks, G, q):
    """Alg. 1 with processing order (1, 2) on a slice stack X (n, n1, n2).

    ranks = (r1, r2), G = (G1, G2) with G1 (n n2, b1) and G2 (n r1, b2),
    q = (q1, q2).  Returns the core C (n, r1, r2) and the factors F1, F2."""
    C = X
    F = []
    for mode, r, Gm, qm in ((1, ranks[0], G[0], q[0]), (2, ranks[1], G[1], q[1])):
        Fm, _ = bki_factor(unfold(C, mode), Gm, qm, r)
        C = mode_product_t(C, Fm, mode)
        F.append(Fm)
    return C, F[0], F[1]


def randomized_gnhtsvt(X, tdims, tau, kind, ranks, G, q, theta=1.0, gamma=4.0):
    """Alg. 4, randomized branch: D(C, L) x_1 F1 x_2 F2 with [C; F1, F2]
    from rsthosvd_bki.  Returns the result and (C, F1, F2)."""
    C, F1, F2 = rsthosvd_bki(X, ranks, G, q)
    Ct, _ = svt.gnhtsvt(C, tdims, tau, kind, theta, gamma)
    return mode_product(mode_product(Ct, F1, 1), F2, 2), (C, F1, F2)


def transformed_randomized_prox(Abar, tau, kind, ranks, G, q, theta=1.0, gamma=4.0):
    """The same operator on the transformed stack Abar = L(A).

    For an orthonormal L along modes 3..d the mode-1 and mode-2 unfoldings of
    Abar are those of A times an orthogonal matrix, so with the Gaussian
    blocks transformed the same way (each block viewed as a stack and
    transformed along its slice index) the Krylov spaces, factors and core
    are those of the spatial form, the core's GNTSVT is the per-slice prox of
    its transformed slices, and the result is L of the spatial result.
    Returns Gbar and (Cbar, F1, F2)."""
    Cbar, F1, F2 = rsthosvd_bki(Abar, ranks, G, q)
    Ct, _ = svt.transformed_prox(Cbar, tau, kind, theta, gamma)
    return mode_product(mode_product(Ct, F1, 1), F2, 2), (Cbar, F1, F2)


def ad_rsthosvd_blbp(X, eps, b, delta_rel, gauss, caps=(None, None)):
    """Alg. "AD-RSTHOSVD-BLBP" (fixed-accuracy Tucker by block Lanczos
    bidiagonalization) with processing order (1, 2) on a slice stack X.

    For each mode: A = the mode unfolding of the current core C; the factor
    F = U^{v} is the basis the block Lanczos loop builds (svt.blbp_basis)
    until its error estimate E falls below eps^2 ||A||_F^2, with deflation
    tolerance delta = delta_rel * ||A||_F and at most min(A's sizes) columns
    (or caps[mode - 1]), with the sign convention of canonical_signs (the
    mode-2 draws act on C x_1 F1^T, so under a rank cap F2 depends on F1's
    signs, which the paper leaves free); then C <- C x_mode F^T.

    gauss(mode, rows, cols, draw) returns the draw-th standard Gaussian
    (rows x cols) block of the mode, rows being the number of columns of
    that mode's unfolding.
    Returns the core C, the factors F1, F2 and the final estimates (E1, E2).

    Reading: the printed algorithm names one tolerance epsilon for every
    mode and compares each mode's E with ||A||_F^2 of that mode's own
    unfolding, so the total error satisfies
    ||X - C x_1 F1 x_2 F2||_F^2 <= E1 + E2 <= 2 eps^2 ||X||_F^2."""
    C = X
    F, E = [], []
    for mode in (1, 2):
        A = unfold(C, mode)
        cap = min(A.shape) if caps[mode - 1] is None else min(caps[mode - 1], *A.shape)
        delta = delta_rel * np.sqrt(float(np.sum(A * A)))
        draws = [0]

        def draw_block(cols, mode=mode, rows=A.shape[1], draws=draws):
            G = gauss(mode, rows, cols, draws[0])
            draws[0] += 1
            return G

        Fm, Em, _ = svt.blbp_basis(A, eps, b, delta, draw_block, cap)
        Fm = canonical_signs(Fm)
        C = mode_product_t(C, Fm, mode)
        F.append(Fm)
        E.append(Em)
    return C, F[0], F[1], tuple(E)


def fixed_accuracy_gnhtsvt(X, tdims, tau, kind, eps, b, delta_rel, gauss, theta=1.0, gamma=4.0,
                           caps=(None, None)):
    """Alg. 4, randomized branch with the fixed-accuracy Tucker form:
    D(C, L) x_1 F1 x_2 F2 with [C; F1, F2] from ad_rsthosvd_blbp.
    Returns the result and (C, F1, F2, (E1, E2))."""
    C, F1, F2, E = ad_rsthosvd_blbp(X, eps, b, delta_rel, gauss, caps)
    Ct, _ = svt.gnhtsvt(C, tdims, tau, kind, theta, gamma)
    return mode_product(mode_product(Ct, F1, 1), F2, 2), (C, F1, F2, E)


def transformed_fixed_accuracy_prox(Abar, tau, kind, eps, b, delta_rel, gauss, theta=1.0,
                                    gamma=4.0, caps=(None, None)):
    """The same operator on the transformed stack Abar = L(A), the form an
    ADMM step evaluates: the factors are built from the unfoldings of Abar
    (those of A times an orthogonal matrix, so the first mode's factor spans
    the same space as in the spatial form when its draws are transformed
    alike), the core's GNTSVT is the per-slice prox of its transformed
    slices.  Returns Gbar and (Cbar, F1, F2, (E1, E2))."""
    Cbar, F1, F2, E = ad_rsthosvd_blbp(Abar, eps, b, delta_rel, gauss, caps)
    Ct, _ = svt.transformed_prox(Cbar, tau, kind, theta, gamma)
    return mode_product(mode_product(Ct, F1, 1), F2, 2), (Cbar, F1, F2, E)
