"""GNHTSVT D_{Phi,tau}(A, L) and its low-rank engines, in float64.

Test infrastructure (see the package docstring).

Definition gNtsvt / Theorem theorem_wtsvt (Sec. 4.2.2): with the T-SVD
A = U *_L S *_L V^T, D_{Phi,tau}(A, L) = U *_L S_{Phi,tau} *_L V^T where every
transformed singular value L(S)^<j>(i, i) is replaced by its scalar prox
Prox_{Phi,tau}.  Because the face-wise product acts slice by slice in the
transform domain, this is: transform, shrink the singular values of every
transformed face slice, rebuild, transform back (Alg. 4, deterministic
branch).  The theorem states it is the minimiser of
tau*||G||_{Phi,L} + ||G - A||_F^2 / 2, with ||G||_{Phi,L} = (1/rho) sum Phi(sigma)
and rho = alpha_3...alpha_d = 1 for the orthonormal DCT.

Three engines compute the transform-domain slice map Abar^<j> -> Gbar^<j>:

* ``slice_prox_full``        full SVD of the slice (Alg. 4, deterministic).
* ``slice_prox_randomized``  Gaussian sketch, q power iterations with
                             re-orthonormalisation, QR, SVD of B = Q^T Abar,
                             shrink, rebuild Q Uhat diag(prox(sigma)) V^T.
                             The sketch and power steps are those of Alg. 1
                             (Gaussian G, (A A^T)^q A G, orthonormal basis),
                             applied per transformed face slice.
* ``slice_prox_adaptive``    Alg. 3 (block Lanczos bidiagonalisation with
                             one-sided reorthogonalisation, defl-QR of
                             Alg. 2, Gaussian refill on deflation, error
                             indicator E) restated for one face slice; its
                             basis U replaces Q above.

Two more engines compress all slices at once with Tucker factors of the two
spatial modes shared by every slice (oracle.tucker): ``tucker`` (Alg. 1,
fixed ranks) and ``ad_tucker`` (Alg. AD-RSTHOSVD-BLBP, fixed accuracy).
"""

import numpy as np
import scipy.linalg

from . import philox, prox as _prox, transform


def _shrink(s, tau, kind, theta, gamma):
    return _prox.prox_scalar(s, tau, kind, theta, gamma)


# ---------------------------------------------------------------- full SVD
def slice_prox_full(Ab, tau, kind, theta=1.0, gamma=4.0):
    """Deterministic branch of Alg. 4 on one transformed face slice."""
    U, s, Vt = np.linalg.svd(Ab, full_matrices=False)
    s2 = _shrink(s, tau, kind, theta, gamma)
    return (U * s2) @ Vt, s, s2


# ------------------------------------------------------------- randomized
def slice_prox_randomized(Ab, Omega, q, tau, kind, theta=1.0, gamma=4.0):
    """Per-slice randomized prox with sketch Omega (n2 x l) and q power steps.

    Steps, in order: Y = Ab Omega; q times { Q = qr(Y); W = qr(Ab^T Q);
    Y = Ab W }; Q = qr(Y); B = Q^T Ab; B = Uhat diag(sigma) V^T;
    Gbar = Q Uhat diag(Prox_{Phi,tau}(sigma)) V^T.
    Returns (Gbar, sigma, shrunk sigma).
    """
    Y = Ab @ Omega
    for _ in range(q):
        Q, _ = np.linalg.qr(Y)
        W, _ = np.linalg.qr(Ab.T @ Q)
        Y = Ab @ W
    Q, _ = np.linalg.qr(Y)
    B = Q.T @ Ab
    Uh, s, Vt = np.linalg.svd(B, full_matrices=False)
    s2 = _shrink(s, tau, kind, theta, gamma)
    return Q @ ((Uh * s2) @ Vt), s, s2


def slice_prox_krylov(Ab, Omega, q, r, tau, kind, theta=1.0, gamma=4.0):
    """Alg. 1's block-Krylov basis on one face slice, then the prox.

    K = [Ab Omega, (Ab Ab^T) Ab Omega, ..., (Ab Ab^T)^q Ab Omega]; Z = orth(K);
    M = Z^T Ab Ab^T Z; U_r = top-r singular vectors of M; F = Z U_r; then the
    prox of F F^T Ab through the SVD of B = F^T Ab.
    """
    blocks = [Ab @ Omega]
    for _ in range(q):
        blocks.append(Ab @ (Ab.T @ blocks[-1]))
    K = np.concatenate(blocks, axis=1)
    Z, _ = np.linalg.qr(K)
    M = Z.T @ Ab @ Ab.T @ Z
    Um, _, _ = np.linalg.svd(M)
    F = Z @ Um[:, :r]
    B = F.T @ Ab
    Uh, s, Vt = np.linalg.svd(B, full_matrices=False)
    s2 = _shrink(s, tau, kind, theta, gamma)
    return F @ ((Uh * s2) @ Vt), s, s2


# --------------------------------------------------------------- adaptive
def defl_qr(A, delta):
    """Alg. 2: pivoted QR A P = Qt Rt; s = largest index with |Rt(s,s)| >= delta;
    R = Rt(1:s, :) P^T; Q = Qt(:, 1:s).  Returns (Q, R, s)."""
    if A.shape[1] == 0:
        return A[:, :0], np.zeros((0, 0)), 0
    Qt, Rt, piv = scipy.linalg.qr(A, mode="economic", pivoting=True)
    d = np.abs(np.diag(Rt))
    keep = np.nonzero(d >= delta)[0]
    s = int(keep[-1]) + 1 if keep.size else 0
    R = np.zeros((s, A.shape[1]))
    R[:, piv] = Rt[:s, :]            # R = Rt(1:s, :) P^T
    return Qt[:, :s], R, s


def blbp_basis(A, eps, b, delta, gauss, cap):
    """Block Lanczos bidiagonalization with deflation and an error estimate:
    the loop of Alg. 3 (one matrix) and of Alg. "AD-RSTHOSVD-BLBP" (one mode
    unfolding).  Returns (U, E, history) with U = U^{v} truncated to cap
    columns and E = ||A||_F^2 - sum ||R^(i)||^2 - sum ||L^(i+1)||^2.

    gauss(cols) returns the next standard Gaussian block (A.shape[1], cols);
    delta is the absolute deflation tolerance.

    Readings of the printed algorithms (their indexing is garbled):
    U^(0) = 0 and L^(1) = 0 (the first step is plain A V^(1)); U^{v} starts
    empty; when defl-QR of the new V block keeps s < b columns, the b - s
    Gaussian refill columns are appended to V^(i+1) itself (and L^(i+1)
    padded with zero columns), so every block stays b wide; the stopping
    test is relative, E < eps^2 ||A||_F^2.
    """
    n1, n2 = A.shape
    normA2 = float(np.sum(A * A))
    E = normA2
    V, _ = np.linalg.qr(gauss(b))
    Vcat = V.copy()
    Ucat = np.zeros((n1, 0))
    U_prev = np.zeros((n1, 0))
    L = np.zeros((0, V.shape[1]))
    hist = []
    if normA2 == 0.0:
        return Ucat, 0.0, hist
    while True:
        U, R, _ = defl_qr(A @ V - U_prev @ L, delta)
        Ucat = np.concatenate([Ucat, U], axis=1)
        E -= float(np.sum(R * R))
        Vn = A.T @ U - V @ R.T
        Vn = Vn - Vcat @ (Vcat.T @ Vn)
        Vn, Lt, s = defl_qr(Vn, delta)
        Vcat = np.concatenate([Vcat, Vn], axis=1)
        E -= float(np.sum(Lt * Lt))
        L = Lt.T                                    # (cols of U) x s
        if s < b and Vcat.shape[1] < n2:
            G = gauss(b - s)
            Vr, _ = np.linalg.qr(G - Vcat @ (Vcat.T @ G))
            Vr = Vr[:, : max(0, min(b - s, n2 - Vcat.shape[1]))]
            Vcat = np.concatenate([Vcat, Vr], axis=1)
            Vn = np.concatenate([Vn, Vr], axis=1)
            L = np.concatenate([L, np.zeros((L.shape[0], Vr.shape[1]))], axis=1)
        hist.append((Ucat.shape[1], E))
        U_prev, V = U, Vn
        if E < eps * eps * normA2 or Ucat.shape[1] >= cap or V.shape[1] == 0:
            break
    return Ucat[:, :cap], E, hist


def adaptive_basis(Ab, eps, b, delta_rel, seed, t, j, max_rank=None):
    """Alg. 3 restated for one face slice: returns (U, E, history).

    The loop is blbp_basis with delta = delta_rel * ||A||_F and the rank cap
    min(n1, n2) (or max_rank).  Gaussian draws use stream STREAM_ADAPTIVE
    with counter words (m//4, j, t, STREAM_ADAPTIVE + 2*draw_index).
    """
    n1, n2 = Ab.shape
    cap = min(n1, n2) if max_rank is None else min(max_rank, n1, n2)
    delta = delta_rel * np.sqrt(float(np.sum(Ab * Ab)))
    draw = 0

    def gauss(cols):
        nonlocal draw
        G = philox.gaussian_block(seed, t, j, n2, cols,
                                  stream=philox.STREAM_ADAPTIVE + 2 * draw)
        draw += 1
        return G

    return blbp_basis(Ab, eps, b, delta, gauss, cap)


def slice_prox_adaptive(Ab, eps, b, delta_rel, seed, t, j, tau, kind,
                        theta=1.0, gamma=4.0, max_rank=None):
    """Prox through the adaptive basis U: B = U^T Ab, SVD, shrink, rebuild."""
    U, E, _ = adaptive_basis(Ab, eps, b, delta_rel, seed, t, j, max_rank=max_rank)
    B = U.T @ Ab
    Uh, s, Vt = np.linalg.svd(B, full_matrices=False)
    s2 = _shrink(s, tau, kind, theta, gamma)
    return U @ ((Uh * s2) @ Vt), s, s2, U.shape[1], E


# ------------------------------------------------------ whole-tensor maps
def transformed_prox(Abar, tau, kind, theta=1.0, gamma=4.0, engine="full",
                     l=None, q=1, seed=0, t=0, eps=0.01, b=10, delta_rel=1e-12,
                     max_rank=None, widths=None, p=0):
    """Apply the chosen slice engine to every transformed face slice.

    Returns (Gbar, info) where info holds per-slice singular values and the
    number of kept (non-zero shrunk) singular values.

    engine "learned": slice j is sketched at its own width widths[j] (the
    randomized engine with q power steps and the Philox block of width
    widths[j]); learned.judge (eps, oversampling p, adaptive cap max_rank)
    decides which sketches the adaptive engine (eps, b, delta_rel, cap
    max_rank) recomputes.  info["fallback"] lists those slices; info["widths"]
    holds each slice's width: the sketch's, or the adaptive basis size.
    """
    n, n1, n2 = Abar.shape
    if engine == "learned":
        from . import learned
        Gbar = np.zeros(Abar.shape, dtype=np.result_type(Abar.dtype, np.float64))
        sig, a2 = [], []
        for j in range(n):
            Ab = np.asarray(Abar[j]).astype(np.result_type(Abar.dtype, np.float64))
            ll = min(int(widths[j]), n1, n2)
            Om = philox.gaussian_block(seed, t, j, n2, ll)
            Gbar[j], s, _ = slice_prox_randomized(Ab, Om, q, tau, kind, theta, gamma)
            sig.append(s)
            a2.append(float(np.sum(Ab * Ab)))
        kept = np.array([min(int(w), n1, n2) for w in widths], dtype=np.int64)
        shrunk = [int(np.count_nonzero(_shrink(sig[j], tau, kind, theta, gamma)))
                  for j in range(n)]
        fb = learned.judge(a2, sig, eps, shrunk, kept, p, max_rank)
        ranks = np.zeros(n, dtype=np.int64)
        for j in range(n):
            if j in set(fb.tolist()):
                Ab = np.asarray(Abar[j]).astype(np.result_type(Abar.dtype, np.float64))
                Gbar[j], s, s2, kept[j], _ = slice_prox_adaptive(Ab, eps, b, delta_rel, seed, t,
                                                                 j, tau, kind, theta, gamma,
                                                                 max_rank)
                sig[j] = s
            ranks[j] = int(np.count_nonzero(_shrink(sig[j], tau, kind, theta, gamma)))
        return Gbar, {"ranks": ranks, "sigma": sig, "fallback": fb, "widths": kept}
    if engine == "tucker":
        # Alg. 4 randomized branch with shared factors of the two spatial
        # modes (oracle.tucker): ranks, block sizes l, q Krylov steps; the
        # Gaussian blocks are drawn per transformed slice (Philox streams 2
        # and 4), stacked by rows
        from . import tucker
        ll = min(int(l), n1, n2)
        G1 = np.concatenate([philox.gaussian_block(seed, t, j, n2, ll, philox.STREAM_TUCKER_1)
                             for j in range(n)], axis=0)
        G2 = np.concatenate([philox.gaussian_block(seed, t, j, ll, ll, philox.STREAM_TUCKER_2)
                             for j in range(n)], axis=0)
        Cbar, F1, F2 = tucker.rsthosvd_bki(np.asarray(Abar, dtype=np.float64), (ll, ll), (G1, G2),
                                           (q, q))
        Ct, info = transformed_prox(Cbar, tau, kind, theta, gamma)
        return tucker.mode_product(tucker.mode_product(Ct, F1, 1), F2, 2), info
    if engine == "ad_tucker":
        # the fixed-accuracy Tucker form (Alg. "AD-RSTHOSVD-BLBP", order
        # (1, 2)): tolerance eps, block size b, deflation delta_rel, rank cap
        # max_rank per mode; draw d of mode m is a Philox block per
        # transformed slice on stream STREAM_AD_TUCKER_m + 2 d, with the
        # slice's share of the unfolding's columns as rows, stacked by rows
        from . import tucker
        base = {1: philox.STREAM_AD_TUCKER_1, 2: philox.STREAM_AD_TUCKER_2}

        def gauss(mode, rows, cols, draw):
            return np.concatenate([philox.gaussian_block(seed, t, j, rows // n, cols,
                                                         base[mode] + 2 * draw)
                                   for j in range(n)], axis=0)

        Cbar, F1, F2, E = tucker.ad_rsthosvd_blbp(np.asarray(Abar, dtype=np.float64), eps, b,
                                                  delta_rel, gauss, (max_rank, max_rank))
        Ct, info = transformed_prox(Cbar, tau, kind, theta, gamma)
        info["tucker_ranks"] = (F1.shape[1], F2.shape[1])
        info["tucker_estimates"] = E
        return tucker.mode_product(tucker.mode_product(Ct, F1, 1), F2, 2), info
    Gbar = np.zeros(Abar.shape, dtype=np.result_type(Abar.dtype, np.float64))
    ranks = np.zeros(n, dtype=np.int64)
    sig = []
    adaptive_ranks = []
    for j in range(n):
        Ab = np.asarray(Abar[j]).astype(np.result_type(Abar.dtype, np.float64))
        if engine == "full":
            Gbar[j], s, s2 = slice_prox_full(Ab, tau, kind, theta, gamma)
        elif engine == "rsvd":
            ll = min(int(l), n1, n2)
            Om = philox.gaussian_block(seed, t, j, n2, ll)
            Gbar[j], s, s2 = slice_prox_randomized(Ab, Om, q, tau, kind, theta, gamma)
        elif engine == "adaptive":
            Gbar[j], s, s2, kept, _ = slice_prox_adaptive(Ab, eps, b, delta_rel, seed, t, j,
                                                          tau, kind, theta, gamma, max_rank)
            adaptive_ranks.append(kept)
        else:
            raise ValueError(engine)
        ranks[j] = int(np.count_nonzero(s2))
        sig.append(s)
    return Gbar, {"ranks": ranks, "sigma": sig, "adaptive_ranks": adaptive_ranks}


def gnhtsvt(A, tdims, tau, kind, theta=1.0, gamma=4.0, engine="full", transform_kind="dct",
            **kw):
    """D_{Phi,tau}(A, L) on a slice stack A (n, n1, n2) (Alg. 4).

    With transform_kind="fft" (U U^H = n I, rho = n3 ... nd) the objective
    tau ||G||_{Phi,L} + ||G - A||_F^2 / 2 equals
    (1/rho) sum_j [tau sum Phi(sigma(Gbar_j)) + ||Gbar_j - Abar_j||_F^2 / 2], so the
    minimiser is again the per-slice prox with the same tau, on complex
    slices (full SVD only).  Slices j and -j of a real tensor are conjugate
    and the prox commutes with conjugation, so the result is real; its
    imaginary part (rounding only) is dropped.
    """
    if transform_kind == "fft" and engine != "full":
        raise ValueError("the DFT transform takes the full-SVD engine")
    Abar = transform.forward(A, tdims, transform_kind)
    Gbar, info = transformed_prox(Abar, tau, kind, theta, gamma, engine, **kw)
    out = transform.inverse(Gbar, tdims, transform_kind)
    return (out.real.copy() if np.iscomplexobj(out) else out), info


def objective(G, A, tdims, tau, kind, theta=1.0, gamma=4.0):
    """tau*||G||_{Phi,L} + ||G - A||_F^2 / 2, with rho = 1 (Theorem theorem_wtsvt)."""
    Gbar = transform.forward(G, tdims)
    val = 0.0
    for j in range(Gbar.shape[0]):
        s = np.linalg.svd(Gbar[j], compute_uv=False)
        val += float(np.sum(_prox.penalty(s, kind, theta, gamma)))
    return tau * val + 0.5 * float(np.sum((G - A) ** 2))
