"""The gradient-domain model (GNHTCTV prior): one ADMM iteration of Alg. 5
with a set Gamma of gradient directions, in float64.

Test infrastructure (see the package docstring).

Definitions (Def. gradient tensor, Def. GNHTCTV):

    nabla_k(A) = A x_k D_{n_k},  D_n the row circulant matrix of (-1, 1, 0, ..., 0),

so (nabla_k A)[.., i_k, ..] = A[.., i_k + 1 (mod n_k), ..] - A[.., i_k, ..], and
Psi(A) = (1/gamma) sum_{k in Gamma} ||nabla_k(A)||_{Phi,L} with gamma = |Gamma|.

Model (Eq. equ_nonconvex): min (1/gamma) sum ||G_k||_{Phi,L} + lambda Upsilon(P_Omega(E))
subject to G_k = nabla_k(L), L + E = M.  One iteration, in the order of Alg. 5:

1. L-update, Eq. coef-tensor: the linear system
       (I + sum_k nabla_k^T nabla_k)(L) = (M - E + Y/mu) + sum_k nabla_k^T(G_k - Lambda_k/mu),
   solved as Eq. gnrhtc-L does: nabla_k is a circular convolution with the
   difference tensor D_k (-1 at the origin, +1 one step back along mode k),
   so the multi-dimensional FFT diagonalises it:
       L = F^{-1}( [F(M - E + Y/mu) + sum_k conj(F(D_k)) . F(G_k - Lambda_k/mu)]
                   / [1 + sum_k conj(F(D_k)) . F(D_k)] ).
2. G-update, Eq. L_prox for every k in Gamma:
       G_k = D_{Phi,tau}(nabla_k(L) + Lambda_k/mu, L),  tau = 1/(gamma mu).
3. E-update, Eq. E_prox_ome / E_prox_ome1, as in the pure-L form (oracle.admm).
4. Multipliers, Eq. lagrange11-22: Y += mu (M - L - E);
   Lambda_k += mu (nabla_k(L) - G_k); mu = min(mu_max, vartheta mu).
5. Eq. convercon: the infinity norms of L - L^t, E - E^t, nabla_k(L) - G_k,
   G_k - G_k^t (each the maximum over k) and M - L - E.

Direction 0 stands for the identity operator (D_0 = I, F(D_0) = 1): Gamma =
{0} is the pure-L prior of the paper's Experiment 2, the form oracle.admm
implements directly.

Tensors are slice stacks (n, n1, n2) with the transformed mode sizes tdims,
as everywhere in the oracle; modes are numbered 1..d as in the paper.
"""

from dataclasses import dataclass, field

import numpy as np

from . import admm, prox as _prox, svt, transform

IDENTITY = 0


@dataclass
class Params(admm.Params):
    modes: tuple = (1, 2)          # Gamma
    transform: str = "dct"         # L: "dct" (orthonormal) or "fft" (the paper's experiments)


@dataclass
class State:
    L: np.ndarray
    E: np.ndarray
    Y: np.ndarray
    G: dict                        # k -> G_k
    Lam: dict                      # k -> Lambda_k
    mu: float
    t: int = 0
    info: dict = field(default_factory=dict)


def _view(S, tdims):
    """The slice stack as an order-d array (nd, ..., n3, n1, n2)."""
    n, n1, n2 = S.shape
    return S.reshape(tuple(reversed(tdims)) + (n1, n2))


def _axis(tdims, k):
    """Axis of mode k (1..d) in the (nd, ..., n3, n1, n2) view."""
    d = 2 + len(tdims)
    if k == 1:
        return d - 2
    if k == 2:
        return d - 1
    if 3 <= k <= d:
        return d - k
    raise ValueError(k)


def mode_sizes(shape, tdims):
    """(n1, n2, n3, ..., nd) of a slice stack of the given shape."""
    return (shape[1], shape[2]) + tuple(int(v) for v in tdims)


def difference_matrix(n):
    """D_n: row i holds -1 in column i and +1 in column i + 1 (mod n)."""
    D = -np.eye(n)
    D[np.arange(n), (np.arange(n) + 1) % n] += 1.0
    return D


def grad(S, tdims, k):
    """nabla_k(S) = S x_k D_{n_k} (Def. gradient tensor); k = 0 is the identity."""
    if k == IDENTITY:
        return np.array(S, dtype=np.float64)
    X = _view(np.asarray(S, dtype=np.float64), tdims)
    ax = _axis(tdims, k)
    return transform.mode_product(X, difference_matrix(X.shape[ax]), ax).reshape(S.shape)


def grad_t(S, tdims, k):
    """nabla_k^T(S) = S x_k D_{n_k}^T, the adjoint of nabla_k."""
    if k == IDENTITY:
        return np.array(S, dtype=np.float64)
    X = _view(np.asarray(S, dtype=np.float64), tdims)
    ax = _axis(tdims, k)
    return transform.mode_product(X, difference_matrix(X.shape[ax]).T, ax).reshape(S.shape)


def difference_tensor(shape, tdims, k):
    """D_k as an order-d array: nabla_k(X) is the circular convolution D_k * X,
    (D_k * X)[i] = sum_m D_k[m] X[i - m], so D_k holds -1 at the origin and +1
    at -e_k (index n_k - 1 along mode k); D_0 is the unit impulse."""
    n, n1, n2 = shape
    Dk = np.zeros(tuple(reversed(tdims)) + (n1, n2))
    if k == IDENTITY:
        Dk[(0,) * Dk.ndim] = 1.0
        return Dk
    ax = _axis(tdims, k)
    Dk[(0,) * Dk.ndim] -= 1.0
    idx = [0] * Dk.ndim
    idx[ax] = Dk.shape[ax] - 1
    Dk[tuple(idx)] += 1.0
    return Dk


def l_update(R0, Rk, tdims, modes):
    """Eq. gnrhtc-L: solve (I + sum_k nabla_k^T nabla_k) L = R0 + sum_k nabla_k^T(R_k)
    by the multi-dimensional FFT; Rk maps k -> R_k."""
    shape = R0.shape
    num = np.fft.fftn(_view(np.asarray(R0, dtype=np.float64), tdims))
    den = np.ones(num.shape)
    for k in modes:
        FD = np.fft.fftn(difference_tensor(shape, tdims, k))
        num = num + np.conj(FD) * np.fft.fftn(_view(np.asarray(Rk[k], dtype=np.float64), tdims))
        den = den + (np.conj(FD) * FD).real
    return np.fft.ifftn(num / den).real.reshape(shape)


def init_state(shape, mu0, modes):
    z = np.zeros(shape, dtype=np.float64)
    return State(L=z.copy(), E=z.copy(), Y=z.copy(), G={k: z.copy() for k in modes},
                 Lam={k: z.copy() for k in modes}, mu=float(mu0), t=0)


def step(st, M, mask, tdims, p):
    """One iteration of Alg. 5 with Gamma = p.modes.  Returns (new state, 5 residuals)."""
    mu = st.mu
    modes = tuple(p.modes)
    gam = len(modes)
    omega = np.asarray(mask, dtype=bool)
    M = np.asarray(M, dtype=np.float64)
    # 1. L-update (Eq. coef-tensor, Eq. gnrhtc-L)
    R0 = M - st.E + st.Y / mu
    L = l_update(R0, {k: st.G[k] - st.Lam[k] / mu for k in modes}, tdims, modes)
    # 2. G-updates (Eq. L_prox), tau = 1/(gamma mu)
    tau = 1.0 / (gam * mu)
    G, gradL, info = {}, {}, {}
    for k in modes:
        gradL[k] = grad(L, tdims, k)
        G[k], info[k] = svt.gnhtsvt(gradL[k] + st.Lam[k] / mu, tdims, tau, p.phi, p.phi_theta,
                                    p.phi_gamma, engine=p.engine, transform_kind=p.transform,
                                    l=p.l, q=p.q, seed=p.seed, t=st.t, eps=p.eps, b=p.b,
                                    delta_rel=p.delta_rel)
    # 3. E-update (Eq. E_prox_ome, E_prox_ome1)
    H = M - L + st.Y / mu
    if p.noise == admm.NOISE_NONE:
        E_on = np.zeros_like(H)
    else:
        E_on = _prox.gnhtt_entrywise(H, p.lam / mu, p.psi, p.psi_theta, p.psi_gamma)
    E = np.where(omega, E_on, H)
    # 4. multipliers and penalty (Eq. lagrange11-22)
    Y = st.Y + mu * (M - L - E)
    Lam = {k: st.Lam[k] + mu * (gradL[k] - G[k]) for k in modes}
    mu_next = min(p.mu_max, p.growth * mu)
    # 5. stopping quantities (Eq. convercon)
    res = np.array([
        np.max(np.abs(L - st.L)),
        np.max(np.abs(E - st.E)),
        max(np.max(np.abs(gradL[k] - G[k])) for k in modes),
        max(np.max(np.abs(G[k] - st.G[k])) for k in modes),
        np.max(np.abs(M - L - E)),
    ])
    new = State(L=L, E=E, Y=Y, G=G, Lam=Lam, mu=mu_next, t=st.t + 1, info=info)
    return new, res


def run(M, mask, tdims, p, callback=None):
    """Alg. 5 loop: iterate until max(residuals) <= tol or max_iter steps."""
    st = init_state(M.shape, p.mu0, tuple(p.modes))
    history = []
    for _ in range(p.max_iter):
        st, res = step(st, M, mask, tdims, p)
        history.append(res)
        if callback is not None:
            callback(st, res)
        if p.tol > 0 and float(np.max(res)) <= p.tol:
            break
    return st, np.array(history)
