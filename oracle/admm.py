"""One ADMM iteration of Alg. 5 in the pure-L form, and the loop around it.

Test infrastructure (see the package docstring).

Model (Eq. orin_nonconvex / Eq. equ_nonconvex) with the "pure L" prior of
the paper's Experiment 2: Gamma holds one direction whose operator is the
identity (nabla -> I), so gamma = |Gamma| = 1 and the split constraint is
G = L.  One iteration, in the order of Alg. 5:

1. L-update, Eq. coef-tensor with nabla = I:
   2 L^{t+1} = (M - E^t + Y^t/mu^t) + (G^t - Lambda^t/mu^t).
2. G-update, Eq. L_prox: G^{t+1} = D_{Phi,tau}(L^{t+1} + Lambda^t/mu^t, L)
   with tau = 1/(gamma mu^t) = 1/mu^t.
3. E-update, Eq. E_prox_ome / E_prox_ome1 with H = M - L^{t+1} + Y^t/mu^t:
   on Omega E = Prox_{psi, lambda/mu^t}(H) entrywise (GNHTT, h = l1);
   off Omega E = H.  Noise-free GNHTC ("lambda set to zero") is read as
   E = 0 on Omega, which enforces P_Omega(L) = P_Omega(M).
4. Multipliers, Eq. lagrange11-22: Y += mu (M - L - E);
   Lambda += mu (L - G); mu = min(mu_max, vartheta mu).
5. Stopping quantities, Eq. convercon (nabla = I): the infinity norms of
   L^{t+1}-L^t, E^{t+1}-E^t, L^{t+1}-G^{t+1}, G^{t+1}-G^t, M-L^{t+1}-E^{t+1}.

Initialisation (Alg. 5): G = E = Lambda = Y = 0; L^0 = 0 (only used by the
first stopping quantity).  M is P_Omega(M): zero off Omega.
"""

from dataclasses import dataclass, field, replace

import numpy as np

from . import prox as _prox, svt

NOISE_NONE = "none"
NOISE_L1 = "l1"        # h = l1 entrywise; psi chosen by psi_kind


@dataclass
class Params:
    phi: str = _prox.MCP           # Phi in GNHTSVT
    phi_theta: float = 1.0
    phi_gamma: float = 4000.0
    psi: str = _prox.MCP           # psi in GNHTT
    psi_theta: float = 1.0
    psi_gamma: float = 4000.0
    noise: str = NOISE_L1
    lam: float = 0.0
    mu0: float = 1e-3
    mu_max: float = 1e10
    growth: float = 1.1
    tol: float = 1e-4
    max_iter: int = 100
    engine: str = "rsvd"          # "full" | "rsvd" | "adaptive" | "tucker"
    l: int = 15                   # sketch width r + p
    q: int = 1                    # power iterations
    seed: int = 0
    eps: float = 0.01             # adaptive engine relative accuracy
    b: int = 10                   # adaptive engine block size
    delta_rel: float = 1e-12


@dataclass
class State:
    L: np.ndarray
    E: np.ndarray
    Y: np.ndarray
    Lam: np.ndarray
    G: np.ndarray
    mu: float
    t: int = 0
    info: dict = field(default_factory=dict)


def init_state(shape, mu0):
    z = np.zeros(shape, dtype=np.float64)
    return State(L=z.copy(), E=z.copy(), Y=z.copy(), Lam=z.copy(), G=z.copy(),
                 mu=float(mu0), t=0)


def default_lambda(n1, n2, tdims, xi=1.0):
    """lambda for the orthonormal transform: xi / sqrt(max(n1, n2)).

    Sec. 6 sets lambda = xi / sqrt(max(n1, n2) * n3 ... nd) for L = FFT, whose
    matrices satisfy U U^H = n_i I, so rho = n3 ... nd and the transformed
    nuclear norm carries a 1/rho factor (Def. gnhtctv).  For the orthonormal
    DCT (rho = 1) the transformed singular values are sqrt(n) times smaller
    than the FFT's and the 1/rho factor is gone, so the nuclear term is
    sqrt(n) times larger relative to ||E||_1; keeping the paper's balance
    multiplies its lambda by sqrt(n3 ... nd), which leaves xi / sqrt(max(n1, n2)).
    `tdims` is accepted for the paper's form and not used.
    """
    return xi / np.sqrt(max(n1, n2))


def step(st, M, mask, tdims, p):
    """One iteration of Alg. 5 (pure-L).  Returns (new state, 5 residuals)."""
    mu = st.mu
    omega = np.asarray(mask, dtype=bool)
    M = np.asarray(M, dtype=np.float64)
    # 1. L-update
    L = 0.5 * ((M - st.E + st.Y / mu) + (st.G - st.Lam / mu))
    # 2. G-update: GNHTSVT with tau = 1/mu
    A = L + st.Lam / mu
    tau = 1.0 / mu
    G, info = svt.gnhtsvt(A, tdims, tau, p.phi, p.phi_theta, p.phi_gamma,
                          engine=p.engine, l=p.l, q=p.q, seed=p.seed, t=st.t,
                          eps=p.eps, b=p.b, delta_rel=p.delta_rel)
    # 3. E-update
    H = M - L + st.Y / mu
    if p.noise == NOISE_NONE:
        E_on = np.zeros_like(H)
    else:
        E_on = _prox.gnhtt_entrywise(H, p.lam / mu, p.psi, p.psi_theta, p.psi_gamma)
    E = np.where(omega, E_on, H)
    # 4. multipliers and penalty
    Y = st.Y + mu * (M - L - E)
    Lam = st.Lam + mu * (L - G)
    mu_next = min(p.mu_max, p.growth * mu)
    # 5. stopping quantities (Eq. convercon with nabla = I)
    res = np.array([
        np.max(np.abs(L - st.L)),
        np.max(np.abs(E - st.E)),
        np.max(np.abs(L - G)),
        np.max(np.abs(G - st.G)),
        np.max(np.abs(M - L - E)),
    ])
    new = State(L=L, E=E, Y=Y, Lam=Lam, G=G, mu=mu_next, t=st.t + 1, info=info)
    return new, res


def run(M, mask, tdims, p, callback=None):
    """Alg. 5 loop: iterate until max(residuals) <= tol or max_iter steps."""
    st = init_state(M.shape, p.mu0)
    history = []
    for _ in range(p.max_iter):
        st, res = step(st, M, mask, tdims, p)
        history.append(res)
        if callback is not None:
            callback(st, res)
        if p.tol > 0 and float(np.max(res)) <= p.tol:
            break
    return st, np.array(history)


def with_(p, **kw):
    return replace(p, **kw)
