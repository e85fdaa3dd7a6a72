"""The one-bit completion model (GNOBHTC): one ADMM iteration of Alg. 6, in
float64.

Test infrastructure (see the package docstring).

Observations (the one-bit model's data): q_k = sign(L*[s_k] + eps_k + xi_k)
for m entries s_k drawn uniformly, with dithers xi_k ~ U[-theta, theta]; by
Prop. one-bitequ theta q_k has the mean of the unquantised sample when
|L*[s_k] + eps_k| <= theta, so theta q_k stands in for it.

Model (Eq. 1bittensorqqqq):
    min (1/2m) sum_k (L[s_k] - theta q_k)^2 + (lambda/gamma) sum_{i in Gamma} ||G_i||_{Phi,L}
        + I{||L||_inf <= alpha}
    s.t. Z = L, G_i = nabla_i(Z),
with the augmented terms <Y, L - Z> + mu/2 ||L - Z||^2 and
<Lambda_i, nabla_i Z - G_i> + mu/2 ||nabla_i Z - G_i||^2, whose signs follow
from the multiplier updates Eq. 1bit-Y.  One iteration, in Alg. 6's order:

1. L-update, Eq. 1bit-L.  The L-subproblem separates over entries: entry e
   sees c_e samples with sum b_e of theta q_k, and minimises over
   [-alpha, alpha] the convex quadratic
       (c_e L^2 - 2 b_e L)/(2m) + Y_e L + mu/2 (L - Z_e)^2,
   whose minimiser is the clip of (m mu Z + J1 - m Y) / (m mu + J2) with
   J1 = sum_k theta q_k P_k (J1[e] = b_e) and J2 = sum_k P_k (J2[e] = c_e).
   These two tensors are the ones the printed update names and leaves
   undefined; this is their derivation.
2. Z-update, Eq. 1bit-Z: (I + sum_i nabla_i^T nabla_i) Z = L + Y/mu +
   sum_i nabla_i^T (G_i - Lambda_i/mu), by the multi-dimensional FFT
   (oracle.ctv.l_update).  The printed right-hand side names L^t; Alg. 6
   updates L first, so the L used is the new one (sequential ADMM).
3. G-update, Eq. 1bit-g: G_i = D_{Phi, lambda/(gamma mu)}(nabla_i(Z) + Lambda_i/mu, L).
4. Multipliers, Eq. 1bit-Y..1bit-MU: Y += mu (L - Z);
   Lambda_i += mu (nabla_i(Z) - G_i); mu = min(mu_max, vartheta mu).
5. Stop test of Alg. 6: ||L^{t+1} - L^t||_F / ||L^t||_F <= varpi.
"""

from dataclasses import dataclass, field

import numpy as np

from . import ctv, prox as _prox, svt


@dataclass
class Params:
    modes: tuple = (1, 2)          # Gamma
    transform: str = "dct"         # L
    phi: str = _prox.MCP
    phi_theta: float = 1.0
    phi_gamma: float = 4000.0
    lam: float = 1.0               # lambda
    theta: float = 1.0             # dither half-width
    alpha: float = 1.0             # ||L||_inf bound
    mu0: float = 1e-6              # Alg. 6 initialisation
    mu_max: float = 1e3
    growth: float = 1.05
    tol: float = 1e-5              # varpi
    max_iter: int = 200
    engine: str = "full"           # GNHTSVT engine: "full" or "rsvd" (oracle.svt)
    l: int = 15                    # rsvd: sketch width
    q: int = 1                     # rsvd: power iterations
    seed: int = 0                  # rsvd: Philox key; the draws of step t use counter t


@dataclass
class State:
    L: np.ndarray
    Z: np.ndarray
    Y: np.ndarray
    G: dict
    Lam: dict
    mu: float
    t: int = 0
    info: dict = field(default_factory=dict)


def sample_tensors(shape, s, q, theta):
    """J1 = sum_k theta q_k P_k and J2 = sum_k P_k for samples at flat
    entries s with signs q."""
    J1 = np.zeros(int(np.prod(shape)))
    J2 = np.zeros(int(np.prod(shape)))
    np.add.at(J1, s, theta * np.asarray(q, dtype=np.float64))
    np.add.at(J2, s, 1.0)
    return J1.reshape(shape), J2.reshape(shape)


def l_update(Z, Y, J1, J2, m, mu, alpha):
    """Eq. 1bit-L: the clip to [-alpha, alpha] of (m mu Z + J1 - m Y) / (m mu + J2)."""
    return np.clip((m * mu * Z + J1 - m * Y) / (m * mu + J2), -alpha, alpha)


def init_state(shape, mu0, modes):
    z = np.zeros(shape, dtype=np.float64)
    return State(L=z.copy(), Z=z.copy(), Y=z.copy(), G={i: z.copy() for i in modes},
                 Lam={i: z.copy() for i in modes}, mu=float(mu0), t=0)


def step(st, J1, J2, m, tdims, p):
    """One iteration of Alg. 6.  Returns (new state, relative change of L)."""
    mu = st.mu
    modes = tuple(p.modes)
    gam = len(modes)
    # 1. L-update (Eq. 1bit-L)
    L = l_update(st.Z, st.Y, J1, J2, m, mu, p.alpha)
    # 2. Z-update (Eq. 1bit-Z)
    Z = ctv.l_update(L + st.Y / mu, {i: st.G[i] - st.Lam[i] / mu for i in modes}, tdims, modes)
    # 3. G-updates (Eq. 1bit-g), threshold lambda/(gamma mu)
    tau = p.lam / (gam * mu)
    G, gradZ, info = {}, {}, {}
    for i in modes:
        gradZ[i] = ctv.grad(Z, tdims, i)
        G[i], info[i] = svt.gnhtsvt(gradZ[i] + st.Lam[i] / mu, tdims, tau, p.phi, p.phi_theta,
                                    p.phi_gamma, engine=p.engine, transform_kind=p.transform,
                                    l=p.l, q=p.q, seed=p.seed, t=st.t)
    # 4. multipliers and penalty (Eq. 1bit-Y .. 1bit-MU)
    Y = st.Y + mu * (L - Z)
    Lam = {i: st.Lam[i] + mu * (gradZ[i] - G[i]) for i in modes}
    mu_next = min(p.mu_max, p.growth * mu)
    # 5. stop quantity of Alg. 6
    nL = np.linalg.norm(st.L)
    rel = np.linalg.norm(L - st.L) / nL if nL > 0 else np.inf
    new = State(L=L, Z=Z, Y=Y, G=G, Lam=Lam, mu=mu_next, t=st.t + 1, info=info)
    return new, rel


def run(shape, s, q, tdims, p, callback=None):
    """Alg. 6 loop on the samples (s, q): until the relative change of L is
    at most tol, or max_iter steps."""
    m = len(s)
    J1, J2 = sample_tensors(shape, s, q, p.theta)
    st = init_state(shape, p.mu0, tuple(p.modes))
    history = []
    for _ in range(p.max_iter):
        st, rel = step(st, J1, J2, m, tdims, p)
        history.append(rel)
        if callback is not None:
            callback(st, rel)
        if p.tol > 0 and rel <= p.tol:
            break
    return st, np.array(history)
