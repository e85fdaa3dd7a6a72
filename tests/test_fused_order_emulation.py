"""CPU emulation (numpy, FP64) of the step grouping the GPU path runs.

Alg. 5 updates L, G, E, then the multipliers.  The GPU splits an iteration at
the slice pass instead: the forward tube pass of iteration t forms L, E, Y and
Abar = L(L + Lambda/mu); the slice pass maps Abar to Gbar; the inverse half
(G = L^{-1}(Gbar), Lambda + mu (L - G)) waits for the next tube pass, which
runs it in the same tile just before the forward half of iteration t + 1 and
writes |L - G| and |G - G_prev| into iteration t's residual slots.  A
recovery ends with the inverse half alone.  This file runs that grouping
with whole-tensor numpy operations and checks it against `oracle.admm.run`
step by step: states and all five residuals (Eq. convercon), for the l1 and
MCP penalties, with and without the sparse noise term."""

import numpy as np
import pytest

from oracle import admm, prox, svt, transform
from paper_2506_09594_gb300 import synth


def _forward_half(M, om, L, E, Y, G, Lam, mu, p):
    """The forward tube pass: Eq. coef-tensor, Eq. E_prox_ome(1), the Y update."""
    L1 = 0.5 * ((M - E + Y / mu) + (G - Lam / mu))
    H = M - L1 + Y / mu
    if p.noise == admm.NOISE_NONE:
        E_on = np.zeros_like(H)
    else:
        E_on = prox.gnhtt_entrywise(H, p.lam / mu, p.psi, p.psi_theta, p.psi_gamma)
    E1 = np.where(om, E_on, H)
    Y1 = Y + mu * (M - L1 - E1)
    res = [np.max(np.abs(L1 - L)), np.max(np.abs(E1 - E)), np.max(np.abs(M - L1 - E1))]
    return L1, E1, Y1, L1 + Lam / mu, res


def _run_grouped_as_on_the_gpu(M, mask, tdims, p, steps):
    om = mask.astype(bool)
    z = np.zeros_like(M)
    L, E, Y, G, Lam = z.copy(), z.copy(), z.copy(), z.copy(), z.copy()
    mu, t = p.mu0, 0
    Gbar, mu_prev = None, None
    rows = []
    for _ in range(steps):
        if Gbar is not None:
            # the fused pass: iteration t-1's inverse half, in the same tile
            G1 = transform.inverse(Gbar, tdims)
            Lam = Lam + mu_prev * (L - G1)
            rows[-1][2] = np.max(np.abs(L - G1))
            rows[-1][3] = np.max(np.abs(G1 - G))
            G = G1
        L, E, Y, X, (rL, rE, rC) = _forward_half(M, om, L, E, Y, G, Lam, mu, p)
        # the slice pass on the transformed stack (Alg. 4, tau = 1/mu)
        Gbar, _ = svt.transformed_prox(transform.forward(X, tdims), 1.0 / mu, p.phi, p.phi_theta,
                                       p.phi_gamma, p.engine, l=p.l, q=p.q, seed=p.seed, t=t)
        rows.append([rL, rE, None, None, rC])
        mu_prev, mu, t = mu, min(p.mu_max, p.growth * mu), t + 1
    # a recovery's last call completes the deferred inverse half
    G1 = transform.inverse(Gbar, tdims)
    Lam = Lam + mu_prev * (L - G1)
    rows[-1][2] = np.max(np.abs(L - G1))
    rows[-1][3] = np.max(np.abs(G1 - G))
    return dict(L=L, E=E, Y=Y, G=G1, Lam=Lam, mu=mu), np.array(rows, dtype=np.float64)


@pytest.mark.parametrize("phi, noise", [(prox.MCP, admm.NOISE_L1), (prox.L1, admm.NOISE_L1),
                                        (prox.MCP, admm.NOISE_NONE)])
def test_deferred_inverse_half_matches_alg5(phi, noise):
    w = synth.WORKLOADS["tubal64_r5"]
    _, M, mask, _ = synth.make_problem(w)
    M, mask = M[:, :24, :20].copy(), mask[:, :24, :20].copy()     # a 24 x 20 x 16 stack
    lam = admm.default_lambda(24, 20, w.tdims)
    p = admm.Params(phi=phi, psi=phi, noise=noise, lam=lam, engine="rsvd", l=8, q=1, seed=5,
                    mu0=0.05, growth=1.2, tol=0.0, max_iter=6)
    st, hist = admm.run(M, mask, w.tdims, p)
    got, rows = _run_grouped_as_on_the_gpu(M, mask, w.tdims, p, 6)
    scale = np.max(np.abs(M))
    for k in ("L", "E", "Y", "G", "Lam"):
        assert np.max(np.abs(got[k] - getattr(st, k))) <= 1e-11 * max(scale, np.max(np.abs(getattr(st, k))))
    assert got["mu"] == pytest.approx(st.mu, rel=1e-15)
    assert rows.shape == hist.shape
    assert np.max(np.abs(rows - hist)) <= 1e-11 * scale
