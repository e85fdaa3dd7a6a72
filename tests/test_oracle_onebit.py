"""Pins of the one-bit completion oracle (Alg. 6, GNOBHTC).

The pins use what the model and the mathematics fix:

* the dithered observations obey Prop. one-bitequ: theta q has the mean of
  the unquantised value (Monte Carlo, several sigma);
* J1, J2 against an explicit loop over the samples;
* the L-step is the minimiser of each entry's box-constrained quadratic
  (bounded scalar minimisation by scipy);
* every step satisfies the optimality identities of its L- and Z-updates,
  rewritten with the new multipliers;
* the G-step threshold lambda/(gamma mu) in the multiplier spectrum;
* recovery of a smooth low-rank tensor improves with the number of samples
  and beats the per-entry average of the samples (empirical).
"""

import numpy as np
import pytest
import scipy.optimize

from oracle import onebit, prox, transform
from paper_2506_09594_gb300 import synth
from shifts import roll_grad_t


def smooth_tensor(n1, n2, n3, rng):
    i1, i2, i3 = np.arange(n1) / n1, np.arange(n2) / n2, np.arange(n3) / n3
    X = np.zeros((n1, n2, n3))
    for r in range(3):
        X += np.einsum("i,j,k->ijk", np.cos(2 * np.pi * (r + 1) * i1 + rng.random() * 6),
                       np.sin(2 * np.pi * (r + 1) * i2 + rng.random() * 6),
                       np.cos(2 * np.pi * r * i3 + rng.random() * 6))
    S = np.ascontiguousarray(np.moveaxis(X, 2, 0))
    return S / np.abs(S).max()


@pytest.mark.parametrize("x", [-0.9, -0.3, 0.0, 0.45, 1.0])
def test_dithered_sign_is_unbiased(x):
    # Prop. one-bitequ: E[theta sign(x + xi)] = x for |x| <= theta
    rng = np.random.default_rng(1)
    theta, m = 1.2, 200000
    s, q = synth.one_bit_observations(np.full((4, 5, 5), x), m, theta, 0.0, rng)
    assert s.min() >= 0 and s.max() < 100 and set(np.unique(q)) <= {-1.0, 1.0}
    est = theta * q.mean()
    sd = theta / np.sqrt(m)
    assert abs(est - x) < 5 * sd


def test_sample_tensors_count_and_sum():
    rng = np.random.default_rng(2)
    shape = (3, 4, 5)
    s = rng.integers(0, 60, 500)
    q = rng.choice([-1.0, 1.0], 500)
    J1, J2 = onebit.sample_tensors(shape, s, q, 0.7)
    W1, W2 = np.zeros(60), np.zeros(60)
    for k in range(500):
        W1[s[k]] += 0.7 * q[k]
        W2[s[k]] += 1
    assert np.allclose(J1.ravel(), W1, atol=1e-12) and np.array_equal(J2.ravel(), W2)


def test_l_step_minimises_each_entry():
    # entry e: min over [-alpha, alpha] of (c L^2 - 2 b L)/(2m) + Y L + mu/2 (L - Z)^2
    rng = np.random.default_rng(3)
    m, mu, alpha = 50, 0.03, 0.8
    Z = rng.uniform(-2, 2, 200)
    Y = rng.uniform(-0.05, 0.05, 200)
    J2 = rng.integers(0, 4, 200).astype(float)
    J1 = rng.uniform(-1, 1, 200) * J2
    L = onebit.l_update(Z, Y, J1, J2, m, mu, alpha)
    assert np.all(np.abs(L) <= alpha)
    for e in range(200):
        def f(x, e=e):
            return (J2[e] * x * x - 2 * J1[e] * x) / (2 * m) + Y[e] * x + 0.5 * mu * (x - Z[e]) ** 2
        r = scipy.optimize.minimize_scalar(f, bounds=(-alpha, alpha), method="bounded",
                                           options={"xatol": 1e-12})
        assert abs(L[e] - r.x) < 1e-7 and f(L[e]) <= f(r.x) + 1e-13


@pytest.mark.parametrize("tk,modes", [("dct", (1, 2)), ("fft", (1, 2, 3))])
def test_every_step_satisfies_its_optimality_identities(tk, modes):
    rng = np.random.default_rng(4)
    tdims = (6,)
    S = smooth_tensor(12, 10, 6, rng)
    s, q = synth.one_bit_observations(S, 3 * S.size, 1.2, 0.05, rng)
    m = len(s)
    p = onebit.Params(modes=modes, transform=tk, phi=prox.L1, lam=2e-3, theta=1.2, alpha=0.9,
                      mu0=1e-3, growth=1.3)
    J1, J2 = onebit.sample_tensors(S.shape, s, q, p.theta)
    st = onebit.init_state(S.shape, p.mu0, modes)
    for _ in range(6):
        new, _ = onebit.step(st, J1, J2, m, tdims, p)
        mu = st.mu
        # Z-update: -Y' + sum nabla^T Lambda' + mu sum nabla^T (G' - G) = 0
        r = -new.Y + sum(roll_grad_t(new.Lam[i] + mu * (new.G[i] - st.G[i]), tdims, i)
                         for i in modes)
        assert np.abs(r).max() < 1e-9 * max(1.0, np.abs(new.Y).max())
        # L-update: (c L - b)/m + Y' + mu (Z' - Z) = 0 where |L| < alpha, and
        # the box's sign conditions where L sits on it
        g = (J2 * new.L - J1) / m + new.Y + mu * (new.Z - st.Z)
        inside = np.abs(new.L) < p.alpha
        scale = max(1.0 / m, np.abs(new.Y).max())
        assert np.abs(g[inside]).max() < 1e-9 * scale
        assert np.all(g[new.L >= p.alpha] <= 1e-9 * scale)
        assert np.all(g[new.L <= -p.alpha] >= -1e-9 * scale)
        st = new


def test_g_step_threshold_is_lambda_over_gamma_mu():
    rng = np.random.default_rng(5)
    tdims, modes = (6,), (1, 2, 3)
    S = smooth_tensor(12, 10, 6, rng)
    s, q = synth.one_bit_observations(S, 3 * S.size, 1.2, 0.05, rng)
    p = onebit.Params(modes=modes, phi=prox.L1, lam=2e-3, theta=1.2, alpha=0.9, mu0=0.02)
    J1, J2 = onebit.sample_tensors(S.shape, s, q, p.theta)
    st = onebit.init_state(S.shape, p.mu0, modes)
    st, _ = onebit.step(st, J1, J2, len(s), tdims, p)    # nonzero L, Z, Y
    new, _ = onebit.step(st, J1, J2, len(s), tdims, p)
    tau = p.lam / (len(modes) * st.mu)
    for i in modes:
        Wb = transform.forward(new.Lam[i] / st.mu, tdims)
        norms = np.array([np.linalg.norm(Wb[j], 2) for j in range(Wb.shape[0])])
        assert norms.max() <= tau * (1 + 1e-10)
        assert abs(norms.max() - tau) < 1e-10 * tau
        # and Lambda_i' / mu is a subgradient of tau ||.||_* at G_i': aligned with it
        Gb = transform.forward(new.G[i], tdims)
        inner = sum(np.sum(Wb[j] * Gb[j]) for j in range(Wb.shape[0]))
        nuc = sum(np.linalg.svd(Gb[j], compute_uv=False).sum() for j in range(Gb.shape[0]))
        assert nuc > 0 and abs(inner - tau * nuc) <= 1e-9 * tau * nuc


def test_recovery_improves_with_samples_and_beats_the_sample_average():
    # smooth CP-rank-3 32x32x8 tensor scaled to max |L*| = 1, dither theta
    # = 1.2, noise 0.05, Gamma = {1, 2}, DFT, l1: the error falls as m grows
    # and stays well below that of the per-entry average of theta q
    rng = np.random.default_rng(0)
    S = smooth_tensor(32, 32, 8, rng)
    errs = []
    for mult in (2, 8, 32):
        s, q = synth.one_bit_observations(S, mult * S.size, 1.2, 0.05, rng)
        p = onebit.Params(modes=(1, 2), transform="fft", phi=prox.L1, lam=1e-3, theta=1.2,
                          alpha=1.0, tol=1e-7, max_iter=400)
        st, hist = onebit.run(S.shape, s, q, (8,), p)
        err = np.linalg.norm(st.L - S) / np.linalg.norm(S)
        J1, J2 = onebit.sample_tensors(S.shape, s, q, 1.2)
        avg = np.where(J2 > 0, J1 / np.maximum(J2, 1), 0.0)
        naive = np.linalg.norm(avg - S) / np.linalg.norm(S)
        assert err < 0.5 * naive, (mult, err, naive)
        errs.append(err)
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.2
