"""Pins of the learned-width oracle (oracle/learned.py) against closed forms,
finite differences and hand-worked examples."""

import numpy as np
import pytest

from oracle import learned as lo


def _params(seed, scale=0.2):
    rng = np.random.default_rng(seed)
    return scale * rng.standard_normal(lo.param_count())


def test_param_count_matches_architecture():
    assert lo.param_count() == 16 * 128 + 128 + 2 * (128 * 128 + 128) + 128 + 1 == 35329


def test_forward_identity_hidden_layers_closed_form():
    # W2 = W3 = I, zero biases: y = w_o . relu(relu(relu(W1 x))) = w_o . relu(W1 x)
    rng = np.random.default_rng(1)
    W1 = rng.standard_normal((128, 16))
    wo = rng.standard_normal((1, 128))
    layers = [(W1, np.zeros(128)), (np.eye(128), np.zeros(128)), (np.eye(128), np.zeros(128)),
              (wo, np.zeros(1))]
    X = rng.standard_normal((7, 16))
    y = lo.forward(lo.pack(layers), X, fp16=False)
    want = np.array([wo[0] @ np.maximum(W1 @ x, 0.0) for x in X])
    np.testing.assert_allclose(y, want, rtol=1e-13, atol=1e-13)


def test_forward_positive_homogeneity_without_biases():
    layers = lo.unpack(_params(2), fp16=False)
    layers = [(W, np.zeros_like(b)) for W, b in layers]
    p = lo.pack(layers)
    X = np.random.default_rng(3).standard_normal((5, 16))
    for a in (0.5, 3.0):
        np.testing.assert_allclose(lo.forward(p, a * X, fp16=False), a * lo.forward(p, X, fp16=False),
                                   rtol=1e-12, atol=1e-12)


def test_forward_bias_only_network():
    # all weights zero: every hidden unit is relu(bias), output = wo . relu(b3) + bo
    layers = [(np.zeros((o, i)), np.full(o, 0.5)) for o, i in lo.layer_shapes()]
    layers[-1] = (np.full((1, 128), 2.0), np.array([-1.0]))
    y = lo.forward(lo.pack(layers), np.ones((3, 16)), fp16=False)
    np.testing.assert_allclose(y, 128 * 2.0 * 0.5 - 1.0)


def test_fp16_rounding_exact_for_representable_weights():
    rng = np.random.default_rng(4)
    p = np.round(_params(4) * 256) / 256          # multiples of 2^-8, |w| < 2: exact in half
    X = rng.standard_normal((6, 16))
    np.testing.assert_array_equal(lo.forward(p, X, fp16=True), lo.forward(p, X, fp16=False))
    q = p + 1e-5                                   # not representable: rounding changes y
    assert np.max(np.abs(lo.forward(q, X, True) - lo.forward(q, X, False))) > 0


@pytest.mark.parametrize("under", [0.0, 0.7])
def test_gradient_matches_central_differences(under):
    rng = np.random.default_rng(5)
    p = _params(5, 0.3)
    X = rng.standard_normal((9, 16))
    t = rng.standard_normal(9)
    _, g = lo.loss_grad(p, X, t, under, fp16=False)
    idx = np.concatenate([rng.choice(lo.param_count(), 60, replace=False),
                          np.arange(lo.param_count() - 129, lo.param_count())])
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (lo.loss(p + e, X, t, under, False) - lo.loss(p - e, X, t, under, False)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_loss_special_cases():
    rng = np.random.default_rng(6)
    p = _params(6)
    X = rng.standard_normal((11, 16))
    y = lo.forward(p, X)
    t = y + rng.uniform(0.1, 1.0, 11)             # every row under-predicted
    mse = np.mean((y - t) ** 2)
    assert lo.loss(p, X, t, 0.0) == pytest.approx(mse, rel=1e-14)
    assert lo.loss(p, X, t, 0.5) == pytest.approx(1.5 * mse, rel=1e-14)
    assert lo.loss(p, X, y - 1.0, 0.5) == pytest.approx(1.0, rel=1e-14)   # over-predicted: weight 1


def test_adam_without_moments_is_sign_descent():
    rng = np.random.default_rng(7)
    p = rng.standard_normal(50)
    g = rng.standard_normal(50)
    m = np.zeros(50)
    v = np.zeros(50)
    for step in (1, 2, 3):
        p2, m, v = lo.adam_step(p, g, m, v, lr=0.01, step=step, beta1=0.0, beta2=0.0, eps=1e-12)
        np.testing.assert_allclose(p2 - p, -0.01 * np.sign(g), rtol=1e-9)
        p = p2


def test_adam_bias_correction_makes_constant_gradient_steps_exactly_lr():
    # Kingma & Ba (2015), Sec. 2-3: with the bias corrections, a gradient that
    # stays constant gives m_hat = g and v_hat = g^2 at every step, so each
    # update is -lr g / (|g| + eps) whatever beta1 and beta2 are; without
    # either correction the early steps are off by (1 - beta^t) factors (rtol
    # 1e-6 covers eps against the smallest |g| and the cancellation in p2 - p)
    rng = np.random.default_rng(8)
    p = rng.standard_normal(40)
    g = rng.standard_normal(40)
    m = np.zeros(40)
    v = np.zeros(40)
    for step in range(1, 6):
        p2, m, v = lo.adam_step(p, g, m, v, lr=0.02, step=step, beta1=0.9, beta2=0.999, eps=1e-12)
        np.testing.assert_allclose(p2 - p, -0.02 * np.sign(g), rtol=1e-6)
        p = p2


def test_adam_minimises_a_quadratic():
    c = np.linspace(-1, 1, 20)
    p = np.zeros(20)
    m = np.zeros(20)
    v = np.zeros(20)
    for step in range(1, 3001):
        p, m, v = lo.adam_step(p, p - c, m, v, lr=0.01, step=step)
    np.testing.assert_allclose(p, c, atol=1e-3)


def test_features_worked_example():
    # row (unsorted) 1, 8, 2, 4 with width 4, kept rank 2, thr 3, thr0 1.5, t/T 0.25;
    # a trailing 100 lies beyond the width and must be ignored
    sig = np.array([[1.0, 8.0, 2.0, 4.0, 100.0]])
    F = lo.features(sig, [2], [4], 3.0, 1.5, 0.25)[0]
    L = np.log(129.0)
    want = np.zeros(16)
    want[0] = np.log(3.0) / L
    want[1] = np.log(4.0) / L
    want[2] = np.log(8.0 / 3.0) / 8
    want[3] = np.log(8.0 / 1.5) / 8
    want[4] = 4.0 / 8.0               # 2nd largest
    want[5] = 1.0 / 8.0               # 4th largest
    want[10] = np.log(3.0) / L        # 8, 4 above 3
    want[11] = np.log(4.0) / L        # 8, 4, 2 above 1.5
    want[12] = np.log(2.0) / L        # 8 above 6
    want[13] = 0.5
    want[14] = np.log(2.0)
    want[15] = 0.25
    np.testing.assert_allclose(F, want, rtol=1e-14, atol=1e-15)


def test_features_degenerate_rows():
    sig = np.array([[0.0, 0.0, 0.0], [5.0, np.nan, -1.0]])
    F = lo.features(sig, [0, 1], [3, 3], 0.0, 2.0, 7.0)
    assert F[0, 2] == -1.0 and F[0, 3] == -1.0 and np.all(F[0, 4:10] == 0)
    assert F[1, 2] == 1.0                      # threshold 0 counts as +infinity ratio
    assert F[1, 14] == 0.0 and F[1, 15] == 1.0
    assert F[1, 10] == pytest.approx(np.log(2.0) / np.log(129.0))   # 5 > 0; NaN, -1 count as 0


def test_features_order_invariant():
    rng = np.random.default_rng(8)
    s = rng.uniform(0, 10, (4, 70))
    w = np.array([70, 33, 9, 1])
    F = lo.features(s, [3, 4, 5, 0], w, 2.0, 2.5, 0.5)
    s2 = s.copy()
    for j in range(4):
        s2[j, :w[j]] = rng.permutation(s[j, :w[j]])
    np.testing.assert_array_equal(F, lo.features(s2, [3, 4, 5, 0], w, 2.0, 2.5, 0.5))


def test_plan_widths_exact_log_ranks():
    p, lmax = 10, 74
    r = np.arange(0, 80)
    width, ids, counts = lo.plan_widths(np.log1p(r), p, lmax)
    want = np.minimum(np.maximum((np.minimum(r, lmax) + p + 7) // 8 * 8, 8), lmax)
    np.testing.assert_array_equal(width, want)
    cls = (width - 1) // 8
    assert np.all(np.diff(cls[ids]) >= 0)
    for c in range(counts.size):             # stable: ids ascending within a class
        sel = ids[cls[ids] == c]
        assert np.all(np.diff(sel) > 0)
    assert counts.sum() == r.size and counts.size == 10


def test_plan_widths_edge_values():
    # p = 6: a predicted rank of 2 fits in 8 columns, 3 needs 16
    w, _, _ = lo.plan_widths(np.array([np.nan, -50.0, 50.0, np.log1p(2.49), np.log1p(2.51)]), 6, 40)
    np.testing.assert_array_equal(w, [40, 8, 40, 8, 16])
    w, _, c = lo.plan_widths(np.array([0.0, 5.0]), 0, 5)   # lmax below 8
    np.testing.assert_array_equal(w, [5, 5])
    assert c.tolist() == [2]


def test_threshold():
    assert lo.threshold(0.5, "l1", 2.0) == 1.0
    assert lo.threshold(0.5, "mcp", 2.0, 4.0) == 1.0
    assert lo.threshold(9.0, "mcp", 1.0, 4.0) == 6.0


def test_judge_worked_example():
    # A = diag(3, 4): ||A||^2 = 25.  A basis that captures the 4 misses
    # E = 9: rejected at eps = 0.5 (9 >= 0.25 * 25), kept at eps = 0.7
    # (9 < 0.49 * 25); a basis capturing both misses nothing; A = 0 is kept;
    # here the shrink kept 1 of width 1 (no margin at p = 1), cap 4
    def J(a2, sig, eps, rank=(1,), width=(1,), p=1, kcap=4):
        return lo.judge(a2, sig, eps, rank, width, p, kcap).tolist()

    assert J([25.0], [[4.0]], 0.5) == [0]
    assert J([25.0], [[4.0]], 0.7) == []
    assert J([25.0, 0.0], [[4.0, 3.0], [0.0]], 1e-3, (1, 0), (1, 1)) == []
    # the boundary itself fails the strict test: E = eps^2 ||A||^2
    assert J([25.0], [[4.0]], 0.6) == [0]
    # the oversampling margin (kept rank <= width - p) or a width at the
    # adaptive cap keeps a sketch that misses energy
    assert J([25.0], [[4.0]], 0.5, (1,), (2,)) == []
    assert J([25.0], [[4.0]], 0.5, (1,), (1,), 1, 1) == []
    assert J([25.0], [[4.0]], 0.5, (2,), (2,)) == [0]


def test_judge_is_the_projection_error_test():
    # E = ||A||^2 - ||Q^T A||^2 equals ||A - Q Q^T A||^2 for orthonormal Q
    # (Pythagoras), so the judge takes Alg. 3's decision computed directly
    rng = np.random.default_rng(7)
    eps = 0.1
    a2, sig, direct = [], [], []
    for j in range(40):
        n1, n2, r, l = 30, 24, int(rng.integers(1, 12)), int(rng.integers(1, 14))
        A = rng.standard_normal((n1, r)) @ rng.standard_normal((r, n2))
        A += 10.0 ** rng.uniform(-4, -1) * rng.standard_normal((n1, n2))
        Q, _ = np.linalg.qr(A @ rng.standard_normal((n2, l)))
        res = np.linalg.norm(A - Q @ (Q.T @ A)) ** 2
        a2.append(np.linalg.norm(A) ** 2)
        sig.append(np.linalg.svd(Q.T @ A, compute_uv=False))
        direct.append(not (res < eps * eps * a2[-1]))
    n = len(a2)
    # no margin (kept rank = width) and no cap: Alg. 3's test alone decides
    got = set(lo.judge(a2, sig, eps, [9] * n, [9] * n, 1, 10 ** 9).tolist())
    assert got == {j for j, d in enumerate(direct) if d}
    assert 0 < len(got) < 40


def test_width_plan_and_feature_invariants_property():
    # widths: within [min(8, lmax), lmax], a multiple of 8 or lmax itself, at
    # least min(rank + p, lmax) for the predicted rank, non-decreasing in the
    # prediction, lmax for NaN; the plan: ids a permutation stably sorted by
    # class, counts per class; features within their stated ranges
    hyp = pytest.importorskip("hypothesis")
    st = hyp.strategies

    @hyp.settings(max_examples=60, deadline=None, derandomize=True)
    @hyp.given(st.lists(st.floats(-30, 30, allow_nan=False, width=32), min_size=1, max_size=40),
               st.integers(0, 20), st.integers(1, 96))
    def check(ys, p, lmax):
        w = [lo.width_of(y, p, lmax) for y in ys]
        for y, wi in zip(ys, w):
            assert min(8, lmax) <= wi <= lmax and (wi % 8 == 0 or wi == lmax)
            r = min(max(float(np.floor(np.expm1(np.clip(np.float32(y), -20, 20)) + 0.5)), 0.0), lmax)
            assert wi >= min(int(r) + p, lmax)
        order = np.argsort(np.asarray(ys, dtype=np.float32), kind="stable")
        assert all(w[a] <= w[b] for a, b in zip(order, order[1:]))
        assert lo.width_of(np.float32("nan"), p, lmax) == lmax
        width, ids, counts = lo.plan_widths(np.asarray(ys, dtype=np.float32), p, lmax)
        assert sorted(ids.tolist()) == list(range(len(ys)))
        cls = (width - 1) // 8
        assert all(cls[a] < cls[b] or (cls[a] == cls[b] and a < b) for a, b in zip(ids, ids[1:]))
        assert counts.sum() == len(ys) and len(counts) == (lmax + 7) // 8
        assert all(counts[c] == np.sum(cls == c) for c in range(len(counts)))

    check()

    @hyp.settings(max_examples=40, deadline=None, derandomize=True)
    @hyp.given(st.integers(1, 12), st.integers(1, 20), st.data())
    def features(n, ld, data):
        rng = np.random.default_rng(n * 50 + ld)
        sig = rng.lognormal(0.0, 2.0, (n, ld)) * (rng.random((n, ld)) < 0.8)
        width = rng.integers(1, ld + 1, n)
        rank = rng.integers(0, 100, n)
        pos = st.one_of(st.just(0.0), st.floats(1e-6, 5.0))
        thr, thr0 = data.draw(pos), data.draw(pos)
        F = lo.features(sig, rank, width, thr, thr0, data.draw(st.floats(-1.0, 2.0)))
        lower = np.array([0, 0, -1, -1] + [0] * 6 + [0, 0, 0, 0, -1, 0], dtype=float)
        upper = np.array([1, 1, 1, 1] + [1] * 6 + [1, 1, 1, 1, 1, 1], dtype=float)
        upper[0] = np.log1p(99) / np.log(129)
        assert np.all(F >= lower - 1e-12) and np.all(F <= upper + 1e-12)

    features()
