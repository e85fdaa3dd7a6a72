"""Learned sketch widths: slice features, the width plan and the
rank-predictor MLP, in float64.

Test infrastructure (see the package docstring).

Not in the paper.  Alg. 1 sketches every slice with one fixed rank and
Alg. 3 grows a basis until its error indicator meets a tolerance; Sec. 7
lists model-driven sketching as future work.  The learned engine predicts a
per-slice sketch width from the previous slice pass:

* ``features``      16 numbers per slice from its previous singular values
                    (any order; only the first ``width`` entries of a row
                    count), kept rank and width, and the shrink thresholds of
                    the previous and the current pass.
* ``forward``       y = MLP(F): 16 -> 128 -> 128 -> 128 -> 1 with ReLU after
                    each hidden layer; the weights (not the biases) are
                    rounded to IEEE half precision first, as the device
                    stores them.
* ``loss_grad``     loss (1/B) sum_r w_r (y_r - t_r)^2 with
                    w_r = 1 + under * [y_r < t_r] (under-prediction costs
                    more), and its gradient by backpropagation; the half
                    rounding of the weights passes gradients straight
                    through.
* ``adam_step``     Adam (Kingma & Ba, 2015) with bias correction.
* ``plan_widths``   l = round_up(round(exp(y) - 1) + p, 8) clipped to
                    [min(8, lmax), lmax], decided in float32 like the device;
                    slice ids stably sorted by width class (l - 1) // 8.
* ``threshold``     the smallest singular value the shrink keeps.
* ``judge``         which learned sketches the plain adaptive method
                    (Alg. 3 per slice) recomputes: a sketch is kept when it
                    meets Alg. 3's stop test (the energy its basis misses,
                    E = ||A||^2 - ||Q^T A||^2 with Q^T A's singular values
                    sig, below eps^2 ||A||^2), or its kept rank is at most
                    l - p (p directions seen beyond every singular value the
                    prox keeps), or l reaches the adaptive basis cap.

Parameter vector: per layer W (out x in, row-major) then b (out), layers in
order 16 -> 128, 128 -> 128, 128 -> 128, 128 -> 1 (35329 values).
"""

import numpy as np

N_FEAT = 16
HIDDEN = 128
LAYERS = 3
POSITIONS = (2, 4, 8, 16, 32, 64)
LOG129 = np.log(129.0)


def layer_shapes():
    ins = [N_FEAT] + [HIDDEN] * LAYERS
    outs = [HIDDEN] * LAYERS + [1]
    return list(zip(outs, ins))


def param_count():
    return sum(o * i + o for o, i in layer_shapes())


def unpack(params, fp16=True):
    """List of (W, b) per layer, W rounded to half precision when fp16."""
    p = np.asarray(params, dtype=np.float64)
    out, off = [], 0
    for o, i in layer_shapes():
        W = p[off:off + o * i].reshape(o, i)
        off += o * i
        b = p[off:off + o]
        off += o
        if fp16:
            W = W.astype(np.float32).astype(np.float16).astype(np.float64)
        out.append((W, b))
    assert off == p.size
    return out


def pack(layers):
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in layers])


def forward(params, X, fp16=True, keep=False):
    """y (B,) = MLP(X); with keep, also the post-ReLU hidden activations."""
    layers = unpack(params, fp16)
    h = np.asarray(X, dtype=np.float64)
    acts = []
    for W, b in layers[:-1]:
        h = np.maximum(h @ W.T + b, 0.0)
        acts.append(h)
    Wo, bo = layers[-1]
    y = (h @ Wo.T + bo)[:, 0]
    return (y, acts) if keep else y


def loss(params, X, t, under, fp16=True):
    y = forward(params, X, fp16)
    w = 1.0 + under * (y < t)
    return float(np.mean(w * (y - t) ** 2))


def loss_grad(params, X, t, under, fp16=True):
    """(loss, gradient with respect to the parameter vector)."""
    X = np.asarray(X, dtype=np.float64)
    B = X.shape[0]
    layers = unpack(params, fp16)
    y, acts = forward(params, X, fp16, keep=True)
    d = y - t
    w = 1.0 + under * (y < t)
    dy = 2.0 * w * d / B                                   # dloss/dy
    grads = [None] * len(layers)
    Wo, _ = layers[-1]
    grads[-1] = (dy[None, :] @ acts[-1], np.array([dy.sum()]))
    dz = np.outer(dy, Wo[0]) * (acts[-1] > 0)              # dloss/dz of the last hidden layer
    for li in range(len(layers) - 2, -1, -1):
        inp = X if li == 0 else acts[li - 1]
        grads[li] = (dz.T @ inp, dz.sum(axis=0))
        if li > 0:
            W, _ = layers[li]
            dz = (dz @ W) * (inp > 0)
    return float(np.mean(w * d * d)), pack(grads)


def adam_step(params, grad, m, v, lr, step, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step; returns (params, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return params - lr * mhat / (np.sqrt(vhat) + eps), m, v


def threshold(tau, kind, theta=1.0, gamma=4.0):
    """Smallest singular value with a nonzero shrink (see prox.prox_scalar)."""
    if kind == "l1" or gamma > tau:
        return tau * theta
    return theta * np.sqrt(gamma * tau)


def features(sig, rank, width, thr, thr0, tfrac):
    """(n, 16) features; row j uses sig[j, :width[j]] (any order)."""
    sig = np.asarray(sig, dtype=np.float64)
    n = sig.shape[0]
    F = np.zeros((n, N_FEAT))
    for j in range(n):
        w = int(min(max(width[j], 1), sig.shape[1]))
        s = sig[j, :w].copy()
        s[~(s > 0)] = 0.0
        s = np.sort(s)[::-1]
        s1 = s[0]
        F[j, 0] = np.log1p(max(int(rank[j]), 0)) / LOG129
        F[j, 1] = np.log(w) / LOG129

        def lratio(a, b):
            if not a > 0:
                return -1.0
            if not b > 0:
                return 1.0
            return float(np.clip(np.log(a / b), -8.0, 8.0) / 8.0)

        F[j, 2] = lratio(s1, thr)
        F[j, 3] = lratio(s1, thr0)
        for q, pos in enumerate(POSITIONS):
            F[j, 4 + q] = s[pos - 1] / s1 if (pos <= w and s1 > 0) else 0.0
        c_now = int(np.sum(s > thr))
        F[j, 10] = np.log1p(c_now) / LOG129
        F[j, 11] = np.log1p(int(np.sum(s > 0.5 * thr))) / LOG129
        F[j, 12] = np.log1p(int(np.sum(s > 2.0 * thr))) / LOG129
        F[j, 13] = (w - c_now) / w
        F[j, 14] = float(np.clip(np.log(thr / thr0), -1.0, 1.0)) if (thr > 0 and thr0 > 0) else 0.0
        F[j, 15] = float(np.clip(tfrac, 0.0, 1.0))
    return F


def width_of(y, p, lmax):
    """Sketch width of one prediction, decided in float32."""
    y = np.float32(y)
    if np.isnan(y):
        r = np.float32(lmax)
    else:
        r = np.floor(np.expm1(np.clip(y, np.float32(-20), np.float32(20))) + np.float32(0.5))
    r = int(min(max(float(r), 0.0), float(lmax)))
    l = (r + p + 7) // 8 * 8
    l = min(l, lmax)
    return max(l, min(8, lmax))


def plan_widths(yhat, p, lmax):
    """(width per slice, slice ids stably sorted by class, class counts)."""
    width = np.array([width_of(y, p, lmax) for y in np.asarray(yhat, dtype=np.float32)],
                     dtype=np.int64)
    cls = (width - 1) // 8
    ids = np.argsort(cls, kind="stable")
    counts = np.bincount(cls, minlength=(lmax + 7) // 8)
    return width, ids, counts


def judge(anorm2, sig, eps, rank, width, p, kcap):
    """Indices of the slices whose learned sketch is rejected.

    anorm2[j] = ||A_j||_F^2; sig[j] = the singular values of B_j = Q_j^T A_j
    (zero padding counts nothing); rank[j] the kept rank after the shrink,
    width[j] the sketch width.  The basis Q_j misses
    E_j = ||A_j||^2 - sum sig_j^2 = ||A_j - Q_j Q_j^T A_j||^2 of the energy
    (Pythagoras).  Kept: E_j < eps^2 ||A_j||^2 (Alg. 3's relative stop rule)
    or A_j = 0, or rank[j] <= width[j] - p, or width[j] >= kcap.
    """
    out = []
    for j, a2 in enumerate(np.asarray(anorm2, dtype=np.float64)):
        cap = float(np.sum(np.asarray(sig[j], dtype=np.float64) ** 2))
        alg3 = not (a2 > 0.0) or a2 - cap < eps * eps * a2
        margin = rank[j] <= width[j] - p
        wide = width[j] >= kcap
        if not (alg3 or margin or wide):
            out.append(j)
    return np.asarray(out, dtype=np.int64)
