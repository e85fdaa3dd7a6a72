"""GPU parity of the learned sketch-width engine and the rank-predictor MLP
(through the C ABI) against the FP64 oracle.

Tolerances: the MLP runs FP16 weights with FP32 accumulation; the oracle
gets the same half-rounded weights, so the outputs differ by FP32 rounding
of sums of at most 129 terms (rel 1e-5 of the output scale), and gradients
likewise (1e-4 of their scale).  Widths, slice orders and counts are
integers: bit-exact, away from the rounding boundaries of exp(y) - 1.  A
slice pass on exactly low-rank slices is exact for every width above the
rank, so it is compared with the full-SVD prox at the FP32 bound 1e-4.
"""

import numpy as np
import pytest

from oracle import learned as lo
from oracle import admm, prox, svt
from paper_2506_09594_gb300 import synth, tr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev(x, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype)


def host(t):
    return t.double().cpu().numpy()


def relF(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def params(seed, scale=0.15):
    rng = np.random.default_rng(seed)
    return (scale * rng.standard_normal(lo.param_count())).astype(np.float32)


def previous_rank_model():
    """An MLP that outputs log(1 + previous kept rank): f0 * log 129 through
    one unit of each hidden layer (exact in half precision up to the
    rounding of log 129)."""
    layers = [(np.zeros((o, i)), np.zeros(o)) for o, i in lo.layer_shapes()]
    layers[0][0][0, 0] = np.log(129.0)
    layers[1][0][0, 0] = 1.0
    layers[2][0][0, 0] = 1.0
    layers[3][0][0, 0] = 1.0
    return lo.pack(layers).astype(np.float32)


def constant_model(r):
    layers = [(np.zeros((o, i)), np.zeros(o)) for o, i in lo.layer_shapes()]
    layers[3][1][0] = np.log1p(r)
    return lo.pack(layers).astype(np.float32)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    tr.load()


# ------------------------------------------------------------------ MLP
@pytest.mark.parametrize("B", [1, 31, 32, 100, 512])
def test_mlp_forward_parity(B):
    p = params(10 + B)
    X = np.random.default_rng(B).standard_normal((B, 16)).astype(np.float32)
    y = host(tr.mlp_forward(dev(p), dev(X)))
    ref = lo.forward(p.astype(np.float64), X.astype(np.float64), fp16=True)
    scale = max(1.0, np.max(np.abs(ref)))
    assert np.max(np.abs(y - ref)) < 1e-5 * scale


@pytest.mark.parametrize("B,under", [(7, 0.0), (64, 0.5), (333, 2.0)])
def test_mlp_loss_grad_parity(B, under):
    p = params(20 + B)
    rng = np.random.default_rng(B + 1)
    X = rng.standard_normal((B, 16)).astype(np.float32)
    t = rng.standard_normal(B).astype(np.float32)
    loss, g = tr.mlp_loss_grad(dev(p), dev(X), dev(t), under)
    rl, rg = lo.loss_grad(p.astype(np.float64), X.astype(np.float64), t.astype(np.float64), under,
                          fp16=True)
    assert abs(float(loss.item()) - rl) < 1e-5 * max(1.0, rl)
    g = host(g)
    assert np.max(np.abs(g - rg)) < 1e-4 * max(1e-3, np.max(np.abs(rg)))


def test_mlp_adam_parity():
    rng = np.random.default_rng(30)
    p = rng.standard_normal(lo.param_count()).astype(np.float32)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    pd, md, vd = dev(p), dev(m), dev(v)
    pr, mr, vr = p.astype(np.float64), m.astype(np.float64), v.astype(np.float64)
    for step in (1, 2, 3):
        g = rng.standard_normal(p.size).astype(np.float32)
        tr.mlp_adam(pd, dev(g), md, vd, lr=1e-2, step=step)
        pr, mr, vr = lo.adam_step(pr, g.astype(np.float64), mr, vr, 1e-2, step)
    assert np.max(np.abs(host(pd) - pr)) < 1e-5 * max(1.0, np.max(np.abs(pr)))


def test_mlp_init_is_seeded_he_uniform():
    a = host(tr.mlp_init(5))
    b = host(tr.mlp_init(5))
    c = host(tr.mlp_init(6))
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    off = 0
    for o, i in lo.layer_shapes():
        W = a[off:off + o * i]
        bias = a[off + o * i:off + o * i + o]
        bound = np.sqrt(6.0 / i)
        assert np.all(np.abs(W) < bound) and np.all(bias == 0)
        if W.size > 1000:   # uniform: variance bound^2 / 3
            assert abs(np.var(W) / (bound ** 2 / 3) - 1) < 0.05
        off += o * i + o


def test_mlp_train_fits_a_teacher():
    # teacher: a random network (oracle forward, FP64); the student trained on
    # the GPU must reach a loss well below the variance of the targets
    rng = np.random.default_rng(40)
    teacher = params(41, 0.1).astype(np.float64)
    X = rng.standard_normal((4096, 16))
    y = lo.forward(teacher, X, fp16=False)
    student = tr.mlp_init(42)
    hist = host(tr.mlp_train(student, dev(X), dev(y), batch=256, steps=1500, lr=2e-3,
                             under_weight=0.0, seed=43))
    final = lo.loss(host(student), X, y, 0.0, fp16=True)
    assert final < 0.05 * np.var(y), (final, np.var(y))
    assert np.mean(hist[-100:]) < 0.1 * np.mean(hist[:20])


# ------------------------------------------------------ features / plan
@pytest.mark.parametrize("dt", [torch.float32, torch.float64])
def test_features_parity(dt):
    rng = np.random.default_rng(50)
    n, ld = 300, 74
    sig = rng.lognormal(0.0, 1.5, (n, ld))
    sig[rng.random((n, ld)) < 0.2] = 0.0
    sig[5, :] = 0.0
    sig[6, :3] = 7.0                               # ties
    width = rng.integers(1, ld + 1, n).astype(np.int32)
    width[:3] = [1, 64, ld]
    rank = rng.integers(0, 80, n).astype(np.int32)
    sig_dev = dev(sig, dt)
    sig_in = host(sig_dev)                          # the values the device holds
    for thr, thr0, tf in [(2.0, 1.7, 0.3), (0.5, 5.0, 1.4), (0.0, 1.0, -0.1)]:
        F = host(tr.features(sig_dev, dev(rank, torch.int32), dev(width, torch.int32),
                             thr, thr0, tf))
        ref = lo.features(sig_in, rank, width, thr, thr0, tf)
        assert np.max(np.abs(F - ref)) < 2e-6, np.unravel_index(np.argmax(np.abs(F - ref)), F.shape)


@pytest.mark.parametrize("n,p,lmax", [(1, 10, 74), (517, 10, 74), (2500, 4, 96), (40, 0, 5),
                                      (1000, 10, 20)])
def test_plan_widths_parity(n, p, lmax):
    rng = np.random.default_rng(n + lmax)
    y = rng.uniform(-1.0, 5.0, n).astype(np.float32)
    # keep exp(y) - 1 away from the rounding boundaries k + 1/2
    r = np.expm1(y.astype(np.float64))
    frac = r - np.floor(r)
    y[np.abs(frac - 0.5) < 1e-3] = np.float32(np.log1p(3.0))
    width, ids, counts = tr.plan_widths(dev(y), p, lmax)
    rw, rids, rcounts = lo.plan_widths(y, p, lmax)
    assert np.array_equal(width.cpu().numpy(), rw)
    assert np.array_equal(ids.cpu().numpy(), rids)
    assert np.array_equal(counts.cpu().numpy(), rcounts)


# ------------------------------------------------------- learned engine
def _learned_handle(dims, rank, oversample, model=None, **kw):
    n = int(np.prod(dims[2:]))
    M = torch.zeros((n, dims[0], dims[1]), dtype=torch.float32, device="cuda")
    mask = torch.ones((n, dims[0], dims[1]), dtype=torch.uint8, device="cuda")
    h = tr.Handle(M, mask, dims, engine=tr.TR_LR_LEARNED, rank=rank, oversample=oversample,
                  phi=tr.TR_PEN_L1, seed=9, **kw)
    if model is not None:
        h.set_model(model)
    return h


def _lowrank(n, n1, n2, seed, hi=30):
    rng = np.random.default_rng(seed)
    ranks = rng.integers(1, hi + 1, n)
    return synth.lowrank_plus_noise_stack(n, n1, n2, ranks, 0.0, seed=seed + 1), ranks


@pytest.mark.parametrize("prec", [tr.TR_PREC_FP32, tr.TR_PREC_BF16X3])
def test_learned_previous_rank_predictor_exact_on_low_rank(prec):
    n, n1, n2 = 48, 96, 80
    Ab, ranks = _lowrank(n, n1, n2, 60)
    # the smallest nonzero singular value of these slices is above 2; rounding
    # noise of the sketched products stays far below tau
    tau = 0.1
    h = _learned_handle((n1, n2, 8, 6), 30, 10, previous_rank_model(), prec=prec)
    ref, _ = svt.transformed_prox(Ab, tau, prox.L1, engine="full")
    Ad = dev(Ab)
    for t in range(3):
        G = host(h.slice_prox(Ad, tau, t))
        assert relF(G, ref) < 1e-4, (t, relF(G, ref))
        _, kept = h.slice_stats()
        assert np.array_equal(kept, ranks)
        w = h.slice_widths()
        if t == 0:
            # no history: the plain adaptive method, whose basis is the rank
            assert np.array_equal(w, ranks)
        else:
            want = np.minimum((ranks + 10 + 7) // 8 * 8, 40)
            # groups smaller than 8 slices run at the next wider width; every
            # sketch captures its slice, so the judge keeps them all
            assert np.all(w >= want) and np.all(w <= 40) and np.all(w % 8 == 0)
            assert np.all(w[want == 40] == 40)
    h.close()


def test_learned_judge_falls_back_to_the_adaptive_engine(tmp_path):
    n, n1, n2 = 40, 90, 100
    Ab, ranks = _lowrank(n, n1, n2, 70)
    tau = 0.1
    # a weights file that always predicts rank 2 (l = 16), read by tr_init
    path = tmp_path / "const2.bin"
    tr.save_model(str(path), constant_model(2))
    h = _learned_handle((n1, n2, n), 30, 10, model_path=str(path).encode())
    ref, _ = svt.transformed_prox(Ab, tau, prox.L1, engine="full")
    Ad = dev(Ab)
    h.slice_prox(Ad, tau, 0)
    G = host(h.slice_prox(Ad, tau, 1))
    assert relF(G, ref) < 1e-4
    # a width-16 sketch captures a slice of rank <= 16 exactly (kept by
    # Alg. 3's test); above that it misses energy with no oversampling
    # margin (kept rank 16 > 16 - 10) below the adaptive cap 40, and the
    # adaptive engine's basis (the rank) replaces it
    np.testing.assert_array_equal(h.slice_widths(), np.where(ranks > 16, ranks, 16))
    h.close()


@pytest.mark.parametrize("prec", [tr.TR_PREC_FP32, tr.TR_PREC_BF16X3])
def test_learned_pass_matches_oracle_with_rejections(tmp_path, prec):
    # slices of rank 3..8 or 24..30 and a constant predictor (rank 2, width
    # 16): a width-16 sketch misses nothing of the low-rank slices (rounding
    # only, far below eps^2 = 1e-4 of the energy) and a third or more of the
    # high-rank ones, whose kept rank 16 leaves no oversampling margin, so
    # both sides take the same decisions; the accepted slices are the
    # randomized prox at width 16, the rejected ones the adaptive engine's,
    # whose deflation keeps exactly the rank (the oracle runs both with the
    # same Philox draws)
    n, n1, n2 = 24, 72, 64
    rng = np.random.default_rng(81)
    ranks = np.where(rng.random(n) < 0.5, rng.integers(3, 9, n), rng.integers(24, 31, n))
    Ab = synth.lowrank_plus_noise_stack(n, n1, n2, ranks, 0.0, seed=82)
    A32 = Ab.astype(np.float32).astype(np.float64)
    tau = 0.05 * np.linalg.svd(A32[0], compute_uv=False)[0]
    path = tmp_path / "const2.bin"
    tr.save_model(str(path), constant_model(2))
    h = _learned_handle((n1, n2, n), 30, 10, model_path=str(path).encode(), prec=prec)
    Ad = dev(Ab)
    h.slice_prox(Ad, tau, 0)
    G = host(h.slice_prox(Ad, tau, 1))
    w = h.slice_widths()
    h.close()
    ref, info = svt.transformed_prox(A32, tau, prox.L1, engine="learned", widths=[16] * n, q=1,
                                     seed=9, t=1, eps=0.01, b=10, delta_rel=1e-5, max_rank=40,
                                     p=10)
    assert sorted(info["fallback"].tolist()) == np.flatnonzero(ranks > 16).tolist()
    np.testing.assert_array_equal(w, info["widths"])
    assert relF(G, ref) < 1e-4, relF(G, ref)


def test_learned_rejects_bad_model_file(tmp_path):
    path = tmp_path / "bad.bin"
    path.write_bytes(b"TRRANK01" + b"\0" * 20)
    with pytest.raises(tr.TrError):
        _learned_handle((40, 40, 4), 10, 10, model_path=str(path).encode())


@pytest.mark.parametrize("model", ["previous_rank", "trained"])
def test_learned_step_recovers_like_the_plain_width(model):
    # A/B on a power-law problem that the ADMM recovers: the learned engine
    # (a hand-built previous-rank predictor, or the shipped trained weights)
    # against the plain fixed width l_max = 74.  Equal recovery error (within
    # 1e-4) with far narrower sketches.
    import os
    if model == "trained" and not os.path.exists(tr.DEFAULT_MODEL):
        pytest.skip("no trained weights file")
    w = synth.Workload("pl", (256, 256, 8, 8), "powerlaw", 0.5, dtype="f32", l=74, q=1,
                       iters=60, seed=4001, noise_model="none")
    X, M, mask, ranks = synth.make_problem(w)
    errs, widths, fbs = {}, {}, {}
    engines = {"rsvd": tr.TR_LR_RSVD, "adaptive": tr.TR_LR_ADAPTIVE, "learned": tr.TR_LR_LEARNED}
    for eng in ("rsvd", "adaptive", "learned"):
        # the adaptive cap: rank + oversample rounded to whole blocks, as the
        # learned engine's fallback (70 of l_max = 74)
        kw = dict(engine=engines[eng], rank=64, oversample=6 if eng == "adaptive" else 10,
                  noise=tr.TR_NOISE_NONE, seed=5, tol=0.0, max_iter=w.iters, growth=1.15)
        h = tr.Handle(dev(M), torch.from_numpy(mask).cuda(), w.dims, **kw)
        if eng == "learned":
            h.set_model(previous_rank_model() if model == "previous_rank"
                         else tr.load_model(tr.DEFAULT_MODEL))
        fbs[eng] = 0
        for _ in range(w.iters):
            fbs[eng] += h.step(info=True)["fallback_slices"]
        errs[eng] = relF(host(h.get_state()["L"]), X)
        widths[eng] = h.slice_widths()
        _, kept = h.slice_stats()
        h.close()
    assert errs["rsvd"] < 5e-3, errs                 # the regime converges
    # every learned slice meets Alg. 3's test or is Alg. 3's own result, so
    # the learned engine recovers as well as the plain adaptive method
    assert errs["learned"] <= errs["adaptive"] + 1e-4, errs
    assert np.all(widths["rsvd"] == 74) and fbs["rsvd"] == 0
    assert widths["learned"].mean() < 0.5 * 74, widths["learned"].mean()
    # the judge kept most slices: fewer fallbacks than slice passes
    assert fbs["learned"] < 0.5 * (w.iters - 1) * 64, fbs["learned"]


@pytest.mark.slow
@pytest.mark.parametrize("model,prec", [("previous_rank", tr.TR_PREC_FP32),
                                        ("trained", tr.TR_PREC_BF16X3),
                                        ("trained", tr.TR_PREC_BF16)])
def test_learned_full_size_sampled(model, prec):
    # the 512 x 512 x 32 x 16 power-law shape (512 slices of rank 2..64,
    # l_max = 64 + 10) in the launch configuration of a step: the first pass
    # is the adaptive method, the second runs at the planned widths.  Every
    # width above the rank gives the exact prox and Alg. 3's judge sends the
    # rest to the adaptive engine, so the kept ranks equal the slice ranks
    # bit for bit on all 512 slices, and four sampled slices match the FP64
    # full-SVD prox (split BF16 at the FP32 bound, plain BF16 products at
    # 1e-3)
    import os
    if model == "trained" and not os.path.exists(tr.DEFAULT_MODEL):
        pytest.skip("no trained weights file")
    n, n1, n2, p, lmax = 512, 512, 512, 10, 74
    ranks = synth.powerlaw_ranks(n, np.random.default_rng(512))
    Ab = synth.lowrank_plus_noise_stack(n, n1, n2, ranks, 0.0, seed=513)
    tau = 0.1        # the smallest nonzero singular value is above 10
    h = _learned_handle((n1, n2, 32, 16), 64, p, prec=prec,
                        **({} if model == "previous_rank"
                           else {"model_path": tr.DEFAULT_MODEL.encode()}))
    if model == "previous_rank":
        h.set_model(previous_rank_model())
    Ad = dev(Ab)
    tol = 1e-3 if prec == tr.TR_PREC_BF16 else 1e-4
    sample = (0, 129, 300, 511)
    refs = {j: svt.slice_prox_full(Ab[j], tau, prox.L1)[0] for j in sample}
    del Ab
    for t in range(2):
        G = h.slice_prox(Ad, tau, t)
        _, kept = h.slice_stats()
        w = h.slice_widths()
        assert np.array_equal(kept, ranks), (t, np.flatnonzero(kept != ranks)[:8])
        # every result rests on a basis at least as wide as the rank (the
        # adaptive basis may keep a few FP32 rounding directions beyond it)
        assert np.all(w >= ranks), (t, np.flatnonzero(w < ranks)[:8])
        if t == 1 and model == "previous_rank":
            want = np.minimum((ranks + p + 7) // 8 * 8, lmax)
            assert np.all(w >= want) and w.mean() < lmax - 20
        for j in sample:
            err = relF(host(G[j]), refs[j])
            assert err < tol, (t, j, err)
        del G
    h.close()
