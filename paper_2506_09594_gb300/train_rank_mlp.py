"""Train the rank predictor of the learned sketch-width engine.

Traces: seeded power-law problems (slice ranks p(r) ~ r^-1.5 on [2, 64];
slices of 128^2, 256^2 and 512^2 in turn) are recovered with the fixed-accuracy engine (Alg. 3 per slice).  Before
each slice pass t >= 1 the features of the previous pass are recorded
(tr_slice_features, exactly what the learned engine will see), and after the
pass the target log(1 + kept rank).  The MLP is then trained on the GPU
(tr_mlp_train: minibatch Adam, under-prediction weighted) and written as a
weights file (tr.save_model).  Everything runs through the C ABI.

    python -m paper_2506_09594_gb300.train_rank_mlp --out rank_mlp.bin
"""

import argparse
import json
import time

import numpy as np

from . import synth, tr


def trace(seed, dims, sr, iters, growth, rank_cap, oversample, eps, block):
    """(features, targets) of one recovery run with the fixed-accuracy engine."""
    import torch
    w = synth.Workload("trace", dims, "powerlaw", sr, dtype="f32", iters=iters, seed=seed,
                       noise_model="none")
    _, M, mask, _ = synth.make_problem(w)
    Md, maskd = torch.from_numpy(M).float().cuda(), torch.from_numpy(mask).cuda()
    h = None
    # the basis cap is rank + oversample rounded up to blocks; on the largest
    # slices a smaller oversample keeps the slice core within shared memory
    for ov in range(oversample, -1, -2):
        try:
            h = tr.Handle(Md, maskd, dims, engine=tr.TR_LR_ADAPTIVE, rank=rank_cap, oversample=ov,
                          adapt_eps=eps, adapt_block=block, noise=tr.TR_NOISE_NONE, tol=0.0,
                          max_iter=iters, growth=growth, seed=seed)
            break
        except tr.TrError:
            continue
    if h is None:
        raise RuntimeError("no basis cap fits for %s" % (dims,))
    feats, targets = [], []
    mu_next = None
    try:
        for t in range(iters):
            if t > 0:
                feats.append(h.slice_features(1.0 / mu_next, t).cpu().numpy())
            info = h.step(info=True)
            mu_next = min(info["mu"] * growth, 1e10)
            if t > 0:
                _, kept = h.slice_stats()
                targets.append(np.log1p(kept.astype(np.float64)))
    finally:
        h.close()
    return np.concatenate(feats), np.concatenate(targets)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--out", required=True)
    ap.add_argument("--seeds", type=int, default=200)
    ap.add_argument("--seed0", type=int, default=3000)
    ap.add_argument("--dims", default="128x128x8x8,256x256x4x4,512x512x2x2",
                    help="comma-separated trace shapes, used in turn")
    ap.add_argument("--iters", type=int, default=60)
    ap.add_argument("--growth", type=float, default=1.1)
    ap.add_argument("--rank-cap", type=int, default=64)
    ap.add_argument("--oversample", type=int, default=10)
    ap.add_argument("--steps", type=int, default=6000)
    ap.add_argument("--batch", type=int, default=1024)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--under", type=float, default=8.0)
    ap.add_argument("--holdout", type=int, default=10)
    args = ap.parse_args(argv)
    import torch

    shapes = [tuple(int(x) for x in d.split("x")) for d in args.dims.split(",")]
    rng = np.random.default_rng(args.seed0)
    t0 = time.time()
    X, Y = [], []
    for k in range(args.seeds + args.holdout):
        seed = args.seed0 + k if k < args.seeds else 4000 + (k - args.seeds)
        sr = float(rng.uniform(0.15, 0.5))
        dims = shapes[k % len(shapes)]
        f, y = trace(seed, dims, sr, args.iters, args.growth, args.rank_cap, args.oversample,
                     0.01, 10)
        X.append(f)
        Y.append(y)
    ntr = sum(x.shape[0] for x in X[:args.seeds])
    Xa = np.concatenate(X).astype(np.float32)
    Ya = np.concatenate(Y).astype(np.float32)
    t_trace = time.time() - t0
    params = tr.mlp_init(args.seed0)
    Xd = torch.from_numpy(Xa[:ntr]).cuda()
    Yd = torch.from_numpy(Ya[:ntr]).cuda()
    hist = tr.mlp_train(params, Xd, Yd, args.batch, args.steps, args.lr, args.under,
                        args.seed0 + 1).cpu().numpy()
    torch.cuda.synchronize()
    t_train = time.time() - t0 - t_trace
    # held-out report: how often the planned width would have kept the rank
    pred = tr.mlp_forward(params, torch.from_numpy(Xa[ntr:]).cuda()).cpu().numpy()
    lmax = args.rank_cap + args.oversample
    width = np.minimum(np.maximum((np.floor(np.expm1(pred) + 0.5).clip(0, lmax).astype(int)
                                   + args.oversample + 7) // 8 * 8, 8), lmax)
    kept = np.rint(np.expm1(Ya[ntr:])).astype(int)
    covered = float(np.mean((kept <= width - args.oversample) | (width == lmax)))
    tr.save_model(args.out, params.cpu().numpy())
    report = {"samples": int(ntr), "holdout_samples": int(Xa.shape[0] - ntr),
              "trace_s": round(t_trace, 1), "train_s": round(t_train, 1),
              "loss_first": float(np.mean(hist[:50])), "loss_last": float(np.mean(hist[-50:])),
              "holdout_covered": covered, "holdout_mean_width": float(width.mean()),
              "lmax": lmax}
    print(json.dumps(report))
    return report


if __name__ == "__main__":
    main()
