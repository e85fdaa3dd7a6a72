"""Graph replay, tube-tile autotuning and batches of uneven problems.

A replayed step runs the same kernels with the same arguments as an eager
step (the schedule is read on the device), and every tube tile computes the
same values, so these are compared bit for bit with the eager single-handle
path, which the parity tests pin to the oracle.  One multi-step comparison
with the oracle itself checks the device schedule (mu, t) end to end.
"""

import numpy as np
import pytest

from oracle import admm
from paper_2506_09594_gb300 import synth, tr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TDT = {"f64": torch.float64, "f32": torch.float32}


def dev(x, dt):
    return torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda", dtype=TDT[dt])


def host(t):
    return t.double().cpu().numpy()


def relF(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def as_dtype(x, dt):
    return x.astype(np.float32).astype(np.float64) if dt == "f32" else x


def problem(dims, seed, rank=4, sr=0.4):
    rng = np.random.default_rng(seed)
    X = synth.lowrank_tensor(dims, rank, rng)[0]
    mask = synth.exact_count_mask(X.size, sr, rng).reshape(X.shape)
    S = synth.exact_count_mask(X.size, 0.05, rng).reshape(X.shape) * rng.uniform(-1, 1, X.shape)
    M = np.where(mask == 1, X + S, 0.0)
    return X, M, mask


def handle(dims, dt, M, mask, **kw):
    return tr.Handle(dev(M, dt), torch.from_numpy(mask).cuda(), dims, **kw)


def states_equal(a, b):
    for k in ("L", "E", "Y", "Lam", "G"):
        if not torch.equal(a[k], b[k]):
            return False, k
    return a["mu"] == b["mu"] and a["t"] == b["t"], "mu/t"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    tr.load()


ENGINES = [("f32", dict(engine=tr.TR_LR_RSVD, rank=8, oversample=4)),
           ("f32", dict(engine=tr.TR_LR_RSVD, rank=8, oversample=4, prec=tr.TR_PREC_BF16)),
           ("f64", dict(engine=tr.TR_LR_RSVD, rank=8, oversample=4)),
           ("f32", dict(engine=tr.TR_LR_ADAPTIVE, rank=8, oversample=4, adapt_block=4))]


@pytest.mark.parametrize("dt,kw", ENGINES)
def test_graph_steps_identical_to_eager(dt, kw):
    dims = (48, 40, 6, 3)
    _, M, mask = problem(dims, 1)
    outs = []
    for graph in (False, True):
        h = handle(dims, dt, M, mask, seed=3, **kw)
        if graph:
            h.graph_mode(True)
        for _ in range(6):
            h.step()
        outs.append(h.get_state())
        launches = h.kernel_launches()
        h.close()
    ok, what = states_equal(outs[0], outs[1])
    assert ok, what
    assert launches > 6


def test_graph_steps_match_oracle():
    dims, dt = (40, 44, 5, 4), "f32"
    _, M, mask = problem(dims, 3 * sum(dims))
    state = synth.random_state(M.shape, seed=9, scale=0.5)
    lam = admm.default_lambda(dims[0], dims[1], dims[2:])
    p = admm.Params(lam=lam, phi_gamma=60.0, psi_gamma=60.0, engine="rsvd", l=10, q=1, seed=4)
    st = admm.State(*(as_dtype(x, dt) for x in state), mu=0.1, t=0)
    for _ in range(5):
        st, _ = admm.step(st, as_dtype(M, dt), mask, tuple(dims[2:]), p)
    h = handle(dims, dt, M, mask, phi_gamma=60.0, psi_gamma=60.0, rank=10, oversample=0,
               power_iters=1, seed=4, **{"lambda": lam})
    h.set_state(*(dev(x, dt) for x in state), mu=0.1, t=0)
    h.graph_mode(True)
    for _ in range(5):       # one eager step, then four replays
        h.step()
    got = h.get_state()
    h.close()
    for name, want in [("L", st.L), ("E", st.E), ("Y", st.Y), ("Lam", st.Lam), ("G", st.G)]:
        assert relF(host(got[name]), want) < 1e-4, (name, relF(host(got[name]), want))
    assert got["t"] == 5 and abs(got["mu"] - st.mu) < 1e-15


def test_learned_engine_graph_steps_identical_to_eager():
    # the learned pass plans widths on the device, so it can be replayed
    dims = (64, 56, 6, 4)
    _, M, mask = problem(dims, 2, rank=5, sr=0.5)
    outs = []
    for graph in (False, True):
        h = handle(dims, "f32", M, mask, engine=tr.TR_LR_LEARNED, rank=24, oversample=8,
                   model_path=tr.DEFAULT_MODEL.encode(), prec=tr.TR_PREC_BF16, mu0=0.05)
        h.graph_mode(graph)
        for _ in range(6):
            h.step()
        info = h.step(info=True)
        outs.append((h.get_state(), h.slice_widths()))
        h.close()
    ok, what = states_equal(outs[0][0], outs[1][0])
    assert ok, what
    assert np.array_equal(outs[0][1], outs[1][1])
    assert info["fallback_slices"] >= 0


@pytest.mark.parametrize("dims,tiles", [((64, 40, 20, 20), (0, 8, 16, 64)),
                                         # 32 slices: tubes short enough for 256-tube tiles; 8000 tubes, a ragged last tile
                                         ((100, 80, 8, 4), (0, 32, 128, 256))])
def test_tube_tiles_compute_identical_steps(dims, tiles):
    _, M, mask = problem(dims, 4)
    outs = []
    for tp in tiles:
        h = handle(dims, "f32", M, mask, rank=8, oversample=4)
        h.set_tube_tile(tp)
        for _ in range(3):
            h.step()
        h.step(info=True)
        outs.append(h.get_state())
        h.close()
    for o in outs[1:]:
        ok, what = states_equal(outs[0], o)
        assert ok, what
    h = handle(dims, "f32", M, mask, rank=8, oversample=4)
    h.step()
    tile, groups = h.autotune(3)
    # FP32 with P % 16 == 0: only tiles the fused pass can prefetch with
    assert tile in (16, 32, 64, 128, 256) and groups in (1, 2, 4)
    assert h.autotune(0) == (tile, groups)      # cached choice
    h.step(info=True)                            # the deferred pass was completed first
    with pytest.raises(tr.TrError):
        h.set_tube_tile(12)
    h.close()


@pytest.mark.parametrize("prec", [tr.TR_PREC_FP32, tr.TR_PREC_BF16])
# 70 slices: uneven ranges; (64, 56): the BF16 forms hand the slice ranges Abar
# as BF16 planes (n2 % 8 == 0, n1 % 4 == 0)
@pytest.mark.parametrize("dims", [(60, 52, 10, 7), (64, 56, 10, 7)])
def test_slice_groups_compute_identical_steps(prec, dims):
    _, M, mask = problem(dims, 6)
    outs = []
    for groups, graph in ((1, False), (2, False), (4, False), (3, True)):
        h = handle(dims, "f32", M, mask, rank=8, oversample=4, prec=prec)
        h.set_slice_groups(groups)
        h.graph_mode(graph)
        for _ in range(4):
            h.step()
        outs.append(h.get_state())
        h.close()
    for o in outs[1:]:
        ok, what = states_equal(outs[0], o)
        assert ok, what
    h = handle(dims, "f32", M, mask, engine=tr.TR_LR_ADAPTIVE, rank=8, oversample=4,
               adapt_block=4)
    with pytest.raises(tr.TrError):
        h.set_slice_groups(2)
    h.close()


BATCH = [((64, 48, 8), "f32", 5, 0.3), ((40, 72, 4, 3), "f32", 3, 0.5),
         ((96, 96, 6), "f32", 6, 0.2), ((33, 29, 5, 2), "f32", 4, 0.4),
         ((50, 50, 12), "f64", 5, 0.35)]


@pytest.mark.parametrize("nstreams,tuned", [(1, False), (3, False), (3, True)])
def test_batch_matches_individual_handles(nstreams, tuned):
    # tuned: every problem's tube tile and slice split autotuned after the
    # first step; launch shapes change, values do not
    probs, prms, singles = [], [], []
    for i, (dims, dt, r, sr) in enumerate(BATCH):
        _, M, mask = problem(dims, 100 + i, rank=r, sr=sr)
        p = tr.default_params(rank=r + 4, oversample=4, seed=7 + i, mu0=0.05,
                              prec=tr.TR_PREC_BF16X3 if i == 2 else tr.TR_PREC_FP32)
        obs, mk = dev(M, dt), torch.from_numpy(mask).cuda()
        probs.append((obs, mk, dims))
        prms.append(p)
        singles.append((dims, dt, M, mask, p))
    b = tr.Batch(probs, prms, nstreams=nstreams)
    for k in range(5):
        b.step()                      # eager first step, then graph launches
        if tuned and k == 0:
            b.autotune(2)
    infos = b.step(info=True)
    assert len(infos) == len(BATCH) and all(x["iter"] == 6 for x in infos)
    assert b.launches() > 0
    for i, (dims, dt, M, mask, p) in enumerate(singles):
        h = tr.Handle(dev(M, dt), torch.from_numpy(mask).cuda(), dims, params=p)
        for _ in range(5):
            h.step()
        ref_info = h.step(info=True)
        ref = h.get_state()
        got = b.handle(i).get_state()
        ok, what = states_equal(ref, got)
        assert ok, (i, what)
        assert np.allclose(ref_info["res_inf"], infos[i]["res_inf"], rtol=0, atol=0)
        h.close()
    b.close()


def test_batch_with_a_learned_problem_matches_its_handle():
    dims = (48, 40, 5, 4)
    _, M, mask = problem(dims, 5, rank=4, sr=0.5)
    p = tr.default_params(engine=tr.TR_LR_LEARNED, rank=16, oversample=8, mu0=0.05,
                          model_path=tr.DEFAULT_MODEL.encode())
    b = tr.Batch([(dev(M, "f32"), torch.from_numpy(mask).cuda(), dims)], p)
    for _ in range(5):
        b.step()
    got = b.handle(0).get_state()
    h = handle(dims, "f32", M, mask, params=p)
    for _ in range(5):
        h.step()
    ok, what = states_equal(h.get_state(), got)
    assert ok, what
    h.close()
    b.close()


def test_graph_replay_with_alternating_observed_buffers():
    # double-buffered inputs: tr_set_observed alternates between two device
    # copies of the same data, each with its own captured step; the iterate
    # and the residuals read back asynchronously (tr_read_residuals) are bit
    # for bit those of replaying one buffer pair
    dims = (48, 40, 6, 3)
    _, M, mask = problem(dims, 11)
    outs, res = [], []
    for alternate in (False, True):
        h = handle(dims, "f32", M, mask, rank=8, oversample=4, seed=5, mu0=0.05)
        bufs = [(dev(M, "f32"), torch.from_numpy(mask).cuda()) for _ in range(2)]
        h.graph_mode(True)
        r = torch.zeros(10 * 8, dtype=torch.float64).pin_memory()
        for k in range(8):
            h.set_observed(*bufs[k % 2 if alternate else 0])
            h.step()
            h.read_residuals(r[10 * k:10 * k + 10])
        torch.cuda.synchronize()
        outs.append(h.get_state())
        res.append(r.clone())
        h.close()
    ok, what = states_equal(outs[0], outs[1])
    assert ok, what
    assert torch.equal(res[0], res[1])
    r = res[0].view(8, 10)
    # deferred steps: this step's ||dL||, ||dE||, ||M-L-E|| in the first half,
    # the previous step's ||L-G||, ||dG|| (completed by the fused pass) in the second
    assert bool((r[:, [2, 3]] == 0).all()), r
    assert bool((r[0, 5:] == 0).all()) and bool((r[:, [5, 6, 9]] == 0).all()), r
    assert float(r[1:, 0].max()) > 0 and float(r[1:, 7].max()) > 0, r
    assert bool(torch.isfinite(r).all()), r


def test_read_residuals_match_a_reported_step():
    dims = (40, 44, 5, 4)
    _, M, mask = problem(dims, 12)
    h = handle(dims, "f32", M, mask, rank=8, oversample=4, seed=6)
    for _ in range(3):
        h.step()
    info = h.step(info=True)                 # runs its inverse pass: all five slots
    r = torch.zeros(10, dtype=torch.float64).pin_memory()
    h.read_residuals(r)
    torch.cuda.synchronize()
    assert np.array_equal(r[:5].numpy(), np.asarray(info["res_inf"]))
    with pytest.raises(ValueError):
        h.read_residuals(torch.zeros(4, dtype=torch.float64))
    h.close()
