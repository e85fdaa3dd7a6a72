"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (relative Frobenius error): 1e-10 for the FP64 path (rounding
order only), 1e-4 for the FP32 path (the stated bound of the FP32 form).
"""

import numpy as np
import pytest

from oracle import admm, philox, prox, svt, transform
from paper_2506_09594_gb300 import synth, tr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-10, "f32": 1e-4}
TDT = {"f64": torch.float64, "f32": torch.float32}


def dev(x, dt):
    return torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda", dtype=TDT[dt])


def host(t):
    return t.double().cpu().numpy()


def relF(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def as_dtype(x, dt):
    """The values the device holds for x: the oracle gets exactly those inputs."""
    return x.astype(np.float32).astype(np.float64) if dt == "f32" else x


def make_handle(dims, dt, M=None, mask=None, **kw):
    n = int(np.prod(dims[2:])) if len(dims) > 2 else 1
    shape = (n, dims[0], dims[1])
    if M is None:
        M = np.zeros(shape)
    if mask is None:
        mask = np.ones(shape, np.uint8)
    Md = dev(M, dt)
    maskd = torch.from_numpy(np.ascontiguousarray(mask)).cuda()
    return tr.Handle(Md, maskd, dims, **kw)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    tr.load()


# ------------------------------------------------------------- transform
@pytest.mark.parametrize("dt", ["f64", "f32"])
@pytest.mark.parametrize("dims", [(7, 5, 3), (9, 4, 5, 3), (3, 3, 2, 2, 2), (6, 5, 64),
                                  (33, 17, 20, 20), (4, 6), (5, 3, 1, 7), (40, 36, 64)])
def test_transform_parity(dims, dt):
    rng = np.random.default_rng(1)
    n = int(np.prod(dims[2:])) if len(dims) > 2 else 1
    X = rng.standard_normal((n, dims[0], dims[1]))
    h = make_handle(dims, dt)
    fwd = host(h.transform_forward(dev(X, dt)))
    inv = host(h.transform_inverse(dev(X, dt)))
    tdims = tuple(dims[2:])
    tol = 1e-13 if dt == "f64" else 3e-6
    assert relF(fwd, transform.forward(X, tdims)) < tol
    assert relF(inv, transform.inverse(X, tdims)) < tol
    back = host(h.transform_inverse(h.transform_forward(dev(X, dt))))
    assert relF(back, X) < tol
    h.close()


# ------------------------------------------------------------ slice prox
SLICE_CASES = [
    # (n, n1, n2, rank, noise, l, q, phi)
    (16, 64, 64, 5, 0.0, 15, 1, "l1"),       # exactly low rank: randomized == exact
    (16, 64, 64, 5, 0.0, 15, 1, "mcp"),
    (6, 70, 45, 8, 0.05, 20, 1, "mcp"),      # ragged tiles, n1 > n2
    (5, 40, 90, 6, 0.1, 16, 2, "l1"),        # n2 > n1, two power steps
    (4, 33, 29, 3, 0.2, 12, 0, "l1"),        # no power step
    (3, 8, 6, 2, 0.1, 20, 1, "mcp"),         # l clamped to min(n1, n2)
    (2, 1, 5, 1, 0.0, 3, 1, "l1"),           # single-row slices
]


@pytest.mark.parametrize("dt", ["f64", "f32"])
@pytest.mark.parametrize("case", SLICE_CASES)
def test_slice_prox_parity(case, dt):
    n, n1, n2, r, noise, l, q, phi = case
    Ab = synth.lowrank_plus_noise_stack(n, n1, n2, r, noise, seed=n1 * 7 + n2)
    s1 = np.linalg.svd(Ab[0], compute_uv=False)[0]
    tau = 0.3 * s1
    kind = prox.L1 if phi == "l1" else prox.MCP
    gamma = 3.0 * tau + 1.0
    dims = (n1, n2, n)
    pen = tr.TR_PEN_L1 if phi == "l1" else tr.TR_PEN_MCP
    h = make_handle(dims, dt, rank=l, oversample=0, power_iters=q, phi=pen, phi_theta=1.0,
                    phi_gamma=gamma, seed=77)
    G = host(h.slice_prox(dev(Ab, dt), tau, t=5))
    ref, info = svt.transformed_prox(Ab, tau, kind, 1.0, gamma, engine="rsvd", l=l, q=q,
                                     seed=77, t=5)
    assert relF(G, ref) < TOL[dt]
    sig, ranks = h.slice_stats()
    ll = min(l, n1, n2)
    for j in range(n):
        # Jacobi leaves singular values in column order: compare them sorted
        assert np.allclose(np.sort(sig[j][:ll])[::-1], info["sigma"][j][:ll],
                           rtol=1e-8 if dt == "f64" else 1e-4,
                           atol=(1e-10 if dt == "f64" else 1e-4) * s1)
    assert np.array_equal(ranks, info["ranks"]) or dt == "f32"
    h.close()


@pytest.mark.parametrize("dt,case", [("f32", (2, 512, 512, 20, 0.01, 74, 1, "mcp")),
                                     ("f32", (3, 300, 420, 12, 0.05, 60, 1, "l1")),
                                     ("f64", (2, 300, 200, 10, 0.01, 40, 1, "l1")),
                                     # exactly rank 5 under a 40-wide sketch: dependent
                                     # columns restart from unit vectors
                                     ("f32", (2, 600, 520, 5, 0.0, 40, 1, "l1")),
                                     ("f64", (2, 600, 64, 3, 0.0, 36, 1, "mcp")),
                                     ("f32", (2, 1000, 700, 30, 0.02, 48, 1, "mcp"))])
def test_slice_prox_large_panels(dt, case):
    # panels too large for the register-resident Gram-Schmidt QR (above 32
    # columns or 512 rows) take the shared-memory Gram-Schmidt QR up to 64
    # columns and 1024 rows, the shared-memory Householder QR beyond
    n, n1, n2, r, noise, l, q, phi = case
    Ab = synth.lowrank_plus_noise_stack(n, n1, n2, r, noise, seed=n1 + n2)
    s1 = np.linalg.svd(Ab[0], compute_uv=False)[0]
    tau = 0.05 * s1
    kind = prox.L1 if phi == "l1" else prox.MCP
    gamma = 3.0 * tau + 1.0
    pen = tr.TR_PEN_L1 if phi == "l1" else tr.TR_PEN_MCP
    h = make_handle((n1, n2, n), dt, rank=l, oversample=0, power_iters=q, phi=pen,
                    phi_gamma=gamma, seed=13)
    G = host(h.slice_prox(dev(Ab, dt), tau, t=1))
    ref, _ = svt.transformed_prox(as_dtype(Ab, dt), tau, kind, 1.0, gamma, engine="rsvd", l=l,
                                  q=q, seed=13, t=1)
    assert relF(G, ref) < TOL[dt]
    h.close()


def test_slice_prox_exact_on_low_rank_matches_full_svd():
    Ab = synth.lowrank_plus_noise_stack(16, 64, 64, 5, 0.0, seed=3)
    h = make_handle((64, 64, 16), "f64", rank=5, oversample=10, phi=tr.TR_PEN_L1)
    G = host(h.slice_prox(dev(Ab, "f64"), 2.0, t=0))
    ref, _ = svt.transformed_prox(Ab, 2.0, prox.L1, engine="full")
    assert relF(G, ref) < 1e-10
    h.close()


# ------------------------------------------------------------- ADMM step
STEP_CASES = [
    # dims, dtype, noise model, penalty, l, mu
    ((64, 64, 16), "f64", "none", "mcp", 15, 0.05),
    ((64, 64, 16), "f32", "l1", "l1", 15, 0.05),
    ((50, 37, 4, 3), "f32", "l1", "mcp", 12, 0.2),
    ((50, 37, 4, 3), "f64", "l1", "mcp", 12, 0.2),
    ((31, 29, 7), "f32", "none", "l1", 9, 1.0),
]


def _problem(dims, seed):
    rng = np.random.default_rng(seed)
    X = synth.lowrank_tensor(dims, 4, rng)[0]
    mask = synth.exact_count_mask(X.size, 0.4, rng).reshape(X.shape)
    S = synth.exact_count_mask(X.size, 0.05, rng).reshape(X.shape) * rng.uniform(-1, 1, X.shape)
    M = np.where(mask == 1, X + S, 0.0)
    return X, M, mask


@pytest.mark.parametrize("case", STEP_CASES)
def test_step_parity_from_random_state(case):
    dims, dt, noise, pen, l, mu = case
    X, M, mask = _problem(dims, seed=sum(dims))
    L0, E0, Y0, La0, G0 = synth.random_state(M.shape, seed=5, scale=0.5)
    kind = prox.L1 if pen == "l1" else prox.MCP
    pen_c = tr.TR_PEN_L1 if pen == "l1" else tr.TR_PEN_MCP
    lam = admm.default_lambda(dims[0], dims[1], dims[2:])
    p = admm.Params(phi=kind, psi=kind, phi_gamma=60.0, psi_gamma=60.0,
                    noise=admm.NOISE_NONE if noise == "none" else admm.NOISE_L1, lam=lam,
                    engine="rsvd", l=l, q=1, seed=11)
    st = admm.State(*(as_dtype(x, dt) for x in (L0, E0, Y0, La0, G0)), mu=mu, t=3)
    ref, res = admm.step(st, as_dtype(M, dt), mask, tuple(dims[2:]), p)
    h = make_handle(dims, dt, M=M, mask=mask, phi=pen_c, psi=pen_c, phi_gamma=60.0,
                    psi_gamma=60.0, noise=tr.TR_NOISE_NONE if noise == "none" else tr.TR_NOISE_L1,
                    rank=l, oversample=0, power_iters=1, seed=11, **{"lambda": lam})
    h.set_state(*(dev(x, dt) for x in (L0, E0, Y0, La0, G0)), mu=mu, t=3)
    info = h.step(info=True)
    got = h.get_state()
    for name, want in [("L", ref.L), ("E", ref.E), ("Y", ref.Y), ("Lam", ref.Lam), ("G", ref.G)]:
        err = relF(host(got[name]), want)
        assert err < TOL[dt], (name, err)
    assert abs(got["mu"] - ref.mu) <= 1e-15 * ref.mu and got["t"] == 4
    assert np.allclose(info["res_inf"], res, rtol=TOL[dt] * 10, atol=TOL[dt] * np.max(res))
    h.close()


@pytest.mark.parametrize("dims,dt", [((64, 64, 16), "f64"), ((50, 37, 4, 3), "f64"),
                                     ((40, 44, 5, 4), "f32"), ((31, 29, 7), "f32")])
def test_fused_steps_match_oracle_and_unfused(dims, dt):
    # Steps taken without info defer the inverse pass into the next step's
    # forward pass (one fused tube kernel).  Four such steps must match the
    # oracle, and match the unfused path (info requested every step).
    X, M, mask = _problem(dims, seed=3 * sum(dims))
    state = synth.random_state(M.shape, seed=9, scale=0.5)
    lam = admm.default_lambda(dims[0], dims[1], dims[2:])
    p = admm.Params(lam=lam, phi_gamma=60.0, psi_gamma=60.0, engine="rsvd", l=10, q=1, seed=4)
    st = admm.State(*(as_dtype(x, dt) for x in state), mu=0.1, t=0)
    for _ in range(4):
        st, _ = admm.step(st, as_dtype(M, dt), mask, tuple(dims[2:]), p)
    outs = []
    for fused in (True, False):
        h = make_handle(dims, dt, M=M, mask=mask, phi_gamma=60.0, psi_gamma=60.0, rank=10,
                        oversample=0, power_iters=1, seed=4, **{"lambda": lam})
        h.set_state(*(dev(x, dt) for x in state), mu=0.1, t=0)
        for _ in range(4):
            h.step(info=not fused)
        outs.append(h.get_state())
        h.close()
    tol = TOL[dt]
    for name, want in [("L", st.L), ("E", st.E), ("Y", st.Y), ("Lam", st.Lam), ("G", st.G)]:
        err = relF(host(outs[0][name]), want)
        assert err < tol, (name, err)
        assert relF(host(outs[0][name]), host(outs[1][name])) < (1e-14 if dt == "f64" else 1e-6)
    assert outs[0]["t"] == 4 and abs(outs[0]["mu"] - st.mu) < 1e-15


def test_recovery_small_workload_matches_oracle():
    w = synth.WORKLOADS["tubal64_r5"]
    X, M, mask, _ = synth.make_problem(w)
    iters = w.iters
    p = admm.Params(phi=prox.MCP, psi=prox.MCP, noise=admm.NOISE_NONE, engine="rsvd", l=w.l,
                    q=w.q, seed=21, tol=0.0, max_iter=iters)
    ref, _ = admm.run(M, mask, w.tdims, p)
    h = make_handle(w.dims, "f64", M=M, mask=mask, noise=tr.TR_NOISE_NONE, rank=w.l,
                    oversample=0, power_iters=w.q, seed=21, tol=0.0, max_iter=iters)
    Lout = torch.empty(M.shape, dtype=torch.float64, device="cuda")
    st, _ = h.recover(Lout)
    L = host(Lout)
    assert relF(L, ref.L) < 1e-8
    e_gpu, e_ref = relF(L, X), relF(ref.L, X)
    assert abs(e_gpu - e_ref) < 1e-8
    h.close()


def test_recover_converges_and_reports_notconv():
    w = synth.WORKLOADS["tubal64_r5"]
    X, M, mask, _ = synth.make_problem(w)
    h = make_handle(w.dims, "f64", M=M, mask=mask, noise=tr.TR_NOISE_NONE, rank=5,
                    oversample=10, seed=2, tol=1e-8, max_iter=400)
    Lout = torch.empty(M.shape, dtype=torch.float64, device="cuda")
    st, info = h.recover(Lout)
    assert st == tr.TR_OK and max(info["res_inf"]) <= 1e-8
    assert relF(host(Lout), X) < 1e-6
    h.close()
    h = make_handle(w.dims, "f64", M=M, mask=mask, noise=tr.TR_NOISE_NONE, tol=1e-12, max_iter=3)
    st, _ = h.recover(None, check=False)
    assert st == tr.TR_ENOTCONV
    h.close()


def test_nan_input_is_reported_and_poisons():
    dims = (16, 12, 4)
    M = np.ones((4, 16, 12))
    M[1, 3, 4] = np.nan
    h = make_handle(dims, "f32", M=M)
    with pytest.raises(tr.TrError) as ei:
        h.step(info=True)
    assert ei.value.status == tr.TR_ENUMERIC
    with pytest.raises(tr.TrError) as ei:
        h.step()
    assert ei.value.status == tr.TR_EINVAL
    z = torch.zeros((4, 16, 12), device="cuda")
    h.set_state(z, z, z, z, z, mu=1.0, t=0)
    h.close()


def test_nan_found_after_graph_replayed_steps():
    # steps without a report (here graph replays) copy the NaN/Inf flag to
    # pinned host memory; once they have completed, the next call reports it
    dims = (16, 12, 4)
    M = np.ones((4, 16, 12))
    M[2, 5, 7] = np.inf
    h = make_handle(dims, "f32", M=M)
    h.graph_mode(True)
    status = None
    for k in range(4):
        if k == 3:
            torch.cuda.synchronize()   # every earlier step has landed by now
        try:
            h.step()
        except tr.TrError as e:
            status = e.status
            break
    assert status == tr.TR_ENUMERIC           # at the latest on the call after the synchronise
    with pytest.raises(tr.TrError) as ei:
        h.step()
    assert ei.value.status == tr.TR_EINVAL       # poisoned until tr_set_state
    z = torch.zeros((4, 16, 12), device="cuda")
    h.set_state(z, z, z, z, z, mu=1.0, t=0)
    h.close()


def test_recover_lagged_stop_matches_per_step_check():
    # tr_recover with tol > 0 checks each step's residuals asynchronously one
    # step late; against stepping with a report every step it returns at most
    # two steps later, and its reported maxima meet tol
    w = synth.WORKLOADS["tubal64_r5"]
    X, M, mask, _ = synth.make_problem(w)
    kw = dict(M=M, mask=mask, noise=tr.TR_NOISE_NONE, rank=5, oversample=10, seed=2, tol=1e-8,
              max_iter=400)
    h = make_handle(w.dims, "f64", **kw)
    first = None
    for it in range(400):
        info = h.step(info=True)
        if max(info["res_inf"]) <= 1e-8:
            first = info["iter"]
            break
    h.close()
    assert first is not None
    for graph in (False, True):
        h = make_handle(w.dims, "f64", **kw)
        h.graph_mode(graph)
        Lout = torch.empty(M.shape, dtype=torch.float64, device="cuda")
        st, info = h.recover(Lout)
        assert st == tr.TR_OK and max(info["res_inf"]) <= 1e-8
        assert first <= info["iter"] <= first + 2, (first, info["iter"])
        assert relF(host(Lout), X) < 1e-6
        h.close()


def test_state_roundtrip():
    dims = (10, 9, 3, 2)
    rng = np.random.default_rng(0)
    h = make_handle(dims, "f64")
    xs = [dev(rng.standard_normal((6, 10, 9)), "f64") for _ in range(5)]
    h.set_state(*xs, mu=0.25, t=7)
    s = h.get_state()
    for k, x in zip(["L", "E", "Y", "Lam", "G"], xs):
        assert torch.equal(s[k], x)
    assert s["mu"] == 0.25 and s["t"] == 7
    h.close()


# ------------------------------------------------- full-size mid workload
@pytest.mark.slow
def test_mid_workload_full_size_step_parity():
    # 200x200x20x20 FP32 (400 slices), the benchmark launch configuration:
    # run the GPU for 55 iterations (tau = 1/mu has fallen to ~5, so singular
    # values survive the shrinkage), then one more step from that state on
    # both sides, compared on every output at full size.
    w = synth.WORKLOADS["tubal200x400_r10"]
    X, M, mask, _ = synth.make_problem(w)
    lam = admm.default_lambda(w.n1, w.n2, w.tdims)
    h = make_handle(w.dims, "f32", M=M, mask=mask, rank=10, oversample=10, power_iters=1,
                    seed=5, **{"lambda": lam})
    for _ in range(55):
        h.step()
    s = h.get_state()
    st = admm.State(L=host(s["L"]), E=host(s["E"]), Y=host(s["Y"]), Lam=host(s["Lam"]),
                    G=host(s["G"]), mu=s["mu"], t=s["t"])
    p = admm.Params(lam=lam, engine="rsvd", l=20, q=1, seed=5)
    M32 = as_dtype(M, "f32")
    ref, res = admm.step(st, M32, mask, w.tdims, p)
    info = h.step(info=True)
    got = h.get_state()
    # The L-update (Eq. coef-tensor) sums terms that can be far larger than L
    # itself; any FP32 evaluation carries a relative error of a few
    # eps32 * kappa_L, kappa_L = || |M| + |E| + |G| + |Y - Lambda|/mu || / ||L||.
    # The bound is the stated 1e-4 or that arithmetic floor, whichever is larger.
    kappa = (np.linalg.norm(np.abs(M32) + np.abs(st.E) + np.abs(st.G)
                            + np.abs(st.Y - st.Lam) / st.mu) / np.linalg.norm(ref.L))
    tol = max(TOL["f32"], 8 * np.finfo(np.float32).eps * kappa)
    errs = {name: relF(host(got[name]), want)
            for name, want in [("L", ref.L), ("E", ref.E), ("Y", ref.Y), ("Lam", ref.Lam),
                               ("G", ref.G)]}
    print("mid full-size step parity: kappa_L %.3g, bound %.3g, errors %s" % (kappa, tol, errs))
    for name, err in errs.items():
        assert err < tol, (name, err, kappa)
    assert info["max_rank"] > 0
    assert np.allclose(info["res_inf"], res, rtol=1e-3, atol=1e-4 * np.max(res))
    h.close()


@pytest.mark.slow
@pytest.mark.parametrize("prec,tol", [(tr.TR_PREC_BF16X3, 1e-4), (tr.TR_PREC_FP32, 1e-4),
                                      (tr.TR_PREC_BF16, 1e-3)])
def test_bench_configuration_full_size_parity(prec, tol):
    # The launch configuration bench.py times, at full size (200x200x20x20
    # FP32, 400 slices, l = 20, q = 1): one eager step, the autotuner (tube
    # tile, slice groups), graph replay, 54 more steps (tau = 1/mu ~ 5, ranks
    # survive the shrinkage).  From that state s0 the GPU takes one eager step
    # and one replay of the captured graph (whose fused tube pass completes
    # the first step); the FP64 oracle takes the same two steps from s0.
    # Every output is compared in relative Frobenius norm and elementwise
    # (largest error over the largest |value|), both against the form's
    # stated bound.
    w = synth.WORKLOADS["tubal200x400_r10"]
    X, M, mask, _ = synth.make_problem(w)
    h = make_handle(w.dims, "f32", M=M, mask=mask, rank=10, oversample=10, power_iters=1,
                    seed=w.seed, prec=prec)
    h.step()
    tile, groups = h.autotune(5)
    h.graph_mode(True)
    for _ in range(54):
        h.step()
    s0 = h.get_state()
    h.step()
    h.step()
    s2 = h.get_state()
    h.close()
    st = admm.State(L=host(s0["L"]), E=host(s0["E"]), Y=host(s0["Y"]), Lam=host(s0["Lam"]),
                    G=host(s0["G"]), mu=s0["mu"], t=s0["t"])
    p = admm.Params(lam=admm.default_lambda(w.n1, w.n2, w.tdims), engine="rsvd", l=20, q=1,
                    seed=w.seed)
    M32 = as_dtype(M, "f32")
    kappa = (np.linalg.norm(np.abs(M32) + np.abs(st.E) + np.abs(st.G)
                            + np.abs(st.Y - st.Lam) / st.mu) / np.linalg.norm(st.L))
    for _ in range(2):
        st, _ = admm.step(st, M32, mask, w.tdims, p)
    report = {"prec": prec, "tile": tile, "groups": groups, "t0": s0["t"], "kappa_L": kappa,
              "tol": tol}
    for name in ("L", "E", "Y", "Lam", "G"):
        want, got = getattr(st, name), host(s2[name])
        report[name] = (relF(got, want), float(np.abs(got - want).max() / np.abs(want).max()))
    print("bench-configuration parity:", report)
    for name in ("L", "E", "Y", "Lam", "G"):
        rel, mabs = report[name]
        assert rel < tol and mabs < tol, (name, report)


# ------------------------------------------- tensor-core (tcgen05) forms
PREC_TOL = {tr.TR_PREC_BF16: 1e-3, tr.TR_PREC_BF16X3: 1e-4}


@pytest.mark.parametrize("prec", [tr.TR_PREC_BF16, tr.TR_PREC_BF16X3])
@pytest.mark.parametrize("case", [(16, 64, 64, 5, 0.0, 15, 1, "l1"), (6, 70, 45, 8, 0.05, 20, 1, "mcp"),
                                  (5, 140, 90, 6, 0.1, 40, 2, "l1"), (4, 33, 29, 3, 0.2, 12, 0, "l1"),
                                  (3, 200, 200, 10, 1e-3, 20, 1, "mcp"),
                                  (3, 200, 160, 50, 1e-3, 80, 1, "l1")])   # 128-column MMA tile
def test_slice_prox_tensor_core_forms(case, prec):
    n, n1, n2, r, noise, l, q, phi = case
    Ab = synth.lowrank_plus_noise_stack(n, n1, n2, r, noise, seed=n1 * 7 + n2 + 1)
    s1 = np.linalg.svd(Ab[0], compute_uv=False)[0]
    tau = 0.3 * s1
    kind = prox.L1 if phi == "l1" else prox.MCP
    gamma = 3.0 * tau + 1.0
    pen = tr.TR_PEN_L1 if phi == "l1" else tr.TR_PEN_MCP
    A32 = as_dtype(Ab, "f32")
    ref, _ = svt.transformed_prox(A32, tau, kind, 1.0, gamma, engine="rsvd", l=l, q=q, seed=31, t=2)
    outs = {}
    for pr in (tr.TR_PREC_FP32, prec):
        h = make_handle((n1, n2, n), "f32", rank=l, oversample=0, power_iters=q, phi=pen,
                        phi_gamma=gamma, seed=31, prec=pr)
        outs[pr] = host(h.slice_prox(dev(Ab, "f32"), tau, t=2))
        h.close()
    err = relF(outs[prec], ref)
    assert err < PREC_TOL[prec], err
    # and against the plain FP32 GPU form
    assert relF(outs[prec], outs[tr.TR_PREC_FP32]) < PREC_TOL[prec]


@pytest.mark.parametrize("prec", [tr.TR_PREC_BF16, tr.TR_PREC_BF16X3])
@pytest.mark.parametrize("case", [(4, 200, 196, 10, 1e-3, 20, 1, "mcp"),   # M tail 72, K tail 4
                                  (3, 132, 100, 8, 1e-2, 48, 1, "l1"),     # 64-column tile
                                  (2, 256, 64, 12, 1e-3, 32, 2, "l1"),     # whole tiles, q = 2
                                  (5, 40, 36, 3, 0.0, 12, 1, "l1"),        # M < 128, K < 64
                                  (3, 96, 320, 6, 1e-2, 24, 1, "mcp")])    # n2 > n1
def test_slice_prox_tensor_core_tma_shapes(case, prec):
    # shapes whose strides allow 3D tensor copies of Abar (n2 a multiple of
    # 4) and of the panels (n1 a multiple of 4), with N <= 64: the products
    # take the TMA-fed tcgen05 kernel, with zero-filled tails in M, N and K
    n, n1, n2, r, noise, l, q, phi = case
    Ab = synth.lowrank_plus_noise_stack(n, n1, n2, r, noise, seed=n1 * 5 + n2 + 3)
    s1 = np.linalg.svd(Ab[0], compute_uv=False)[0]
    tau = 0.2 * s1
    kind = prox.L1 if phi == "l1" else prox.MCP
    gamma = 3.0 * tau + 1.0
    pen = tr.TR_PEN_L1 if phi == "l1" else tr.TR_PEN_MCP
    A32 = as_dtype(Ab, "f32")
    ref, _ = svt.transformed_prox(A32, tau, kind, 1.0, gamma, engine="rsvd", l=l, q=q, seed=41, t=6)
    h = make_handle((n1, n2, n), "f32", rank=l, oversample=0, power_iters=q, phi=pen,
                    phi_gamma=gamma, seed=41, prec=prec)
    G = host(h.slice_prox(dev(Ab, "f32"), tau, t=6))
    h.close()
    err = relF(G, ref)
    assert err < PREC_TOL[prec], err
    assert np.abs(G - ref).max() < PREC_TOL[prec] * np.abs(ref).max()


@pytest.mark.parametrize("prec", [tr.TR_PREC_BF16, tr.TR_PREC_BF16X3])
@pytest.mark.parametrize("case", [(4, 200, 200, 10, 1e-3, 20, 1, "mcp"),  # M tail 72, K tail 8
                                  (3, 132, 104, 8, 1e-2, 48, 1, "l1"),    # 64-column tile
                                  (2, 256, 64, 12, 1e-3, 32, 2, "l1"),    # whole tiles, q = 2
                                  (5, 40, 40, 3, 0.0, 12, 1, "l1"),       # M < 64, K < 64
                                  (2, 72, 136, 5, 1e-2, 16, 1, "l1"),     # an MN box wholly past M
                                  (3, 96, 320, 6, 1e-2, 24, 1, "mcp")])   # n2 > n1
def test_slice_prox_bf16_planes(case, prec):
    # A handle whose steps write Abar as BF16 planes (n2 and n1 n2 multiples
    # of 8, l <= 64) runs its products on the planes: 128-byte swizzled K-major
    # tiles for Abar X, MN-major tiles for Abar^T Q.  The eager profile takes
    # that path from an FP32 Abar; tr_slice_prox converts Abar in shared
    # memory instead.  Both split each element the same way and form the same
    # three partial products (summed in another order), so the two agree to
    # FP32 rounding noise, and both meet the oracle at the form's tolerance.
    n, n1, n2, r, noise, l, q, phi = case
    Ab = synth.lowrank_plus_noise_stack(n, n1, n2, r, noise, seed=n1 * 3 + n2 + 5)
    s1 = np.linalg.svd(Ab[0], compute_uv=False)[0]
    tau = 0.2 * s1
    kind = prox.L1 if phi == "l1" else prox.MCP
    gamma = 3.0 * tau + 1.0
    pen = tr.TR_PEN_L1 if phi == "l1" else tr.TR_PEN_MCP
    ref, _ = svt.transformed_prox(as_dtype(Ab, "f32"), tau, kind, 1.0, gamma, engine="rsvd", l=l,
                                  q=q, seed=43, t=3)
    h = make_handle((n1, n2, n), "f32", rank=l, oversample=0, power_iters=q, phi=pen,
                    phi_gamma=gamma, seed=43, prec=prec)
    A = dev(Ab, "f32")
    G_conv = host(h.slice_prox(A, tau, t=3))
    out = torch.empty_like(A)
    kern = h.profile_slice_pass(A, tau, 3, reps=1, out=out)
    G_pl = host(out)
    h.close()
    names = [k for k, _ in kern]
    assert sum("planes" in k for k in names) == 2 + 2 * q, names
    assert relF(G_pl, G_conv) < 1e-5, relF(G_pl, G_conv)
    err = relF(G_pl, ref)
    assert err < PREC_TOL[prec], err
    assert np.abs(G_pl - ref).max() < PREC_TOL[prec] * np.abs(ref).max()


@pytest.mark.parametrize("prec", [tr.TR_PREC_BF16, tr.TR_PREC_BF16X3])
# (96, 80): the steps hand the slice pass Abar as BF16 planes; (90, 80): n1 is
# not a multiple of 4, so Abar stays FP32 and the products convert it
@pytest.mark.parametrize("dims", [(96, 80, 5, 4), (90, 80, 5, 4)])
def test_step_tensor_core_forms(prec, dims):
    # The BF16 form keeps the sketch in BF16: its subspace matches the FP32
    # one only where the transformed slices' spectra decay beyond the sketch
    # width (the regime the randomized engine is for).  So the iterate here is
    # structured -- L and G near the low-rank truth, small multipliers --
    # rather than white noise (a flat spectrum, where any perturbation of the
    # sketch moves the captured subspace).
    X, M, mask = _problem(dims, seed=77)
    rs = np.random.default_rng(2)
    noise = lambda s: s * rs.standard_normal(M.shape)
    state = [X + noise(0.01), noise(0.01), noise(0.05), noise(0.05), X + noise(0.01)]
    lam = admm.default_lambda(dims[0], dims[1], dims[2:])
    p = admm.Params(lam=lam, phi_gamma=60.0, psi_gamma=60.0, engine="rsvd", l=12, q=1, seed=8)
    st = admm.State(*(as_dtype(x, "f32") for x in state), mu=0.2, t=1)
    ref, _ = admm.step(st, as_dtype(M, "f32"), mask, tuple(dims[2:]), p)
    h = make_handle(dims, "f32", M=M, mask=mask, phi_gamma=60.0, psi_gamma=60.0, rank=12,
                    oversample=0, power_iters=1, seed=8, prec=prec, **{"lambda": lam})
    h.set_state(*(dev(x, "f32") for x in state), mu=0.2, t=1)
    h.step(info=True)
    got = h.get_state()
    # L, E, Y are elementwise in the (identical) state: FP32 rounding only.
    for name, want in [("L", ref.L), ("E", ref.E), ("Y", ref.Y)]:
        assert relF(host(got[name]), want) < 1e-5, name
    # G is the prox output: the form's tolerance.
    errG = relF(host(got["G"]), ref.G)
    assert errG < PREC_TOL[prec], errG
    # Lambda_new - Lambda_ref = mu (G_ref - G): bounded through G's error.
    dLam = np.linalg.norm(host(got["Lam"]) - ref.Lam)
    assert dLam <= 0.2 * np.linalg.norm(host(got["G"]) - ref.G) * 1.001 + 1e-6 * np.linalg.norm(ref.Lam)
    h.close()


# --------------------------------------------------- adaptive engine (Alg. 3)
@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_adaptive_engine_matches_oracle_on_low_rank_slices(dt):
    # exact ranks 3, 7, 12, 5: block Lanczos stops cleanly (E -> 0) and
    # deflates at the exact rank, so both sides take the same steps
    n1, n2, b, kcap = 60, 48, 4, 24
    ranks = [3, 7, 12, 5]
    Ab = synth.lowrank_plus_noise_stack(4, n1, n2, ranks, 0.0, seed=12)
    tau = 0.4
    delta = 1e-11 if dt == "f64" else 1e-5
    ref, info = svt.transformed_prox(as_dtype(Ab, dt), tau, prox.L1, engine="adaptive", eps=1e-4,
                                     b=b, delta_rel=delta, seed=9, t=3, max_rank=kcap)
    h = make_handle((n1, n2, 4), dt, engine=tr.TR_LR_ADAPTIVE, adapt_block=b, adapt_eps=1e-4,
                    rank=kcap, oversample=0, phi=tr.TR_PEN_L1, seed=9)
    G = host(h.slice_prox(dev(Ab, dt), tau, t=3))
    assert relF(G, ref) < TOL[dt]
    full, _ = svt.transformed_prox(Ab, tau, prox.L1, engine="full")
    assert relF(G, full) < (1e-9 if dt == "f64" else 1e-4)
    h.close()


def test_adaptive_engine_accuracy_bound_on_noisy_slices():
    # E < eps^2 ||A||^2 at the stop, so ||A - U U^T A|| < eps ||A||, and the l1
    # prox is nonexpansive: ||D(A) - D(U U^T A)|| <= eps ||A|| per slice
    n, n1, n2, b, kcap, eps = 6, 80, 70, 5, 40, 0.05
    Ab = synth.lowrank_plus_noise_stack(n, n1, n2, 8, 0.02, seed=4)
    h = make_handle((n1, n2, n), "f32", engine=tr.TR_LR_ADAPTIVE, adapt_block=b, adapt_eps=eps,
                    rank=kcap, oversample=0, phi=tr.TR_PEN_L1, seed=2)
    G = host(h.slice_prox(dev(Ab, "f32"), 0.5, t=0))
    full, _ = svt.transformed_prox(Ab, 0.5, prox.L1, engine="full")
    for j in range(n):
        assert np.linalg.norm(G[j] - full[j]) <= eps * np.linalg.norm(Ab[j]) * 1.01
    h.close()


def test_adaptive_engine_step_parity():
    dims = (40, 36, 3, 4)
    X, M, mask = _problem(dims, seed=5)
    state = [X, np.zeros_like(X), np.zeros_like(X), np.zeros_like(X), X]
    lam = admm.default_lambda(dims[0], dims[1], dims[2:])
    p = admm.Params(lam=lam, phi_gamma=60.0, psi_gamma=60.0, engine="adaptive", eps=1e-4, b=4,
                    delta_rel=1e-11, seed=6)
    st = admm.State(*state, mu=0.3, t=0)
    ref, _ = admm.step(st, M, mask, tuple(dims[2:]), p)
    h = make_handle(dims, "f64", M=M, mask=mask, phi_gamma=60.0, psi_gamma=60.0, rank=36,
                    oversample=0, engine=tr.TR_LR_ADAPTIVE, adapt_block=4, adapt_eps=1e-4, seed=6,
                    **{"lambda": lam})
    h.set_state(*(dev(x, "f64") for x in state), mu=0.3, t=0)
    h.step(info=True)
    got = h.get_state()
    for name, want in [("L", ref.L), ("E", ref.E), ("G", ref.G)]:
        assert relF(host(got[name]), want) < 1e-9, name
    h.close()


# ------------------------------------------------------------- edge cases
def test_zero_problem_stays_zero():
    # M = 0: every iterate stays exactly 0 (no NaN from 0/0 in the prox or the
    # sketch of an all-zero slice), ranks are 0
    dims = (40, 36, 5, 3)
    h = make_handle(dims, "f32", rank=8, oversample=4)
    for _ in range(3):
        info = h.step(info=True)
    s = h.get_state()
    for k in ("L", "E", "Y", "Lam", "G"):
        assert float(s[k].abs().max()) == 0.0, k
    assert info["max_rank"] == 0 and max(info["res_inf"]) == 0.0
    h.close()


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_no_shrink_gives_the_rank_l_projection(dt):
    # tau = 0 with l1: Prox is the identity, so Gbar = Q Q^T Abar, the sketch's
    # rank-l projection, as in the oracle's randomized engine
    Ab = synth.lowrank_plus_noise_stack(5, 50, 44, 6, 0.2, seed=8)
    h = make_handle((50, 44, 5), dt, rank=12, oversample=0, power_iters=1,
                    phi=tr.TR_PEN_L1, seed=21)
    G = host(h.slice_prox(dev(Ab, dt), 0.0, t=3))
    ref, _ = svt.transformed_prox(as_dtype(Ab, dt), 0.0, prox.L1, engine="rsvd", l=12, q=1,
                                  seed=21, t=3)
    assert relF(G, ref) < TOL[dt]
    h.close()


def test_sketch_width_clamped_to_slice_size():
    # rank + oversample above min(n1, n2): the sketch takes every column, so
    # the randomized prox is the exact (full-SVD) prox
    Ab = synth.lowrank_plus_noise_stack(4, 30, 20, 20, 0.0, seed=9)
    h = make_handle((30, 20, 4), "f64", rank=25, oversample=10, phi=tr.TR_PEN_L1)
    G = host(h.slice_prox(dev(Ab, "f64"), 0.5, t=0))
    ref, _ = svt.transformed_prox(Ab, 0.5, prox.L1, engine="full")
    assert relF(G, ref) < 1e-10
    sig, _ = h.slice_stats()
    assert sig.shape[1] == 20
    h.close()


def test_single_slice_order3():
    # n3 = 1: one slice, the transform is the identity
    X, M, mask = _problem((40, 30, 1), seed=12)
    lam = admm.default_lambda(40, 30, (1,))
    p = admm.Params(lam=lam, engine="rsvd", l=8, q=1, seed=2)
    st = admm.State(*synth.random_state(M.shape, seed=3, scale=0.5), mu=0.5, t=0)
    ref, _ = admm.step(admm.State(*(as_dtype(x, "f32") for x in (st.L, st.E, st.Y, st.Lam, st.G)),
                                  mu=0.5, t=0), as_dtype(M, "f32"), mask, (1,), p)
    h = make_handle((40, 30, 1), "f32", M=M, mask=mask, rank=8, oversample=0, seed=2,
                    **{"lambda": lam})
    h.set_state(*(dev(x, "f32") for x in (st.L, st.E, st.Y, st.Lam, st.G)), mu=0.5, t=0)
    h.step(info=True)
    got = h.get_state()
    for name, want in [("L", ref.L), ("G", ref.G), ("Lam", ref.Lam)]:
        assert relF(host(got[name]), want) < TOL["f32"], name
    h.close()


@pytest.mark.slow
@pytest.mark.parametrize("prec", [tr.TR_PREC_FP32, tr.TR_PREC_BF16X3, tr.TR_PREC_BF16])
def test_precision_config_full_size_sampled(prec):
    # 1024 x 1024 x 64 FP32 stack, rank 32 + noise, l = 48, q = 1, on the GPU
    # in the launch configuration of a step; the FP64 oracle recomputes four
    # sampled slices (all 64 would take minutes), and the mixed forms are also
    # compared with the plain FP32 GPU form on the whole stack
    n, n1, n2, r, l = 64, 1024, 1024, 32, 48
    Ab = synth.lowrank_plus_noise_stack(n, n1, n2, r, 1e-2, seed=1024)
    A32 = as_dtype(Ab, "f32")
    tau = 0.05 * np.linalg.svd(A32[0], compute_uv=False)[0]
    outs = {}
    for pr in sorted({tr.TR_PREC_FP32, prec}):
        h = make_handle((n1, n2, n), "f32", rank=l, oversample=0, power_iters=1,
                        phi=tr.TR_PEN_L1, seed=17, prec=pr)
        outs[pr] = host(h.slice_prox(dev(Ab, "f32"), tau, t=4))
        h.close()
    tol = PREC_TOL.get(prec, TOL["f32"])
    for j in (0, 17, 40, 63):
        Om = philox.gaussian_block(17, 4, j, n2, l)
        ref, _, _ = svt.slice_prox_randomized(A32[j], Om, 1, tau, prox.L1)
        assert relF(outs[prec][j], ref) < tol, (j, relF(outs[prec][j], ref))
    assert relF(outs[prec], outs[tr.TR_PREC_FP32]) < tol
