"""The bench's oracle-parity check (CPU): one step of the FP64 oracle from a
state s0 against a candidate state s1.  Lambda is judged by its derived bound,
||dLambda|| <= mu (||dL|| + ||dG||) + tol ||Lambda|| (Lambda+ = Lambda + mu (L - G)),
the other outputs by the relative tolerance.  No GPU involved."""

import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from oracle import admm  # noqa: E402
from paper_2506_09594_gb300 import synth  # noqa: E402

W = synth.WORKLOADS["tubal64_r5"]   # 64 x 64 x 16 FP64, noise-free model


def _states():
    _, M, mask, _ = synth.make_problem(W)
    p = admm.Params(lam=admm.default_lambda(W.n1, W.n2, W.tdims), engine="rsvd", l=W.l, q=W.q,
                    seed=W.seed, noise=admm.NOISE_NONE)
    st = admm.init_state(M.shape, p.mu0)
    for _ in range(55):   # past the first steps, where tau = 1/mu zeroes G
        st, _ = admm.step(st, M, mask, W.tdims, p)
    nxt, _ = admm.step(st, M, mask, W.tdims, p)
    as_dict = lambda s: {"L": s.L.copy(), "E": s.E.copy(), "Y": s.Y.copy(), "Lam": s.Lam.copy(),
                         "G": s.G.copy(), "mu": s.mu, "t": s.t}
    return M, mask, as_dict(st), as_dict(nxt)


def test_exact_step_passes_and_reports_the_lambda_bound():
    M, mask, s0, s1 = _states()
    out = bench.oracle_parity(W, M, mask, (s0, s1), 1e-10, steps=1, noise_model="none")
    assert out["pass"] and out["steps"] == 1
    for name in ("L", "E", "Y", "Lam", "G"):
        assert out[name]["rel_F"] == 0.0
    assert "bound_mu_dL_dG" in out["Lam"]


def test_lambda_judged_by_its_derived_bound():
    M, mask, s0, s1 = _states()
    assert np.linalg.norm(s1["G"]) > 0
    rng = np.random.default_rng(5)
    dG = 5e-11 * np.linalg.norm(s1["G"]) * rng.standard_normal(s1["G"].shape) / np.sqrt(s1["G"].size)
    # consistent: Lambda carries mu times G's error, as the update makes it;
    # G is within the tolerance, Lambda's relative error is not, the bound holds
    good = dict(s1, G=s1["G"] + dG, Lam=s1["Lam"] - s0["mu"] * dG)
    out = bench.oracle_parity(W, M, mask, (s0, good), 1e-10, steps=1, noise_model="none")
    assert out["G"]["rel_F"] < 1e-10 < out["Lam"]["rel_F"]
    assert out["pass"]
    # inconsistent: an error in Lambda that the step's G and L do not explain
    dLam = 1e-6 * np.linalg.norm(s1["Lam"]) * rng.standard_normal(s1["Lam"].shape) / np.sqrt(s1["Lam"].size)
    bad = dict(s1, Lam=s1["Lam"] + dLam)
    assert not bench.oracle_parity(W, M, mask, (s0, bad), 1e-10, steps=1, noise_model="none")["pass"]
    # and a G error beyond the tolerance fails however Lambda looks
    worse = dict(s1, G=s1["G"] + 1e4 * dG, Lam=s1["Lam"] - s0["mu"] * 1e4 * dG)
    assert not bench.oracle_parity(W, M, mask, (s0, worse), 1e-10, steps=1, noise_model="none")["pass"]
