"""GPU parity of the one-bit completion step (tr_onebit_*, Alg. 6) against
the FP64 oracle (oracle/onebit.py) with the same randomized per-slice prox
(Philox sketches of iteration t): one step from a random state, and a run
whose recovery error must match the oracle's.  Tolerances: one step 1e-9
(FP64) and 1e-4 (FP32) relative Frobenius; the run's recovery errors within
0.01 of each other.
"""

import numpy as np
import pytest

from oracle import onebit, prox
from paper_2506_09594_gb300 import synth, tr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TDT = {"f64": torch.float64, "f32": torch.float32}
TOL = {"f64": 1e-9, "f32": 1e-4}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    tr.load()


def smooth(dims, rng):
    n1, n2, n3 = dims
    i1, i2, i3 = np.arange(n1) / n1, np.arange(n2) / n2, np.arange(n3) / n3
    X = np.zeros((n1, n2, n3))
    for r in range(3):
        X += np.einsum("i,j,k->ijk", np.cos(2 * np.pi * (r + 1) * i1 + rng.random() * 6),
                       np.sin(2 * np.pi * (r + 1) * i2 + rng.random() * 6),
                       np.cos(2 * np.pi * r * i3 + rng.random() * 6))
    S = np.ascontiguousarray(np.moveaxis(X, 2, 0))
    return S / np.abs(S).max()


def relF(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def dev(x, dt):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda", TDT[dt])


@pytest.mark.parametrize("dt", ["f64", "f32"])
@pytest.mark.parametrize("modes", [(1, 2), (1, 2, 3)])
def test_onebit_step_matches_oracle(dt, modes):
    rng = np.random.default_rng(3)
    dims = (36, 30, 8)
    S = smooth(dims, rng)
    s, q = synth.one_bit_observations(S, 4 * S.size, 1.2, 0.05, rng)
    kw = dict(lam=2e-3, theta=1.2, alpha=0.9, phi=prox.MCP, phi_gamma=50.0)
    p = onebit.Params(modes=modes, engine="rsvd", l=12, q=1, seed=7, mu0=0.05, **kw)
    J1, J2 = onebit.sample_tensors(S.shape, s, q, p.theta)
    def draw(scale):
        x = scale * rng.standard_normal(S.shape)
        return x.astype(np.float32).astype(np.float64) if dt == "f32" else x

    # the state the device holds, exactly, in both precisions
    st = onebit.State(L=draw(0.3), Z=draw(0.3), Y=draw(0.01), G={i: draw(0.1) for i in modes},
                      Lam={i: draw(0.01) for i in modes}, mu=0.05, t=4)
    ref, rel_ref = onebit.step(st, J1, J2, len(s), (8,), p)
    ob = tr.OneBit(dims, torch.from_numpy(s).cuda(), torch.from_numpy(q.astype(np.int8)).cuda(),
                   dtype=TDT[dt], modes=list(modes), rank=12, oversample=0, power_iters=1, seed=7,
                   mu0=0.05, phi=tr.TR_PEN_MCP, **{"lambda": 2e-3, "theta": 1.2, "alpha": 0.9,
                                                  "phi_gamma": 50.0})
    ob.set_state(dev(st.L, dt), dev(st.Z, dt), dev(st.Y, dt),
                 dev(np.stack([st.G[i] for i in modes]), dt),
                 dev(np.stack([st.Lam[i] for i in modes]), dt), mu=0.05, t=4)
    rel = ob.step(rel=True)
    got = ob.get_state()
    for name in ("L", "Z", "Y"):
        g = got[name].double().cpu().numpy()
        assert relF(g, getattr(ref, name)) < TOL[dt], (name, relF(g, getattr(ref, name)))
    for q_, i in enumerate(modes):
        assert relF(got["G"][q_].double().cpu().numpy(), ref.G[i]) < TOL[dt], ("G", i)
        assert relF(got["Lam"][q_].double().cpu().numpy(), ref.Lam[i]) < TOL[dt], ("Lam", i)
    assert abs(rel - rel_ref) < 10 * TOL[dt] * max(1.0, rel_ref)
    assert got["mu"] == pytest.approx(0.05 * 1.05) and got["t"] == 5
    ob.close()


def test_onebit_run_recovers_like_the_oracle():
    rng = np.random.default_rng(0)
    dims = (32, 32, 8)
    S = smooth(dims, rng)
    s, q = synth.one_bit_observations(S, 8 * S.size, 1.2, 0.05, rng)
    # sketch width 32 = the slice size: the randomized prox is exact here
    p = onebit.Params(modes=(1, 2), engine="rsvd", l=32, q=1, seed=2, phi=prox.L1, lam=1e-3,
                      theta=1.2, alpha=1.0, tol=0.0, max_iter=300)
    ref, _ = onebit.run(S.shape, s, q, (8,), p)
    ob = tr.OneBit(dims, torch.from_numpy(s).cuda(), torch.from_numpy(q.astype(np.int8)).cuda(),
                   dtype=torch.float64, modes=[1, 2], rank=32, oversample=0, power_iters=1,
                   seed=2, phi=tr.TR_PEN_L1, **{"lambda": 1e-3, "theta": 1.2, "alpha": 1.0})
    for _ in range(300):
        ob.step()
    L = ob.get_state()["L"].cpu().numpy()
    e_gpu, e_ref = relF(L, S), relF(ref.L, S)
    assert abs(e_gpu - e_ref) < 0.01 and e_gpu < 0.42      # oracle: 0.38 (DCT)
    ob.close()
