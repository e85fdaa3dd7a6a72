"""GPU parity of the gradient-domain ADMM step (tr_ctv_*, Alg. 5 with a set
Gamma of gradient directions) against the FP64 oracle (oracle/ctv.py) with
the same randomized per-slice prox (Philox sketches of iteration t): one
step from a random state, and a completion run of a smooth low-rank tensor.
Tolerances: one step 1e-9 (FP64) and 1e-4 (FP32) relative Frobenius, the
residuals alike; the run 1e-6 from the oracle's iterate and 1e-5 from the
truth (the oracle reaches 1.2e-7).
"""

import numpy as np
import pytest

from oracle import admm, ctv, prox
from paper_2506_09594_gb300 import tr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TDT = {"f64": torch.float64, "f32": torch.float32}
TOL = {"f64": 1e-9, "f32": 1e-4}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    tr.load()


def relF(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def dev(x, dt):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda", TDT[dt])


@pytest.mark.parametrize("dt", ["f64", "f32"])
@pytest.mark.parametrize("modes,noise", [((1, 2), admm.NOISE_L1), ((1, 2, 4), admm.NOISE_NONE)])
def test_ctv_step_matches_oracle(dt, modes, noise):
    rng = np.random.default_rng(5)
    dims, tdims = (36, 30, 5, 4), (5, 4)
    shape = (20, 36, 30)

    def draw(scale):
        x = scale * rng.standard_normal(shape)
        return x.astype(np.float32).astype(np.float64) if dt == "f32" else x

    mask = (rng.random(shape) < 0.6).astype(np.uint8)
    M = np.where(mask == 1, draw(1.0), 0.0)
    st = ctv.State(L=draw(0.5), E=draw(0.1), Y=draw(0.05), G={k: draw(0.3) for k in modes},
                   Lam={k: draw(0.05) for k in modes}, mu=0.4, t=2)
    p = ctv.Params(modes=modes, transform="dct", engine="rsvd", l=12, q=1, seed=8, phi=prox.MCP,
                   phi_gamma=30.0, psi=prox.MCP, psi_gamma=30.0, noise=noise, lam=0.2)
    ref, res_ref = ctv.step(st, M, mask, tdims, p)
    c = tr.Ctv(dev(M, dt), torch.from_numpy(mask).cuda(), dims, modes=list(modes), rank=12,
               oversample=0, power_iters=1, seed=8, phi=tr.TR_PEN_MCP, phi_gamma=30.0,
               psi=tr.TR_PEN_MCP, psi_gamma=30.0,
               noise=tr.TR_NOISE_L1 if noise == admm.NOISE_L1 else tr.TR_NOISE_NONE,
               **{"lambda": 0.2})
    c.set_state(dev(st.L, dt), dev(st.E, dt), dev(st.Y, dt),
                dev(np.stack([st.G[k] for k in modes]), dt),
                dev(np.stack([st.Lam[k] for k in modes]), dt), mu=0.4, t=2)
    res = c.step(info=True)
    got = c.get_state()
    for name in ("L", "E", "Y"):
        g = got[name].double().cpu().numpy()
        want = getattr(ref, name)
        assert relF(g, want) < TOL[dt], (name, relF(g, want))
    for q, k in enumerate(modes):
        assert relF(got["G"][q].double().cpu().numpy(), ref.G[k]) < TOL[dt], ("G", k)
        assert relF(got["Lam"][q].double().cpu().numpy(), ref.Lam[k]) < TOL[dt], ("Lam", k)
    assert np.allclose(res, res_ref, rtol=100 * TOL[dt], atol=100 * TOL[dt])
    assert got["mu"] == pytest.approx(0.44) and got["t"] == 3
    c.close()


def test_ctv_run_completes_a_smooth_tensor():
    rng = np.random.default_rng(0)
    n1, n2, n3 = 32, 32, 8
    i1, i2, i3 = np.arange(n1) / n1, np.arange(n2) / n2, np.arange(n3) / n3
    X = np.zeros((n1, n2, n3))
    for r in range(3):
        X += np.einsum("i,j,k->ijk", np.cos(2 * np.pi * (r + 1) * i1 + rng.random() * 6),
                       np.sin(2 * np.pi * (r + 1) * i2 + rng.random() * 6),
                       np.cos(2 * np.pi * r * i3 + rng.random() * 6))
    S = np.ascontiguousarray(np.moveaxis(X, 2, 0))
    mask = rng.random(S.shape) < 0.5
    M = np.where(mask, S, 0.0)
    # sketch width 32 = the slice size: the randomized prox is exact here
    p = ctv.Params(modes=(1, 2), transform="dct", engine="rsvd", l=32, q=1, seed=4, phi=prox.L1,
                   noise=admm.NOISE_NONE, mu0=1e-2, growth=1.1, tol=0.0, max_iter=150)
    ref, _ = ctv.run(M, mask, (n3,), p)
    c = tr.Ctv(dev(M, "f64"), torch.from_numpy(mask.astype(np.uint8)).cuda(), (n1, n2, n3),
               modes=[1, 2], rank=32, oversample=0, power_iters=1, seed=4, phi=tr.TR_PEN_L1,
               noise=tr.TR_NOISE_NONE, mu0=1e-2, growth=1.1)
    for _ in range(150):
        c.step()
    L = c.get_state()["L"].cpu().numpy()
    assert relF(L, ref.L) < 1e-6
    assert relF(L, S) < 1e-5
    c.close()
