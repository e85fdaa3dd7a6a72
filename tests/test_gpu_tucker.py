"""GPU parity of the shared-Tucker randomized prox (tr_slice_prox_tucker,
Alg. 1 with processing order (1, 2) + Alg. 4 randomized branch) against
the FP64 oracle (oracle/tucker.py, transform-domain form).

The GPU orthonormalises the Krylov block by Gram-Schmidt and takes the top
singular vectors of Z^T A A^T Z by one-sided Jacobi, the oracle by
Householder and LAPACK.  Both order the factor columns by decreasing
singular value with the canonical sign (largest-magnitude entry positive),
so on inputs whose retained singular values are distinct and well separated
the factors agree column by column, and so do the mode-2 sketch and the
result.  Tolerances: FP64 1e-10, FP32 1e-4 (relative Frobenius).
"""

import numpy as np
import pytest

from oracle import prox, svt, tucker
from paper_2506_09594_gb300 import tr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TDT = {"f64": torch.float64, "f32": torch.float32}
TOL = {"f64": 1e-10, "f32": 1e-4}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    tr.load()


def dev(x, dt):
    return torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda", dtype=TDT[dt])


def as_dtype(x, dt):
    return x.astype(np.float32).astype(np.float64) if dt == "f32" else x


def relF(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def handle(dims, dt, phi, gamma=40.0):
    n = int(np.prod(dims[2:]))
    M = torch.zeros((n, dims[0], dims[1]), dtype=TDT[dt], device="cuda")
    mask = torch.ones((n, dims[0], dims[1]), dtype=torch.uint8, device="cuda")
    return tr.Handle(M, mask, dims, phi=phi, phi_gamma=gamma, rank=8, oversample=4)


def shared_plus_noise(n, n1, n2, s1, s2, noise, rng, graded=False):
    P, _ = np.linalg.qr(rng.standard_normal((n1, s1)))
    Q, _ = np.linalg.qr(rng.standard_normal((n2, s2)))
    S = 3.0 * rng.standard_normal((n, s1, s2))
    if graded:   # distinct, well separated singular values in both modes
        S = S * np.geomspace(4.0, 1.0, s1)[None, :, None] * np.geomspace(3.0, 1.0, s2)[None, None, :]
    return np.einsum("ia,jab,kb->jik", P, S, Q) + noise * rng.standard_normal((n, n1, n2)), P, Q


def colmajor(G, dt):
    # a column-major (rows x cols) block as a (cols, rows) row-major tensor
    return dev(G.T, dt)


@pytest.mark.parametrize("dt", ["f64", "f32"])
@pytest.mark.parametrize("kind", [prox.L1, prox.MCP])
def test_tucker_prox_matches_oracle(dt, kind):
    # noisy stack with graded shared spectra: the r retained directions of
    # each mode are distinct and well separated, so the factors (signs
    # canonical) agree column by column and the mode-2 sketch sees the same
    # core; the noise directions beyond r are dropped by both
    rng = np.random.default_rng(11)
    dims = (40, 36, 5, 4)
    n, n1, n2 = 20, 40, 36
    r1, r2, b1, b2, q1, q2 = 6, 5, 4, 4, 1, 1
    Ab, _, _ = shared_plus_noise(n, n1, n2, 6, 5, 1e-3, rng, graded=True)
    Ab = as_dtype(Ab, dt)
    G1 = as_dtype(rng.standard_normal((n * n2, b1)), dt)
    G2 = as_dtype(rng.standard_normal((n * r1, b2)), dt)
    tau = 0.5
    want, (_, F1w, F2w) = tucker.transformed_randomized_prox(Ab, tau, kind, (r1, r2), (G1, G2),
                                                             (q1, q2), gamma=40.0)
    h = handle(dims, dt, tr.TR_PEN_L1 if kind == prox.L1 else tr.TR_PEN_MCP)
    got, F1, F2 = h.slice_prox_tucker(dev(Ab, dt), tau, (r1, r2), (b1, b2), (q1, q2),
                                      colmajor(G1, dt), colmajor(G2, dt), factors=True)
    got = got.double().cpu().numpy()
    assert relF(got, want) < TOL[dt], relF(got, want)
    F1 = F1.double().cpu().numpy()
    F2 = F2.double().cpu().numpy()
    # with distinct spectra and canonical signs the factors themselves agree
    assert relF(F1, F1w) < 100 * TOL[dt] and relF(F2, F2w) < 100 * TOL[dt]
    assert np.linalg.norm(F1.T @ F1 - np.eye(r1)) < 50 * TOL[dt]
    assert np.linalg.norm(F2.T @ F2 - np.eye(r2)) < 50 * TOL[dt]
    h.close()


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_tucker_prox_exact_on_shared_spaces(dt):
    # slices sharing column and row spaces of dimensions 5 and 3: with
    # r = (5, 3) the factors capture them, and the result is the
    # deterministic prox of every transformed slice (full SVD)
    rng = np.random.default_rng(12)
    dims = (48, 30, 6, 2)
    n = 12
    Ab, P, Q = shared_plus_noise(n, 48, 30, 5, 3, 0.0, rng)
    Ab = as_dtype(Ab, dt)
    want, _ = svt.transformed_prox(Ab, 0.3, prox.L1)
    h = handle(dims, dt, tr.TR_PEN_L1)
    G1 = rng.standard_normal((n * 30, 3))
    G2 = rng.standard_normal((n * 5, 2))
    got, F1, F2 = h.slice_prox_tucker(dev(Ab, dt), 0.3, (5, 3), (3, 2), (1, 1), colmajor(G1, dt),
                                      colmajor(G2, dt), factors=True)
    assert relF(got.double().cpu().numpy(), want) < TOL[dt]
    F1 = F1.double().cpu().numpy()
    F2 = F2.double().cpu().numpy()
    assert np.linalg.norm(P - F1 @ (F1.T @ P)) < 10 * TOL[dt]
    assert np.linalg.norm(Q - F2 @ (F2.T @ Q)) < 10 * TOL[dt]
    h.close()


def test_tucker_prox_rejects_bad_arguments():
    h = handle((16, 12, 4), "f32", tr.TR_PEN_L1)
    A = torch.zeros((4, 16, 12), device="cuda")
    G = torch.zeros(1024, device="cuda")
    for ranks, blocks, kry in (((13, 4), (4, 4), (3, 0)),     # r1 > min(n1, n2)
                               ((4, 4), (2, 2), (0, 0)),      # (q+1) b < r
                               ((4, 4), (20, 4), (1, 0)),     # (q+1) b > 32
                               ((4, 4), (4, 4), (-1, 0))):    # negative Krylov steps
        with pytest.raises(tr.TrError):
            h.slice_prox_tucker(A, 0.1, ranks, blocks, kry, G, G)
    h.close()


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_tucker_engine_step_matches_oracle(dt):
    # one ADMM step of the TR_LR_TUCKER engine (r = b = l = 6, q = 1) against
    # oracle.admm.step(engine="tucker") with the same Philox blocks, on an
    # exactly low-rank stack whose slices share graded spaces of dimension 6
    # (every retained direction well separated), fully observed, noise-free:
    # the step's prox input is L(X)
    from oracle import admm, transform
    rng = np.random.default_rng(21)
    dims, tdims = (40, 36, 5, 4), (5, 4)
    n = 20
    Xbar, _, _ = shared_plus_noise(n, 40, 36, 6, 6, 0.0, rng, graded=True)
    X = as_dtype(transform.inverse(Xbar, tdims), dt)
    mask = np.ones(X.shape, dtype=np.uint8)
    zero = np.zeros_like(X)
    p = admm.Params(phi=prox.MCP, psi=prox.MCP, phi_gamma=30.0, psi_gamma=30.0,
                    noise=admm.NOISE_NONE, lam=0.1, engine="tucker", l=6, q=1, seed=9)
    ref, _ = admm.step(admm.State(X, zero, zero, zero, X, mu=0.5, t=3), X, mask, tdims, p)
    h = tr.Handle(dev(X, dt), torch.from_numpy(mask).cuda(), dims, engine=tr.TR_LR_TUCKER,
                  rank=6, oversample=0, power_iters=1, seed=9, phi=tr.TR_PEN_MCP,
                  psi=tr.TR_PEN_MCP, phi_gamma=30.0, psi_gamma=30.0, noise=tr.TR_NOISE_NONE,
                  **{"lambda": 0.1})
    Z = dev(zero, dt)
    h.set_state(dev(X, dt), Z, Z, Z, dev(X, dt), mu=0.5, t=3)
    h.step()
    got = h.get_state()
    for name, want in [("L", ref.L), ("E", ref.E), ("Y", ref.Y), ("Lam", ref.Lam), ("G", ref.G)]:
        g = got[name].double().cpu().numpy()
        if np.linalg.norm(want) == 0:
            assert np.linalg.norm(g) <= TOL[dt], name
        else:
            assert relF(g, want) < TOL[dt], (name, relF(g, want))
    h.close()


def test_tucker_engine_graph_steps_identical_to_eager():
    rng = np.random.default_rng(22)
    dims = (48, 40, 6, 3)
    X = rng.standard_normal((18, 48, 40))
    mask = (rng.random(X.shape) < 0.5).astype(np.uint8)
    M = np.where(mask == 1, X, 0.0)
    outs = []
    for graph in (False, True):
        h = tr.Handle(dev(M, "f32"), torch.from_numpy(mask).cuda(), dims, engine=tr.TR_LR_TUCKER,
                      rank=6, oversample=0, power_iters=1, seed=3, mu0=0.05)
        h.graph_mode(graph)
        for _ in range(5):
            h.step()
        outs.append(h.get_state())
        h.close()
    for k in ("L", "E", "Y", "Lam", "G"):
        assert torch.equal(outs[0][k], outs[1][k]), k
