"""GPU parity of the gradient-domain building blocks (tr_grad,
tr_gradient_solve) against the FP64 oracle (oracle/ctv.py): the periodic
differences nabla_k and nabla_k^T, and the solve of
(I + sum_{k in Gamma} nabla_k^T nabla_k) X = R (Eq. coef-tensor, Eq. gnrhtc-L),
on ragged shapes of orders 2 to 4 that span several 64 x 64 product tiles.
Tolerances: differences to 1e-14 (FP64) and 1e-6 (FP32) of the largest entry; the solve 1e-12
(FP64) and 1e-5 (FP32) relative to the largest entry.
"""

import numpy as np
import pytest

from oracle import ctv
from paper_2506_09594_gb300 import tr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TDT = {"f64": torch.float64, "f32": torch.float32}
SHAPES = [(37, 29, 5, 3), (70, 66, 4), (130, 9), (16, 80, 1, 6)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    tr.load()


def stack(dims, rng):
    n = int(np.prod(dims[2:])) if len(dims) > 2 else 1
    return rng.standard_normal((n, dims[0], dims[1]))


@pytest.mark.parametrize("dt", ["f64", "f32"])
@pytest.mark.parametrize("dims", SHAPES)
def test_grad_matches_oracle(dt, dims):
    rng = np.random.default_rng(1)
    X = stack(dims, rng)
    Xd = torch.from_numpy(X).to("cuda", TDT[dt])
    Xh = Xd.double().cpu().numpy()
    for k in range(1, len(dims) + 1):
        for adj in (False, True):
            got = tr.grad(Xd, dims, k, adjoint=adj).double().cpu().numpy()
            want = (ctv.grad_t if adj else ctv.grad)(Xh, tuple(dims[2:]), k)
            tol = (1e-14 if dt == "f64" else 1e-6) * np.abs(want).max()
            assert np.abs(got - want).max() <= tol, (k, adj)


@pytest.mark.parametrize("dt", ["f64", "f32"])
@pytest.mark.parametrize("dims,modes", [((37, 29, 5, 3), (1, 2, 3, 4)), ((70, 66, 4), (1, 2)),
                                        ((70, 66, 4), (3,)), ((130, 9), (1, 2)),
                                        ((16, 80, 1, 6), (2, 4)), ((37, 29, 5, 3), ())])
def test_gradient_solve_matches_oracle(dt, dims, modes):
    rng = np.random.default_rng(2)
    R = stack(dims, rng)
    Rd = torch.from_numpy(R).to("cuda", TDT[dt])
    got = tr.gradient_solve(Rd, dims, modes).double().cpu().numpy()
    Rh = Rd.double().cpu().numpy()
    want = ctv.l_update(Rh, {k: np.zeros_like(Rh) for k in modes}, tuple(dims[2:]), modes)
    tol = 1e-12 if dt == "f64" else 1e-5
    assert np.abs(got - want).max() <= tol * np.abs(want).max()
