"""tr_slice_prox_noalloc against tr_slice_prox.

The no-allocation entry point serves callers that cannot call cudaMalloc
(latency-critical host loops, code inside another framework's memory pool).
It must produce what the handle-based slice pass produces, on two calls in
a row (its fixed scratch array keeps the previous call's contents), and must
refuse a problem whose scratch exceeds the fixed array.  Before the checked
calls, one call of a larger shape with a wider sketch on an all-NaN stack
leaves NaN across the array at other offsets than the checked shape uses,
so a read of anything the checked call did not write itself shows up.
This file sorts last so that a run stopping at the first failure has run
every other test first.
"""

import numpy as np
import pytest

from paper_2506_09594_gb300 import synth, tr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _stack(n, n1, n2, dtype):
    Ab = synth.lowrank_plus_noise_stack(n, n1, n2, 6, 0.05, seed=n * n1 + n2)
    return torch.from_numpy(Ab).to("cuda", dtype)


@pytest.mark.parametrize("dtype,tol", [(torch.float32, 1e-4), (torch.float64, 1e-10)])
def test_noalloc_matches_handle_slice_prox_twice(dtype, tol):
    tr.load()
    n, n1, n2, l, q = 24, 70, 45, 16, 1
    Ab = _stack(n, n1, n2, dtype)
    tau = 0.3 * float(torch.linalg.matrix_norm(Ab[0], ord=2))
    M = torch.zeros((n, n1, n2), dtype=dtype, device="cuda")
    mask = torch.ones((n, n1, n2), dtype=torch.uint8, device="cuda")
    h = tr.Handle(M, mask, (n1, n2, n), rank=l, oversample=0, power_iters=q,
                  phi=tr.TR_PEN_MCP, phi_theta=1.0, phi_gamma=3 * tau + 1, seed=99)
    ref = h.slice_prox(Ab, tau, t=7)
    torch.cuda.synchronize()
    h.close()
    # leave NaN in the shared array: 24 slices of 96 x 96 at sketch width 48
    junk = torch.full((24, 96, 96), float("nan"), dtype=dtype, device="cuda")
    tr.slice_prox_noalloc(junk, torch.empty_like(junk), 48, 1, tau, 3, seed=5)
    torch.cuda.synchronize()
    for call in range(2):
        out = torch.full_like(Ab, float("nan"))
        tr.slice_prox_noalloc(Ab, out, l, q, tau, 7, seed=99, phi=tr.TR_PEN_MCP, theta=1.0,
                              gamma=3 * tau + 1)
        torch.cuda.synchronize()
        err = float(torch.linalg.norm(out - ref) / torch.linalg.norm(ref))
        assert err < tol, (call, err)


def test_noalloc_refuses_oversized_problem():
    tr.load()
    n, n1, n2 = 400, 200, 200          # needs ~19 MB of scratch at l = 20
    Ab = torch.zeros((n, n1, n2), dtype=torch.float32, device="cuda")
    Gb = torch.empty_like(Ab)
    with pytest.raises(tr.TrError) as ei:
        tr.slice_prox_noalloc(Ab, Gb, 20, 1, 1.0, 0)
    assert ei.value.status == tr.TR_EUNSUPPORTED
    assert "bytes" in str(ei.value)
