"""CPU emulation (numpy) of the rank-l rebuild kernel's work split.

For slices above the fused rebuild's size, Gbar = Z Qb^T (n1 x l times
l x n2) runs in `rank_update_kernel`: one CTA of 256 threads per BT x BT
output tile (BT = 256, 128 or 64), both panels' tile rows staged k-major
and zero-filled past the ragged edge, and tasks of 8 rows x 4 columns taken
by thread t, t + 256, ... with the task's (row group, column group) advanced
incrementally (step 256 = step_r row groups + step_c column groups, with a
carry).  This file replays that split for every CTA and thread and checks
that each output element is written exactly once, that no read leaves the
staged tile, and that the result equals Z Qb^T, on ragged sizes."""

import numpy as np
import pytest


def _replay(Z, Qb, BT):
    n1, l = Z.shape
    n2 = Qb.shape[0]
    C = np.zeros((n1, n2))
    writes = np.zeros((n1, n2), np.int64)
    for r0 in range(0, n1, BT):
        for c0 in range(0, n2, BT):
            tr, tc = min(n1 - r0, BT), min(n2 - c0, BT)
            Zk = np.zeros((l, BT))
            Qk = np.zeros((l, BT))
            Zk[:, :tr] = Z[r0:r0 + tr].T
            Qk[:, :tc] = Qb[c0:c0 + tc].T
            RG, CG = (tr + 7) // 8, (tc + 3) // 4
            step_r, step_c = 256 // CG, 256 % CG
            for tid in range(256):
                rg, cg = tid // CG, tid % CG
                t = tid
                while t < RG * CG:
                    assert (rg, cg) == divmod(t, CG)
                    assert rg * 8 + 8 <= BT and cg * 4 + 4 <= BT     # reads stay in the tile
                    acc = Zk[:, rg * 8:rg * 8 + 8].T @ Qk[:, cg * 4:cg * 4 + 4]
                    for i in range(8):
                        if rg * 8 + i >= tr:
                            break
                        for jj in range(4):
                            col = c0 + cg * 4 + jj
                            if col < c0 + tc:
                                C[r0 + rg * 8 + i, col] = acc[i, jj]
                                writes[r0 + rg * 8 + i, col] += 1
                    rg += step_r
                    cg += step_c
                    if cg >= CG:
                        cg -= CG
                        rg += 1
                    t += 256
    return C, writes


@pytest.mark.parametrize("n1, n2, l, BT", [(200, 200, 20, 256), (300, 130, 7, 128),
                                           (37, 513, 5, 64), (520, 260, 12, 256),
                                           (65, 64, 3, 64)])
def test_every_output_written_once_and_equal_to_the_product(n1, n2, l, BT):
    rng = np.random.default_rng(n1 + n2 + l + BT)
    Z = rng.standard_normal((n1, l))
    Qb = rng.standard_normal((n2, l))
    C, writes = _replay(Z, Qb, BT)
    assert writes.min() == 1 and writes.max() == 1
    assert np.abs(C - Z @ Qb.T).max() <= 1e-12 * max(1.0, np.abs(Z @ Qb.T).max())
