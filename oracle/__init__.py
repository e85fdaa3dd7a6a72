"""FP64 CPU oracle for the per-iteration low-rank proximal step of the
GNRHTC / GNHTC ADMM of "Accelerating Large-Scale Regularized High-Order
Tensor Recovery" (arXiv 2506.09594).

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import or run it.  The CUDA library never calls it and shares no code with
it: no kernels, headers, helpers, tables or constant generators.  The only
module both sides use is the seeded input generator
``paper_2506_09594_gb300.synth``, which holds none of the method's
arithmetic.

Everything here is plain numpy in float64, written step by step in the
paper's order and notation:

* ``philox``    Philox4x32-10 counters + Box-Muller Gaussians (the sketch
                matrices the method draws, Alg. 1 "draw a Gaussian random
                matrix").
* ``transform`` the invertible transform L = x_3 U_3 ... x_d U_d with the
                orthonormal DCT-II or the DFT of the paper's experiments
                (Sec. 2, Eq. trans / orth), and face slices X^<j> (Sec. 2).
* ``prox``      scalar proximal maps Prox_{psi,mu} (Eq. equ_gst1) for the
                l1 and MCP penalties, and GNHTT (Sec. 4.2.1).
* ``svt``       GNHTSVT D_{Phi,tau}(A, L): the deterministic branch of
                Alg. 4 (full SVD of every transformed face slice), the
                per-slice randomized branch (Gaussian sketch, power
                iterations, QR, small SVD of Q^T A), and the per-slice
                fixed-accuracy block-Lanczos engine restated from Alg. 3.
* ``admm``      one iteration of Alg. 5 in the pure-L form (Gamma = {I})
                and the loop around it.
* ``learned``   the learned sketch-width engine (not in the paper): slice
                features, width plan, certificate and the rank-predictor
                MLP (forward, backpropagation, Adam).
* ``tucker``    the paper's own randomized GNHTSVT: shared Tucker factors of
                the two spatial modes by Alg. 1 (R-STHOSVD-BKI, block Krylov
                space, orthonormal basis, top singular vectors of
                Z^T A A^T Z, sequential truncation), then the deterministic
                GNTSVT of the core (Alg. 4, randomized branch); and the
                fixed-accuracy form, Alg. AD-RSTHOSVD-BLBP.
* ``ctv``       the gradient-domain prior (GNHTCTV): difference operators
                nabla_k, the FFT-diagonalised L-update (Eq. coef-tensor,
                Eq. gnrhtc-L) and one iteration of Alg. 5 with a set Gamma
                of gradient directions.
* ``onebit``    the one-bit completion model GNOBHTC: one iteration of
                Alg. 6 (box-constrained L-step derived from Eq.
                1bittensorqqqq, FFT Z-step, GNHTSVT G-steps).

Parity status: every function is pinned by ``tests/test_oracle_*.py``
against closed forms, brute force, library routines it does not itself
call, or published known-answer vectors, except where a docstring says
"parity unpinned".
"""

from . import philox, transform, prox, svt, admm, learned, tucker, ctv, onebit  # noqa: F401
