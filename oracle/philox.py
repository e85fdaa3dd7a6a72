"""Philox4x32-10 and Box-Muller Gaussians for the sketch matrices.

Test infrastructure (see the package docstring).

Alg. 1 and Alg. 3 each "draw a Gaussian random matrix".  So that the CPU
oracle and the GPU path draw the *same* matrix, both sides implement one
counter-based generator from its published definition:

* Philox4x32-10: Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
  easy as 1, 2, 3", SC'11.  A 128-bit counter (four 32-bit words) and a
  64-bit key (two words) go through ten rounds.  Each round multiplies word
  0 and word 2 by two fixed odd multipliers, producing 64-bit products
  (hi, lo); the new counter is (hi_b ^ c1 ^ k0, lo_b, hi_a ^ c3 ^ k1, lo_a)
  where (hi_a, lo_a) comes from word 0 and (hi_b, lo_b) from word 2.  The
  key words are advanced by two Weyl increments before every round but the
  first.
* Box-Muller: Box & Muller (1958).  Two uniforms (u1, u2) in (0, 1] give
  r = sqrt(-2 ln u1) and the pair (r cos 2 pi u2, r sin 2 pi u2).

Sketch element addressing (shared *definition*, not shared code): the
sketch Omega for ADMM iteration ``t``, face slice ``j`` and stream ``s`` is
an (n2 x l) matrix.  Element (k, c) has linear index m = c*n2 + k
(column-major).  Counter = (m // 4, j, t, s), key = (seed mod 2^32,
seed div 2^32).  The four output words w0..w3 become u_i = (w_i + 1/2)/2^32
and the four Gaussians (z0, z1) from (u0, u1), (z2, z3) from (u2, u3);
element m takes z_{m mod 4}.
"""

import numpy as np

# Philox4x32 multipliers and Weyl key increments (Salmon et al., SC'11).
PHILOX_M0 = np.uint64(0xD2511F53)
PHILOX_M1 = np.uint64(0xCD9E8D57)
PHILOX_W0 = np.uint64(0x9E3779B9)
PHILOX_W1 = np.uint64(0xBB67AE85)
_MASK32 = np.uint64(0xFFFFFFFF)
_SHIFT32 = np.uint64(32)

# Stream tags (fourth counter word).
STREAM_SKETCH = 0      # the sketch Omega of the randomized range finder
STREAM_ADAPTIVE = 1    # the start block and refills of the adaptive engine
STREAM_TUCKER_1 = 2    # the mode-1 Gaussian block of the shared-Tucker engine
STREAM_TUCKER_2 = 4    # the mode-2 Gaussian block of the shared-Tucker engine
STREAM_AD_TUCKER_1 = 0x10000  # mode-1 start block and refills of the fixed-accuracy
                              # Tucker engine: stream STREAM_AD_TUCKER_1 + 2*draw
STREAM_AD_TUCKER_2 = 0x20000  # the same for mode 2


def philox4x32_10(counter, key):
    """Ten Philox4x32 rounds.

    counter: integer array (..., 4) of 32-bit words; key: (..., 2) (or (2,)).
    Returns a uint64 array (..., 4) holding the four 32-bit output words.
    """
    ctr = np.asarray(counter, dtype=np.uint64) & _MASK32
    k = np.asarray(key, dtype=np.uint64) & _MASK32
    c0, c1, c2, c3 = ctr[..., 0], ctr[..., 1], ctr[..., 2], ctr[..., 3]
    k0, k1 = k[..., 0], k[..., 1]
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + PHILOX_W0) & _MASK32
            k1 = (k1 + PHILOX_W1) & _MASK32
        prod_a = c0 * PHILOX_M0          # < 2^64: exact in uint64
        prod_b = c2 * PHILOX_M1
        hi_a, lo_a = prod_a >> _SHIFT32, prod_a & _MASK32
        hi_b, lo_b = prod_b >> _SHIFT32, prod_b & _MASK32
        c0, c1, c2, c3 = (hi_b ^ c1 ^ k0), lo_b, (hi_a ^ c3 ^ k1), lo_a
    return np.stack([c0, c1, c2, c3], axis=-1)


def uniform_open01(words):
    """Map 32-bit words to (0, 1]: u = (w + 1/2) / 2^32, in float64."""
    return (np.asarray(words, dtype=np.float64) + 0.5) * 2.0 ** -32


def box_muller(u1, u2):
    """Box & Muller (1958): two uniforms -> two independent N(0, 1)."""
    r = np.sqrt(-2.0 * np.log(u1))
    theta = 2.0 * np.pi * u2
    return r * np.cos(theta), r * np.sin(theta)


def gaussian_block(seed, t, j, rows, cols, stream=STREAM_SKETCH):
    """The (rows x cols) Gaussian matrix drawn at iteration t for slice j.

    Element (k, c) uses linear index m = c*rows + k (column-major); see the
    module docstring for the counter layout.
    """
    seed = int(seed)
    key = np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint64)
    m = np.arange(rows * cols, dtype=np.uint64)
    groups = m // np.uint64(4)
    ngroups = int(groups[-1]) + 1 if rows * cols else 0
    g = np.arange(ngroups, dtype=np.uint64)
    ctr = np.stack([g,
                    np.full_like(g, np.uint64(j)),
                    np.full_like(g, np.uint64(t)),
                    np.full_like(g, np.uint64(stream))], axis=-1)
    w = philox4x32_10(ctr, key)
    u = uniform_open01(w)
    z0, z1 = box_muller(u[:, 0], u[:, 1])
    z2, z3 = box_muller(u[:, 2], u[:, 3])
    z = np.stack([z0, z1, z2, z3], axis=-1).reshape(-1)
    vals = z[: rows * cols]
    # column-major: element (k, c) at m = c*rows + k
    return vals.reshape(cols, rows).T.copy()
