"""Seeded synthetic workloads shaped like the paper's recovery problems.

This module only builds *inputs*: ground-truth tensors with a prescribed
transform-domain tubal rank, observation masks, noise and outliers.  It
holds none of the recovery method's arithmetic; the low-rank construction
uses scipy's inverse DCT, a library routine neither the CUDA path nor the
CPU oracle calls.  Both the tests and the benchmark draw their inputs here.

Layout: every tensor is returned as its face-slice stack (n, n1, n2) in C
order, n = n3*...*nd, slice index j = i3 + n3*(i4 + n4*(...)) (i3 fastest),
which is exactly the device layout the C ABI expects.

Recipes (Sec. 6 "Experimental Datasets" protocol: data normalised to a fixed
scale, impulse noise added at ratio NR, then SR * prod(n_i) entries sampled
at random to form P_Omega(M)):

* transform-domain slices Xbar^<j> = A_j B_j^T / sqrt(r_j), A_j (n1 x r_j),
  B_j (n2 x r_j) i.i.d. N(0, 1), so entries have unit variance; then
  X* = L^{-1}(Xbar) with the orthonormal DCT-II along modes 3..d;
* Gaussian noise N(0, sigma^2) on every entry;
* sparse outliers: exactly round(outlier_ratio * N) entries (uniform,
  without replacement) receive an added U(-1, 1) value;
* mask: exactly round(SR * N) entries observed, uniform without replacement;
* M = P_Omega(X* + noise + outliers) (zero off Omega).
"""

from dataclasses import dataclass, field

import numpy as np
import scipy.fft


@dataclass
class Workload:
    name: str
    dims: tuple            # (n1, n2, n3, ..., nd)
    rank: object           # int, or "powerlaw"
    sr: float              # sampling ratio
    noise_sigma: float = 0.0
    outlier_ratio: float = 0.0
    dtype: str = "f32"
    l: int = 0             # sketch width r + oversampling
    q: int = 1             # power iterations
    iters: int = 50
    seed: int = 1000
    noise_model: str = "l1"     # "none" (GNHTC) or "l1" (GNRHTC)
    extra: dict = field(default_factory=dict)

    @property
    def n1(self):
        return self.dims[0]

    @property
    def n2(self):
        return self.dims[1]

    @property
    def tdims(self):
        return tuple(self.dims[2:])

    @property
    def nslices(self):
        n = 1
        for v in self.dims[2:]:
            n *= v
        return n

    @property
    def numel(self):
        return self.n1 * self.n2 * self.nslices


WORKLOADS = {
    # order-3 FP64 64x64x16, tubal rank 5, 50% observed, noise-free, l = 5+10.
    "tubal64_r5": Workload("tubal64_r5", (64, 64, 16), 5, 0.5, dtype="f64",
                           l=15, q=1, iters=50, seed=1000, noise_model="none"),
    # order-4 FP32 200x200x20x20 (400 slices), rank 10, sigma 1e-3, 5% outliers,
    # 30% observed, l = 10+10.
    "tubal200x400_r10": Workload("tubal200x400_r10", (200, 200, 20, 20), 10, 0.3,
                                 noise_sigma=1e-3, outlier_ratio=0.05, dtype="f32",
                                 l=20, q=1, iters=100, seed=1001, noise_model="l1"),
    # order-3 1024x1024x64, rank 32, 20% observed, l = 32+10 padded to 48.
    "tubal1024x64_r32": Workload("tubal1024x64_r32", (1024, 1024, 64), 32, 0.2,
                                 dtype="f32", l=48, q=1, iters=20, seed=1002,
                                 noise_model="none"),
    # order-4 512x512x32x16, power-law slice ranks in [2, 64], 15% observed.
    "tubal512x512_powerlaw": Workload("tubal512x512_powerlaw", (512, 512, 32, 16),
                                      "powerlaw", 0.15, dtype="f32", l=74, q=1,
                                      iters=20, seed=3000, noise_model="none"),
}


def powerlaw_ranks(n, rng, lo=2, hi=64, alpha=1.5):
    """Discrete power law p(r) ~ r^-alpha on [lo, hi]."""
    r = np.arange(lo, hi + 1)
    p = r.astype(np.float64) ** -alpha
    p /= p.sum()
    return rng.choice(r, size=n, p=p)


def _idct_modes(Xbar, tdims):
    """Inverse orthonormal DCT-II along every transformed mode of a stack."""
    n, n1, n2 = Xbar.shape
    v = Xbar.reshape(tuple(reversed(tdims)) + (n1, n2))
    nt = len(tdims)
    for axis in range(nt):
        v = scipy.fft.idct(v, type=2, norm="ortho", axis=axis)
    return v.reshape(n, n1, n2)


def lowrank_tensor(dims, ranks, rng):
    """Slice stack X* whose transformed slices have the given ranks."""
    n1, n2 = dims[0], dims[1]
    tdims = tuple(dims[2:])
    n = int(np.prod(tdims)) if tdims else 1
    if np.isscalar(ranks):
        ranks = np.full(n, int(ranks))
    Xbar = np.empty((n, n1, n2), dtype=np.float64)
    for j in range(n):
        r = int(ranks[j])
        A = rng.standard_normal((n1, r))
        B = rng.standard_normal((n2, r))
        Xbar[j] = (A @ B.T) / np.sqrt(r)
    return _idct_modes(Xbar, tdims), np.asarray(ranks)


def exact_count_mask(numel, ratio, rng):
    """Exactly round(ratio * numel) True entries, uniform without replacement."""
    k = int(round(ratio * numel))
    idx = rng.permutation(numel)[:k]
    m = np.zeros(numel, dtype=np.uint8)
    m[idx] = 1
    return m


def make_problem(w, seed=None):
    """Build (X*, M, mask, ranks) for workload `w` as float64 / uint8 stacks."""
    rng = np.random.default_rng(w.seed if seed is None else seed)
    n, n1, n2 = w.nslices, w.n1, w.n2
    if w.rank == "powerlaw":
        ranks = powerlaw_ranks(n, rng)
    else:
        ranks = int(w.rank)
    X, ranks = lowrank_tensor(w.dims, ranks, rng)
    obs = X.copy()
    if w.noise_sigma > 0:
        obs += w.noise_sigma * rng.standard_normal(obs.shape)
    if w.outlier_ratio > 0:
        om = exact_count_mask(obs.size, w.outlier_ratio, rng).reshape(obs.shape)
        obs += om * rng.uniform(-1.0, 1.0, size=obs.shape)
    mask = exact_count_mask(obs.size, w.sr, rng).reshape(obs.shape)
    M = np.where(mask == 1, obs, 0.0)
    return X, M, mask, ranks


def random_state(shape, seed, scale=1.0):
    """Random iterate (L, E, Y, Lambda, G) for per-step parity tests."""
    rng = np.random.default_rng(seed)
    return [scale * rng.standard_normal(shape) for _ in range(5)]


def lowrank_plus_noise_stack(n, n1, n2, rank, noise, seed):
    """A transform-domain stack with slices of the given rank plus noise."""
    rng = np.random.default_rng(seed)
    out = np.empty((n, n1, n2))
    for j in range(n):
        r = int(rank[j]) if not np.isscalar(rank) else int(rank)
        A = rng.standard_normal((n1, r))
        B = rng.standard_normal((n2, r))
        out[j] = A @ B.T / np.sqrt(max(r, 1))
    out += noise * rng.standard_normal(out.shape)
    return out


def one_bit_observations(Lstar, m, theta, noise_sd, rng):
    """Dithered one-bit samples of a tensor (the observation model of the
    one-bit completion model): m entries drawn uniformly with replacement,
    y_k = Lstar[s_k] + eps_k with eps_k ~ N(0, noise_sd^2), and
    q_k = sign(y_k + xi_k) with dither xi_k ~ U[-theta, theta] (sign(0) = +1).
    Returns (s, q): flat entry indices (int64) and signs (+-1, float64)."""
    flat = np.asarray(Lstar, dtype=np.float64).ravel()
    s = rng.integers(0, flat.size, size=int(m))
    y = flat[s] + noise_sd * rng.standard_normal(int(m))
    xi = rng.uniform(-theta, theta, size=int(m))
    q = np.where(y + xi >= 0.0, 1.0, -1.0)
    return s.astype(np.int64), q
