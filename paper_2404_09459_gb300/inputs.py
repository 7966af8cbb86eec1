"""Seeded synthetic matrix pairs (input generation only; no GSV arithmetic).

A pair is built with planted generalized singular values, the construction the
paper uses for its synthetic experiments (Section 4.1: G1 = U Sigma1 R,
G2 = V Sigma2 R with orthonormalised Gaussian U, V, sorted uniform alpha,
beta = sqrt(1 - alpha^2)), made real-valued and numerically low-rank:

    G1 = U_r diag(alpha) D O_r + sigma N1,    G2 = V_r diag(beta) D O_r + sigma N2

U_r (m x r), V_r (p x r) Haar column-orthonormal, O_r (r x n) orthonormal rows,
D = diag(d_1..d_r) the singular scale of the shared factor R = D O_r, N1, N2
i.i.d. N(0, 1).  Without noise the r non-trivial GSV pairs are exactly
(alpha_i, beta_i) and the singular values of the stack [G1; G2] are d_i.

Used by the tests (the oracle and the GPU see the same arrays) and by the
benchmark.  The `torch` backend builds the same recipe on a CUDA device with
torch's generator (different random stream) for pairs too large for the host.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class PairSpec:
    """Shape and spectrum of one synthetic pair plus the solver parameters."""
    m: int
    p: int
    n: int
    r: int
    alpha: str = "uniform"      # "linspace" (0.99 .. 0.01) or "uniform" (U(0,1) sorted desc)
    decay: str = "exp10"        # "logspace02" (1..100), "exp10" exp(-i/10), "pow15" i^-1.5
    sigma: float = 1e-6
    k: int = 0                  # target rank (0: use r)
    oversample: int = 10
    q: int = 1
    seed: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def kk(self) -> int:
        return self.k if self.k else self.r

    @property
    def l(self) -> int:
        return self.kk + self.oversample


# Workloads.  `PAIR_FP64_SMALL` is the plain FP64 pair, `PAIR_TF32_LARGE` the single
# large mixed-precision pair, `PAIR_BF16_STRESS` the slow-decay precision stress pair.
PAIR_FP64_SMALL = PairSpec(m=2000, p=2000, n=200, r=20, alpha="linspace", decay="logspace02",
                           sigma=1e-8, k=20, oversample=10, q=1, seed=0)
PAIR_TF32_LARGE = PairSpec(m=20000, p=15000, n=1000, r=50, alpha="uniform", decay="exp10",
                           sigma=1e-6, k=50, oversample=10, q=2, seed=0)
PAIR_BF16_STRESS = PairSpec(m=120000, p=80000, n=4000, r=200, alpha="uniform", decay="pow15",
                            sigma=1e-4, k=200, oversample=20, q=3, seed=0)


def planted_alpha(spec: PairSpec, rng: np.random.Generator) -> np.ndarray:
    if spec.alpha == "linspace":
        a = np.linspace(0.99, 0.01, spec.r)
    elif spec.alpha == "uniform":
        a = np.sort(rng.uniform(0.0, 1.0, spec.r))[::-1].copy()
    else:
        raise ValueError(spec.alpha)
    return a


def planted_scale(spec: PairSpec) -> np.ndarray:
    i = np.arange(1, spec.r + 1, dtype=np.float64)
    if spec.decay == "logspace02":
        return np.logspace(0.0, 2.0, spec.r)
    if spec.decay == "exp10":
        return np.exp(-i / 10.0)
    if spec.decay == "pow15":
        return i ** -1.5
    raise ValueError(spec.decay)


def _haar_columns(rng: np.random.Generator, rows: int, cols: int) -> np.ndarray:
    a = rng.standard_normal((rows, cols))
    q, r = np.linalg.qr(a)
    return q * np.sign(np.diag(r))[None, :]


def planted_pair(spec: PairSpec, dtype=np.float64):
    """Numpy pair (G1, G2, alpha_true, beta_true) for `spec` (host memory)."""
    rng = np.random.default_rng(np.random.SeedSequence([spec.seed, spec.m, spec.p, spec.n, spec.r]))
    alpha = planted_alpha(spec, rng)
    beta = np.sqrt((1.0 - alpha) * (1.0 + alpha))
    d = planted_scale(spec)
    U = _haar_columns(rng, spec.m, spec.r)
    V = _haar_columns(rng, spec.p, spec.r)
    O = _haar_columns(rng, spec.n, spec.r).T
    G1 = (U * (alpha * d)[None, :]) @ O
    G2 = (V * (beta * d)[None, :]) @ O
    if spec.sigma:
        G1 += spec.sigma * rng.standard_normal(G1.shape)
        G2 += spec.sigma * rng.standard_normal(G2.shape)
    return G1.astype(dtype), G2.astype(dtype), alpha, beta


def planted_pair_torch(spec: PairSpec, device="cuda", dtype=None):
    """The same recipe built with torch on `device` (for pairs too large for numpy)."""
    import torch
    dtype = dtype or torch.float32
    g = torch.Generator(device=device)
    g.manual_seed(int(spec.seed) * 1000003 + spec.m * 7 + spec.p * 11 + spec.n * 13 + spec.r)
    rng = np.random.default_rng(np.random.SeedSequence([spec.seed, spec.m, spec.p, spec.n, spec.r]))
    alpha = planted_alpha(spec, rng)
    beta = np.sqrt((1.0 - alpha) * (1.0 + alpha))
    d = planted_scale(spec)

    def haar(rows, cols):
        # the thin QR of the Gaussian block runs on the host (numpy / LAPACK)
        return torch.from_numpy(_haar_columns(rng, rows, cols)).to(device)

    U = haar(spec.m, spec.r)
    V = haar(spec.p, spec.r)
    O = haar(spec.n, spec.r).T.contiguous()
    ad = torch.tensor(alpha * d, device=device)
    bd = torch.tensor(beta * d, device=device)
    out = []
    for basis, w, rows in ((U, ad, spec.m), (V, bd, spec.p)):
        G = torch.empty(rows, spec.n, device=device, dtype=dtype)
        step = 8192
        for r0 in range(0, rows, step):
            r1 = min(rows, r0 + step)
            blk = (basis[r0:r1] * w[None, :]) @ O
            if spec.sigma:
                blk += spec.sigma * torch.randn(r1 - r0, spec.n, generator=g, device=device,
                                                dtype=torch.float64)
            G[r0:r1] = blk.to(dtype)
        out.append(G)
    return out[0], out[1], alpha, beta


def full_gmp_pair(m: int, p: int, n: int, seed: int = 0, rank_frac: float = 0.6, dtype=np.float64):
    """The paper's own synthetic pair (Section 4.1), real-valued: G1 = U diag(alpha) R and
    G2 = V diag(beta) R with U (m x n), V (p x n) orthonormalised Gaussian, R (n x n) Gaussian
    and rank(G1) = rank(G2) = round(rank_frac min(m, p, n)).  So n - rank(G2) pairs have
    alpha = 1 (beta = 0), n - rank(G1) have alpha = 0 (beta = 1), and the rest take sorted
    U(0, 1) values, with beta = sqrt(1 - alpha^2).  The stack [G1; G2] has full rank n: every
    one of the n pairs is resolved (r = n), and each side needs a basis of its full rank.
    Returns (G1, G2, alpha, beta), alpha descending."""
    if m < n or p < n:
        raise ValueError("the construction needs m >= n and p >= n")
    rng = np.random.default_rng(np.random.SeedSequence([seed, m, p, n, 4101]))
    r = int(round(rank_frac * min(m, p, n)))
    n_one, n_zero = n - r, n - r
    n_mid = n - n_one - n_zero
    if n_mid < 0:
        raise ValueError("rank_frac must be at least 0.5")
    mid = np.sort(rng.uniform(0.0, 1.0, n_mid))[::-1]
    alpha = np.concatenate([np.ones(n_one), mid, np.zeros(n_zero)])
    beta = np.sqrt((1.0 - alpha) * (1.0 + alpha))
    U = _haar_columns(rng, m, n)
    V = _haar_columns(rng, p, n)
    R = rng.standard_normal((n, n))
    G1 = (U * alpha[None, :]) @ R
    G2 = (V * beta[None, :]) @ R
    return G1.astype(dtype), G2.astype(dtype), alpha, beta


def _haar_columns_complex(rng: np.random.Generator, rows: int, cols: int) -> np.ndarray:
    a = rng.standard_normal((rows, cols)) + 1j * rng.standard_normal((rows, cols))
    q, r = np.linalg.qr(a)
    d = np.diag(r)
    return q * (d / np.abs(d))[None, :]


def planted_pair_complex(spec: PairSpec, dtype=np.complex128):
    """The planted recipe over C: G1 = U_r diag(alpha) D O_r + sigma N1, G2 = V_r diag(beta) D O_r
    + sigma N2 with U_r, V_r complex Haar column-orthonormal, O_r complex orthonormal rows and
    N circularly symmetric complex Gaussian (E |N_ij|^2 = 1).  Returns (G1, G2, alpha, beta)."""
    rng = np.random.default_rng(np.random.SeedSequence([spec.seed, spec.m, spec.p, spec.n, spec.r, 7001]))
    alpha = planted_alpha(spec, rng)
    beta = np.sqrt((1.0 - alpha) * (1.0 + alpha))
    d = planted_scale(spec)
    U = _haar_columns_complex(rng, spec.m, spec.r)
    V = _haar_columns_complex(rng, spec.p, spec.r)
    O = _haar_columns_complex(rng, spec.n, spec.r).conj().T
    G1 = (U * (alpha * d)[None, :]) @ O
    G2 = (V * (beta * d)[None, :]) @ O
    if spec.sigma:
        for G in (G1, G2):
            G += spec.sigma * (rng.standard_normal(G.shape) + 1j * rng.standard_normal(G.shape)) / np.sqrt(2.0)
    return G1.astype(dtype), G2.astype(dtype), alpha, beta


def full_gmp_pair_complex(m: int, p: int, n: int, seed: int = 0, rank_frac: float = 0.6, dtype=np.complex128):
    """The paper's own synthetic pair of Section 4.1 as the paper states it, over C: as
    full_gmp_pair with complex orthonormalised Gaussian U, V and a complex Gaussian R."""
    if m < n or p < n:
        raise ValueError("the construction needs m >= n and p >= n")
    rng = np.random.default_rng(np.random.SeedSequence([seed, m, p, n, 4102]))
    r = int(round(rank_frac * min(m, p, n)))
    n_one = n_zero = n - r
    n_mid = n - n_one - n_zero
    if n_mid < 0:
        raise ValueError("rank_frac must be at least 0.5")
    mid = np.sort(rng.uniform(0.0, 1.0, n_mid))[::-1]
    alpha = np.concatenate([np.ones(n_one), mid, np.zeros(n_zero)])
    beta = np.sqrt((1.0 - alpha) * (1.0 + alpha))
    U = _haar_columns_complex(rng, m, n)
    V = _haar_columns_complex(rng, p, n)
    R = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(2.0)
    G1 = (U * alpha[None, :]) @ R
    G2 = (V * beta[None, :]) @ R
    return G1.astype(dtype), G2.astype(dtype), alpha, beta


def uneven_batch(npairs: int = 256, seed: int = 0, m_range=(2000, 30000), n_range=(100, 1000),
                 r_range=(10, 100), oversample: int = 10, q: int = 1, sigma: float = 1e-9):
    """Specs of a batch of uneven pairs: m, p ~ U[m_range], n ~ U[n_range],
    r ~ U[r_range] (clipped so that k + oversample <= min(m, p, n)), seed per pair.
    sigma = 1e-9 keeps every planted scale exp(-i/10), i <= 100, far above the noise floor
    sigma (sqrt(M) + sqrt(n)); at 1e-6 the tail of ranks above ~70 would sit in the noise and its
    GSVs would be noise-determined."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, npairs, 4242]))
    specs = []
    for i in range(npairs):
        m = int(rng.integers(m_range[0], m_range[1] + 1))
        p = int(rng.integers(m_range[0], m_range[1] + 1))
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        r = int(rng.integers(r_range[0], r_range[1] + 1))
        r = min(r, min(m, p, n) - oversample)
        specs.append(PairSpec(m=m, p=p, n=n, r=r, alpha="uniform", decay="exp10", sigma=sigma,
                              k=r, oversample=oversample, q=q, seed=seed * 100003 + i))
    return specs


def learned_pairs(npairs: int, seed: int = 0, sigma: float = 1e-9, m_range=(2000, 30000), n_range=(100, 1000),
                  r_range=(10, 100), oversample: int = 10):
    """Pairs of the learned-proposal workload: the uneven-batch laws (m, p, n, r, alpha, exp(-i/10)
    scale) with noise sigma; at sigma = 1e-6 the noise alone would be ~2e-3 of ||G||_F, above
    the 1e-4 residual tolerance the labels are taken at, so every basis narrower than n would miss."""
    return uneven_batch(npairs, seed, m_range=m_range, n_range=n_range, r_range=r_range, oversample=oversample,
                        q=1, sigma=sigma)


def mlp_init(seed: int = 0) -> np.ndarray:
    """Initial parameters of the 64-128-128-37 network (flat float32, W1 | b1 | W2 | b2 | W3 | b3,
    row-major): He-normal weights N(0, 2 / fan_in), zero biases."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 6412837]))
    parts = []
    for fin, fout in ((64, 128), (128, 128), (128, 37)):
        parts.append(rng.standard_normal(fin * fout) * np.sqrt(2.0 / fin))
        parts.append(np.zeros(fout))
    return np.concatenate(parts).astype(np.float32)


def aligned_rows(G, row_bytes: int = 16):
    """The same matrix stored with its row stride padded to a multiple of `row_bytes` (a view of
    a zero-padded torch tensor or numpy array): the layout the tensor-memory-accelerator
    products need to read G in place."""
    per = max(1, row_bytes // G.element_size()) if hasattr(G, "element_size") else max(1, row_bytes // G.itemsize)
    rows, n = G.shape
    ld = -(-n // per) * per
    if ld == n:
        return G
    if hasattr(G, "new_zeros"):
        buf = G.new_zeros((rows, ld))
    else:
        buf = np.zeros((rows, ld), dtype=G.dtype)
    buf[:, :n] = G
    return buf[:, :n]
