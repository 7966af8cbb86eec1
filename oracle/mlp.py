"""Plain FP64 CPU oracle of the learned (k, q) proposal (test infrastructure).

Only the tests, the smoke check and the CPU legs of the benchmark may import
this module; the product path never does.  It shares no code with the CUDA
path.  The proposal replaces the search over (k, q) of the fixed-rank method
(projector theorem of Section 3 with q power steps) by a classifier that reads
a cheap probe of the pair; Algorithm 1 (the adaptive range finder of Section 2)
stays the judge: it labels the training pairs and it is the fallback whenever
the proposed basis misses the residual tolerance.

Readings taken here (the paper has no learned component; each is also listed in
the design notes):
  * Probe features.  Per side s with G_s (M x n): Omega_p is the n x 64
    Gaussian of Philox stream 0x20000; Y = G Omega_p; mu_i = eigenvalues of
    Y^T Y, descending; g2 = ||G||_F^2.  Since E||G w||^2 = ||G||_F^2 for a
    Gaussian w, mu_i / (64 g2) ~ sigma_i^2 / sum sigma^2: dimensionless energy
    fractions of the leading 64 directions.  The 64 features are log10 of
    mu_1, mu_3, ..., mu_63 over 64 g2 (32 per side, side 1 first), clipped to
    [-12, 1]: an energy fraction of 1e-12 is far below the 1e-8 that a 1e-4
    relative residual leaves, and the clip keeps rounding-level eigenvalues
    (about 1e-16 of the largest in FP64) out of the features.  A 64-column
    probe shows where a side's energy falls off for ranks up to about 64; with
    16 columns the leading 16 fractions of a pair are the same for every rank
    above 16 under a fixed decay law, so the rank could not be read off.
  * Network: 64 -> 128 -> 128 -> 37, ReLU, inputs standardised by a fixed
    mean and standard deviation (from the training set); logits 0..31 are
    the k bucket (bucket b covers k = 4b+1 .. 4b+4), logits 32..36 are
    q = 0..4.  Loss: mean softmax cross-entropy of the two heads, summed.
    Adam (Kingma & Ba, ICLR 2015) with bias correction.
  * Labels at tolerance tol (relative cumulated residual, as Algorithm 1):
    k_ad = the larger of the two sides' basis sizes from Algorithm 1 with
    blocks of 4; the k bucket is the one holding max(k_ad - oversample, 1);
    q is the smallest q in 0..4 whose fixed-rank bases (k = top of the
    bucket, l = k + oversample) meet tol on both sides; if none does the
    bucket is raised (at most three times) and the search repeated.
"""
from __future__ import annotations

import numpy as np

from . import gsvd as O
from .philox import gaussian

IN, HID, KCLS, QCLS = 64, 128, 32, 5
OUT = KCLS + QCLS
PROBE_COLS = 64
K_BUCKET = 4
FEAT_MIN, FEAT_MAX = -12.0, 1.0
STREAM_PROBE = O.STREAM_PROBE
SHAPES = (("W1", (IN, HID)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)),
          ("W3", (HID, OUT)), ("b3", (OUT,)))
NPARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta) -> dict:
    """Flat parameter vector (the order of SHAPES, each row-major) -> dict of arrays."""
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.size == NPARAMS
    out, o = {}, 0
    for name, shape in SHAPES:
        size = int(np.prod(shape))
        out[name] = theta[o:o + size].reshape(shape)
        o += size
    return out


def pack(d: dict) -> np.ndarray:
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SHAPES])


# ------------------------------------------------------------------ features

def side_features(G: np.ndarray, seed: int, pair: int, side: int) -> np.ndarray:
    G = np.asarray(G, dtype=np.float64)
    n = G.shape[1]
    Om = gaussian(n, PROBE_COLS, seed, pair, side, STREAM_PROBE)
    Y = G @ Om
    g2 = float(np.sum(G * G))
    mu = np.linalg.eigvalsh(Y.T @ Y)[::-1]
    with np.errstate(divide="ignore"):
        f = np.log10(np.maximum(mu[0::2], 0.0) / (PROBE_COLS * g2))
    return np.clip(f, FEAT_MIN, FEAT_MAX)


def probe_features(G1, G2, seed: int, pair: int = 0) -> np.ndarray:
    """The 64 probe features of the pair (side 1 then side 2)."""
    return np.concatenate([side_features(G1, seed, pair, 0), side_features(G2, seed, pair, 1)])


# ------------------------------------------------------------------ network

def _relu(x):
    return np.maximum(x, 0.0)


def forward(theta, norm, X, bf16_weights: bool = False):
    """Logits (B x 37) and the activations.  norm = (mean[64], std[64]).
    bf16_weights: the weight matrices rounded to bfloat16 first (biases kept), the
    inference form."""
    p = unpack(theta)
    if bf16_weights:
        for name in ("W1", "W2", "W3"):
            p[name] = O.round_bf16(p[name]).astype(np.float64)
    mean, std = (np.asarray(a, dtype=np.float64) for a in norm)
    Xh = (np.asarray(X, dtype=np.float64) - mean) / std
    a1 = Xh @ p["W1"] + p["b1"]
    h1 = _relu(a1)
    a2 = h1 @ p["W2"] + p["b2"]
    h2 = _relu(a2)
    z = h2 @ p["W3"] + p["b3"]
    return z, dict(Xh=Xh, a1=a1, h1=h1, a2=a2, h2=h2, p=p)


def _log_softmax(z):
    zm = z - z.max(axis=1, keepdims=True)
    return zm - np.log(np.exp(zm).sum(axis=1, keepdims=True))


def loss_grad(theta, norm, X, yk, yq):
    """Mean cross-entropy of both heads and its gradient (flat, the order of SHAPES)."""
    z, c = forward(theta, norm, X)
    B = z.shape[0]
    yk = np.asarray(yk, dtype=np.int64)
    yq = np.asarray(yq, dtype=np.int64)
    lk = _log_softmax(z[:, :KCLS])
    lq = _log_softmax(z[:, KCLS:])
    rows = np.arange(B)
    loss = -(lk[rows, yk].mean() + lq[rows, yq].mean())
    dz = np.concatenate([np.exp(lk), np.exp(lq)], axis=1)
    dz[rows, yk] -= 1.0
    dz[rows, KCLS + yq] -= 1.0
    dz /= B
    p = c["p"]
    g = {"W3": c["h2"].T @ dz, "b3": dz.sum(axis=0)}
    d2 = (dz @ p["W3"].T) * (c["a2"] > 0)
    g["W2"] = c["h1"].T @ d2
    g["b2"] = d2.sum(axis=0)
    d1 = (d2 @ p["W2"].T) * (c["a1"] > 0)
    g["W1"] = c["Xh"].T @ d1
    g["b1"] = d1.sum(axis=0)
    return float(loss), pack(g)


def adam_step(theta, m, v, grad, t: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step t >= 1); returns new (theta, m, v)."""
    m = beta1 * np.asarray(m, dtype=np.float64) + (1 - beta1) * grad
    v = beta2 * np.asarray(v, dtype=np.float64) + (1 - beta2) * grad * grad
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    return np.asarray(theta, dtype=np.float64) - lr * mh / (np.sqrt(vh) + eps), m, v


def predict(theta, norm, X, bf16_weights: bool = True):
    """(k bucket, q) by argmax of each head."""
    z, _ = forward(theta, norm, np.atleast_2d(X), bf16_weights)
    return z[:, :KCLS].argmax(axis=1), z[:, KCLS:].argmax(axis=1)


def plan(z, quantile: float = 0.9):
    """The learned solve's decision from network outputs z (B x (KCLS + QCLS)): the k bucket is
    the smallest one whose cumulative softmax probability reaches `quantile` (an undersized basis
    costs an Algorithm 1 fallback, an oversized one only columns), q the most probable class
    (the first on ties).  Returns (k bucket, q) arrays."""
    z = np.atleast_2d(np.asarray(z, dtype=np.float64))
    zk = z[:, :KCLS]
    p = np.exp(zk - zk.max(axis=1, keepdims=True))
    p /= p.sum(axis=1, keepdims=True)
    kb = np.empty(z.shape[0], dtype=np.int64)
    for i in range(z.shape[0]):
        c = 0.0
        b = 0
        for b in range(KCLS):
            c += p[i, b]
            if c >= quantile:
                break
        kb[i] = b
    return kb, z[:, KCLS:].argmax(axis=1)


# ------------------------------------------------------------------ labels

def k_of_bucket(b: int) -> int:
    return K_BUCKET * (int(b) + 1)


def bucket_of_k(k: int) -> int:
    return int(np.clip((int(k) - 1) // K_BUCKET, 0, KCLS - 1))


def fixed_residual(G, k: int, oversample: int, q: int, seed: int, pair: int, side: int) -> float:
    """Relative residual ||G - Q Q^T G||_F / ||G||_F of the fixed-rank basis."""
    G = np.asarray(G, dtype=np.float64)
    Q = O.basis_fixed(G, min(k + oversample, min(G.shape)), q, seed, pair, side)
    return float(np.linalg.norm(G - Q @ (Q.T @ G)) / np.linalg.norm(G))


def labels(G1, G2, tol: float, seed: int, pair: int = 0, oversample: int = 10):
    """(k bucket, q, k_ad) of the pair under the label rule of the module docstring."""
    k_ad = max(O.adaptive_basis(G, tol, K_BUCKET, seed, pair, s)[0].shape[1] for s, G in enumerate((G1, G2)))
    kb = bucket_of_k(max(k_ad - oversample, 1))
    for _ in range(4):
        k = k_of_bucket(kb)
        for q in range(5):
            if all(fixed_residual(G, k, oversample, q, seed, pair, s) <= tol for s, G in enumerate((G1, G2))):
                return kb, q, k_ad
        if kb == KCLS - 1:
            break
        kb += 1
    return kb, 4, k_ad
