"""Training driver of the learned (k, q) proposal.

Orchestration only: the probe features, the labels (Algorithm 1 and the fixed-rank
bases, in FP64 on the GPU), the network's forward and backward passes and the Adam
steps all run in the library's kernels through the C ABI.

Label rule (the paper has no learned component; this is the reading the network is
trained to): at residual tolerance tol, k_ad is the larger of the two sides' basis
sizes from Algorithm 1 with blocks of 4; the k bucket is the one holding
max(k_ad - oversample, 1); q is the smallest q in 0..4 whose fixed-rank bases
(k = top of the bucket, l = k + oversample) meet tol on both sides (cumulated
residual of Section 2); if none does, the bucket is raised (at most three times).
The labels are computed in FP64: the cumulated residual cancels below about
sqrt(u) ||G||_F, ~3e-4 with FP32 data, which could not certify tol = 1e-4.
"""
from __future__ import annotations

import struct
import time

import numpy as np

from . import (FLAG_BASIS_ONLY, MLP_HID, MLP_IN, MLP_KBUCKET, MLP_KCLS, MLP_PARAMS, MLP_QCLS, Context,
               GsvdRandError)
from .inputs import mlp_init, planted_pair_torch


def bucket_of_k(k: int) -> int:
    return int(np.clip((int(k) - 1) // MLP_KBUCKET, 0, MLP_KCLS - 1))


def k_of_bucket(b: int) -> int:
    return MLP_KBUCKET * (int(b) + 1)


class Labeler:
    """Features and labels of pairs (FP64 device tensors) with two reusable contexts."""

    def __init__(self, tol: float = 1e-4, oversample: int = 10, device: int = 0):
        self.tol, self.os, self.device = tol, oversample, device
        self.ca = Context("fp64", device=device, adaptive=True, block_b=MLP_KBUCKET, tol=tol, flags=FLAG_BASIS_ONLY)
        self.cf = Context("fp64", device=device, flags=FLAG_BASIS_ONLY)

    def close(self):
        self.ca.close()
        self.cf.close()

    def adaptive_cols(self, G1, G2, seed: int) -> int:
        try:
            self.ca.solve(G1, G2, 1, 0, 0, seed)
        except GsvdRandError as e:
            if e.name != "TOL_MISS":
                raise
        return max(self.ca.basis_cols())

    def label(self, G1, G2, seed: int):
        """(k bucket, q, k_ad)."""
        k_ad = self.adaptive_cols(G1, G2, seed)
        lmax = min(G1.shape[0], G2.shape[0], G1.shape[1], 224)
        kb = bucket_of_k(max(k_ad - self.os, 1))
        for _ in range(4):
            k = max(1, min(k_of_bucket(kb), lmax - self.os))
            for q in range(5):
                out = self.cf.solve(G1, G2, k, self.os, q, seed)
                if max(out["resid"]) <= self.tol:
                    return kb, q, k_ad
            if kb == MLP_KCLS - 1 or k_of_bucket(kb) >= lmax - self.os:
                break
            kb += 1
        return kb, MLP_QCLS - 1, k_ad


def make_dataset(specs, tol: float = 1e-4, oversample: int = 10, device: int = 0, features_prec: str = "fp64"):
    """Features X (N x 64 float32), labels yk, yq (int32) and k_ad of the pairs `specs`
    (each generated on the device from its seed, labelled, then freed)."""
    import torch
    lab = Labeler(tol, oversample, device)
    fctx = Context(features_prec, device=device)
    X = np.zeros((len(specs), MLP_IN), np.float32)
    yk = np.zeros(len(specs), np.int32)
    yq = np.zeros(len(specs), np.int32)
    kad = np.zeros(len(specs), np.int32)
    try:
        for i, s in enumerate(specs):
            G1, G2, _, _ = planted_pair_torch(s, device=f"cuda:{device}", dtype=torch.float64)
            g1, g2 = (G1, G2) if features_prec == "fp64" else (G1.float(), G2.float())
            X[i] = fctx.probe_features(g1, g2, s.seed).cpu().numpy()
            yk[i], yq[i], kad[i] = lab.label(G1, G2, s.seed)
            del G1, G2, g1, g2
    finally:
        lab.close()
        fctx.close()
    return X, yk, yq, kad


def train(X, yk, yq, epochs: int = 200, batch: int = 256, lr: float = 1e-3, seed: int = 0, device: int = 0,
          ctx: Context | None = None):
    """FP32 training on the device.  Returns (params, norm, per-epoch mean loss)."""
    import torch
    dev = f"cuda:{device}"
    X = np.asarray(X, np.float32)
    N = X.shape[0]
    B = min(batch, N)
    mean = X.mean(axis=0)
    std = np.maximum(X.std(axis=0), 1e-3)
    norm = torch.from_numpy(np.concatenate([mean, std]).astype(np.float32)).to(dev)
    params = torch.from_numpy(mlp_init(seed)).to(dev)
    m = torch.zeros(MLP_PARAMS, dtype=torch.float32, device=dev)
    v = torch.zeros_like(m)
    Xd = torch.from_numpy(X).to(dev)
    ykd = torch.from_numpy(np.asarray(yk, np.int32)).to(dev)
    yqd = torch.from_numpy(np.asarray(yq, np.int32)).to(dev)
    rng = np.random.default_rng(np.random.SeedSequence([seed, 771]))
    own = ctx is None
    ctx = ctx or Context("fp32", device=device)
    hist, t = [], 0
    try:
        for _ in range(epochs):
            steps = N // B
            order = torch.from_numpy(rng.permutation(N)[:steps * B].astype(np.int32)).to(dev)
            losses = ctx.mlp_train(params, m, v, norm, Xd, ykd, yqd, order, B, t, lr)
            t += steps
            hist.append(float(losses.mean().item()))
    finally:
        if own:
            ctx.close()
    return params, norm, np.array(hist)


def predict(params, norm, X, bf16: bool = True, device: int = 0, ctx: Context | None = None,
            quantile: float | None = None):
    """(k bucket, q): argmax of each head, or for k the smallest bucket whose cumulative
    softmax probability reaches `quantile` (the learned solve's rule with 0.9)."""
    import torch
    own = ctx is None
    ctx = ctx or Context("fp32", device=device)
    try:
        z = ctx.mlp_forward(params, norm, torch.as_tensor(np.asarray(X, np.float32)).to(params.device), bf16)
    finally:
        if own:
            ctx.close()
    if quantile is not None:  # the learned solve's own rule, run by the library on the device
        ctx2 = ctx if not own else Context("fp32", device=device)
        try:
            plan = ctx2.mlp_plan(z.contiguous(), quantile)
        finally:
            if own:
                ctx2.close()
        return plan[:, 2], plan[:, 1]
    z = z.cpu().numpy()
    return z[:, :MLP_KCLS].argmax(axis=1), z[:, MLP_KCLS:].argmax(axis=1)


def constant_net(kb: int, q: int):
    """Parameters and normalisation of a network that proposes bucket kb and q for every pair
    (zero weights, biases that put more than 0.999 of each head's softmax mass there): the plain
    fixed-rank method run through the learned pipeline (same probes, fixed-rank group, residual
    sums and Algorithm 1 fallback), so that a comparison isolates what the trained network adds."""
    th = np.zeros(MLP_PARAMS, np.float32)
    b3 = MLP_PARAMS - (MLP_KCLS + MLP_QCLS)
    th[b3 + int(kb)] = 12.0
    th[b3 + MLP_KCLS + int(q)] = 12.0
    return th, np.concatenate([np.zeros(MLP_IN), np.ones(MLP_IN)]).astype(np.float32)


def save(path: str, params, norm):
    """The network file gsvd_rand_mlp_load reads."""
    p = np.asarray(params.cpu().numpy() if hasattr(params, "cpu") else params, np.float32)
    nm = np.asarray(norm.cpu().numpy() if hasattr(norm, "cpu") else norm, np.float32)
    assert p.size == MLP_PARAMS and nm.size == 2 * MLP_IN
    with open(path, "wb") as f:
        f.write(b"GSVDMLP1")
        f.write(struct.pack("<4i", MLP_IN, MLP_HID, MLP_KCLS, MLP_QCLS))
        f.write(nm.astype("<f4").tobytes())
        f.write(p.astype("<f4").tobytes())


def timed_solves(specs, make_ctx, k_cap: int, oversample: int, device: int = 0, plans=None):
    """Per-pair device-synchronised wall time of ctx.solve over FP64 pairs (generation not
    timed), with each solve's residuals and, for learned contexts, its plan.  plans: optional
    (k, q) per pair for a fixed-rank context (k_cap and q = 1 otherwise)."""
    import torch
    rows = []
    with make_ctx() as ctx:
        for i, s in enumerate(specs):
            k, q = plans[i] if plans is not None else (k_cap, 1)
            G1, G2, _, _ = planted_pair_torch(s, device=f"cuda:{device}", dtype=torch.float64)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            try:
                out = ctx.solve(G1, G2, k, oversample, q, s.seed)
                status = "ok"
            except GsvdRandError as e:
                out, status = dict(resid=(np.nan, np.nan), r=0), e.name
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            plan = ctx.last_plan() if getattr(ctx, "_learned", False) else None
            rows.append(dict(seconds=dt, resid=out["resid"], r=out.get("r", 0), status=status, plan=plan))
            del G1, G2
    return rows
