"""Plain FP64 CPU oracle for the randomized GSV method (test infrastructure).

This module is the slow, obviously-correct statement of what the GPU library
computes.  Only the tests, the smoke check and the CPU-baseline leg of the
benchmark may import it; the product path never does.  It shares no code with
the CUDA path: dense linear algebra here is NumPy/LAPACK (Householder QR,
SVD), the CUDA path uses CholeskyQR2 and its own kernels.

Readings of the paper taken here (each also listed in the design notes):
  * The "reduced QR" of the stacked compressed pair (Algorithm 2) is realised
    as a rank-revealing thin SVD truncated to r columns, because the stack
    [Q1^T G1; Q2^T G2] has fewer rows than columns in the fixed-rank setting
    and an unpivoted reduced QR would make the factor orthogonal, so that the
    singular values of L1 would all be one.
  * alpha and beta are both taken as singular values of the two blocks of the
    orthonormal factor and paired by order (the CS decomposition), instead of
    beta = sqrt(1 - alpha^2), which loses relative accuracy as alpha -> 1.
  * The power iterations (q) are subspace iteration with re-orthonormalisation
    after every product, as in Halko, Martinsson & Tropp (2011), Alg. 4.4; the
    paper cites that work for the basis extraction but does not list q.
  * The stopping test of Algorithm 1 is relative: ||(I - QQ^T) G||_F <= tol ||G||_F.
  * Alpha is sorted non-increasing and beta non-decreasing (eq. (ab) of Section 1).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .philox import gaussian

# Philox stream ids (fourth counter word); the same values are fixed in the C header.
STREAM_FIXED = 0          # the n x (k+p) test matrix of the fixed-rank solve
STREAM_ADAPTIVE = 0x10000  # + block index i: Omega_i of Algorithm 1
STREAM_PROBE = 0x20000     # the 64-column probe sketch of the learned proposal


def orth(Y: np.ndarray) -> np.ndarray:
    """Orthonormal basis of range(Y) by Householder reduced QR (LAPACK geqrf/orgqr)."""
    q, _ = np.linalg.qr(Y, mode="reduced")
    return q


def cs_values(Zr: np.ndarray, m: int):
    """GSV pairs from an orthonormal-column matrix Zr = [Z1; Z2] split after row m.

    By the CS decomposition (Golub & Van Loan, Thm 2.5.2; used for the GSVD by
    Paige & Saunders, cited in Section 1), Z1 = U1 C W^T and Z2 = U2 S W^T with
    C^2 + S^2 = I, so alpha = sigma(Z1) and beta = sigma(Z2), paired by sorting
    alpha non-increasing and beta non-decreasing (eq. (ab)).
    """
    r = Zr.shape[1]
    Z1, Z2 = Zr[:m], Zr[m:]
    a = np.linalg.svd(Z1, compute_uv=False) if Z1.size else np.zeros(0)
    b = np.linalg.svd(Z2, compute_uv=False) if Z2.size else np.zeros(0)
    a = np.concatenate([a, np.zeros(r - a.size)])
    b = np.concatenate([b, np.zeros(r - b.size)])
    alpha = np.sort(a)[::-1].copy()
    beta = np.sort(b).copy()
    return alpha, beta


def gsv_from_stack(S: np.ndarray, m: int, r: int):
    """GSVs of the pair whose stack is S = [A1 (m rows); A2], truncated to rank r.

    Thin SVD S = Z Sigma W^T (LAPACK gesdd), keep the leading r left singular
    vectors, then the CS split (Section 1 definition, eq. (gsvd1); Algorithm 2
    with the rank-revealing reading of its reduced QR).
    """
    Z, s, _ = np.linalg.svd(S, full_matrices=False)
    r = min(r, Z.shape[1])
    return cs_values(Z[:, :r], m) + (s,)


def direct_gsvd(G1: np.ndarray, G2: np.ndarray, r: int | None = None):
    """Direct dense GSVD of {G1 (m x n), G2 (p x n)}: the plain definition.

    With r = n and a Grassman matrix pair (rank [G1; G2] = n) this is the
    reduced GSVD of eq. (gsvd1); for a numerically rank-r pair it returns the r
    GSV pairs of the rank-r truncation of the stack.  Returns (alpha, beta).
    """
    G1 = np.asarray(G1, dtype=np.float64)
    G2 = np.asarray(G2, dtype=np.float64)
    n = G1.shape[1]
    r = n if r is None else r
    alpha, beta, _ = gsv_from_stack(np.vstack([G1, G2]), G1.shape[0], r)
    return alpha, beta


def pencil_gsvd(G1: np.ndarray, G2: np.ndarray):
    """Brute force for tiny full-rank pairs: alpha^2 are the eigenvalues of the
    symmetric-definite pencil (G1^T G1, G1^T G1 + G2^T G2); beta^2 those of
    (G2^T G2, same).  Independent of the SVD/CS route (Van Loan 1976, cited [23])."""
    A1 = G1.T @ G1
    A2 = G2.T @ G2
    Bm = A1 + A2
    a2 = sla.eigh(A1, Bm, eigvals_only=True)
    b2 = sla.eigh(A2, Bm, eigvals_only=True)
    alpha = np.sqrt(np.clip(a2, 0.0, None))[::-1].copy()
    beta = np.sqrt(np.clip(b2, 0.0, None))
    return alpha, beta


def round_bf16(x) -> np.ndarray:
    """Each entry rounded to the nearest FP32, then to the nearest bfloat16 (8-bit
    significand), ties to even both times; returned as float32.

    bfloat16 keeps the upper 16 bits of an IEEE binary32 word.  Round half to even on
    the 16 dropped bits: add 0x7FFF plus the lowest kept bit, then clear the dropped
    bits (a carry into the exponent is the correct round-up across a binade).
    """
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float64).astype(np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def basis_fixed(G: np.ndarray, l: int, q: int, seed: int, pair: int = 0, side: int = 0,
                omega_round: str | None = None):
    """Fixed-rank randomized range finder with q power iterations.

    Y = G Omega (Omega n x l Gaussian, Theorem 3 with l = k + p), Q = orth(Y);
    then q times: Z = orth(G^T Q), Q = orth(G Z)  (subspace iteration,
    Halko-Martinsson-Tropp 2011 Alg. 4.4).  Returns Q (M x l).
    omega_round="bf16" draws the same Omega rounded to bfloat16 (round_bf16), the test
    matrix of the BF16 mode: still Gaussian up to a 2^-8 relative perturbation.
    """
    n = G.shape[1]
    Om = gaussian(n, l, seed, pair, side, STREAM_FIXED)
    if omega_round == "bf16":
        Om = round_bf16(Om).astype(np.float64)
    elif omega_round is not None:
        raise ValueError(f"unknown omega_round {omega_round!r}")
    Q = orth(G @ Om)
    for _ in range(q):
        Z = orth(G.T @ Q)
        Q = orth(G @ Z)
    return Q


def rand_gsvd(G1, G2, k: int, oversample: int, q: int, seed: int, pair: int = 0,
              omega_round: str | None = None):
    """Algorithm 2 with the fixed-rank basis extraction: the method as the GPU runs it.

    For each side s: Q_s = basis_fixed(G_s), B_s = Q_s^T G_s; then the GSVs of
    the compressed pair from the stack [B1; B2] truncated to r = k.
    Returns a dict with alpha, beta (k each), the relative residuals
    ||G_s - Q_s B_s||_F / ||G_s||_F, and the intermediate Q_s, B_s.
    """
    G1 = np.asarray(G1, dtype=np.float64)
    G2 = np.asarray(G2, dtype=np.float64)
    l = k + oversample
    out = {}
    Bs = []
    for s, G in enumerate((G1, G2)):
        Q = basis_fixed(G, l, q, seed, pair, s, omega_round)
        B = Q.T @ G
        out[f"Q{s + 1}"] = Q
        out[f"B{s + 1}"] = B
        out[f"resid{s + 1}"] = np.linalg.norm(G - Q @ B) / max(np.linalg.norm(G), 1e-300)
        Bs.append(B)
    alpha, beta, svals = gsv_from_stack(np.vstack(Bs), Bs[0].shape[0], k)
    out.update(alpha=alpha, beta=beta, stack_svals=svals)
    return out


def rand_gsvd_factors(G1, G2, k: int, oversample: int, q: int, seed: int, pair: int = 0,
                      omega_round: str | None = None):
    """The GSVD factors of the randomized method (the recovery that follows Algorithm 2 in
    Section 2, in the rank-revealing reading): with S = [B1; B2] = Zr Sigma_r Wr^T (thin SVD
    truncated to r = k) and the SVD Z1 = U1 C Vh of its first block, U = Q1 U1, R = Vh Zr^T S
    and V = Q2 Z2 Vh^T diag(1 / beta), so that G1 ~ U diag(alpha) R and G2 ~ V diag(beta) R
    (G_s ~ Q_s B_s).  A column whose alpha (beta) is zero is left zero in U (V).  Columns and
    rows are ordered by alpha non-increasing.  omega_round as in basis_fixed.
    Returns dict(U, V, R, alpha, beta)."""
    out = rand_gsvd(G1, G2, k, oversample, q, seed, pair, omega_round)
    Q1, Q2, B1, B2 = out["Q1"], out["Q2"], out["B1"], out["B2"]
    S = np.vstack([B1, B2])
    l1 = B1.shape[0]
    Z, _, _ = np.linalg.svd(S, full_matrices=False)
    Zr = Z[:, :k]
    _, _, Vh = np.linalg.svd(Zr[:l1], full_matrices=False)
    ZW = Zr @ Vh.T                  # [Z1; Z2] W: column norms alpha_i, beta_i
    a = np.linalg.norm(ZW[:l1], axis=0)
    b = np.linalg.norm(ZW[l1:], axis=0)
    order = np.argsort(-a, kind="stable")
    ZW, a, b = ZW[:, order], a[order], b[order]
    U = Q1 @ (ZW[:l1] / np.where(a > 0, a, np.inf))
    V = Q2 @ (ZW[l1:] / np.where(b > 0, b, np.inf))
    R = ZW.T @ S
    return dict(U=U, V=V, R=R, alpha=a, beta=b)


def adaptive_basis(G, tol: float, b: int, seed: int, pair: int = 0, side: int = 0,
                   max_cols: int | None = None):
    """Algorithm 1 (BasisExt), blocked adaptive range finder.

    Loop over blocks i: draw Omega_i (n x b); Y_i = (I - Q Q^T)(G Omega_i),
    projected twice (the second projection is re-orthogonalisation, on which
    the paper is silent); P_i = orth(Y_i), then once more
    P_i = orth((I - Q Q^T) P_i) so that Q stays orthonormal when Y_i is
    numerically rank-deficient (its extra columns are then directions
    orthogonal to Q and to range(G), which add zero rows to Q^T G and leave
    the GSVs unchanged); Q = [Q, P_i]; stop when the
    cumulated residual sqrt(||G||_F^2 - sum_i ||P_i^T G||_F^2) (Section 2, the
    cumulated form of ||(I - QQ^T) G||_F) is <= tol * ||G||_F or Q has
    min(M, n) columns.  Returns (Q, list of relative residual estimates).
    """
    G = np.asarray(G, dtype=np.float64)
    M, n = G.shape
    cap = min(M, n) if max_cols is None else min(max_cols, M, n)
    g2 = float(np.sum(G * G))
    acc = 0.0
    Q = np.zeros((M, 0))
    hist = []
    i = 0
    while Q.shape[1] < cap:
        bi = min(b, cap - Q.shape[1])
        Om = gaussian(n, bi, seed, pair, side, STREAM_ADAPTIVE + i)
        Y = G @ Om
        for _ in range(2):
            Y = Y - Q @ (Q.T @ Y)
        P = orth(Y)
        P = orth(P - Q @ (Q.T @ P))
        Q = np.hstack([Q, P])
        acc += float(np.sum((P.T @ G) ** 2))
        est = np.sqrt(max(g2 - acc, 0.0)) / np.sqrt(g2) if g2 > 0 else 0.0
        hist.append(est)
        i += 1
        if est <= tol:
            break
    return Q, hist


def rand_gsvd_adaptive(G1, G2, tol: float, b: int, seed: int, r: int, pair: int = 0,
                       max_cols: int | None = None):
    """Algorithm 2 on the bases of Algorithm 1 (adaptive range finder per side).

    Q_s = adaptive_basis(G_s, tol, b) (blocks of b columns until the cumulated
    relative residual is <= tol or the column cap is reached), B_s = Q_s^T G_s,
    then the GSVs of the stack [B1; B2] truncated to min(r, l1 + l2).  Returns a
    dict with alpha, beta, the column counts l1, l2 and the residual estimate
    histories of both sides.
    """
    out = {"hist": []}
    Bs, ls = [], []
    for s, G in enumerate((G1, G2)):
        G = np.asarray(G, dtype=np.float64)
        Q, hist = adaptive_basis(G, tol, b, seed, pair, s, max_cols)
        Bs.append(Q.T @ G)
        ls.append(Q.shape[1])
        out["hist"].append(hist)
    S = np.vstack(Bs)
    rr = min(r, S.shape[0])
    alpha, beta, _ = gsv_from_stack(S, ls[0], rr)
    out.update(alpha=alpha, beta=beta, l1=ls[0], l2=ls[1])
    return out


def metrics(alpha, beta, pad_to_n: int = 0, pad_mode: int = 0):
    """Comparative quantities of Section 1 from GSV pairs.

    theta_l = arctan(alpha_l / beta_l) - pi/4, taken as atan2(alpha, beta) - pi/4
      so that beta = 0 gives +pi/4 (antisymmetric angular distance);
    rho_l = alpha_l / beta_l (+inf when beta_l = 0) (relative significance);
    P_{1,l} = alpha_l^2 / sum alpha^2, P_{2,l} = beta_l^2 / sum beta^2
      (generalized fractions of eigenexpression);
    D_i = -(1 / log N) sum_l P_{i,l} log P_{i,l}, with 0 log 0 = 0
      (generalized normalized Shannon entropy), N = number of pairs.
    pad_to_n > 0 pads to that many pairs as Algorithm 2 does: pad_mode 0 appends
    (alpha, beta) = (0, 1) (the l1 <= l2 branch), pad_mode 1 prepends (1, 0).
    """
    a = np.asarray(alpha, dtype=np.float64)
    b = np.asarray(beta, dtype=np.float64)
    if pad_to_n and pad_to_n > a.size:
        extra = pad_to_n - a.size
        if pad_mode == 0:
            a = np.concatenate([a, np.zeros(extra)])
            b = np.concatenate([b, np.ones(extra)])
        else:
            a = np.concatenate([np.ones(extra), a])
            b = np.concatenate([np.zeros(extra), b])
    N = a.size
    theta = np.arctan2(a, b) - np.pi / 4
    with np.errstate(divide="ignore"):
        rho = np.where(b == 0, np.inf, a / np.where(b == 0, 1.0, b))
    out = dict(theta=theta, rho=rho)
    for name, x in (("1", a), ("2", b)):
        x2 = x * x
        tot = x2.sum()
        P = x2 / tot if tot > 0 else np.zeros_like(x2)
        with np.errstate(divide="ignore", invalid="ignore"):
            terms = np.where(P > 0, P * np.log(np.where(P > 0, P, 1.0)), 0.0)
        D = -terms.sum() / np.log(N) if N > 1 else np.nan
        out["P" + name] = P
        out["D" + name] = D
    return out


def gsv_error(alpha_ref, beta_ref, alpha, beta):
    """Per-pair GSV error e_i = max(|alpha_i - alpha_ref_i|, |beta_i - beta_ref_i|):
    the error of the unit-norm pair, the paper's accuracy measure (Table 1,
    Corollary "error-bounds")."""
    return np.maximum(np.abs(np.asarray(alpha) - alpha_ref), np.abs(np.asarray(beta) - beta_ref))


def perturbation_E(G1, G2, G1t, G2t):
    """E = sqrt(2) ||Delta G||_F min(||G^+||_2, ||G~^+||_2) of Section 3 (the
    bound of Lemma "per" and Theorem "exp"), G = [G1; G2]."""
    G = np.vstack([G1, G2])
    Gt = np.vstack([G1t, G2t])
    dG = np.linalg.norm(Gt - G)
    inv = min(1.0 / np.linalg.svd(G, compute_uv=False)[-1],
              1.0 / np.linalg.svd(Gt, compute_uv=False)[-1])
    return np.sqrt(2.0) * dG * inv


def alg2_literal(B1: np.ndarray, B2: np.ndarray):
    """Algorithm 2 steps after the basis extraction, literally, for the case the
    paper assumes: the compressed stack [B1; B2] ((l1 + l2) x n) has full column
    rank n.  Reduced QR [B1; B2] = [L1; L2] R~; singular values of the smaller
    block; zero padding to n; the other GSV from sqrt(1 - x^2).
    Returns (alpha, beta) of length n.  Used to pin the rank-revealing reading:
    on full-rank stacks it must agree with `gsv_from_stack(..., r=n)`."""
    l1, n = B1.shape
    l2 = B2.shape[0]
    Lq, _ = np.linalg.qr(np.vstack([B1, B2]), mode="reduced")
    L1, L2 = Lq[:l1], Lq[l1:]
    if l1 <= l2:
        a = np.sort(np.linalg.svd(L1, compute_uv=False))[::-1]
        alpha = np.concatenate([a, np.zeros(n - a.size)])
        beta = np.sqrt(np.clip(1.0 - alpha ** 2, 0.0, None))
    else:
        b = np.sort(np.linalg.svd(L2, compute_uv=False))
        beta = np.concatenate([np.zeros(n - b.size), b])
        alpha = np.sqrt(np.clip(1.0 - beta ** 2, 0.0, None))
    return alpha, beta


# ----------------------------------------------------------------------------------------------
# Complex pairs.  Section 1 states the GSVD over C (eq. (gsvd1): G1 = U Sigma1 R, G2 = V Sigma2 R
# with unitary U, V) and the synthetic experiments of Section 4.1 are complex; the randomized
# method is the same with conjugate transposes and a complex Gaussian test matrix.
# ----------------------------------------------------------------------------------------------
def gaussian_complex(n: int, l: int, seed: int, pair: int = 0, side: int = 0, stream: int = STREAM_FIXED):
    """Complex Gaussian test matrix (n x l): Omega[j, c] = g[j, 2c] + i g[j, 2c + 1], g the real
    Philox/Box-Muller stream of an n x 2l matrix, so that the real and imaginary parts of each
    entry are the two normals of one Box-Muller pair (independent, circularly symmetric)."""
    g = gaussian(n, 2 * l, seed, pair, side, stream)
    return g[:, 0::2] + 1j * g[:, 1::2]


def basis_fixed_complex(G, l: int, q: int, seed: int, pair: int = 0, side: int = 0):
    """The fixed-rank range finder over C: Y = G Omega, Q = orth(Y); q times Z = orth(G^H Q),
    Q = orth(G Z) (complex Householder QR)."""
    n = G.shape[1]
    Q = orth(G @ gaussian_complex(n, l, seed, pair, side, STREAM_FIXED))
    for _ in range(q):
        Z = orth(G.conj().T @ Q)
        Q = orth(G @ Z)
    return Q


def rand_gsvd_complex(G1, G2, k: int, oversample: int, q: int, seed: int, pair: int = 0):
    """Algorithm 2 over C with the fixed-rank bases: B_s = Q_s^H G_s, then the GSVs of the
    stack [B1; B2] truncated to r = k (thin SVD and CS split, as gsv_from_stack; the singular
    values of complex blocks are real).  Returns alpha, beta (k each), the relative residuals
    ||G_s - Q_s B_s||_F / ||G_s||_F, Q_s and B_s."""
    G1 = np.asarray(G1, dtype=np.complex128)
    G2 = np.asarray(G2, dtype=np.complex128)
    l = k + oversample
    out, Bs = {}, []
    for s, G in enumerate((G1, G2)):
        Q = basis_fixed_complex(G, l, q, seed, pair, s)
        B = Q.conj().T @ G
        out[f"Q{s + 1}"] = Q
        out[f"B{s + 1}"] = B
        out[f"resid{s + 1}"] = np.linalg.norm(G - Q @ B) / max(np.linalg.norm(G), 1e-300)
        Bs.append(B)
    alpha, beta, svals = gsv_from_stack(np.vstack(Bs), Bs[0].shape[0], k)
    out.update(alpha=alpha, beta=beta, stack_svals=svals)
    return out


def direct_gsvd_complex(G1, G2, r: int | None = None):
    """The direct dense GSVD of a complex pair (thin SVD of the stack, CS split)."""
    G1 = np.asarray(G1, dtype=np.complex128)
    G2 = np.asarray(G2, dtype=np.complex128)
    r = G1.shape[1] if r is None else r
    alpha, beta, _ = gsv_from_stack(np.vstack([G1, G2]), G1.shape[0], r)
    return alpha, beta


def pencil_gsvd_complex(G1, G2):
    """Brute force for tiny full-rank complex pairs: alpha^2 are the eigenvalues of the
    Hermitian-definite pencil (G1^H G1, G1^H G1 + G2^H G2), beta^2 those of (G2^H G2, same)."""
    A1 = G1.conj().T @ G1
    A2 = G2.conj().T @ G2
    Bm = A1 + A2
    a2 = sla.eigh(A1, Bm, eigvals_only=True)
    b2 = sla.eigh(A2, Bm, eigvals_only=True)
    return np.sqrt(np.clip(a2, 0.0, None))[::-1].copy(), np.sqrt(np.clip(b2, 0.0, None))


def realify(G) -> np.ndarray:
    """The real 2m x 2n matrix of a complex m x n one, each entry a + ib as the 2 x 2 block
    [[a, -b], [b, a]]: the representation of C as real 2 x 2 matrices, a ring homomorphism
    (products and conjugate transposes carry over), so every singular value of G appears twice
    in it and every GSV of a complex pair twice in the real pair."""
    G = np.asarray(G, dtype=np.complex128)
    m, n = G.shape
    R = np.empty((2 * m, 2 * n))
    R[0::2, 0::2] = G.real
    R[0::2, 1::2] = -G.imag
    R[1::2, 0::2] = G.imag
    R[1::2, 1::2] = G.real
    return R
