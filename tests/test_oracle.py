"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test targets a mistake a plausible implementation could make (a dropped
term, a wrong sign or index, a transposed operand, a swapped sin/cos, a wrong
sort order); none re-types the oracle's own formula.
"""
import os

import numpy as np
import pytest
from scipy import stats

from oracle import gsvd as O
from oracle.philox import gaussian, philox4x32_10, philox_words
from paper_2404_09459_gb300.inputs import PairSpec, full_gmp_pair, planted_pair, planted_scale

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rng(seed):
    return np.random.default_rng(seed)


def _full_rank_pair(rng, m, p, n, alpha=None, cond=10.0):
    """G1 = U diag(alpha) R, G2 = V diag(beta) R with a nonsingular R (n x n)."""
    if alpha is None:
        alpha = np.sort(rng.uniform(0.02, 0.98, n))[::-1]
    beta = np.sqrt(1.0 - alpha ** 2)
    U, _ = np.linalg.qr(rng.standard_normal((m, n)))
    V, _ = np.linalg.qr(rng.standard_normal((p, n)))
    A, _ = np.linalg.qr(rng.standard_normal((n, n)))
    Bq, _ = np.linalg.qr(rng.standard_normal((n, n)))
    R = A @ np.diag(np.logspace(0, np.log10(cond), n)) @ Bq
    return U @ np.diag(alpha) @ R, V @ np.diag(beta) @ R, alpha, beta


# ---------------------------------------------------------------- Philox / Omega

def test_philox_known_answers():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for row in rows:
        v = [int(x, 16) for x in row]
        out = philox4x32_10(*v[0:4], *v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_philox_counter_fields_are_independent():
    # Changing any counter word or the key changes the words (no aliasing of fields).
    base = [int(x[0]) for x in philox_words(1, seed=7, pair=3, side=1, stream=5)]
    for kw in (dict(seed=8, pair=3, side=1, stream=5), dict(seed=7, pair=4, side=1, stream=5),
               dict(seed=7, pair=3, side=0, stream=5), dict(seed=7, pair=3, side=1, stream=6),
               dict(seed=7 + (1 << 32), pair=3, side=1, stream=5)):
        assert [int(x[0]) for x in philox_words(1, **kw)] != base


def test_gaussian_is_standard_normal():
    z = gaussian(400, 250, seed=3).ravel()
    assert abs(z.mean()) < 0.01
    assert abs(z.var() - 1.0) < 0.01
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # the two outputs of one Box-Muller step are uncorrelated
    assert abs(np.corrcoef(z[0::2], z[1::2])[0, 1]) < 0.01


def test_gaussian_box_muller_geometry():
    # Each (z0, z1) pair is (r cos t, r sin t) with r^2 = -2 ln u1 and t = 2 pi u2,
    # u1, u2 in (0, 1): the radius must exceed 0 and the angle must be uniform.
    z = gaussian(1000, 2, seed=11)
    r2 = z[:, 0] ** 2 + z[:, 1] ** 2
    # r^2 of a 2-D standard normal is chi^2 with 2 dof = Exp(mean 2)
    assert stats.kstest(r2, "expon", args=(0, 2.0)).pvalue > 1e-3
    ang = np.mod(np.arctan2(z[:, 1], z[:, 0]), 2 * np.pi) / (2 * np.pi)
    assert stats.kstest(ang, "uniform").pvalue > 1e-3
    # slot 0 is the cosine branch: the angle from the first word pair of counter 0
    w = philox_words(1, seed=11)
    u2 = ((int(w[2][0]) >> 5) * 2.0 ** 26 + (int(w[3][0]) >> 6)) * 2.0 ** -53
    t = np.mod(np.arctan2(z[0, 1], z[0, 0]), 2 * np.pi)
    assert abs(t - 2 * np.pi * u2) < 1e-12


def test_gaussian_flat_index_order():
    # The stream depends only on the row-major flat index: (3 x 5) and (5 x 3) share values.
    a = gaussian(3, 5, seed=1).ravel()
    b = gaussian(5, 3, seed=1).ravel()
    np.testing.assert_array_equal(a, b)
    c = gaussian(4, 7, seed=1).ravel()  # odd total, last slot-0 only
    np.testing.assert_array_equal(c[:15], a)


# ---------------------------------------------------------------- direct GSVD

def test_direct_recovers_planted_full_rank():
    rng = _rng(0)
    G1, G2, a, b = _full_rank_pair(rng, 40, 30, 12, cond=100.0)
    al, be = O.direct_gsvd(G1, G2)
    np.testing.assert_allclose(al, a, atol=1e-12)
    np.testing.assert_allclose(be, b, atol=1e-12)


@pytest.mark.parametrize("seed", range(5))
def test_direct_matches_pencil_brute_force(seed):
    rng = _rng(100 + seed)
    n = int(rng.integers(2, 9))
    G1 = rng.standard_normal((int(rng.integers(n, 12)), n))
    G2 = rng.standard_normal((int(rng.integers(n, 12)), n))
    al, be = O.direct_gsvd(G1, G2)
    ap, bp = O.pencil_gsvd(G1, G2)
    np.testing.assert_allclose(al, ap, atol=1e-10)
    np.testing.assert_allclose(be, bp, atol=1e-10)


def test_direct_n1_closed_form():
    rng = _rng(5)
    g1 = rng.standard_normal((7, 1))
    g2 = rng.standard_normal((4, 1))
    al, be = O.direct_gsvd(g1, g2)
    den = np.sqrt(np.sum(g1 ** 2) + np.sum(g2 ** 2))
    assert abs(al[0] - np.linalg.norm(g1) / den) < 1e-15
    assert abs(be[0] - np.linalg.norm(g2) / den) < 1e-15


def test_direct_swap_and_invariances():
    rng = _rng(6)
    G1 = rng.standard_normal((15, 6))
    G2 = rng.standard_normal((11, 6))
    al, be = O.direct_gsvd(G1, G2)
    # swapping the pair swaps the roles and reverses the order
    a2, b2 = O.direct_gsvd(G2, G1)
    np.testing.assert_allclose(a2, be[::-1], atol=1e-13)
    np.testing.assert_allclose(b2, al[::-1], atol=1e-13)
    # orthogonal transform of the rows of one matrix
    H, _ = np.linalg.qr(rng.standard_normal((15, 15)))
    a3, b3 = O.direct_gsvd(H @ G1, G2)
    np.testing.assert_allclose(a3, al, atol=1e-13)
    # right multiplication by a nonsingular matrix (full-rank pair)
    X = rng.standard_normal((6, 6)) + 3 * np.eye(6)
    a4, b4 = O.direct_gsvd(G1 @ X, G2 @ X)
    np.testing.assert_allclose(a4, al, atol=1e-11)
    np.testing.assert_allclose(b4, be, atol=1e-11)


def test_direct_unit_norm_and_order():
    rng = _rng(7)
    for _ in range(5):
        G1 = rng.standard_normal((20, 9))
        G2 = rng.standard_normal((13, 9))
        al, be = O.direct_gsvd(G1, G2)
        np.testing.assert_allclose(al ** 2 + be ** 2, 1.0, atol=1e-13)
        assert np.all(np.diff(al) <= 1e-15) and np.all(np.diff(be) >= -1e-15)
        assert np.all((al >= 0) & (al <= 1 + 1e-15) & (be >= 0) & (be <= 1 + 1e-15))


def test_direct_exact_ones_and_zeros():
    # eq. (ab): directions only in G1 give alpha = 1, beta = 0; only in G2 give (0, 1)
    rng = _rng(8)
    n = 6
    R = rng.standard_normal((n, n)) + 4 * np.eye(n)
    U, _ = np.linalg.qr(rng.standard_normal((10, n)))
    V, _ = np.linalg.qr(rng.standard_normal((9, n)))
    a = np.array([1.0, 1.0, 0.8, 0.3, 0.0, 0.0])
    b = np.sqrt(1 - a ** 2)
    al, be = O.direct_gsvd(U @ np.diag(a) @ R, V @ np.diag(b) @ R)
    np.testing.assert_allclose(al, a, atol=1e-12)
    np.testing.assert_allclose(be, b, atol=1e-12)


def test_paper_full_pair_workload_recovers_planted():
    # Section 4.1's synthetic pair (real-valued): rank(G1) = rank(G2) = 60% of n, so 40% of the
    # pairs are (1, 0), 40% are (0, 1) and the rest uniform; the stack has full rank and all n
    # pairs are resolved (r = n).  The direct GSVD and the randomized method with a full basis
    # per side (k = n, no oversampling: each side's sketch has exact rank 0.6 n < l) both give
    # the planted values.
    G1, G2, a, b = full_gmp_pair(120, 90, 40, seed=3)
    assert np.linalg.matrix_rank(G1) == 24 and np.linalg.matrix_rank(G2) == 24
    assert np.sum(a == 1.0) == 16 and np.sum(a == 0.0) == 16
    al, be = O.direct_gsvd(G1, G2, r=40)
    np.testing.assert_allclose(al, a, atol=1e-12)
    np.testing.assert_allclose(be, b, atol=1e-12)
    for q in (0, 1):
        out = O.rand_gsvd(G1, G2, 40, 0, q, seed=7)
        assert np.max(O.gsv_error(a, b, out["alpha"], out["beta"])) < 1e-12
        assert out["resid1"] < 1e-13 and out["resid2"] < 1e-13


def test_gsvd_factors_reconstruct_and_match_the_planted_R():
    # the recovery after Algorithm 2 (Section 2): G1 = U diag(alpha) R, G2 = V diag(beta) R with
    # orthonormal U, V.  On a planted noise-free pair G1 = U_r diag(alpha) D O_r the shared factor
    # is R = D O_r up to row signs (the GSVs are distinct), so R R^T = D^2 with the planted scales
    spec = PairSpec(m=200, p=150, n=60, r=10, alpha="uniform", decay="exp10", sigma=0.0, k=10,
                    oversample=5, q=1, seed=4)
    G1, G2, a, b = planted_pair(spec)
    f = O.rand_gsvd_factors(G1, G2, 10, 5, 1, seed=3)
    np.testing.assert_allclose(f["alpha"], a, atol=1e-12)
    np.testing.assert_allclose(f["beta"], b, atol=1e-12)
    assert np.linalg.norm(G1 - (f["U"] * f["alpha"]) @ f["R"]) <= 1e-12 * np.linalg.norm(G1)
    assert np.linalg.norm(G2 - (f["V"] * f["beta"]) @ f["R"]) <= 1e-12 * np.linalg.norm(G2)
    np.testing.assert_allclose(f["U"].T @ f["U"], np.eye(10), atol=1e-12)
    np.testing.assert_allclose(f["V"].T @ f["V"], np.eye(10), atol=1e-12)
    d = planted_scale(spec)
    np.testing.assert_allclose(f["R"] @ f["R"].T, np.diag(d ** 2), atol=1e-12)


def test_alg2_literal_matches_rank_revealing_reading():
    # When the compressed stack has full column rank (the paper's setting) the
    # literal Algorithm 2 (reduced QR, SVD of the smaller block, sqrt(1 - x^2))
    # and the rank-revealing reading give the same GSVs, for both branches.
    rng = _rng(9)
    for (l1, l2) in ((5, 9), (9, 5)):
        n = 7
        B1 = rng.standard_normal((l1, n))
        B2 = rng.standard_normal((l2, n))
        a_lit, b_lit = O.alg2_literal(B1, B2)
        a_rr, b_rr = O.direct_gsvd(B1, B2, r=n)
        np.testing.assert_allclose(a_lit, a_rr, atol=1e-12)
        np.testing.assert_allclose(b_lit, b_rr, atol=1e-12)


# ---------------------------------------------------------------- randomized (Algorithm 2)

def test_randomized_exact_on_exact_rank_pair():
    # eq. (gsvd-reduced): when Q1, Q2 span the column spaces exactly, the
    # compressed pair has the same GSVs.  Noise-free rank-r pair, l >= r.
    spec = PairSpec(m=300, p=250, n=80, r=12, alpha="uniform", decay="exp10", sigma=0.0,
                    k=12, oversample=6, q=0, seed=3)
    G1, G2, a, b = planted_pair(spec)
    for q in (0, 1, 2):
        out = O.rand_gsvd(G1, G2, 12, 6, q, seed=1)
        np.testing.assert_allclose(out["alpha"], a, atol=1e-12)
        np.testing.assert_allclose(out["beta"], b, atol=1e-12)
        assert out["resid1"] < 1e-13 and out["resid2"] < 1e-13
    al, be = O.direct_gsvd(G1, G2, r=12)
    np.testing.assert_allclose(al, a, atol=1e-12)


def test_randomized_on_small_planted_workload():
    # the small FP64 workload shape, scaled down: within the noise of the truth
    spec = PairSpec(m=400, p=400, n=60, r=10, alpha="linspace", decay="logspace02", sigma=1e-8,
                    k=10, oversample=10, q=1, seed=0)
    G1, G2, a, b = planted_pair(spec)
    out = O.rand_gsvd(G1, G2, 10, 10, 1, seed=0)
    assert np.max(O.gsv_error(a, b, out["alpha"], out["beta"])) < 1e-6
    al, be = O.direct_gsvd(G1, G2, r=10)
    assert np.max(O.gsv_error(al, be, out["alpha"], out["beta"])) < 1e-10


def test_theorem3_expected_residual_bound():
    # Theorem 3: E ||(I - Q1 Q1^T) G1||_F^2 <= eta (k/(p-1) + 1) sum_{j>k} alpha_j^2,
    # eta = sigma_max(G1^T G1 + G2^T G2); q = 0, Omega Gaussian with k + p columns.
    rng = _rng(10)
    n, k, p = 30, 6, 4
    alpha = np.sort(np.concatenate([rng.uniform(0.6, 0.95, k), rng.uniform(0.0, 0.15, n - k)]))[::-1]
    G1, G2, a, b = _full_rank_pair(rng, 60, 50, n, alpha=alpha, cond=3.0)
    eta = np.linalg.eigvalsh(G1.T @ G1 + G2.T @ G2)[-1]
    bound = eta * (k / (p - 1) + 1) * np.sum(alpha[k:] ** 2)
    res = []
    for s in range(200):
        Q = O.basis_fixed(G1, k + p, 0, seed=s)
        res.append(np.linalg.norm(G1 - Q @ (Q.T @ G1)) ** 2)
    assert np.mean(res) <= bound
    # and the bound is not vacuous: the residual is far below ||G1||_F^2
    assert np.mean(res) < 0.5 * np.linalg.norm(G1) ** 2


def test_residual_falls_with_rank_fig2():
    # Fig. 2: the GSV error falls as the basis residual falls (here: as k grows).
    spec = PairSpec(m=300, p=300, n=100, r=40, alpha="uniform", decay="exp10", sigma=1e-7,
                    k=0, oversample=4, q=0, seed=4)
    G1, G2, a, b = planted_pair(spec)
    errs, res = [], []
    for k in (10, 20, 30, 40):
        out = O.rand_gsvd(G1, G2, k, 4, 0, seed=2)
        errs.append(np.max(O.gsv_error(a[:k], b[:k], out["alpha"], out["beta"])))
        res.append(out["resid1"] + out["resid2"])
    assert all(res[i + 1] < res[i] for i in range(3))
    assert errs[-1] < errs[0]


# ---------------------------------------------------------------- Algorithm 1 (adaptive)

def test_adaptive_equals_one_shot_qr_lemma_c2():
    # Lemma c2: the blocked basis equals the reduced QR of G [Omega_1 ... Omega_j]
    # up to column signs (full column rank sketch).
    rng = _rng(11)
    G = rng.standard_normal((50, 24))
    Q, hist = O.adaptive_basis(G, tol=1e-14, b=5, seed=4, max_cols=15)
    assert Q.shape[1] == 15
    Om = np.hstack([gaussian(24, 5, 4, 0, 0, O.STREAM_ADAPTIVE + i) for i in range(3)])
    Qs, _ = np.linalg.qr(G @ Om)
    signs = np.sign(np.sum(Q * Qs, axis=0))
    np.testing.assert_allclose(Q, Qs * signs[None, :], atol=1e-11)


def test_adaptive_cumulated_residual_and_stop():
    spec = PairSpec(m=200, p=200, n=90, r=17, sigma=0.0, seed=5)
    G1, _, _, _ = planted_pair(spec)
    Q, hist = O.adaptive_basis(G1, tol=1e-9, b=4, seed=1)
    # stops once the rank is covered: ceil(17/4) = 5 blocks
    assert Q.shape[1] == 20 and len(hist) == 5
    assert hist[-1] <= 1e-9 and all(h > 1e-9 for h in hist[:-1])
    # the cumulated estimate equals the plain residual ||(I - QQ^T)G||_F / ||G||_F
    for j, h in enumerate(hist[:-1]):
        Qj = Q[:, : 4 * (j + 1)]
        direct = np.linalg.norm(G1 - Qj @ (Qj.T @ G1)) / np.linalg.norm(G1)
        assert abs(direct - h) < 1e-7
    np.testing.assert_allclose(Q.T @ Q, np.eye(20), atol=1e-12)


def test_adaptive_full_when_tolerance_unreachable():
    # Lemma c2, second part: with l = n the basis reproduces G exactly.
    rng = _rng(12)
    G = rng.standard_normal((30, 12))
    Q, hist = O.adaptive_basis(G, tol=0.0, b=5, seed=2)
    assert Q.shape[1] == 12
    assert np.linalg.norm(G - Q @ (Q.T @ G)) < 1e-12 * np.linalg.norm(G)


def test_adaptive_gsvd_recovers_planted_pairs():
    # Algorithm 1 + Algorithm 2 on a noise-free pair of exact rank 13: the bases
    # cover the rank (ceil(13 / 5) = 3 blocks per side) and the GSVs are the
    # planted ones (Section 2: exact when the basis captures range(G_s)).
    spec = PairSpec(m=160, p=120, n=70, r=13, alpha="uniform", decay="exp10", sigma=0.0, seed=21)
    G1, G2, at, bt = planted_pair(spec)
    # the cumulated residual sqrt(||G||^2 - sum ||P_i^T G||^2) cannot resolve less than about
    # sqrt(u) ||G|| (cancellation), so the tolerance sits above 1e-8
    out = O.rand_gsvd_adaptive(G1, G2, tol=1e-6, b=5, seed=3, r=13)
    assert out["l1"] == 15 and out["l2"] == 15
    assert all(h[-1] <= 1e-6 for h in out["hist"]) and all(h[-2] > 1e-2 for h in out["hist"])
    assert np.max(O.gsv_error(at, bt, out["alpha"], out["beta"])) < 1e-11


# ---------------------------------------------------------------- metrics (Section 1)

def test_metrics_equal_significance():
    a = np.full(8, 1 / np.sqrt(2))
    m = O.metrics(a, a.copy())
    np.testing.assert_allclose(m["theta"], 0.0, atol=1e-15)
    np.testing.assert_allclose(m["P1"], 1 / 8, atol=1e-15)
    assert abs(m["D1"] - 1.0) < 1e-14 and abs(m["D2"] - 1.0) < 1e-14
    np.testing.assert_allclose(m["rho"], 1.0, atol=1e-15)


def test_metrics_single_genelet():
    a = np.array([1.0, 0.0, 0.0, 0.0])
    b = np.array([0.0, 1.0, 1.0, 1.0])
    m = O.metrics(a, b)
    assert m["D1"] == 0.0  # all expression captured by one genelet
    assert abs(m["D2"] - np.log(3) / np.log(4)) < 1e-15
    assert m["theta"][0] == pytest.approx(np.pi / 4) and m["rho"][0] == np.inf
    assert m["theta"][1] == pytest.approx(-np.pi / 4)


def test_metrics_ranges_and_swap():
    rng = _rng(13)
    al, be = O.direct_gsvd(rng.standard_normal((20, 9)), rng.standard_normal((14, 9)))
    m = O.metrics(al, be)
    assert np.all(np.diff(m["theta"]) <= 1e-15)
    assert np.all(np.abs(m["theta"]) <= np.pi / 4 + 1e-15)
    assert abs(m["P1"].sum() - 1) < 1e-14 and abs(m["P2"].sum() - 1) < 1e-14
    assert 0 <= m["D1"] <= 1 and 0 <= m["D2"] <= 1
    # theta is tan-consistent with rho
    np.testing.assert_allclose(np.tan(m["theta"] + np.pi / 4), m["rho"], rtol=1e-12)
    ms = O.metrics(be[::-1], al[::-1])
    np.testing.assert_allclose(ms["theta"], -m["theta"][::-1], atol=1e-15)
    np.testing.assert_allclose(ms["P1"], m["P2"][::-1], atol=1e-15)
    assert abs(ms["D1"] - m["D2"]) < 1e-15


def test_metrics_padding_closed_form():
    rng = _rng(14)
    a = np.sort(rng.uniform(0.1, 0.9, 6))[::-1]
    b = np.sqrt(1 - a ** 2)
    m = O.metrics(a, b)
    mp = O.metrics(a, b, pad_to_n=20, pad_mode=0)
    # appended (0, 1) pairs: P1 keeps its values, D1 rescales by log r / log n
    np.testing.assert_allclose(mp["P1"][:6], m["P1"], atol=1e-15)
    assert abs(mp["D1"] - m["D1"] * np.log(6) / np.log(20)) < 1e-14
    np.testing.assert_allclose(mp["theta"][6:], -np.pi / 4, atol=1e-15)
    mq = O.metrics(a, b, pad_to_n=20, pad_mode=1)
    np.testing.assert_allclose(mq["theta"][:14], np.pi / 4, atol=1e-15)
    assert abs(mq["D2"] - m["D2"] * np.log(6) / np.log(20)) < 1e-14


def test_perturbation_bounds_lemma_per_and_theorem_exp():
    # Lemma "per" / Corollary: max GSV error <= E; Theorem "exp" (i): |dtheta| <= arcsin(2E)
    rng = _rng(15)
    for s in range(5):
        G1, G2, a, b = _full_rank_pair(rng, 30, 25, 8, cond=5.0)
        eps = 10.0 ** (-4 - s)
        G1t = G1 + eps * rng.standard_normal(G1.shape)
        G2t = G2 + eps * rng.standard_normal(G2.shape)
        E = O.perturbation_E(G1, G2, G1t, G2t)
        at, bt = O.direct_gsvd(G1t, G2t)
        assert np.sqrt(np.sum((at - a) ** 2 + (bt - b) ** 2)) <= E
        th = O.metrics(a, b)["theta"]
        tht = O.metrics(at, bt)["theta"]
        assert np.max(np.abs(th - tht)) <= np.arcsin(min(1.0, 2 * E))


def test_perturbation_E_closed_form_on_a_diagonal_pair():
    # G1 = diag(a1 d1, a2 d2), G2 = diag(b1 d1, b2 d2) (a_i^2 + b_i^2 = 1): the stack [G1; G2] has
    # orthogonal columns of norms d1, d2, so ||G^+||_2 = 1 / d2 for d1 > d2.  Adding eps to entry
    # (2, 2) of G1 gives ||Delta G||_F = eps and a second column of norm
    # sqrt((a2 d2 + eps)^2 + (b2 d2)^2) > d2, whose inverse is the smaller of the two pseudo-inverse
    # norms: E = sqrt(2) eps / sqrt((a2 d2 + eps)^2 + (b2 d2)^2), written out by hand.
    a1, a2, d1, d2, eps = 0.8, 0.6, 2.0, 0.5, 1e-3
    b1, b2 = 0.6, 0.8
    G1 = np.diag([a1 * d1, a2 * d2])
    G2 = np.diag([b1 * d1, b2 * d2])
    G1t = G1.copy()
    G1t[1, 1] += eps
    # (a2 d2 + eps)^2 + (b2 d2)^2 = 0.301^2 + 0.4^2 = 0.250601
    E_hand = np.sqrt(2.0) * 1e-3 / np.sqrt(0.250601)
    assert abs(O.perturbation_E(G1, G2, G1t, G2) - E_hand) <= 1e-15 * E_hand
    # symmetric in which pair is taken as the reference
    assert abs(O.perturbation_E(G1t, G2, G1, G2) - E_hand) <= 1e-15 * E_hand
    # and the Lemma's bound holds on it: the perturbed pair of the second column is
    # ((a2 d2 + eps), b2 d2) / its norm, the first pair is unchanged
    nrm = np.sqrt(0.250601)
    at, bt = np.array([a1, 0.301 / nrm]), np.array([b1, 0.4 / nrm])
    got_a, got_b = O.direct_gsvd(G1t, G2)
    np.testing.assert_allclose(got_a, at, atol=1e-15)
    np.testing.assert_allclose(got_b, bt, atol=1e-15)
    assert np.sqrt(np.sum((at - [a1, a2]) ** 2 + (bt - [b1, b2]) ** 2)) <= E_hand


def test_power_iterations_keep_small_directions():
    # Subspace iteration must re-orthonormalise after every product: with a
    # spectrum spanning 1 .. 1e-8 and q = 4 the plain powered sketch
    # (G G^T)^q G Omega loses the weak directions to rounding, while the
    # re-orthonormalised iteration keeps all r GSV pairs to ~eps / 1e-8.
    rng = _rng(16)
    m, p, n, r = 200, 180, 60, 12
    d = np.logspace(0, -8, r)
    a = np.sort(rng.uniform(0.05, 0.95, r))[::-1]
    b = np.sqrt(1 - a ** 2)
    U, _ = np.linalg.qr(rng.standard_normal((m, r)))
    V, _ = np.linalg.qr(rng.standard_normal((p, r)))
    Ot, _ = np.linalg.qr(rng.standard_normal((n, r)))
    G1 = (U * (a * d)) @ Ot.T
    G2 = (V * (b * d)) @ Ot.T
    out = O.rand_gsvd(G1, G2, r, 4, 4, seed=3)
    assert np.max(O.gsv_error(a, b, out["alpha"], out["beta"])) < 1e-5


def test_round_bf16_ties_carries_and_bound():
    # bfloat16 keeps 8 significand bits: spacing 2^-7 on [1, 2).  Values are written
    # from that spacing, not from the rounding formula.
    x = np.array([1.0, -2.5, 0.0, 1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, 1 + 2.0 ** -8 + 2.0 ** -20,
                  2 - 2.0 ** -9, -(1 + 2.0 ** -8 + 2.0 ** -20), 3.0 * 2.0 ** -130])
    want = np.array([1.0, -2.5, 0.0, 1.0, 1 + 2.0 ** -6, 1 + 2.0 ** -7,
                     2.0, -(1 + 2.0 ** -7), 3.0 * 2.0 ** -130], dtype=np.float32)
    np.testing.assert_array_equal(O.round_bf16(x), want)
    # FP32 first: 1 + 2^-8 + 2^-30 rounds to 1 + 2^-8 in FP32 (a tie in BF16, to even 1.0),
    # while rounding the FP64 value directly to 8 bits would give 1 + 2^-7
    assert O.round_bf16(np.array([1 + 2.0 ** -8 + 2.0 ** -30]))[0] == np.float32(1.0)
    rng = _rng(21)
    v = rng.standard_normal(20000) * 10.0 ** rng.uniform(-6, 6, 20000)
    r = O.round_bf16(v).astype(np.float64)
    f = v.astype(np.float32).astype(np.float64)
    assert np.all(np.abs(r - f) <= 2.0 ** -8 * np.abs(f))  # unit roundoff of an 8-bit significand
    # the 256 representable significands of a binade map to themselves
    grid = 1.0 + np.arange(128) / 128.0
    np.testing.assert_array_equal(O.round_bf16(grid), grid.astype(np.float32))


def test_round_bf16_matches_torch_conversion():
    torch = pytest.importorskip("torch")
    rng = _rng(22)
    v = (rng.standard_normal(50000) * 10.0 ** rng.uniform(-3, 3, 50000)).astype(np.float32)
    ref = torch.from_numpy(v).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(O.round_bf16(v), ref)


def test_bf16_omega_sketch_stays_a_range_finder():
    # The rounded test matrix is a 2^-8 relative perturbation of a Gaussian one: on an
    # exact-rank pair the randomized GSVs still equal the planted ones.
    rng = _rng(23)
    m, p, n, r = 120, 100, 40, 6
    a = np.sort(rng.uniform(0.1, 0.9, r))[::-1]
    b = np.sqrt(1 - a ** 2)
    U, _ = np.linalg.qr(rng.standard_normal((m, r)))
    V, _ = np.linalg.qr(rng.standard_normal((p, r)))
    Ot, _ = np.linalg.qr(rng.standard_normal((n, r)))
    d = np.linspace(1, 0.3, r)
    G1 = (U * (a * d)) @ Ot.T
    G2 = (V * (b * d)) @ Ot.T
    plain = O.rand_gsvd(G1, G2, r, 4, 0, seed=5)
    rounded = O.rand_gsvd(G1, G2, r, 4, 0, seed=5, omega_round="bf16")
    assert np.max(O.gsv_error(a, b, rounded["alpha"], rounded["beta"])) < 1e-12
    assert np.max(O.gsv_error(plain["alpha"], plain["beta"], rounded["alpha"], rounded["beta"])) < 1e-12
    with pytest.raises(ValueError):
        O.rand_gsvd(G1, G2, r, 4, 0, seed=5, omega_round="fp8")


# ---------------------------------------------------------------- complex pairs (Section 1 over C)
def _full_rank_pair_complex(rng, m, p, n, alpha=None, cond=10.0):
    """G1 = U diag(alpha) R, G2 = V diag(beta) R over C: U, V with orthonormal columns, R nonsingular."""
    if alpha is None:
        alpha = np.sort(rng.uniform(0.02, 0.98, n))[::-1]
    beta = np.sqrt(1.0 - alpha ** 2)

    def cgauss(r, c):
        return rng.standard_normal((r, c)) + 1j * rng.standard_normal((r, c))

    U, _ = np.linalg.qr(cgauss(m, n))
    V, _ = np.linalg.qr(cgauss(p, n))
    A, _ = np.linalg.qr(cgauss(n, n))
    Bq, _ = np.linalg.qr(cgauss(n, n))
    R = A @ np.diag(np.logspace(0, np.log10(cond), n)) @ Bq
    return U @ np.diag(alpha) @ R, V @ np.diag(beta) @ R, alpha, beta


def test_complex_direct_gsvd_matches_planted_and_hermitian_pencil():
    # the planted GSVs of a complex pair, and brute force by the Hermitian-definite pencil
    # (a transpose in place of the conjugate transpose makes the pencil non-Hermitian and fails)
    rng = _rng(40)
    for n in (1, 3, 6):
        G1, G2, a, b = _full_rank_pair_complex(rng, 9, 8, n)
        ad, bd = O.direct_gsvd_complex(G1, G2)
        np.testing.assert_allclose(ad, a, atol=1e-12)
        np.testing.assert_allclose(bd, b, atol=1e-12)
        ap, bp = O.pencil_gsvd_complex(G1, G2)
        np.testing.assert_allclose(ap, a, atol=1e-10)
        np.testing.assert_allclose(np.sort(bp), np.sort(b), atol=1e-10)
        # exchanging the two matrices exchanges alpha and beta
        a2, b2 = O.direct_gsvd_complex(G2, G1)
        np.testing.assert_allclose(a2, np.sort(b)[::-1], atol=1e-12)


def test_complex_gsvs_appear_twice_in_the_realified_pair():
    # C as real 2 x 2 blocks is a ring homomorphism: the real oracle on (realify(G1), realify(G2))
    # returns every complex GSV twice; the block signs are pinned by realify(A) realify(B) = realify(AB)
    rng = _rng(41)
    G1, G2, a, b = _full_rank_pair_complex(rng, 12, 10, 5)
    ar, br = O.direct_gsvd(O.realify(G1), O.realify(G2))
    np.testing.assert_allclose(ar[0::2], a, atol=1e-12)
    np.testing.assert_allclose(ar[1::2], a, atol=1e-12)
    np.testing.assert_allclose(br[0::2], np.sort(b), atol=1e-12)
    A = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
    B = rng.standard_normal((3, 2)) + 1j * rng.standard_normal((3, 2))
    np.testing.assert_allclose(O.realify(A) @ O.realify(B), O.realify(A @ B), atol=1e-14)
    np.testing.assert_allclose(O.realify(A.conj().T), O.realify(A).T, atol=0)


def test_complex_gaussian_test_matrix_is_circular():
    # independent N(0, 1) real and imaginary parts: E|w|^2 = 2, E w^2 = 0, uncorrelated parts
    W = O.gaussian_complex(400, 50, seed=12, pair=3, side=1)
    x, y = W.real.ravel(), W.imag.ravel()
    assert stats.kstest(x, "norm").pvalue > 1e-3 and stats.kstest(y, "norm").pvalue > 1e-3
    assert abs(np.mean(np.abs(W) ** 2) - 2.0) < 0.05
    assert abs(np.mean(W ** 2)) < 0.05
    assert abs(np.corrcoef(x, y)[0, 1]) < 0.03
    # the sketch of the realified pair by the realified test matrix is the realified sketch
    G = _rng(42).standard_normal((7, 400)) + 1j * _rng(43).standard_normal((7, 400))
    np.testing.assert_allclose(O.realify(G) @ O.realify(W), O.realify(G @ W), atol=1e-10)


@pytest.mark.parametrize("q", [0, 1, 2])
def test_complex_randomized_equals_planted_on_exact_rank(q):
    # exact rank r with l >= r: the bases capture the ranges, so the randomized GSVs are the
    # planted ones; q >= 1 runs the power steps with G^H (a plain transpose loses the range)
    from paper_2404_09459_gb300.inputs import planted_pair_complex
    spec = PairSpec(m=120, p=90, n=40, r=8, alpha="uniform", decay="exp10", sigma=0.0, k=8, oversample=4,
                    q=q, seed=44)
    G1, G2, a, b = planted_pair_complex(spec)
    out = O.rand_gsvd_complex(G1, G2, 8, 4, q, seed=9)
    np.testing.assert_allclose(out["alpha"], a, atol=1e-10)
    np.testing.assert_allclose(out["beta"], b, atol=1e-10)
    assert out["resid1"] < 1e-12 and out["resid2"] < 1e-12


def test_paper_complex_full_pair_recovered():
    # Section 4.1's synthetic pair as the paper states it (complex U, V, R): 40% of the pairs at
    # (1, 0), 40% at (0, 1), 20% uniform; all n pairs are resolved with k = n
    from paper_2404_09459_gb300.inputs import full_gmp_pair_complex
    G1, G2, a, b = full_gmp_pair_complex(150, 130, 50, seed=2)
    d_a, d_b = O.direct_gsvd_complex(G1, G2)
    np.testing.assert_allclose(d_a, a, atol=1e-12)
    out = O.rand_gsvd_complex(G1, G2, 50, 0, 0, seed=5)
    np.testing.assert_allclose(out["alpha"], a, atol=1e-10)
    np.testing.assert_allclose(out["beta"], b, atol=1e-10)


@pytest.mark.parametrize("q", [1, 2])
def test_complex_power_steps_span_the_powered_sketch(q):
    # subspace iteration (Halko, Martinsson & Tropp 2011, Alg. 4.4) spans range((G G^H)^q G Omega)
    # in exact arithmetic; on a full-rank, mildly conditioned G the two bases agree to rounding
    # (a power step taken with G^T instead of G^H spans another subspace)
    rng = _rng(45)
    U, _ = np.linalg.qr(rng.standard_normal((60, 40)) + 1j * rng.standard_normal((60, 40)))
    V, _ = np.linalg.qr(rng.standard_normal((40, 40)) + 1j * rng.standard_normal((40, 40)))
    G = (U * np.linspace(1.0, 0.1, 40)[None, :]) @ V.conj().T
    Q = O.basis_fixed_complex(G, 10, q, seed=3, pair=1, side=0)
    W = O.gaussian_complex(40, 10, seed=3, pair=1, side=0)
    P, _ = np.linalg.qr(np.linalg.matrix_power(G @ G.conj().T, q) @ G @ W)
    sines = np.linalg.norm(P - Q @ (Q.conj().T @ P), 2)
    assert sines < 1e-10, sines
