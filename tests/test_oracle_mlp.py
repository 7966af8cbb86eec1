"""Pins of the learned-proposal oracle (oracle/mlp.py) against mathematics it must obey.

Gradients against central finite differences, the cross-entropy at zero weights
(log C per head), Adam's first steps in closed form, probe features against
their invariances and a rank-one closed form, and labels on exact-rank pairs.
"""
import numpy as np
import pytest

from oracle import gsvd as O
from oracle import mlp as L
from oracle.philox import gaussian


def _theta(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(L.NPARAMS) * scale


def _batch(seed, B=9):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((B, L.IN)) * 2.0 - 1.0
    norm = (rng.standard_normal(L.IN) * 0.5, rng.uniform(0.5, 2.0, L.IN))
    return X, norm, rng.integers(0, L.KCLS, B), rng.integers(0, L.QCLS, B)


def test_param_count_and_layout():
    assert L.NPARAMS == 64 * 128 + 128 + 128 * 128 + 128 + 128 * 37 + 37
    th = np.arange(L.NPARAMS, dtype=np.float64)
    p = L.unpack(th)
    assert p["W1"][0, 1] == 1.0 and p["W1"][1, 0] == 128.0  # row-major, W1 first
    assert p["b3"][-1] == L.NPARAMS - 1
    np.testing.assert_array_equal(L.pack(p), th)


def test_gradient_matches_central_differences():
    th = _theta(1)
    X, norm, yk, yq = _batch(2)
    _, g = L.loss_grad(th, norm, X, yk, yq)
    rng = np.random.default_rng(3)
    idx = np.concatenate([rng.choice(L.NPARAMS, 60, replace=False), [L.NPARAMS - 1, 0, 8192]])
    h = 1e-6
    for i in idx:
        e = np.zeros(L.NPARAMS)
        e[i] = h
        fd = (L.loss_grad(th + e, norm, X, yk, yq)[0] - L.loss_grad(th - e, norm, X, yk, yq)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 + 1e-5 * abs(fd), (i, fd, g[i])


def test_zero_weights_give_uniform_heads():
    X, norm, yk, yq = _batch(4, B=6)
    loss, g = L.loss_grad(np.zeros(L.NPARAMS), norm, X, yk, yq)
    assert abs(loss - (np.log(32) + np.log(5))) < 1e-12
    p = L.unpack(g)
    # d loss / d b3 = mean over the batch of (uniform probabilities - one-hot)
    want = np.concatenate([np.full(32, 1 / 32), np.full(5, 1 / 5)])
    for b in range(6):
        want[yk[b]] -= 1 / 6
        want[32 + yq[b]] -= 1 / 6
    np.testing.assert_allclose(p["b3"], want, atol=1e-15)
    assert np.all(p["W1"] == 0) and np.all(p["W3"] == 0)  # ReLU of zero blocks every path
    assert abs(p["b3"][:32].sum()) < 1e-15 and abs(p["b3"][32:].sum()) < 1e-15


def test_adam_first_steps_closed_form():
    g1 = np.array([0.5, -2.0, 1e-3])
    g2 = np.array([-1.0, 0.0, 1e-3])
    th, m, v = L.adam_step(np.zeros(3), np.zeros(3), np.zeros(3), g1, 1, lr=0.01)
    # step 1: m^ = g, v^ = g^2  ->  update -lr g / (|g| + eps)
    np.testing.assert_allclose(th, -0.01 * g1 / (np.abs(g1) + 1e-8), rtol=1e-12)
    th2, _, _ = L.adam_step(th, m, v, g2, 2, lr=0.01)
    m2 = 0.9 * 0.1 * g1 + 0.1 * g2
    v2 = 0.999 * 0.001 * g1 ** 2 + 0.001 * g2 ** 2
    step = 0.01 * (m2 / (1 - 0.81)) / (np.sqrt(v2 / (1 - 0.999 ** 2)) + 1e-8)
    np.testing.assert_allclose(th2, th - step, rtol=1e-12)


def test_bf16_inference_rounds_weights_only():
    th = _theta(5)
    X, norm, _, _ = _batch(6)
    z, _ = L.forward(th, norm, X)
    zb, _ = L.forward(th, norm, X, bf16_weights=True)
    assert 0 < np.max(np.abs(z - zb)) < 0.05 * np.max(np.abs(z))
    p = L.unpack(th)
    for n in ("W1", "W2", "W3"):
        p[n] = O.round_bf16(p[n])
    np.testing.assert_allclose(L.forward(L.pack(p), norm, X)[0], zb, rtol=0, atol=1e-12)


def _pair(seed, m=300, p=260, n=90, r=6, decay=0.5):
    rng = np.random.default_rng(seed)
    a = np.sort(rng.uniform(0.1, 0.9, r))[::-1]
    b = np.sqrt(1 - a ** 2)
    U, _ = np.linalg.qr(rng.standard_normal((m, r)))
    V, _ = np.linalg.qr(rng.standard_normal((p, r)))
    Ot, _ = np.linalg.qr(rng.standard_normal((n, r)))
    d = decay ** np.arange(r)
    return (U * (a * d)) @ Ot.T, (V * (b * d)) @ Ot.T


def test_features_scale_invariant_and_swap_symmetric():
    G1, G2 = _pair(7)
    f = L.probe_features(G1, G2, seed=3, pair=2)
    assert f.shape == (64,)
    np.testing.assert_allclose(L.probe_features(37.0 * G1, 1e-3 * G2, 3, 2), f, atol=1e-9)
    # side 2 draws its own probe (side index 1): swapping the matrices swaps the sides only
    # when the probes are swapped too, so compare each half with a direct evaluation
    np.testing.assert_allclose(L.side_features(G2, 3, 2, 1), f[32:], atol=0)
    np.testing.assert_allclose(L.side_features(G1, 3, 2, 0), f[:32], atol=0)


def test_features_rank_one_closed_form_and_rank_floor():
    rng = np.random.default_rng(8)
    u, v = rng.standard_normal(200), rng.standard_normal(70)
    G = 3.0 * np.outer(u, v)
    f = L.side_features(G, 5, 1, 0)
    assert f.shape == (32,)
    Om = gaussian(70, 64, 5, 1, 0, L.STREAM_PROBE)
    w = Om.T @ v / np.linalg.norm(v)  # Y = 3 |u| |v| u^ w^T, Y^T Y = g2 w w^T
    np.testing.assert_allclose(f[0], np.log10(w @ w / 64), atol=1e-10)
    assert np.all(f[1:] == L.FEAT_MIN)  # nothing beyond rank one


def test_features_show_ranks_up_to_the_probe_width():
    # orthonormal U, V and equal singular values: Y^T Y = Omega^T V V^T Omega, whose nonzero
    # eigenvalues are those of the r x r Wishart matrix W = (V^T Omega)(V^T Omega)^T, so the
    # features are exactly log10 of W's eigenvalues over 64 r (g2 = r), every other one, and the
    # rank shows as the first clipped feature: feature t is clipped exactly when 2 t >= r
    rng = np.random.default_rng(11)
    n = 150
    for r in (6, 23, 40, 63):
        U, _ = np.linalg.qr(rng.standard_normal((300, r)))
        V, _ = np.linalg.qr(rng.standard_normal((n, r)))
        G = U @ V.T
        f = L.side_features(G, 4, 0, 1)
        Om = gaussian(n, 64, 4, 0, 1, L.STREAM_PROBE)
        B = V.T @ Om
        lam = np.sort(np.linalg.eigvalsh(B @ B.T))[::-1]
        want = np.log10(lam[0::2] / (64 * r))
        t = np.arange(32)
        np.testing.assert_allclose(f[2 * t < r], want, atol=1e-9)
        assert np.all(f[2 * t >= r] == L.FEAT_MIN)


def test_labels_on_exact_rank_pair():
    # exact rank r: Algorithm 1 with blocks of 4 stops at the first multiple of 4 >= r (the
    # residual is then at rounding level), and a q = 0 fixed-rank basis with l >= r is exact
    G1, G2 = _pair(9, r=6)
    kb, q, k_ad = L.labels(G1, G2, tol=1e-6, seed=1, oversample=4)
    assert k_ad == 8
    assert q == 0 and kb == L.bucket_of_k(8 - 4) == 0
    assert L.k_of_bucket(kb) + 4 >= 6


def test_labels_need_power_steps_on_flat_tail():
    # a flat spectrum just below the target directions: q = 0 leaves the residual above tol
    rng = np.random.default_rng(10)
    m, n = 400, 120
    U, _ = np.linalg.qr(rng.standard_normal((m, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    s = np.concatenate([np.full(8, 1.0), np.full(n - 8, 2e-4)])
    G1 = (U * s) @ V.T
    G2 = (np.roll(U, 7, axis=0) * s) @ V.T
    kb, q, k_ad = L.labels(G1, G2, tol=3e-2, seed=2, oversample=4)
    assert q >= 1 or L.k_of_bucket(kb) + 4 >= k_ad
    k = L.k_of_bucket(kb)
    for side, G in enumerate((G1, G2)):
        assert L.fixed_residual(G, k, 4, q, 2, 0, side) <= 3e-2
    with pytest.raises(AssertionError):
        L.unpack(np.zeros(5))


def test_plan_rule_on_known_probabilities():
    # logits log(p): cumulative probabilities 0.5, 0.8, 0.95, ... -> the 0.9 quantile is bucket 2,
    # the 0.5 quantile bucket 0, the 0.8 quantile bucket 1 (reached exactly), q the argmax (first
    # of two equal maxima)
    p = np.zeros(L.KCLS)
    p[:4] = [0.5, 0.3, 0.15, 0.05]
    zk = np.log(np.where(p > 0, p, 1e-300))
    zq = np.array([0.0, 2.0, 2.0, 1.0, -1.0])
    z = np.concatenate([zk, zq])[None, :]
    for qt, want in ((0.9, 2), (0.5, 0), (0.8 - 1e-12, 1), (0.999, 3)):
        kb, q = L.plan(z, qt)
        assert kb[0] == want and q[0] == 1
    # a flat k head reaches the quantile at bucket ceil(0.9 KCLS) - 1; the last bucket when never reached
    z2 = np.zeros((1, L.KCLS + 5))
    assert L.plan(z2, 0.9)[0][0] == int(np.ceil(0.9 * L.KCLS)) - 1
    assert L.plan(z2, 1.0 + 1e-9)[0][0] == L.KCLS - 1
