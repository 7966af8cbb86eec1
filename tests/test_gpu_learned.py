"""The learned (k, q) proposal on the GPU vs its FP64 oracle (oracle/mlp.py), through the C ABI.

Probe features, forward (FP32 and BF16 weights), loss and gradient, Adam steps and the
training loop against the oracle on the same inputs; labels from the GPU's Algorithm 1
against the oracle's; the learned solve with a fixed proposal (no fallback and fallback)
against the oracle's fixed-rank and adaptive GSVs.
"""
import os
import tempfile

import numpy as np
import pytest

from oracle import gsvd as O
from oracle import mlp as L
from paper_2404_09459_gb300.inputs import PairSpec, mlp_init, planted_pair

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2404_09459_gb300 as P  # noqa: E402
from paper_2404_09459_gb300 import learn  # noqa: E402

P._build.build()
DEV = "cuda"


def _net(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    th = mlp_init(seed).astype(np.float64) * scale + rng.standard_normal(L.NPARAMS) * 0.01
    norm = np.concatenate([rng.standard_normal(64) * 0.3 - 3.0, rng.uniform(0.5, 3.0, 64)])
    return th.astype(np.float32), norm.astype(np.float32)


def _t(a, dt=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV, dt)


SPECS = [PairSpec(m=700, p=520, n=150, r=12, alpha="uniform", decay="exp10", sigma=1e-9, k=12, oversample=6, q=1,
                  seed=3),
         PairSpec(m=333, p=401, n=97, r=30, alpha="uniform", decay="pow15", sigma=1e-7, k=20, oversample=6, q=1,
                  seed=4)]


@pytest.mark.parametrize("prec", ["fp64", "tf32x3", "fp32"])
@pytest.mark.parametrize("spec", SPECS, ids=["exp10", "pow15"])
def test_probe_features_match_oracle(spec, prec):
    G1, G2, _, _ = planted_pair(spec)
    ref = L.probe_features(G1, G2, spec.seed)
    dt = torch.float64 if prec == "fp64" else torch.float32
    with P.Context(prec) as ctx:
        got = ctx.probe_features(_t(G1, dt), _t(G2, dt), spec.seed).cpu().numpy()
        host = ctx.probe_features(G1 if prec == "fp64" else G1.astype(np.float32),
                                  G2 if prec == "fp64" else G2.astype(np.float32), spec.seed)
    if prec != "tf32x3":
        # same products either way (a host input is staged with 16-byte rows, which moves an
        # FP32 input with n % 4 != 0 from the CUDA-core to the tensor-core products)
        np.testing.assert_array_equal(got, host)
    else:
        np.testing.assert_allclose(host[ref > -5.0], ref[ref > -5.0], rtol=0, atol=2e-3)
    # FP64: eigenvalues to ~1e-13 relative, the features then rounded to FP32 (half an ulp of
    # |f| <= 12 is below 5e-7); FP32 data: ~1e-6 relative in the energies near the top, more
    # for small ones whose Gram entries cancel
    keep = ref > (-10.0 if prec == "fp64" else -5.0)
    tol = 1e-6 if prec == "fp64" else 2e-3
    np.testing.assert_allclose(got[keep], ref[keep], rtol=0, atol=tol)
    assert np.all((got >= L.FEAT_MIN) & (got <= L.FEAT_MAX))


@pytest.mark.parametrize("bf16", [False, True])
@pytest.mark.parametrize("B", [1, 37])
def test_forward_matches_oracle(B, bf16):
    th, norm = _net(1)
    X = np.random.default_rng(2).uniform(-12, 1, (B, 64)).astype(np.float32)
    ref, _ = L.forward(th, (norm[:64], norm[64:]), X, bf16_weights=bf16)
    with P.Context("fp32") as ctx:
        z = ctx.mlp_forward(_t(th), _t(norm), _t(X), bf16).cpu().numpy()
    np.testing.assert_allclose(z, ref, rtol=1e-4, atol=1e-4 * np.max(np.abs(ref)))
    # the argmax the solve takes, where the oracle's top two differ by more than the tolerance
    for head in (slice(0, 32), slice(32, 37)):
        r = ref[:, head]
        srt = np.sort(r, axis=1)
        clear = srt[:, -1] - srt[:, -2] > 1e-3 * np.max(np.abs(ref))
        np.testing.assert_array_equal(z[clear][:, head].argmax(1), r[clear].argmax(1))


def test_loss_and_gradient_match_oracle():
    th, norm = _net(3)
    rng = np.random.default_rng(4)
    B = 53
    X = rng.uniform(-12, 1, (B, 64)).astype(np.float32)
    yk, yq = rng.integers(0, 32, B).astype(np.int32), rng.integers(0, 5, B).astype(np.int32)
    loss_ref, g_ref = L.loss_grad(th, (norm[:64], norm[64:]), X, yk, yq)
    with P.Context("fp32") as ctx:
        loss, g = ctx.mlp_loss_grad(_t(th), _t(norm), _t(X), _t(yk, torch.int32), _t(yq, torch.int32))
    g = g.cpu().numpy()
    assert abs(loss - loss_ref) <= 1e-5 * abs(loss_ref)
    scale = np.max(np.abs(g_ref))
    np.testing.assert_allclose(g, g_ref, rtol=1e-3, atol=1e-5 * scale)
    # every block of the flat layout, not only the largest entries
    o = 0
    for name, shape in L.SHAPES:
        size = int(np.prod(shape))
        blk = slice(o, o + size)
        assert np.linalg.norm(g[blk] - g_ref[blk]) <= 1e-4 * np.linalg.norm(g_ref[blk]) + 1e-7, name
        o += size


def test_adam_and_training_steps_match_oracle():
    th, norm = _net(5, scale=0.5)
    rng = np.random.default_rng(6)
    N, B, steps, lr = 96, 32, 4, 3e-3
    X = rng.uniform(-12, 1, (N, 64)).astype(np.float32)
    yk, yq = rng.integers(0, 32, N).astype(np.int32), rng.integers(0, 5, N).astype(np.int32)
    order = rng.permutation(N)[: steps * B].astype(np.int32) if steps * B <= N else \
        np.concatenate([rng.permutation(N) for _ in range(2)])[: steps * B].astype(np.int32)
    ref, m, v = th.astype(np.float64), np.zeros(L.NPARAMS), np.zeros(L.NPARAMS)
    nrm = (norm[:64], norm[64:])
    losses = []
    for i in range(steps):
        rows = order[i * B:(i + 1) * B]
        lo, g = L.loss_grad(ref, nrm, X[rows], yk[rows], yq[rows])
        losses.append(lo)
        ref, m, v = L.adam_step(ref, m, v, g, i + 1, lr)
    with P.Context("fp32") as ctx:
        pt, mt, vt = _t(th), torch.zeros(L.NPARAMS, device=DEV), torch.zeros(L.NPARAMS, device=DEV)
        hist = ctx.mlp_train(pt, mt, vt, _t(norm), _t(X), _t(yk, torch.int32), _t(yq, torch.int32),
                             _t(order, torch.int32), B, 0, lr).cpu().numpy()
        # the single-step entry points agree with the fused training loop
        p2, m2, v2 = _t(th), torch.zeros(L.NPARAMS, device=DEV), torch.zeros(L.NPARAMS, device=DEV)
        for i in range(steps):
            rows = order[i * B:(i + 1) * B]
            _, g = ctx.mlp_loss_grad(p2, _t(norm), _t(X[rows]), _t(yk[rows], torch.int32),
                                     _t(yq[rows], torch.int32))
            ctx.mlp_adam(p2, m2, v2, g, i + 1, lr)
    np.testing.assert_allclose(hist, losses, rtol=1e-4)
    # Adam moves each weight by about lr per step whatever the gradient's size, so compare
    # the displacement from the start with a tolerance of a small fraction of lr
    d_ref = ref - th
    d = pt.cpu().numpy().astype(np.float64) - th
    assert np.max(np.abs(d - d_ref)) <= 0.02 * lr * steps
    np.testing.assert_array_equal(pt.cpu().numpy(), p2.cpu().numpy())


def _fixed_net(kb, q):
    """A network whose heads ignore the features: zero weights, biases picking (kb, q)."""
    th = np.zeros(L.NPARAMS, np.float32)
    b3 = L.NPARAMS - 37
    th[b3 + kb] = 12.0  # softmax mass > 0.999: above the 0.9 quantile the solve takes
    th[b3 + 32 + q] = 12.0
    return th, np.concatenate([np.zeros(64), np.ones(64)]).astype(np.float32)


def test_learned_solve_uses_proposal_or_falls_back():
    # planted rank 20 above every k asked for, so that all returned pairs are signal pairs
    spec = PairSpec(m=900, p=700, n=160, r=20, alpha="uniform", decay="exp10", sigma=1e-10, k=16, oversample=8,
                    q=1, seed=11)
    G1, G2, _, _ = planted_pair(spec)
    g1, g2 = _t(G1, torch.float64), _t(G2, torch.float64)
    tol = 1e-6
    # adequate proposal: bucket 3 (k = 16, l = 24 >= r), q = 1 -> the fixed-rank solve, no fallback
    th, norm = _fixed_net(3, 1)
    with P.Context("fp64", use_learned=True, tol=tol, block_b=8) as ctx:
        ctx.mlp_set(th, norm)
        out = ctx.solve(g1, g2, 64, spec.oversample, 0, spec.seed)
        assert ctx.last_plan() == (16, 1, False)
    ref = O.rand_gsvd(G1, G2, 16, spec.oversample, 1, spec.seed)
    assert out["r"] == 16 and max(out["resid"]) <= tol
    assert np.max(O.gsv_error(ref["alpha"], ref["beta"], out["alpha"].cpu().numpy(), out["beta"].cpu().numpy())) < 1e-10
    # too small a proposal (k = 4, l = 12 < r): residual misses, Algorithm 1 solves the pair
    th, norm = _fixed_net(0, 0)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "net.bin")
        learn.save(path, th, norm)
        with P.Context("fp64", use_learned=True, mlp_path=path, tol=tol, block_b=8) as ctx:
            out = ctx.solve(g1, g2, 64, spec.oversample, 0, spec.seed)
            k, q, fb = ctx.last_plan()
            l1, l2 = ctx.basis_cols()
    assert (k, q, fb) == (4, 0, True)
    ref = O.rand_gsvd_adaptive(G1, G2, tol, 8, spec.seed, 4)
    assert (l1, l2) == (ref["l1"], ref["l2"])
    assert max(out["resid"]) <= tol
    assert np.max(O.gsv_error(ref["alpha"], ref["beta"], out["alpha"].cpu().numpy(), out["beta"].cpu().numpy())) < 1e-10
    with P.Context("fp64", use_learned=True) as ctx:
        with pytest.raises(P.GsvdRandError) as e:
            ctx.solve(g1, g2, 8, 4, 0, 1)
    assert e.value.name == "ARG"


@pytest.mark.parametrize("spec", [
    PairSpec(m=500, p=420, n=120, r=9, alpha="uniform", decay="exp10", sigma=0.0, k=9, oversample=4, q=1, seed=21),
    PairSpec(m=640, p=500, n=140, r=30, alpha="uniform", decay="exp10", sigma=1e-9, k=30, oversample=10, q=1,
             seed=22)], ids=["exact_rank", "graded"])
def test_labels_match_oracle(spec):
    G1, G2, _, _ = planted_pair(spec)
    tol = 1e-4
    ref = L.labels(G1, G2, tol, spec.seed, oversample=spec.oversample)
    lab = learn.Labeler(tol, spec.oversample)
    try:
        got = lab.label(_t(G1, torch.float64), _t(G2, torch.float64), spec.seed)
    finally:
        lab.close()
    assert tuple(int(x) for x in got) == tuple(int(x) for x in ref)


def test_grouped_learned_plans_and_fallback():
    # the learned proposal for a whole group: every pair proposes k = 16, q = 1 (a fixed network),
    # capped by each pair's k (its rank here, so that every returned pair is a planted one): the
    # pairs of rank 16 and 12 are solved by the fixed-rank group, the rank-30 pair misses tol with
    # k = 16 and is solved again by the grouped Algorithm 1 (mixed precision: tol above the ~4e-4
    # floor of the residual estimate)
    from paper_2404_09459_gb300.inputs import aligned_rows
    specs = [PairSpec(m=900, p=700, n=160, r=16, alpha="uniform", decay="exp10", sigma=1e-10, k=16, oversample=8,
                      seed=31),
             PairSpec(m=1300, p=800, n=200, r=30, alpha="uniform", decay="exp10", sigma=1e-10, k=30, oversample=8,
                      seed=32),
             PairSpec(m=600, p=640, n=120, r=12, alpha="uniform", decay="exp10", sigma=1e-10, k=12, oversample=8,
                      seed=33)]
    mats = [planted_pair(s)[:2] for s in specs]
    pairs = [dict(G1=aligned_rows(_t(G1)), G2=aligned_rows(_t(G2)), k=s.k, oversample=8, q=0, seed=s.seed, pair=i)
             for i, (s, (G1, G2)) in enumerate(zip(specs, mats))]
    tol, b = 2e-3, 8
    th, norm = _fixed_net(3, 1)
    with P.Context("tf32x3", use_learned=True, tol=tol, block_b=b) as ctx:
        ctx.mlp_set(th, norm)
        outs = ctx.solve_grouped(pairs)
        plans = ctx.grouped_plans(len(pairs))
    assert plans == [(16, 1, 0), (16, 1, 1), (12, 1, 0)]
    for i, (s, (G1, G2), out) in enumerate(zip(specs, mats, outs)):
        assert out["status"] == 0 and max(out["resid"]) <= tol
        if plans[i][2]:
            ref = O.rand_gsvd_adaptive(G1, G2, tol, b, s.seed, s.k, pair=i, max_cols=min(s.m, s.p, s.n, 128))
        else:
            ref = O.rand_gsvd(G1, G2, plans[i][0], 8, 1, s.seed, pair=i)
        assert out["r"] == s.k
        e = O.gsv_error(ref["alpha"], ref["beta"], out["alpha"].cpu().numpy(), out["beta"].cpu().numpy())
        assert np.max(e) <= 1e-4, (i, np.max(e))


def test_grouped_probe_features_match_oracle():
    # the probes of a learned group run as one grouped pass (3xTF32 products, batched Grams): the
    # features of every pair, with its own Philox word, against the oracle's probe of that pair
    # (the single probe's FP32 targets); a pair too narrow for the probe (n < 16) keeps zeros
    from paper_2404_09459_gb300.inputs import aligned_rows
    specs = SPECS + [PairSpec(m=1500, p=900, n=260, r=40, alpha="uniform", decay="exp10", sigma=1e-8, k=40,
                              oversample=8, seed=35),
                     PairSpec(m=400, p=300, n=12, r=6, alpha="uniform", decay="exp10", sigma=1e-8, k=4,
                              oversample=2, seed=36)]
    mats = [planted_pair(s)[:2] for s in specs]
    pairs = [dict(G1=aligned_rows(_t(G1)), G2=aligned_rows(_t(G2)), k=min(s.k, s.n - 2), oversample=2, q=0,
                  seed=s.seed, pair=i) for i, (s, (G1, G2)) in enumerate(zip(specs, mats))]
    th, norm = _fixed_net(3, 1)
    with P.Context("tf32x3", use_learned=True, tol=2e-3, block_b=8) as ctx:
        ctx.mlp_set(th, norm)
        try:
            ctx.solve_grouped(pairs)
        except P.GsvdRandError as e:
            assert e.name == "ARG"  # the narrow pair
        got = ctx.grouped_features(len(pairs))
    for i, (s, (G1, G2)) in enumerate(zip(specs[:-1], mats[:-1])):
        ref = L.probe_features(G1, G2, s.seed, pair=i)
        keep = ref > -5.0
        np.testing.assert_allclose(got[i][keep], ref[keep], rtol=0, atol=2e-3)
        assert np.all((got[i] >= L.FEAT_MIN) & (got[i] <= L.FEAT_MAX))
    assert np.all(got[-1] == 0.0)


def test_plan_on_device_matches_oracle_rule():
    # the learned solves' (k, q) decision runs on the device (gsvd_rand_mlp_plan); both sides take
    # it in FP64 from the same FP32 logits
    rng = np.random.default_rng(5)
    z = (rng.standard_normal((300, 37)) * 3.0).astype(np.float32)
    z[:20, :32] = 0.0  # flat k heads
    z[20:40, 32:] = 1.0  # q ties: the first class
    with P.Context("fp32") as ctx:
        for qt in (0.9, 0.5, 0.99):
            plan = ctx.mlp_plan(_t(z), qt)
            kb, q = L.plan(z.astype(np.float64), qt)
            np.testing.assert_array_equal(plan[:, 2], kb)
            np.testing.assert_array_equal(plan[:, 1], q)
            np.testing.assert_array_equal(plan[:, 0], 4 * (kb + 1))


def test_grouped_learned_gain_over_algorithm1_and_fixed_rank():
    # what the trained network gains over the method without it: labels from the FP64 Algorithm 1
    # (at half the solve's tolerance: the FP32 residual estimate of the mixed solve then has a
    # margin), the network trained on the GPU by the library's kernels, then one held-out group
    # solved three ways, every pair certified within tol on both sides: (1) the learned group
    # (probes, network, per-pair plans, fixed-rank group, Algorithm 1 for misses); (2) the plain
    # fixed-rank method at the one (k, q) the training labels need at most, as a constant proposal
    # through the same pipeline (probes, fixed-rank group with the same residual sums, Algorithm 1
    # for the pairs it leaves above tol); (3) the grouped Algorithm 1 alone (b = 16).  The learned
    # group runs more pairs per second than both
    from paper_2404_09459_gb300.inputs import aligned_rows, learned_pairs, planted_pair_torch
    tol, os_, b = 2e-3, 10, 16
    law = dict(m_range=(4000, 12000), n_range=(300, 600))
    tr = learned_pairs(160, seed=11, **law)
    ho = learned_pairs(96, seed=12, **law)
    X, yk, yq, _ = learn.make_dataset(tr, tol / 2, os_, 0, features_prec="tf32x3")
    params, norm, hist = learn.train(X, yk, yq, epochs=120, batch=64, lr=2e-3)
    assert hist[-1] < hist[0]
    mats = [tuple(aligned_rows(G) for G in planted_pair_torch(s, device=DEV, dtype=torch.float32)[:2]) for s in ho]
    kb_fix, q_fix = int(yk.max()), int(yq.max())
    pl = [dict(G1=G1, G2=G2, k=128 - os_, oversample=os_, q=1, seed=s.seed, pair=i)
          for i, (s, (G1, G2)) in enumerate(zip(ho, mats))]

    def timed(ctx):
        ctx.solve_grouped(pl)  # graphs captured, products tuned
        ts = []
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            t0.record()
            outs = ctx.solve_grouped(pl)
            t1.record()
            torch.cuda.synchronize()
            ts.append(t0.elapsed_time(t1))
        assert all(o["status"] == 0 and max(o["resid"]) <= tol for o in outs)
        return float(np.median(ts))

    with P.Context("tf32x3", use_learned=True, tol=tol, block_b=b) as ctx:
        ctx.mlp_set(params.cpu().numpy(), norm.cpu().numpy())
        t_learned = timed(ctx)
        fb_learned = np.mean([p_[2] for p_ in ctx.grouped_plans(len(ho))])
    with P.Context("tf32x3", use_learned=True, tol=tol, block_b=b) as ctx:
        ctx.mlp_set(*_fixed_net(kb_fix, q_fix))
        t_plain = timed(ctx)
        plans = ctx.grouped_plans(len(ho))
        fb_plain = np.mean([p_[2] for p_ in plans])
        assert all(p_[0] == min(learn.k_of_bucket(kb_fix), 128 - os_) and p_[1] == q_fix for p_ in plans)
    with P.Context("tf32x3", adaptive=True, tol=tol, block_b=b) as ctx:
        t_adaptive = timed(ctx)
    print(f"learned {t_learned:.2f} ms (fallback {fb_learned:.2f}), fixed rank k {learn.k_of_bucket(kb_fix)} "
          f"q {q_fix} {t_plain:.2f} ms (fallback {fb_plain:.2f}), Algorithm 1 {t_adaptive:.2f} ms")
    assert t_learned < t_adaptive and t_learned < t_plain