"""Grouped solves (one launch per step for a whole batch, replayed from a CUDA graph)
against the FP64 oracle, through the C ABI (needs a CUDA GPU).

Tolerance: the mixed-precision target, per-pair GSV error
e_i = max(|alpha_i - alpha_ref_i|, |beta_i - beta_ref_i|) <= 1e-4 (3xTF32 products,
FP64 CholeskyQR Grams and FP64 compressed-pair GSVD), 1e-3 for single-pass TF32.
"""
import numpy as np
import pytest

from oracle import gsvd as O
from paper_2404_09459_gb300.inputs import PairSpec, aligned_rows, planted_pair

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2404_09459_gb300 as P  # noqa: E402

P._build.build()

TOL = {"tf32": 1e-3, "tf32x3": 1e-4}


def _dev(a):
    # rows padded to 16 bytes: the grouped products read G in place through TMA
    return aligned_rows(torch.from_numpy(np.ascontiguousarray(a)).to("cuda", torch.float32))


def _specs(seed, count, wide=False):
    """Uneven pairs: m, p, n, rank, oversample and q all differ; `wide` adds bases with
    l = k + oversample > 64 (the second CholeskyQR class) and stacks L = 2 l > 128 (the
    packed-triangle eigensolver)."""
    rng = np.random.default_rng(seed)
    specs = []
    for i in range(count):
        m, p = (int(x) for x in rng.integers(300, 2500, 2))
        n = int(rng.integers(90, 420))
        r = int(rng.integers(4, 36))
        os_ = int(rng.choice([4, 8, 10]))
        if wide and i % 2 == 0:
            r = int(rng.integers(56, 70))
            n = max(n, r + 40)
            os_ = 10
        specs.append(PairSpec(m=m, p=p, n=n, r=r, alpha="uniform", decay="exp10", sigma=1e-6, k=r,
                              oversample=os_, q=int(rng.integers(0, 3)), seed=500 + i))
    return specs


def _pairs(specs, mats):
    return [dict(G1=_dev(G1), G2=_dev(G2), k=s.kk, oversample=s.oversample, q=s.q, seed=s.seed, pair=i)
            for i, (s, (G1, G2)) in enumerate(zip(specs, mats))]


def _check_vs_oracle(prec, specs, mats, outs):
    for i, (s, (G1, G2), out) in enumerate(zip(specs, mats, outs)):
        assert out["status"] == 0 and out["r"] == s.kk
        ref = O.rand_gsvd(G1, G2, s.kk, s.oversample, s.q, s.seed, pair=i)
        a = np.asarray(out["alpha"].cpu() if hasattr(out["alpha"], "cpu") else out["alpha"])
        b = np.asarray(out["beta"].cpu() if hasattr(out["beta"], "cpu") else out["beta"])
        e = O.gsv_error(ref["alpha"], ref["beta"], a, b)
        assert np.max(e) <= TOL[prec], (i, s, np.max(e))
        dth = np.abs(np.arctan2(a, b) - np.arctan2(ref["alpha"], ref["beta"]))
        assert np.max(dth) <= max(1e-4, TOL[prec])
        assert np.all(np.diff(a) <= 0) and np.all(np.diff(b) >= 0)
        # cumulated residual sqrt(||G||^2 - ||B||^2) / ||G||: ||B||^2 carries the relative error
        # of the products (2^-10 for single-pass TF32) and of the FP32 basis' orthogonality, so
        # the estimate is held on the squared scale
        rtol = 4e-3 if prec == "tf32" else 1e-4
        for sd in range(2):
            assert abs(out["resid"][sd] ** 2 - ref[f"resid{sd + 1}"] ** 2) <= rtol, (i, sd, out["resid"])


@pytest.mark.parametrize("prec", ["tf32x3", "tf32"])
def test_grouped_uneven_pairs_match_oracle(prec):
    # single-pass TF32 truncates G to 10 mantissa bits: planted scales below ~1e-3 of the
    # largest (ranks above ~60 with the exp(-i/10) law) are beyond it, so it takes the
    # narrower pairs; 3xTF32 takes the wide ones too
    specs = _specs(11, 7, wide=prec == "tf32x3")
    mats = [planted_pair(s)[:2] for s in specs]
    with P.Context(prec) as ctx:
        outs = ctx.solve_grouped(_pairs(specs, mats))
        info = ctx.grouped_info()
    _check_vs_oracle(prec, specs, mats, outs)
    assert info["captures"] == 1 and info["replays"] == 1 and info["launches"] > 20
    for st, ps in info["tuned"]:
        assert st >= 2 and ps in (1, 2)


def test_grouped_replays_graph_bit_identical_and_host_outputs():
    specs = _specs(12, 6)
    mats = [planted_pair(s)[:2] for s in specs]
    pairs = _pairs(specs, mats)
    with P.Context("tf32x3") as ctx:
        first = ctx.solve_grouped(pairs)
        second = ctx.solve_grouped(pairs)           # same inputs, new output buffers: replay
        host = ctx.solve_grouped(pairs, host_out=True)
        info = ctx.grouped_info()
    assert info["captures"] == 1 and info["replays"] == 3
    for a, b, c in zip(first, second, host):
        np.testing.assert_array_equal(a["alpha"].cpu().numpy(), b["alpha"].cpu().numpy())
        np.testing.assert_array_equal(a["beta"].cpu().numpy(), b["beta"].cpu().numpy())
        np.testing.assert_array_equal(a["alpha"].cpu().numpy(), np.asarray(c["alpha"]))
        np.testing.assert_array_equal(a["beta"].cpu().numpy(), np.asarray(c["beta"]))
        assert a["resid"] == c["resid"]
    _check_vs_oracle("tf32x3", specs, mats, host)


def test_grouped_agrees_with_single_and_worker_solves():
    specs = _specs(13, 5, wide=True)
    mats = [planted_pair(s)[:2] for s in specs]
    pairs = _pairs(specs, mats)
    with P.Context("tf32x3") as ctx:
        grouped = ctx.solve_grouped(pairs)
        workers = ctx.solve_batched(pairs, workers=3)
    for g, w in zip(grouped, workers):
        # both are within 1e-4 of the oracle; they differ only in rounding (Gram chunking)
        e = O.gsv_error(w["alpha"].cpu().numpy(), w["beta"].cpu().numpy(), g["alpha"].cpu().numpy(),
                        g["beta"].cpu().numpy())
        assert np.max(e) <= 2e-4


def test_grouped_new_batch_recaptures_and_bad_pair_is_left_out():
    specs = _specs(14, 4)
    mats = [planted_pair(s)[:2] for s in specs]
    pairs = _pairs(specs, mats)
    with P.Context("tf32x3") as ctx:
        good = ctx.solve_grouped(pairs)
        bad = dict(pairs[1])
        bad["k"] = 10_000  # k + oversample > n
        with pytest.raises(P.GsvdRandError) as e:
            ctx.solve_grouped([pairs[0], bad, pairs[2], pairs[3]])
        assert e.value.name == "ARG"
        again = ctx.solve_grouped([pairs[0], pairs[2], pairs[3]])
        info = ctx.grouped_info()
    assert info["captures"] == 3
    np.testing.assert_array_equal(good[0]["alpha"].cpu().numpy(), again[0]["alpha"].cpu().numpy())


def test_grouped_refuses_fp64_contexts():
    specs = _specs(15, 1)
    mats = [planted_pair(s)[:2] for s in specs]
    with P.Context("fp64") as ctx:
        pairs = [dict(G1=aligned_rows(torch.from_numpy(G1).cuda()), G2=aligned_rows(torch.from_numpy(G2).cuda()), k=s.kk,
                      oversample=s.oversample, q=s.q, seed=s.seed) for s, (G1, G2) in zip(specs, mats)]
        with pytest.raises(P.GsvdRandError) as e:
            ctx.solve_grouped(pairs)
        assert e.value.name == "UNSUPPORTED"


def test_grouped_leaves_out_pairs_with_unaligned_rows():
    specs = _specs(16, 3)
    specs[1] = PairSpec(m=500, p=400, n=101, r=8, k=8, oversample=6, q=1, seed=7)
    mats = [planted_pair(s)[:2] for s in specs]
    pairs = _pairs(specs, mats)
    pairs[1]["G1"] = torch.from_numpy(mats[1][0]).to("cuda", torch.float32)  # 404-byte rows
    with P.Context("tf32x3") as ctx:
        with pytest.raises(P.GsvdRandError) as e:
            outs = ctx.solve_grouped(pairs)
        assert e.value.name == "ARG"
        outs = ctx.solve_grouped([pairs[0], pairs[2]])
    _check_vs_oracle("tf32x3", [specs[0]], [mats[0]], outs[:1])


def test_grouped_limits_widest_basis_small_tiles_and_q0():
    # l = 128 (the widest grouped basis: two 128-column accumulators and the A ring fill the
    # tensor memory; a 256-row stack), pairs shorter than one 128-row tile, q = 0 everywhere
    specs = [PairSpec(m=900, p=700, n=300, r=60, alpha="uniform", decay="exp10", sigma=1e-10, k=60,
                      oversample=68, q=0, seed=31),
             PairSpec(m=100, p=90, n=64, r=6, alpha="uniform", decay="exp10", sigma=1e-6, k=6,
                      oversample=4, q=0, seed=32),
             PairSpec(m=130, p=257, n=41, r=9, alpha="uniform", decay="exp10", sigma=1e-6, k=9,
                      oversample=7, q=0, seed=33)]
    mats = [planted_pair(s)[:2] for s in specs]
    with P.Context("tf32x3") as ctx:
        outs = ctx.solve_grouped(_pairs(specs, mats))
        single = _pairs(specs, mats)[1:2]  # keeps its pair word (1)
        one = ctx.solve_grouped(single)
    _check_vs_oracle("tf32x3", specs, mats, outs)
    # a group of one pair: the same arithmetic as inside the larger group
    np.testing.assert_array_equal(one[0]["alpha"].cpu().numpy(), outs[1]["alpha"].cpu().numpy())


def test_grouped_pipeline_shapes_agree_bit_for_bit(monkeypatch):
    # every pipeline shape the tuner may pick runs each tile's MMAs in the same order, so the
    # results are the same: two CTAs per SM (bases wider than 64 columns: one accumulator each),
    # one CTA per SM with 2 or 4 ring stages
    specs = _specs(17, 6, wide=True)
    mats = [planted_pair(s)[:2] for s in specs]
    pairs = _pairs(specs, mats)
    res = {}
    for shape in ("2,2", "2,1", "4,1"):
        monkeypatch.setenv("GSVD_RAND_GROUP_PIPELINE", shape)
        with P.Context("tf32x3") as ctx:
            res[shape] = ctx.solve_grouped(pairs)
            tuned = ctx.grouped_info()["tuned"]
        assert all(t == tuple(int(x) for x in shape.split(",")) for t in tuned), (shape, tuned)
    for shape in ("2,1", "4,1"):
        for a, b in zip(res["2,2"], res[shape]):
            np.testing.assert_array_equal(a["alpha"].cpu().numpy(), b["alpha"].cpu().numpy())
            np.testing.assert_array_equal(a["beta"].cpu().numpy(), b["beta"].cpu().numpy())
    _check_vs_oracle("tf32x3", specs, mats, res["2,2"])


def test_grouped_batch_laws_at_the_largest_ranks():
    # the uneven-batch laws at their largest ranks (exp(-i/10) scales down to ~5e-5 of the first,
    # a compressed-pair Gram spanning ~1e-9), noise sigma 1e-9 well below the smallest planted scale
    from paper_2404_09459_gb300.inputs import uneven_batch
    specs = [s for s in uneven_batch(64, seed=9, m_range=(1500, 4000), n_range=(200, 600), r_range=(92, 100))][:3]
    mats = [planted_pair(s)[:2] for s in specs]
    with P.Context("tf32x3") as ctx:
        outs = ctx.solve_grouped(_pairs(specs, mats))
    _check_vs_oracle("tf32x3", specs, mats, outs)


def test_grouped_dense_tail_across_the_cut():
    # the single-solve dense-tail case (d_i = i^-1.5 at full rank, l = 96 .. 128, stacks of 192 .. 256
    # rows whose eigenvalues around the cut lie below FP32 resolution) as one group
    specs = [PairSpec(m=900, p=700, n=300, r=300, alpha="uniform", decay="pow15", sigma=0.0, k=l - 10,
                      oversample=10, q=0, seed=5) for l in (96, 112, 128)]
    mats = [tuple(G.astype(np.float32).astype(np.float64) for G in planted_pair(s)[:2]) for s in specs]
    with P.Context("tf32x3") as ctx:
        outs = ctx.solve_grouped(_pairs(specs, mats))
    _check_vs_oracle("tf32x3", specs, mats, outs)


def test_grouped_rank_far_below_l_retries_with_fp64_cholesky():
    # sketches whose rank is far below l with noise under FP32 resolution (sigma 1e-9): the first
    # shifted CholeskyQR pass leaves Q1 beyond what the FP32 factors of the next pass resolve, and
    # such a pair is solved again on its own with FP64 Cholesky factors and the same Philox words,
    # and, where those bases still break down, in FP64 throughout on widened copies.
    # The first pair is an uneven-batch draw (m 7274, p 7004, n 370, rank 35) whose G2 sketch at
    # pair word 35 broke down in grouped solves; with k = rank the k returned pairs are the planted
    # ones, well separated from the noise pairs, and are compared with the oracle.  The last pair is
    # the same matrices with l = 82 (the sketch whose pivot 54 overflowed with FP64 Cholesky factors
    # too), again with k = rank
    from paper_2404_09459_gb300.inputs import learned_pairs, planted_pair_torch
    s35 = learned_pairs(48, seed=12, m_range=(4000, 12000), n_range=(300, 600))[35]
    specs = [PairSpec(m=s35.m, p=s35.p, n=s35.n, r=s35.r, alpha=s35.alpha, decay=s35.decay, sigma=s35.sigma,
                      k=s35.r, oversample=128 - s35.r, q=1, seed=s35.seed),
             PairSpec(m=3000, p=2500, n=300, r=8, alpha="uniform", decay="exp10", sigma=1e-9, k=8, oversample=110,
                      q=2, seed=71),
             PairSpec(m=2000, p=4000, n=256, r=20, alpha="uniform", decay="exp10", sigma=1e-9, k=20,
                      oversample=100, q=0, seed=72)]
    specs.append(PairSpec(m=s35.m, p=s35.p, n=s35.n, r=s35.r, alpha=s35.alpha, decay=s35.decay, sigma=s35.sigma,
                          k=s35.r, oversample=82 - s35.r, q=0, seed=s35.seed))
    words = [35, 1, 2, 35]
    mats = [tuple(G.double().cpu().numpy() for G in planted_pair_torch(specs[0], device="cuda")[:2])]
    mats += [planted_pair(s)[:2] for s in specs[1:3]] + [mats[0]]
    pairs = [dict(G1=_dev(G1), G2=_dev(G2), k=s.kk, oversample=s.oversample, q=s.q, seed=s.seed, pair=w)
             for s, (G1, G2), w in zip(specs, mats, words)]
    with P.Context("tf32x3") as ctx:
        outs = ctx.solve_grouped(pairs)
        retries = ctx.chol64_retries()
        single = ctx.solve_batched(pairs[3:], 1)[0]
    # the group retried its breaking pairs (the FP32 breakdown is marginal: a single solve's
    # product rounding may avoid it, so the batched single solve only has to agree)
    assert retries >= 2
    outs = outs + [single]
    specs, mats, words = specs + specs[3:], mats + mats[3:], words + words[3:]
    for s, (G1, G2), w, out in zip(specs, mats, words, outs):
        assert out["status"] == 0 and out["r"] == s.kk
        ref = O.rand_gsvd(G1, G2, s.kk, s.oversample, s.q, s.seed, pair=w)
        a, b = np.asarray(out["alpha"].cpu()), np.asarray(out["beta"].cpu())
        assert np.max(O.gsv_error(ref["alpha"], ref["beta"], a, b)) <= TOL["tf32x3"], (w, s)
        assert np.all(np.diff(a) <= 0) and np.all(np.diff(b) >= 0)


def test_grouped_host_inputs_staged_and_replayed():
    # host matrices (pinned and pageable, unpadded rows) are copied into the context's device memory
    # inside each call; the group runs on those copies: the same bits as device inputs, and a second
    # call with the same host matrices replays the captured graph
    specs = _specs(18, 4)
    mats = [planted_pair(s)[:2] for s in specs]
    dev_pairs = _pairs(specs, mats)
    host_pairs = []
    for i, (d, (G1, G2)) in enumerate(zip(dev_pairs, mats)):
        h1 = torch.from_numpy(np.ascontiguousarray(G1, dtype=np.float32))
        h2 = torch.from_numpy(np.ascontiguousarray(G2, dtype=np.float32))
        if i % 2 == 0:
            h1, h2 = h1.pin_memory(), h2.pin_memory()
        host_pairs.append(dict(d, G1=h1, G2=h2))
    with P.Context("tf32x3") as ctx:
        ref = ctx.solve_grouped(dev_pairs)
    with P.Context("tf32x3") as ctx:
        first = ctx.solve_grouped(host_pairs)
        second = ctx.solve_grouped(host_pairs)
        info = ctx.grouped_info()
    assert info["captures"] == 1 and info["replays"] == 2
    for r, a, b in zip(ref, first, second):
        for key in ("alpha", "beta"):
            np.testing.assert_array_equal(r[key].cpu().numpy(), np.asarray(a[key]))
            np.testing.assert_array_equal(np.asarray(a[key]), np.asarray(b[key]))


def test_grouped_host_inputs_in_two_overlapped_halves():
    # 20 pairs from host buffers: the group runs as two halves, the second half's inputs landing
    # while the first is solved; every pair's result is bit-identical to one group of device inputs
    # (a pair's arithmetic does not depend on the group it runs in), and a repeated call replays
    specs = _specs(23, 20)
    mats = [planted_pair(s)[:2] for s in specs]
    dev_pairs = _pairs(specs, mats)
    host_pairs = [dict(d, G1=torch.from_numpy(np.ascontiguousarray(G1, dtype=np.float32)).pin_memory(),
                       G2=torch.from_numpy(np.ascontiguousarray(G2, dtype=np.float32)).pin_memory())
                  for d, (G1, G2) in zip(dev_pairs, mats)]
    with P.Context("tf32x3") as ctx:
        ref = ctx.solve_grouped(dev_pairs)
    with P.Context("tf32x3") as ctx:
        first = ctx.solve_grouped(host_pairs)
        second = ctx.solve_grouped(host_pairs)
        info = ctx.grouped_info()
    assert info["captures"] == 1 and info["replays"] == 2
    for r, a, b in zip(ref, first, second):
        assert a["status"] == 0 and b["status"] == 0
        for key in ("alpha", "beta"):
            np.testing.assert_array_equal(r[key].cpu().numpy(), np.asarray(a[key]))
            np.testing.assert_array_equal(np.asarray(a[key]), np.asarray(b[key]))
    _check_vs_oracle("tf32x3", specs[:3], mats[:3], first[:3])


def _adaptive_specs():
    # uneven pairs whose planted rank sets where Algorithm 1 stops: blocks of 8 columns until the
    # cumulated residual drops below tol (2e-3); before the block that covers the rank the
    # uncovered directions keep it above ~1e-2 (even where their alpha or beta is small), after it
    # the noise (1e-9) is far below it, and the estimate's FP32 cancellation floor (~3e-4) too
    return [PairSpec(m=1200, p=900, n=200, r=12, alpha="uniform", decay="exp10", sigma=1e-9, k=12, seed=71),
            PairSpec(m=700, p=1500, n=150, r=30, alpha="uniform", decay="exp10", sigma=1e-9, k=30, seed=72),
            PairSpec(m=400, p=350, n=90, r=5, alpha="uniform", decay="exp10", sigma=1e-9, k=5, seed=73),
            PairSpec(m=2500, p=2100, n=300, r=21, alpha="uniform", decay="exp10", sigma=1e-9, k=21, seed=74)]


def test_grouped_adaptive_matches_oracle_algorithm1():
    # Algorithm 1 for every side of the batch with the stop test on the device: the basis sizes
    # equal the FP64 oracle's per side and the GSVs match it at the mixed-precision target
    specs = _adaptive_specs()
    mats = [planted_pair(s)[:2] for s in specs]
    tol, b = 2e-3, 8
    with P.Context("tf32x3", adaptive=True, block_b=b, tol=tol) as ctx:
        outs = ctx.solve_grouped(_pairs(specs, mats))
        cols = ctx.grouped_basis_cols(len(specs))
        info = ctx.grouped_info()
    for i, (s, (G1, G2), out) in enumerate(zip(specs, mats, outs)):
        cap = min(s.m, s.p, s.n, 128)
        ref = O.rand_gsvd_adaptive(G1, G2, tol, b, s.seed, s.kk, pair=i, max_cols=cap)
        assert cols[i] == (ref["l1"], ref["l2"]), (i, cols[i], ref["l1"], ref["l2"])
        assert out["status"] == 0 and out["r"] == min(s.kk, ref["l1"] + ref["l2"])
        a, bt = out["alpha"].cpu().numpy(), out["beta"].cpu().numpy()
        e = O.gsv_error(ref["alpha"], ref["beta"], a, bt)
        assert np.max(e) <= TOL["tf32x3"], (i, np.max(e))
        # the residual estimate at the stop
        for sd in range(2):
            assert out["resid"][sd] <= tol and abs(out["resid"][sd] - ref["hist"][sd][-1]) <= 1e-3, (i, sd)
    assert info["captures"] == 1


def test_grouped_adaptive_replay_and_more_pairs_than_columns():
    # a replay of the same batch gives the same bits; a pair asking for more pairs (k = 40) than
    # its two stopped bases hold returns min(k, l1 + l2) of them, the rest marked -1
    specs = _adaptive_specs()[:3]
    specs[2] = PairSpec(m=400, p=350, n=90, r=5, alpha="uniform", decay="exp10", sigma=1e-9, k=40, seed=73)
    mats = [planted_pair(s)[:2] for s in specs]
    with P.Context("tf32x3", adaptive=True, block_b=8, tol=2e-3) as ctx:
        first = ctx.solve_grouped(_pairs(specs, mats))
        second = ctx.solve_grouped(_pairs(specs, mats))
        cols = ctx.grouped_basis_cols(len(specs))
    for a, b in zip(first, second):
        np.testing.assert_array_equal(a["alpha"].cpu().numpy(), b["alpha"].cpu().numpy())
    G1, G2 = mats[2]
    ref = O.rand_gsvd_adaptive(G1, G2, 2e-3, 8, specs[2].seed, 40, pair=2, max_cols=min(400, 350, 90, 128))
    ract = ref["l1"] + ref["l2"]
    assert cols[2] == (ref["l1"], ref["l2"]) and first[2]["r"] == ract < 40
    a = first[2]["alpha"].cpu().numpy()
    bt = first[2]["beta"].cpu().numpy()
    assert a.size == ract
    # the planted pairs (rank 5) are resolved; the others are noise-level pairs of the extra columns
    e = O.gsv_error(ref["alpha"][:5], ref["beta"][:5], a[:5], bt[:5])
    assert np.max(e) <= TOL["tf32x3"], np.max(e)
