"""GPU path vs the FP64 oracle, through the C ABI (needs a CUDA GPU).

Tolerances (stated by the method's accuracy targets): per-pair GSV error
e_i = max(|alpha_i - alpha_ref_i|, |beta_i - beta_ref_i|) <= 1e-10 on the FP64
path and <= 1e-4 on the mixed-precision paths; antisymmetric angular distance
within 1e-4 rad.  Philox words are compared bit for bit.
"""
import numpy as np
import pytest

from oracle import gsvd as O
from oracle.philox import gaussian, philox_words
from paper_2404_09459_gb300.inputs import (PAIR_FP64_SMALL, PAIR_TF32_LARGE, PairSpec, aligned_rows, full_gmp_pair,
                                          planted_pair, planted_pair_torch)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2404_09459_gb300 as P  # noqa: E402

P._build.build()

# tf32 (single-pass TF32 tensor products) truncates every operand to 10 mantissa
# bits in hardware; it is the fast mode with a looser bound.  tf32x3 is the
# mixed-precision form held to the 1e-4 target.
TOL = {"fp64": 1e-10, "fp32": 1e-4, "tf32": 1e-3, "tf32x3": 1e-4, "bf16": 1e-4}
DT = {"fp64": torch.float64}


def _dev(a, prec):
    dt = torch.float64 if prec == "fp64" else torch.float32
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt)


def _bf16(a):
    """FP64 host matrix -> BF16 CPU tensor (to nearest FP32, then to nearest BF16)."""
    return torch.from_numpy(np.ascontiguousarray(a)).to(torch.float32).to(torch.bfloat16)


def _solve(prec, G1, G2, spec, **kw):
    with P.Context(prec, **kw) as ctx:
        out = ctx.solve(_dev(G1, prec), _dev(G2, prec), spec.kk, spec.oversample, spec.q, spec.seed)
    return out["alpha"].cpu().numpy(), out["beta"].cpu().numpy(), out


def _check(prec, G1, G2, spec, ref=None, **kw):
    ref = ref or O.rand_gsvd(G1, G2, spec.kk, spec.oversample, spec.q, spec.seed)
    a, b, out = _solve(prec, G1, G2, spec, **kw)
    e = O.gsv_error(ref["alpha"], ref["beta"], a, b)
    dth = np.abs(np.arctan2(a, b) - np.arctan2(ref["alpha"], ref["beta"]))
    assert np.max(e) <= TOL[prec], (prec, np.max(e), e)
    assert np.max(dth) <= max(1e-4, TOL[prec])
    # alpha non-increasing, beta non-decreasing; within exact ties (a multiple GSV) the pairs are
    # values only, each within the mode's tolerance, so neighbours may swap by up to that much
    assert np.all(np.diff(a) <= TOL[prec]) and np.all(np.diff(b) >= -TOL[prec])
    return a, b, out, ref


# ---------------------------------------------------------------- generator

def test_philox_words_bit_exact():
    with P.Context("fp64") as ctx:
        for seed, pair, side, stream in ((0, 0, 0, 0), (123456789012345, 7, 1, 0x10003), (2**64 - 1, 2**32 - 1, 1, 5)):
            w = ctx.philox(4099, seed, pair, side, stream)
            ref = np.stack(philox_words(4099, seed, pair, side, stream), axis=1)
            np.testing.assert_array_equal(w, ref)


@pytest.mark.parametrize("n,l", [(200, 30), (97, 13), (1, 1)])
def test_gaussian_matches_oracle(n, l):
    with P.Context("fp64") as ctx:
        g = ctx.gaussian(n, l, seed=42, pair=3, side=1)
        gd = ctx.gaussian(n, l, seed=42, pair=3, side=1, device_out=True).cpu().numpy()
    ref = gaussian(n, l, 42, 3, 1)
    np.testing.assert_allclose(g, ref, rtol=0, atol=1e-13)
    np.testing.assert_array_equal(g, gd)


# ---------------------------------------------------------------- FP64 path

def test_fp64_small_pair_full_size():
    """The plain FP64 workload at its full size (m = p = 2000, n = 200, k = 20, os = 10, q = 1)."""
    G1, G2, at, bt = planted_pair(PAIR_FP64_SMALL)
    a, b, out, ref = _check("fp64", G1, G2, PAIR_FP64_SMALL)
    assert abs(out["resid"][0] - ref["resid1"]) < 1e-6 and abs(out["resid"][1] - ref["resid2"]) < 1e-6


@pytest.mark.parametrize("m,p,n,k,os_,q", [(333, 257, 97, 7, 5, 2), (130, 70, 65, 60, 4, 0),
                                          (64, 64, 64, 1, 0, 1), (1000, 90, 300, 33, 11, 3)])
def test_fp64_ragged_shapes(m, p, n, k, os_, q):
    spec = PairSpec(m=m, p=p, n=n, r=min(k + 3, n), alpha="uniform", decay="exp10", sigma=1e-7, k=k,
                    oversample=os_, q=q, seed=m + n)
    G1, G2, _, _ = planted_pair(spec)
    _check("fp64", G1, G2, spec)


def test_fp64_exact_rank_equals_planted():
    spec = PairSpec(m=500, p=400, n=150, r=15, alpha="uniform", decay="exp10", sigma=0.0, k=15,
                    oversample=5, q=1, seed=9)
    G1, G2, at, bt = planted_pair(spec)
    a, b, _ = _solve("fp64", G1, G2, spec)
    assert np.max(O.gsv_error(at, bt, a, b)) < 1e-11


def test_fp64_deterministic_and_host_buffers():
    spec = PairSpec(m=400, p=300, n=100, r=10, sigma=1e-8, k=10, oversample=6, q=1, seed=5)
    G1, G2, _, _ = planted_pair(spec)
    a1, b1, _ = _solve("fp64", G1, G2, spec)
    a2, b2, _ = _solve("fp64", G1, G2, spec)
    np.testing.assert_array_equal(a1, a2)
    with P.Context("fp64") as ctx:  # host (numpy) inputs and outputs
        out = ctx.solve(G1, G2, spec.kk, spec.oversample, spec.q, spec.seed)
    assert isinstance(out["alpha"], np.ndarray)
    np.testing.assert_array_equal(out["alpha"], a1)
    np.testing.assert_array_equal(out["beta"], b1)


# ---------------------------------------------------------------- mixed paths

def test_fp32_simt_reduced_large_pair():
    spec = PairSpec(m=4000, p=3000, n=400, r=30, alpha="uniform", decay="exp10", sigma=1e-6, k=30,
                    oversample=10, q=2, seed=2)
    G1, G2, _, _ = planted_pair(spec)
    _check("fp32", G1, G2, spec)


@pytest.mark.parametrize("prec", ["tf32x3", "tf32"])
@pytest.mark.parametrize("m,p,n,k,os_,q", [(4000, 3000, 400, 30, 10, 2), (1000, 777, 200, 50, 14, 1),
                                          (130, 300, 36, 5, 3, 3)])
def test_tensor_core_ragged(prec, m, p, n, k, os_, q):
    spec = PairSpec(m=m, p=p, n=n, r=min(k + 2, n), alpha="uniform", decay="exp10", sigma=1e-6, k=k,
                    oversample=os_, q=q, seed=m + p)
    G1, G2, _, _ = planted_pair(spec)
    _check(prec, G1, G2, spec)


def _odd_ld(a):
    """FP32 device matrix whose row stride (n + 1 floats) is not a multiple of 16 bytes: the
    tensor-core products cannot read it through TMA, so the solve takes the CUDA-core products."""
    t = torch.empty((a.shape[0], a.shape[1] + 1), dtype=torch.float32, device="cuda")
    t[:, :a.shape[1]] = torch.from_numpy(np.ascontiguousarray(a)).to("cuda", torch.float32)
    return t[:, :a.shape[1]]


# every layout the solve records its bases in: FP64 row-major Q (fp64), FP32 row-major Q (fp32,
# and tf32 on an unaligned input, which takes the CUDA-core products), FP32 transposed Q (tf32x3,
# bf16 with BF16 storage of G)
@pytest.mark.parametrize("prec,layout", [("fp64", "plain"), ("tf32x3", "plain"), ("fp32", "plain"),
                                         ("tf32", "odd_ld"), ("bf16", "plain")])
def test_gsvd_factors_match_oracle(prec, layout):
    # U, V, R of the recovery after Algorithm 2: the products U diag(alpha) R and V diag(beta) R
    # do not depend on the bases' rotations, so they are compared with the oracle's element by
    # element; U and V have orthonormal columns
    spec = PairSpec(m=3000, p=2500, n=300, r=20, alpha="uniform", decay="exp10", sigma=1e-8, k=20,
                    oversample=8, q=1, seed=41)
    G1, G2, _, _ = planted_pair(spec)
    if prec == "bf16":
        # parity on the BF16-rounded pair with the BF16-rounded Omega (the mode's own inputs)
        G1, G2 = (O.round_bf16(G).astype(np.float64) for G in (G1, G2))
        ref = O.rand_gsvd_factors(G1, G2, 20, 8, 1, spec.seed, omega_round="bf16")
        g1, g2 = (torch.from_numpy(np.ascontiguousarray(G)).to("cuda", torch.float32).to(torch.bfloat16)
                  for G in (G1, G2))
    else:
        ref = O.rand_gsvd_factors(G1, G2, 20, 8, 1, spec.seed)
        g1, g2 = ((_odd_ld(G) if layout == "odd_ld" else _dev(G, prec)) for G in (G1, G2))
    flags = P.FLAG_BF16_SPLIT_POWER if prec == "bf16" else 0
    with P.Context(prec, flags=flags) as ctx:
        out = ctx.solve(g1, g2, 20, 8, 1, spec.seed)
        f = ctx.factors()
        U, V, R = (f[x].cpu().numpy() for x in "UVR")
        a, b = out["alpha"].cpu().numpy(), out["beta"].cpu().numpy()
        ctx.metrics(out["alpha"], out["beta"])  # takes the workspace: the factors are gone
        with pytest.raises(P.GsvdRandError) as e:
            ctx.factors()
        assert e.value.name == "ARG"
    assert U.shape == (3000, 20) and V.shape == (2500, 20) and R.shape == (20, 300)
    assert np.max(O.gsv_error(ref["alpha"], ref["beta"], a, b)) <= TOL[prec]
    tol = TOL[prec]
    for F, s, Fr, sr, G in ((U, a, ref["U"], ref["alpha"], G1), (V, b, ref["V"], ref["beta"], G2)):
        rec, rec_ref = (F * s) @ R, (Fr * sr) @ ref["R"]
        assert np.linalg.norm(rec - rec_ref) <= tol * np.linalg.norm(G), np.linalg.norm(rec - rec_ref)
        keep = s > 1e-3
        otol = 1e-9 if prec == "fp64" else 1e-4  # the bases' orthonormality: FP64 or FP32 Q
        assert np.max(np.abs(F[:, keep].T @ F[:, keep] - np.eye(keep.sum()))) <= otol


def test_single_solve_product_shapes_tuned_and_pinned_agree(monkeypatch):
    # a single solve's two-side products are tuned like the grouped ones (pipeline depth, one or
    # two CTAs per SM); every shape runs each tile's MMAs in the same order: the same bits
    spec = PairSpec(m=4000, p=3000, n=400, r=30, alpha="uniform", decay="exp10", sigma=1e-6, k=30,
                    oversample=10, q=1, seed=21)
    G1, G2, _, _ = planted_pair(spec)
    res = {}
    for shape in (None, "2,2", "4,1"):
        if shape:
            monkeypatch.setenv("GSVD_RAND_GROUP_PIPELINE", shape)
        with P.Context("tf32x3") as ctx:
            out = ctx.solve(_dev(G1, "tf32x3"), _dev(G2, "tf32x3"), 30, 10, 1, 21)
            shapes = ctx.product_shapes()
        if shape:
            assert all(sh == tuple(int(x) for x in shape.split(",")) for sh in shapes), shapes
        else:
            assert all(sh[0] >= 2 and sh[1] in (1, 2) for sh in shapes), shapes
        res[shape] = out["alpha"].cpu().numpy()
    np.testing.assert_array_equal(res[None], res["2,2"])
    np.testing.assert_array_equal(res[None], res["4,1"])


def test_tf32x3_unaligned_rows_use_cuda_cores():
    # n = 97: a row stride TMA cannot address; device inputs then run the FP32 CUDA-core products
    spec = PairSpec(m=500, p=400, n=97, r=12, sigma=1e-6, k=12, oversample=6, q=1, seed=4)
    G1, G2, _, _ = planted_pair(spec)
    _check("tf32x3", G1, G2, spec)


@pytest.mark.parametrize("prec,m,p,n,k,os_", [("tf32x3", 3000, 2500, 400, 70, 10), ("fp64", 6000, 5000, 300, 20, 8)])
def test_separate_kernel_cholqr(prec, m, p, n, k, os_):
    # l = 80 > 64 (mixed) and 6000-row FP64 sides: CholeskyQR2 as separate kernels instead of the
    # single persistent kernel
    spec = PairSpec(m=m, p=p, n=n, r=k + 2, alpha="uniform", decay="exp10", sigma=1e-7, k=k, oversample=os_,
                    q=1, seed=m)
    G1, G2, _, _ = planted_pair(spec)
    _check(prec, G1, G2, spec)


# Algorithm 1 bases.  The pairs are chosen so that the cumulated residual falls from above
# 1e-2 to far below tol within one block on both sides (the stop is an integer decision
# taken from floating-point values computed differently on each side).
ADAPTIVE_CASES = [
    ("fp64", PairSpec(m=1500, p=1200, n=300, r=40, alpha="uniform", decay="exp10", sigma=1e-12, seed=31), 16, 1e-6, 40),
    ("tf32x3", PairSpec(m=3000, p=2500, n=400, r=30, alpha="uniform", decay="exp10", sigma=1e-8, seed=32), 12, 1e-3, 30),
    ("tf32x3", PairSpec(m=4000, p=3000, n=500, r=60, alpha="uniform", decay="exp10", sigma=1e-8, seed=33), 64, 1e-3, 60),
    # b = 100 (the paper's block): separate-kernel CholeskyQR and a 200 x 200 small eigenproblem
    ("tf32x3", PairSpec(m=5000, p=4000, n=600, r=90, alpha="uniform", decay="logspace02", sigma=1e-8, seed=34), 100, 1e-3, 90),
]


@pytest.mark.parametrize("prec,spec,b,tol,k", ADAPTIVE_CASES)
def test_adaptive_basis_matches_oracle(prec, spec, b, tol, k):
    G1, G2, _, _ = planted_pair(spec)
    ref = O.rand_gsvd_adaptive(G1, G2, tol=tol, b=b, seed=7, r=k)
    with P.Context(prec, adaptive=True, block_b=b, tol=tol) as ctx:
        out = ctx.solve(_dev(G1, prec), _dev(G2, prec), k, 0, 0, 7)
        l1, l2 = ctx.basis_cols()
    assert (l1, l2) == (ref["l1"], ref["l2"])
    assert out["r"] == min(k, l1 + l2)
    a, b_ = out["alpha"].cpu().numpy(), out["beta"].cpu().numpy()
    e = O.gsv_error(ref["alpha"], ref["beta"], a, b_)
    assert np.max(e) <= TOL[prec], np.max(e)
    assert max(out["resid"]) <= tol


@pytest.mark.parametrize("prec,sigma,q", [("fp64", 1e-12, 1), ("fp64", 1e-12, 0), ("fp32", 1e-8, 0), ("tf32x3", 1e-8, 0),
                                           ("tf32x3", 0.0, 0)])
def test_rank_deficient_sketch(prec, sigma, q):
    # k equals the planted rank and the oversampled columns see only noise below the data's
    # precision (or none): the sketch is numerically rank-deficient.  Small Householder
    # columns must not overflow the reflector, and no weak direction may leave the basis.
    spec = PairSpec(m=4000, p=3000, n=500, r=60, alpha="uniform", decay="exp10", sigma=sigma, k=60,
                    oversample=4, q=q, seed=33)
    G1, G2, _, _ = planted_pair(spec)
    _check(prec, G1, G2, spec)


def _batch_specs(count, seed):
    rng = np.random.default_rng(seed)
    specs = []
    for i in range(count):
        m, p = (int(x) for x in rng.integers(400, 3000, 2))
        n = int(rng.integers(100, 400))
        r = int(rng.integers(5, 40))
        specs.append(PairSpec(m=m, p=p, n=n, r=r, alpha="uniform", decay="exp10", sigma=1e-6, k=r,
                              oversample=8, q=1, seed=100 + i))
    return specs


@pytest.mark.parametrize("prec", ["fp64", "tf32x3"])
def test_batched_uneven_pairs_match_oracle(prec):
    specs = _batch_specs(10, 5 if prec == "fp64" else 6)
    mats = [planted_pair(s)[:2] for s in specs]
    pairs = [dict(G1=_dev(G1, prec), G2=_dev(G2, prec), k=s.kk, oversample=s.oversample, q=s.q, seed=s.seed,
                  pair=i) for i, (s, (G1, G2)) in enumerate(zip(specs, mats))]
    with P.Context(prec) as ctx:
        outs = ctx.solve_batched(pairs, workers=4)
        again = ctx.solve_batched(pairs, workers=3)
    for i, (s, (G1, G2), out) in enumerate(zip(specs, mats, outs)):
        assert out["status"] == 0 and out["r"] == s.kk
        ref = O.rand_gsvd(G1, G2, s.kk, s.oversample, s.q, s.seed, pair=i)
        e = O.gsv_error(ref["alpha"], ref["beta"], out["alpha"].cpu().numpy(), out["beta"].cpu().numpy())
        assert np.max(e) <= TOL[prec], (i, np.max(e))
        np.testing.assert_array_equal(out["alpha"].cpu().numpy(), again[i]["alpha"].cpu().numpy())


def test_batched_equals_single_solves_and_reports_per_pair_status():
    specs = _batch_specs(5, 7)
    mats = [planted_pair(s)[:2] for s in specs]
    pairs = [dict(G1=_dev(G1, "tf32x3"), G2=_dev(G2, "tf32x3"), k=s.kk, oversample=s.oversample, q=s.q,
                  seed=s.seed, pair=0) for s, (G1, G2) in zip(specs, mats)]
    with P.Context("tf32x3") as ctx:
        outs = ctx.solve_batched(pairs, workers=2)
        for s, (G1, G2), out in zip(specs, mats, outs):
            single = ctx.solve(_dev(G1, "tf32x3"), _dev(G2, "tf32x3"), s.kk, s.oversample, s.q, s.seed)
            np.testing.assert_array_equal(single["alpha"].cpu().numpy(), out["alpha"].cpu().numpy())
        # one bad pair (k + oversample > n) fails alone; the others still run
        bad = dict(pairs[1])
        bad["k"] = 500
        with pytest.raises(P.GsvdRandError) as e:
            ctx.solve_batched([pairs[0], bad, pairs[2]], workers=2)
        assert e.value.name == "ARG"


@pytest.mark.parametrize("prec,q", [("fp64", 0), ("tf32x3", 1), ("fp64", 1)])
def test_paper_full_pair_workload(prec, q):
    # Section 4.1's synthetic pair: rank(G1) = rank(G2) = 60 of n = 100, 40 pairs (1, 0), 40 pairs
    # (0, 1), 20 uniform; the stack has full rank, so all n pairs are resolved (k = n, no
    # oversampling: each side's sketch has exact rank 60 in a basis of 100, L = 200).  The FP32
    # eigensolver start replaces the vectors it sets aside in a multiple eigenvalue (here the 40-fold
    # 1 and 0 of Z1^T Z1) by inverse iteration within that eigenspace.
    G1, G2, a, b = full_gmp_pair(300, 260, 100, seed=3)
    if prec != "fp64":  # the oracle takes the FP32-stored pair the GPU reads
        G1, G2 = G1.astype(np.float32).astype(np.float64), G2.astype(np.float32).astype(np.float64)
    spec = PairSpec(m=300, p=260, n=100, r=100, k=100, oversample=0, q=q, seed=11)
    al, be, out, ref = _check(prec, G1, G2, spec)
    assert out["r"] == 100
    # the exact blocks: within the mode's tolerance of the planted 1s and 0s
    tol = 1e-10 if prec == "fp64" else 1e-4
    assert np.max(np.abs(al[:40] - 1.0)) <= tol and np.max(np.abs(be[:40])) <= tol
    assert np.max(np.abs(al[60:])) <= tol and np.max(np.abs(be[60:] - 1.0)) <= tol


@pytest.mark.parametrize("l", [80, 96, 112, 128])
@pytest.mark.parametrize("prec", ["fp32", "tf32x3"])
def test_dense_tail_across_the_cut(prec, l):
    # slow decay d_i = i^-1.5 at full rank: the k-th singular value of the stack is 1e-3 .. 8e-4 of
    # the first, so the eigenvalues of K = S S^T around the cut (k-th and (k+1)-th) lie near 1e-6 of
    # the largest, below what the FP32 eigensolver start resolves, and a dense run of them (the
    # whole tail of K, L - k + a few tens of columns, more than 128 for l >= 96) has to be split
    # across the cut in the refinement
    spec = PairSpec(m=900, p=700, n=300, r=300, alpha="uniform", decay="pow15", sigma=0.0, k=l - 10,
                    oversample=10, q=0, seed=5)
    G1, G2, _, _ = planted_pair(spec)
    G1, G2 = G1.astype(np.float32).astype(np.float64), G2.astype(np.float32).astype(np.float64)
    _check(prec, G1, G2, spec)


def test_fp32_cholesky_breakdown_repeated_with_fp64_factors():
    # rank 19 in a basis of 29 with the noise (1e-9) under FP32 resolution: kappa(Y) ~ 1e6, so
    # the first shifted CholeskyQR pass can leave Q1 beyond what an FP32 Gram resolves; the FP32
    # factors of the next pass then break down and the solve is repeated with FP64 factors.
    # This draw (built on the device, as the batch bench builds it) broke down in FP32 on GB300.
    spec = PairSpec(m=6845, p=19105, n=267, r=19, alpha="uniform", decay="exp10", sigma=1e-9, k=19,
                    oversample=10, q=1, seed=100018)
    G1, G2 = (aligned_rows(G) for G in planted_pair_torch(spec, device="cuda", dtype=torch.float32)[:2])
    pair = dict(G1=G1, G2=G2, k=19, oversample=10, q=1, seed=spec.seed, pair=15)
    with P.Context("tf32x3") as ctx:
        out = ctx.solve_batched([pair], workers=1)[0]
        retries = ctx.chol64_retries()
    with P.Context("tf32x3", flags=P.FLAG_CHOL_FP64) as ctx:
        f64 = ctx.solve_batched([pair], workers=1)[0]
        assert ctx.chol64_retries() == 0
    assert retries in (0, 1, 2)
    if retries == 1:
        # the repeated solve is the FP64-factor solve
        np.testing.assert_array_equal(out["alpha"].cpu().numpy(), f64["alpha"].cpu().numpy())
    ref = O.rand_gsvd(G1.double().cpu().numpy(), G2.double().cpu().numpy(), 19, 10, 1, spec.seed, pair=15)
    for o in (out, f64):
        e = O.gsv_error(ref["alpha"], ref["beta"], o["alpha"].cpu().numpy(), o["beta"].cpu().numpy())
        assert np.max(e) <= TOL["tf32x3"], np.max(e)
    # an input NaN breaks every form: repeated with FP64 factors, then in FP64 throughout on
    # widened copies, then reported
    bad = G1.clone()
    bad[3, 7] = float("nan")
    with P.Context("tf32x3") as ctx:
        with pytest.raises(P.GsvdRandError) as e:
            ctx.solve(bad, G2, 19, 10, 1, spec.seed)
        assert e.value.name == "NONFINITE"
        assert ctx.chol64_retries() == 2


def test_adaptive_cap_reached_reports_tol_miss():
    # 256-column cap below n = 300 with a noisy pair: the tolerance cannot be met
    spec = PairSpec(m=600, p=500, n=300, r=20, sigma=1e-2, seed=35)
    G1, G2, _, _ = planted_pair(spec)
    with P.Context("fp64", adaptive=True, block_b=64, tol=1e-6) as ctx:
        with pytest.raises(P.GsvdRandError) as e:
            ctx.solve(_dev(G1, "fp64"), _dev(G2, "fp64"), 20, 0, 0, 1)
        assert e.value.name == "TOL_MISS"
        assert ctx.basis_cols() == (256, 256)


def test_bf16_adaptive_refused_and_unaligned_inputs_staged():
    spec = PairSpec(m=200, p=200, n=64, r=5, sigma=1e-6, k=5, oversample=3, q=1, seed=4)
    G1, G2, _, _ = planted_pair(spec)
    g1, g2 = _bf16(G1).cuda(), _bf16(G2).cuda()
    with P.Context("bf16", adaptive=1, block_b=8, tol=1e-2) as ctx:
        with pytest.raises(P.GsvdRandError) as e:
            ctx.solve(g1, g2, 5, 0, 0, 1)
    assert e.value.name == "UNSUPPORTED"
    wide = torch.zeros(200, 68, dtype=torch.bfloat16, device="cuda")
    wide[:, 1:65] = g1
    with P.Context("bf16") as ctx:
        ref = ctx.solve(g1, g2, 5, 3, 1, 4)
        # base 2 bytes past a 16-byte boundary: staged into the workspace, same result
        got = ctx.solve(wide[:, 1:65], g2, 5, 3, 1, 4)
        host = ctx.solve(_bf16(G1), _bf16(G2), 5, 3, 1, 4)
    torch.testing.assert_close(got["alpha"], ref["alpha"], rtol=0, atol=0)
    np.testing.assert_array_equal(host["alpha"], ref["alpha"].cpu().numpy())


def test_tf32x3_large_pair_full_size():
    """The single large pair at full size (m = 20000, p = 15000, n = 1000, k = 50, os = 10, q = 2),
    in the mixed-precision form the benchmark times (3xTF32 tensor products)."""
    G1, G2, _, _ = planted_pair(PAIR_TF32_LARGE)
    ref = O.rand_gsvd(G1, G2, PAIR_TF32_LARGE.kk, PAIR_TF32_LARGE.oversample, PAIR_TF32_LARGE.q,
                      PAIR_TF32_LARGE.seed)
    _check("tf32x3", G1, G2, PAIR_TF32_LARGE, ref=ref)
    _check("tf32", G1, G2, PAIR_TF32_LARGE, ref=ref)


# ---------------------------------------------------------------- wide compressed pairs
# L = l1 + l2 above 128 runs the packed-triangle eigensolver (shared memory up to
# L = 318, global scratch above).

@pytest.mark.parametrize("prec,m,p,n,k,os_,q", [
    ("fp64", 3000, 2600, 400, 90, 10, 1),      # L = 200
    ("tf32x3", 5000, 4100, 600, 110, 14, 1),   # L = 248
    ("fp32", 3000, 2500, 500, 170, 10, 1),     # L = 360: matrix in global scratch
    ("tf32x3", 4000, 3500, 600, 140, 12, 1),   # l = 152 > 128: Q = Y R^-1 on the tensor cores
], ids=["L200-fp64", "L248-tf32x3", "L360-fp32", "l152-tf32x3"])
def test_wide_compressed_pair(prec, m, p, n, k, os_, q):
    # scale law logspace(0, 2) over r = k planted pairs: every returned pair is a signal pair well
    # above the noise (a noise-determined pair has an arbitrary alpha and would interleave with the
    # others in the sorted output); the oversampled columns carry noise only, so the eigensolver's
    # noise-complement path runs too
    spec = PairSpec(m=m, p=p, n=n, r=k, alpha="uniform", decay="logspace02", sigma=1e-7, k=k, oversample=os_, q=q,
                    seed=m + k)
    G1, G2, _, _ = planted_pair(spec)
    ref = O.rand_gsvd(G1, G2, spec.kk, spec.oversample, spec.q, spec.seed)
    a, b, _ = _solve(prec, G1, G2, spec)
    e = O.gsv_error(ref["alpha"], ref["beta"], a, b)
    assert np.max(e) <= TOL[prec], (np.max(e), e)
    assert np.all(np.diff(a) <= 0) and np.all(np.diff(b) >= 0)
    assert np.max(np.abs(a ** 2 + b ** 2 - 1)) < 1e-10


# ---------------------------------------------------------------- BF16 mode
# G is stored in BF16.  Parity is against the oracle run on the same BF16-rounded G
# (converted exactly to FP64) with the same BF16-rounded Omega, so that the error is
# that of the GPU arithmetic: FP32 accumulation, FP32 CholeskyQR data and the power
# steps' BF16 operands.  The storage error itself (vs the unrounded FP64 pair) is
# the precision stress the bench reports; it is not a parity quantity.

def _check_bf16(G1, G2, spec, flags=0, gate=None):
    b1, b2 = _bf16(G1), _bf16(G2)
    ref = O.rand_gsvd(b1.double().numpy(), b2.double().numpy(), spec.kk, spec.oversample, spec.q, spec.seed,
                      omega_round="bf16")
    with P.Context("bf16", flags=flags) as ctx:
        out = ctx.solve(b1.cuda(), b2.cuda(), spec.kk, spec.oversample, spec.q, spec.seed)
    a, b = out["alpha"].cpu().numpy(), out["beta"].cpu().numpy()
    gate = spec.kk if gate is None else gate
    e = O.gsv_error(ref["alpha"], ref["beta"], a, b)[:gate]
    dth = np.abs(np.arctan2(a, b) - np.arctan2(ref["alpha"], ref["beta"]))[:gate]
    assert np.max(e) <= TOL["bf16"], (np.max(e), e)
    assert np.max(dth) <= 1e-4
    assert np.all(np.diff(a) <= 0) and np.all(np.diff(b) >= 0)
    return a, b, ref


BF16_CASES = [
    PairSpec(m=3000, p=2500, n=300, r=12, alpha="uniform", decay="exp10", sigma=1e-6, k=12, oversample=8, q=1,
             seed=1),  # n not a multiple of 8: G staged into an aligned copy
    PairSpec(m=4100, p=3000, n=520, r=20, alpha="uniform", decay="exp10", sigma=1e-6, k=20, oversample=10, q=2,
             seed=2),  # ragged row tiles and K tail
    PairSpec(m=2000, p=1800, n=200, r=20, alpha="uniform", decay="exp10", sigma=1e-6, k=20, oversample=10, q=0,
             seed=3),  # projection straight after the sketch
]


@pytest.mark.parametrize("flags", [0, P.FLAG_BF16_SPLIT_POWER])
@pytest.mark.parametrize("spec", BF16_CASES, ids=lambda s: f"m{s.m}n{s.n}q{s.q}")
def test_bf16_matches_oracle_on_rounded_inputs(spec, flags):
    G1, G2, _, _ = planted_pair(spec)
    _check_bf16(G1, G2, spec, flags)


def test_bf16_slow_decay_gated_above_noise_floor():
    """Slow decay d_i = i^-1.5 with sigma = 1e-5: pairs whose scale is below ten times the
    noise floor sigma (sqrt(M) + sqrt(n)) are noise-determined and not gated."""
    spec = PairSpec(m=5000, p=4000, n=777, r=50, alpha="uniform", decay="pow15", sigma=1e-5, k=50,
                    oversample=14, q=2, seed=4)
    G1, G2, _, _ = planted_pair(spec)
    floor = spec.sigma * (np.sqrt(spec.m) + np.sqrt(spec.n))
    gate = int(np.sum(np.arange(1, spec.r + 1) ** -1.5 >= 10 * floor))
    assert gate >= 15
    for flags in (0, P.FLAG_BF16_SPLIT_POWER):
        _check_bf16(G1, G2, spec, flags, gate=gate)


def test_bf16_large_pair_full_size():
    """The single large pair (m = 20000, p = 15000, n = 1000, k = 50, os = 10, q = 2) stored in BF16."""
    G1, G2, _, _ = planted_pair(PAIR_TF32_LARGE)
    _check_bf16(G1, G2, PAIR_TF32_LARGE)
    _check_bf16(G1, G2, PAIR_TF32_LARGE, P.FLAG_BF16_SPLIT_POWER)


def test_bf16_stress_full_size():
    """The precision-stress pair at full size (m = 120000, p = 80000, n = 4000, r = 200, d_i = i^-1.5,
    sigma = 1e-4, k = 200, os = 20, q = 3; l = 220, L = 440) with G in BF16 and split power steps.
    The noise floor sigma (sqrt(m) + sqrt(n)) = 0.041 buries all but the leading pairs: those with
    d_i >= 10x the floor are held to 1e-4, the noise-determined rest is checked for validity."""
    from paper_2404_09459_gb300.inputs import PAIR_BF16_STRESS as S, planted_pair_torch
    G1, G2, _, _ = planted_pair_torch(S)
    b1, b2 = G1.to(torch.bfloat16), G2.to(torch.bfloat16)
    del G1, G2
    with P.Context("bf16", flags=P.FLAG_BF16_SPLIT_POWER) as ctx:
        out = ctx.solve(b1, b2, S.kk, S.oversample, S.q, S.seed)
    a, b = out["alpha"].cpu().numpy(), out["beta"].cpu().numpy()
    ref = O.rand_gsvd(b1.double().cpu().numpy(), b2.double().cpu().numpy(), S.kk, S.oversample, S.q, S.seed,
                      omega_round="bf16")
    floor = S.sigma * (np.sqrt(S.m) + np.sqrt(S.n))
    gate = int(np.sum(np.arange(1, S.r + 1) ** -1.5 >= 10 * floor))
    e = O.gsv_error(ref["alpha"], ref["beta"], a, b)
    assert gate >= 1 and np.max(e[:gate]) <= TOL["bf16"], e[:gate]
    assert np.all(np.diff(a) <= 0) and np.all(np.diff(b) >= 0)
    assert np.all((a >= 0) & (a <= 1 + 1e-12) & (b >= 0) & (b <= 1 + 1e-12))
    assert np.max(np.abs(a ** 2 + b ** 2 - 1)) < 1e-10
    # noise-determined pairs: reported, held only to ten times the target (measured max 1.3e-4)
    assert np.max(e) <= 10 * TOL["bf16"], (np.max(e), np.median(e))


# ---------------------------------------------------------------- metrics

@pytest.mark.parametrize("pad_to_n,pad_mode", [(0, 0), (40, 0), (40, 1)])
def test_metrics_match_oracle(pad_to_n, pad_mode):
    rng = np.random.default_rng(3)
    a = np.ascontiguousarray(np.sort(rng.uniform(0, 1, 17))[::-1])
    a[0] = 1.0
    b = np.sqrt(1 - a ** 2)
    ref = O.metrics(a, b, pad_to_n, pad_mode)
    with P.Context("fp64") as ctx:
        got = ctx.metrics(a, b, pad_to_n, pad_mode)
        gd = ctx.metrics(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), pad_to_n, pad_mode)
    for key in ("theta", "P1", "P2"):
        np.testing.assert_allclose(got[key], ref[key], rtol=0, atol=1e-14)
        np.testing.assert_allclose(gd[key].cpu().numpy(), ref[key], rtol=0, atol=1e-14)
    fin = np.isfinite(ref["rho"])
    np.testing.assert_allclose(got["rho"][fin], ref["rho"][fin], rtol=1e-14)
    assert np.all(np.isinf(got["rho"][~fin]))
    assert abs(float(got["D1"]) - ref["D1"]) < 1e-14 and abs(float(got["D2"]) - ref["D2"]) < 1e-14


# ---------------------------------------------------------------- errors

def test_error_codes():
    spec = PairSpec(m=100, p=80, n=40, r=5, sigma=0.0, k=5, oversample=3, q=1, seed=1)
    G1, G2, _, _ = planted_pair(spec)
    with P.Context("fp64") as ctx:
        with pytest.raises(P.GsvdRandError) as e:
            ctx.solve(_dev(G1, "fp64"), _dev(G2, "fp64"), 38, 10, 1, 0)  # l > n
        assert e.value.name == "ARG"
        with pytest.raises(P.GsvdRandError) as e:
            ctx.solve(_dev(np.zeros_like(G1), "fp64"), _dev(G2, "fp64"), 5, 3, 1, 0)
        assert e.value.name == "BREAKDOWN"
        bad = G1.copy()
        bad[3, 7] = np.nan
        with pytest.raises(P.GsvdRandError) as e:
            ctx.solve(_dev(bad, "fp64"), _dev(G2, "fp64"), 5, 3, 1, 0)
        assert e.value.name == "NONFINITE"
        # the context stays usable after device-reported errors
        out = ctx.solve(_dev(G1, "fp64"), _dev(G2, "fp64"), 5, 3, 1, 0)
        assert out["r"] == 5
        with pytest.raises(P.GsvdRandError) as e:
            ctx.metrics(np.array([1.0]), np.array([0.0]))
        assert e.value.name == "ARG"


def test_bf16_low_noise_config3_shape():
    """The precision-stress shape (m = 120000, p = 80000, n = 4000, r = 200, d_i = i^-1.5, k = 200,
    os = 20, q = 3; L = 440) at low noise, sigma = 1e-7: the noise floor sigma (sqrt(m) + sqrt(n))
    = 4.1e-5 lies below the planted tail (d_200 = 3.5e-4), so most pairs are resolved and gated, and
    the cut between the 200th and 201st eigenvalue of K (about 1e-7 of the largest apart from the
    noise) lies below FP32 resolution."""
    from paper_2404_09459_gb300.inputs import PAIR_BF16_STRESS
    from dataclasses import replace
    S = replace(PAIR_BF16_STRESS, sigma=1e-7, seed=7)
    G1, G2, _, _ = planted_pair_torch(S)
    b1, b2 = G1.to(torch.bfloat16), G2.to(torch.bfloat16)
    del G1, G2
    with P.Context("bf16", flags=P.FLAG_BF16_SPLIT_POWER) as ctx:
        out = ctx.solve(b1, b2, S.kk, S.oversample, S.q, S.seed)
    a, b = out["alpha"].cpu().numpy(), out["beta"].cpu().numpy()
    ref = O.rand_gsvd(b1.double().cpu().numpy(), b2.double().cpu().numpy(), S.kk, S.oversample, S.q, S.seed,
                      omega_round="bf16")
    floor = S.sigma * (np.sqrt(S.m) + np.sqrt(S.n))
    gate = int(np.sum(np.arange(1, S.r + 1) ** -1.5 >= 10 * floor))
    e = O.gsv_error(ref["alpha"], ref["beta"], a, b)
    print("gate", gate, "max", e[:gate].max(), "per decile", [float(e[i:i + 20].max()) for i in range(0, 200, 20)])
    assert gate >= 20
    assert np.max(e[:gate]) <= TOL["bf16"], (gate, np.max(e[:gate]), np.argmax(e[:gate]))
    dth = np.abs(np.arctan2(a, b) - np.arctan2(ref["alpha"], ref["beta"]))[:gate]
    assert np.max(dth) <= 1e-4
