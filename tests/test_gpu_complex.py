"""Complex pairs (Section 1's GSVD over C; Section 4.1's complex synthetic pairs) on the GPU
against the complex FP64 oracle, through the C ABI (needs a CUDA GPU).

Tolerances as for real pairs: per-pair GSV error e_i = max(|alpha_i - alpha_ref_i|,
|beta_i - beta_ref_i|) <= 1e-10 on the FP64 path, <= 1e-4 on the 3xTF32 and FP32 paths, 1e-3
with single-pass TF32; antisymmetric angular distance within 1e-4 rad.  The oracle runs the
complex method directly (complex Householder QR and SVD); the library runs the realified pair.
"""
import numpy as np
import pytest

from oracle import gsvd as O
from paper_2404_09459_gb300.inputs import PairSpec, full_gmp_pair_complex, planted_pair_complex

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2404_09459_gb300 as P  # noqa: E402

P._build.build()

TOL = {"fp64": 1e-10, "fp32": 1e-4, "tf32": 1e-3, "tf32x3": 1e-4}


def _inputs(G1, G2, prec):
    """The stored pair the GPU reads and the same pair for the oracle (complex64 rounding on the
    mixed paths)."""
    if prec == "fp64":
        return G1, G2, G1, G2
    c1, c2 = G1.astype(np.complex64), G2.astype(np.complex64)
    return c1, c2, c1.astype(np.complex128), c2.astype(np.complex128)


def _check(prec, G1, G2, k, os_, q, seed, device=True):
    g1, g2, o1, o2 = _inputs(G1, G2, prec)
    ref = O.rand_gsvd_complex(o1, o2, k, os_, q, seed)
    if device:
        g1, g2 = torch.from_numpy(np.ascontiguousarray(g1)).cuda(), torch.from_numpy(np.ascontiguousarray(g2)).cuda()
    with P.Context(prec) as ctx:
        out = ctx.solve_complex(g1, g2, k, os_, q, seed)
    a = np.asarray(out["alpha"].cpu() if hasattr(out["alpha"], "cpu") else out["alpha"])
    b = np.asarray(out["beta"].cpu() if hasattr(out["beta"], "cpu") else out["beta"])
    assert out["r"] == k
    e = O.gsv_error(ref["alpha"], ref["beta"], a, b)
    assert np.max(e) <= TOL[prec], (prec, np.max(e), e)
    dth = np.abs(np.arctan2(a, b) - np.arctan2(ref["alpha"], ref["beta"]))
    assert np.max(dth) <= max(1e-4, TOL[prec])
    assert np.all(np.diff(a) <= TOL[prec]) and np.all(np.diff(b) >= -TOL[prec])
    # the cumulated residual of the realified pair is the complex pair's (||rho(M)||_F^2 = 2 ||M||_F^2);
    # ||B||^2 carries the products' relative error, so it is held on the squared scale (2^-10 for
    # single-pass TF32, as for real pairs)
    rtol = 1e-8 if prec == "fp64" else (4e-3 if prec == "tf32" else 1e-4)
    for s in range(2):
        assert abs(out["resid"][s] ** 2 - ref[f"resid{s + 1}"] ** 2) <= rtol, (s, out["resid"], ref[f"resid{s + 1}"])
    return a, b, ref


@pytest.mark.parametrize("q", [0, 1, 2])
@pytest.mark.parametrize("prec", ["fp64", "tf32x3", "fp32", "tf32"])
def test_complex_planted_pair_matches_oracle(prec, q):
    spec = PairSpec(m=700, p=520, n=150, r=14, alpha="uniform", decay="exp10", sigma=1e-8, k=14, oversample=8,
                    q=q, seed=61)
    G1, G2, _, _ = planted_pair_complex(spec)
    _check(prec, G1, G2, 14, 8, q, seed=17)


@pytest.mark.parametrize("prec", ["fp64", "tf32x3"])
def test_complex_ragged_shapes(prec):
    # odd n (rows of the realified matrix 2n), few rows per basis column, l close to n
    for (m, p, n, r, k, os_, q) in ((301, 257, 101, 9, 9, 6, 1), (90, 70, 40, 10, 10, 20, 1), (64, 200, 33, 5, 5, 3, 2)):
        spec = PairSpec(m=m, p=p, n=n, r=r, alpha="uniform", decay="exp10", sigma=1e-9, k=k, oversample=os_, q=q,
                        seed=m + n)
        G1, G2, _, _ = planted_pair_complex(spec)
        _check(prec, G1, G2, k, os_, q, seed=5)


@pytest.mark.parametrize("q", [0, 1])
@pytest.mark.parametrize("prec", ["fp64", "tf32x3"])
def test_paper_complex_full_pair(prec, q):
    # Section 4.1's complex synthetic pair: 40% of the pairs at (1, 0), 40% at (0, 1), 20% uniform,
    # each side of rank 60% of n; all n pairs resolved with k = n (the realified stack has 4n rows)
    G1, G2, a, b = full_gmp_pair_complex(150, 130, 50, seed=3)
    al, be, _ = _check(prec, G1, G2, 50, 0, q, seed=11)
    tol = TOL[prec]
    assert np.max(np.abs(al[:10] - 1.0)) <= tol and np.max(np.abs(be[:10])) <= tol
    assert np.max(np.abs(al[40:])) <= tol and np.max(np.abs(be[40:] - 1.0)) <= tol


def test_complex_host_inputs_and_refusals():
    spec = PairSpec(m=400, p=350, n=90, r=8, alpha="uniform", decay="exp10", sigma=1e-8, k=8, oversample=6, q=1,
                    seed=62)
    G1, G2, _, _ = planted_pair_complex(spec)
    _check("fp64", G1, G2, 8, 6, 1, seed=4, device=False)   # host (numpy) inputs and outputs
    _check("tf32x3", G1, G2, 8, 6, 1, seed=4, device=False)
    c1 = torch.from_numpy(G1.astype(np.complex64)).cuda()
    c2 = torch.from_numpy(G2.astype(np.complex64)).cuda()
    with P.Context("tf32x3", adaptive=True) as ctx:
        with pytest.raises(P.GsvdRandError) as e:
            ctx.solve_complex(c1, c2, 8, 6, 1, 4)
        assert e.value.name == "UNSUPPORTED"
    with P.Context("tf32x3") as ctx:
        with pytest.raises(P.GsvdRandError) as e:
            ctx.solve_complex(c1, c2, 85, 6, 1, 4)  # k + oversample > n
        assert e.value.name == "ARG"
        with pytest.raises(P.GsvdRandError):
            ctx.factors()  # no factors after a complex solve
