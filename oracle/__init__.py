"""FP64 CPU oracle of the randomized GSV method — TEST INFRASTRUCTURE ONLY.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline / reference legs
of `bench.py` may import this package.  The GPU library never calls it and
shares no code with it; when the CUDA extension is missing the library fails
instead of falling back here.

Contents and what each follows (paper: Xu, Shen, Li, Gao, Li, "Randomized
algorithms for GSVs", arXiv:2404.09459):
  philox.gaussian      Gaussian test matrices Omega (Algorithm 1; Theorem 3)
  gsvd.direct_gsvd     the reduced GSVD of eq. (gsvd1) by SVD + CS split
  gsvd.pencil_gsvd     brute force for tiny pairs (symmetric-definite pencil)
  gsvd.rand_gsvd       Algorithm 2 with the fixed-rank basis of Theorem 3 + q power steps
  gsvd.adaptive_basis  Algorithm 1 (BasisExt) with the cumulated residual of Section 2
  gsvd.rand_gsvd_adaptive  Algorithm 2 on the Algorithm 1 bases
  gsvd.metrics         theta, rho, P1, P2, D1, D2 of Section 1
  gsvd.perturbation_E  the E of Lemma "per" / Theorem "exp" (Section 3)
  gsvd.rand_gsvd_complex, direct_gsvd_complex, pencil_gsvd_complex, gaussian_complex
                       the same over C (eq. (gsvd1) is stated over C; Section 4.1 is complex)
  gsvd.realify         the real 2 x 2-block form of a complex matrix (a pin of the complex path)

Every function is pinned by a `-m "not gpu"` test against values fixed by the
paper or by mathematics (known-answer vectors, closed forms, invariants,
brute force); none is "parity unpinned".
"""
from . import philox, gsvd  # noqa: F401
