"""gsvd_rand_metrics_noalloc against gsvd_rand_metrics and the FP64 oracle (needs a CUDA GPU).

The no-allocation entry point keeps its scratch in a fixed static device array;
here two calls in a row must each agree with the allocating entry point to
rounding (the entropy sums are added in another order) and with the oracle's
Section 1 formulas, leave the device's free memory unchanged, and refuse sizes
above the fixed limit.

Tolerances against the oracle: theta and P to 1e-14 absolute, rho to 1e-14
relative (one division or atan2 per entry, a few ulps); D_1, D_2 to 4e-12: each
is a sum of N <= 32768 terms P log P of magnitude <= 1/e, summed in another
order, so the rounding differences stay below N u = 3.6e-12.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2404_09459_gb300 as P  # noqa: E402
from oracle import gsvd as O  # noqa: E402

P._build.build()

KEYS = ("theta", "rho", "P1", "P2")


def _pairs(r, seed):
    rng = np.random.default_rng(seed)
    a = np.sort(rng.uniform(0, 1, r))[::-1].copy()
    a[0] = 1.0
    a[-1] = 0.0
    return a, np.sqrt(1 - a ** 2)


def _close(got, ref):
    for key in KEYS:
        g = np.asarray(got[key].cpu() if hasattr(got[key], "cpu") else got[key])
        fin = np.isfinite(ref[key])
        np.testing.assert_allclose(g[fin], ref[key][fin], rtol=1e-14, atol=1e-14)
        assert np.all(np.isinf(g[~fin]))
    for key in ("D1", "D2"):
        assert abs(float(got[key]) - float(ref[key])) <= 1e-13, key


def _close_oracle(got, a, b, pad_to_n, pad_mode):
    ref = O.metrics(a, b, pad_to_n, pad_mode)
    for key in KEYS:
        g = np.asarray(got[key].cpu() if hasattr(got[key], "cpu") else got[key])
        fin = np.isfinite(ref[key])
        if key == "rho":
            np.testing.assert_allclose(g[fin], ref[key][fin], rtol=1e-14, atol=0)
        else:
            np.testing.assert_allclose(g[fin], ref[key][fin], rtol=0, atol=1e-14)
        assert np.all(np.isinf(g[~fin]))
    for key in ("D1", "D2"):
        assert abs(float(got[key]) - float(ref[key])) <= 4e-12, key


@pytest.mark.parametrize("r,pad_to_n,pad_mode", [(17, 0, 0), (17, 40, 0), (17, 40, 1), (3000, 5000, 1),
                                                 (20000, P.NOALLOC_MAX_N, 0)])
def test_host_buffers_two_calls_match_allocating_entry_point(r, pad_to_n, pad_mode):
    a, b = _pairs(r, r + pad_to_n)
    with P.Context("fp64") as ctx:
        ref = ctx.metrics(a, b, pad_to_n, pad_mode)
    first = P.metrics_noalloc(a, b, pad_to_n, pad_mode)
    second = P.metrics_noalloc(a, b, pad_to_n, pad_mode)
    _close(first, ref)
    _close(second, ref)
    _close_oracle(first, a, b, pad_to_n, pad_mode)
    _close_oracle(second, a, b, pad_to_n, pad_mode)
    for key in KEYS:
        np.testing.assert_array_equal(first[key], second[key])


def test_device_buffers_two_calls_allocate_nothing():
    r, N = 2500, 4096
    a, b = _pairs(r, 7)
    da, db = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    with P.Context("fp64") as ctx:
        ref = ctx.metrics(a, b, N, 0)
    outs = [{k: torch.full((N,), -7.0, dtype=torch.float64, device="cuda") for k in KEYS} for _ in range(2)]
    for o in outs:
        o["D"] = torch.zeros(2, dtype=torch.float64, device="cuda")
    stream = torch.cuda.Stream()
    P.metrics_noalloc(a, b, N, 0, stream=stream)  # first call on the device: scratch set-up
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    got = [P.metrics_noalloc(da, db, N, 0, stream=stream, out=o) for o in outs]
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free_before
    for g in got:
        _close(g, ref)
        _close_oracle(g, a, b, N, 0)


def test_size_above_limit_is_refused():
    a, b = _pairs(10, 1)
    with pytest.raises(P.GsvdRandError) as e:
        P.metrics_noalloc(a, b, P.NOALLOC_MAX_N + 1, 0)
    assert e.value.name == "TOO_LARGE"
    with pytest.raises(P.GsvdRandError) as e:
        P.metrics_noalloc(a[:1], b[:1])  # N = 1: the entropy needs log N > 0
    assert e.value.name == "ARG"
    # the scratch is still good after a refusal
    with P.Context("fp64") as ctx:
        ref = ctx.metrics(a, b)
    _close(P.metrics_noalloc(a, b), ref)
