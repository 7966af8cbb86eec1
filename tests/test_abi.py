"""The C-ABI library builds for sm_103a, loads, and exports every symbol the
header declares (no GPU needed; no compute call is made)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gsvd_rand.h")


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(gsvd_rand_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2404_09459_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("gsvd_rand_create", "gsvd_rand_solve", "gsvd_rand_metrics", "gsvd_rand_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_match_header():
    import paper_2404_09459_gb300 as P
    assert sorted(P.EXPORTS) == sorted(set(P.EXPORTS))
    assert set(P.EXPORTS) <= set(_declared())


def test_config_init_defaults(lib):
    import paper_2404_09459_gb300 as P
    cfg = P._Config()
    lib.gsvd_rand_config_init.argtypes = [ctypes.POINTER(P._Config)]
    assert lib.gsvd_rand_config_init(ctypes.byref(cfg)) == 0
    assert cfg.prec == P.PREC["tf32"] and cfg.block_b == 100 and abs(cfg.tol - 1e-4) < 1e-18
    assert lib.gsvd_rand_config_init(None) == -1


def test_noalloc_limit_matches_header():
    import paper_2404_09459_gb300 as P
    m = re.search(r"#define GSVD_RAND_NOALLOC_MAX_N (\d+)", open(HEADER).read())
    assert m and int(m.group(1)) == P.NOALLOC_MAX_N
