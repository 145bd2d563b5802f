"""The C-ABI library without a GPU: it loads, exports every symbol the header
declares, its host-side parameter functions agree with the oracle, and bad
arguments are rejected before any device work."""
import ctypes as C
import glob
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(qw_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_entry_points():
    names = _declared_functions()
    for must in ("qw_build_index", "qw_run_workload", "qw_hash", "qw_index_free"):
        assert must in names


def test_library_exports_every_declared_symbol(qwlib):
    lib = C.CDLL(qwlib.LIB_PATH)
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"
    assert set(_declared_functions()) == set(qwlib.EXPORTED)


def test_version(qwlib):
    assert "sm_103a" in qwlib.qw_version()


def test_collision_probability_matches_oracle(qwlib, orc):
    for w in (1.0, 2.719, 4.0):
        for r in (0.2, 1.0, 2.0, 5.0):
            assert abs(qwlib.collision_probability(r, w) - orc.collision_prob(r, w)) < 1e-14
    assert math.isnan(qwlib.collision_probability(0.0, 4.0))


@pytest.mark.parametrize("m,w,c,n,v", [(16, 4.0, 2, 10_000, 100), (64, 4.0, 2, 1_000_000, 100),
                                       (64, 2.719, 2, 54_387, 100), (64, 4.0, 3, 4_000_000, 100),
                                       (127, 1.5, 2, 10_000_000, 10), (8, 4.0, 2, 50, 100)])
def test_threshold_matches_oracle(qwlib, orc, m, w, c, n, v):
    assert qwlib.collision_threshold(m, w, c, n, v) == orc.threshold(m, w, c, n, v)


def test_threshold_rejects_bad_arguments(qwlib):
    assert qwlib.collision_threshold(0, 4.0, 2, 100, 10) == -1
    assert qwlib.collision_threshold(8, -1.0, 2, 100, 10) == -1
    assert qwlib.collision_threshold(8, 4.0, 1, 100, 10) == -1


def test_argument_errors_without_device(qwlib):
    L = qwlib.load()
    h = C.c_void_p()
    p = qwlib.qw_index_params(m=8, w=4.0, c=2, v=100, l=0, delta=0.0)
    assert L.qw_build_index(None, 10, 4, None, None, C.byref(p), 0, None, C.byref(h)) == qwlib.QW_ERR_ARG
    assert b"null" in L.qw_last_error()
    fake = C.c_void_p(16)
    for bad in (qwlib.qw_index_params(m=0, w=4.0, c=2, v=1), qwlib.qw_index_params(m=200, w=4.0, c=2),
                qwlib.qw_index_params(m=8, w=0.0, c=2), qwlib.qw_index_params(m=8, w=4.0, c=1),
                qwlib.qw_index_params(m=8, w=4.0, c=2, v=-1), qwlib.qw_index_params(m=8, w=4.0, c=2, l=9)):
        assert L.qw_build_index(fake, 10, 4, fake, fake, C.byref(bad), 0, None, C.byref(h)) == qwlib.QW_ERR_ARG
    assert L.qw_build_index(fake, 0, 4, fake, fake, C.byref(p), 0, None, C.byref(h)) == qwlib.QW_ERR_ARG
    assert L.qw_build_index(fake, 10, 4, fake, fake, C.byref(p), 7, None, C.byref(h)) == qwlib.QW_ERR_ARG
    qp = qwlib.qw_query_params()
    assert L.qw_run_workload(None, fake, 1, 1, C.byref(qp), fake, fake, None, 0, None) == qwlib.QW_ERR_ARG
    assert L.qw_workload_candidates(None, fake, 1, 1, C.byref(qp), fake, None, None, 0, None) == qwlib.QW_ERR_ARG
    assert L.qw_hash(None, 1, 1, fake, fake, 1, 1.0, fake, None, None) == qwlib.QW_ERR_ARG
    assert L.qw_hash(fake, -1, 1, fake, fake, 1, 1.0, fake, None, None) == qwlib.QW_ERR_ARG
    assert L.qw_index_get_info(None, None) == qwlib.QW_ERR_ARG
    assert L.qw_index_profile(None, None, 0) == qwlib.QW_ERR_ARG
    L.qw_index_free(None)  # no-op


def test_binding_rejects_bad_tensors(qwlib):
    torch = pytest.importorskip("torch")
    x = torch.zeros((4, 3), dtype=torch.float32)
    with pytest.raises(ValueError):
        qwlib._f32(x.double(), "x")
    with pytest.raises(ValueError):
        qwlib._f32(x.t(), "x")


def test_product_path_has_no_oracle_import():
    """The package never imports, links or executes the oracle."""
    pkg = os.path.join(ROOT, "paper_1907_11803_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*"), recursive=True):
        if path.endswith((".py", ".cu", ".cuh", ".h")):
            text = open(path).read()
            code = re.sub(r"(#|//).*", "", text)
            assert not re.search(r"\bimport\s+oracle|from\s+oracle|liboracle|qwlsh_oracle", code), path


def test_l2_split_arguments_of_the_binding(qwlib):
    """query(l2=...) maps to the ABI's l2_mode / l2_index_permille fields."""
    assert qwlib._l2_fields(None) == {"l2_mode": qwlib.QW_L2_OFF, "l2_index_permille": 0}
    assert qwlib._l2_fields("off") == {"l2_mode": qwlib.QW_L2_OFF, "l2_index_permille": 0}
    assert qwlib._l2_fields("model") == {"l2_mode": qwlib.QW_L2_MODEL, "l2_index_permille": 0}
    assert qwlib._l2_fields(250) == {"l2_mode": qwlib.QW_L2_SPLIT, "l2_index_permille": 250}
    for bad in (True, 0.5, "half"):
        with pytest.raises(ValueError):
            qwlib._l2_fields(bad)
    qp = qwlib.qw_query_params(**qwlib._l2_fields(990))
    assert qp.l2_mode == qwlib.QW_L2_SPLIT and qp.l2_index_permille == 990
    assert list(qp.reserved) == [0]


def test_host_bitmaps_need_bitmaps_without_device(qwlib):
    """The argument check runs before any device work."""
    L = qwlib.load()
    h = C.c_void_p()
    fake = C.c_void_p(16)
    p = qwlib.qw_index_params(m=8, w=4.0, c=2, v=10, host_bitmaps=1)
    assert L.qw_build_index(fake, 10, 4, fake, fake, C.byref(p), 0, None, C.byref(h)) == qwlib.QW_ERR_ARG
    assert b"host_bitmaps" in L.qw_last_error()
