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


def test_qalsh_collision_probability_matches_oracle(qwlib, orc):
    for w in (1.0, 2.719, 4.0):
        for r in (0.2, 1.0, 2.0, 5.0):
            assert abs(qwlib.qw_qalsh_collision_probability(r, w) - orc.qalsh_prob(r, w)) < 1e-15
    assert math.isnan(qwlib.qw_qalsh_collision_probability(-1.0, 4.0))


@pytest.mark.parametrize("m,w,c,n,v", [(16, 2.719, 2, 10_000, 100), (64, 2.719, 2, 1_000_000, 700),
                                       (64, 1.0, 3, 4_000_000, 100), (8, 2.719, 2, 50, 100)])
def test_qalsh_threshold_matches_oracle(qwlib, orc, m, w, c, n, v):
    """Section 3.1's rule l = ceil(alpha m) with QALSH's p1 = P(1), p2 = P(c)."""
    assert qwlib.qw_qalsh_collision_threshold(m, w, c, n, v) == orc.qalsh_threshold(m, w, c, n, v)


def test_family_arguments_without_device(qwlib):
    L = qwlib.load()
    h = C.c_void_p()
    fake = C.c_void_p(16)
    for bad, word in ((qwlib.qw_index_params(m=8, w=2.7, c=2, v=10, family=2), b"family"),
                      (qwlib.qw_index_params(m=8, w=2.7, c=2, v=10, family=1, bitmaps=1), b"bitmaps"),
                      (qwlib.qw_index_params(m=8, w=2.7, c=2, v=10, family=1, projection=1), b"FP64")):
        assert L.qw_build_index(fake, 10, 4, fake, fake, C.byref(bad), 0, None, C.byref(h)) == qwlib.QW_ERR_ARG
        assert word in L.qw_last_error()


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


def test_start_model_argument_errors_without_device(qwlib):
    """The start-model, feature and bandwidth calls reject bad arguments before
    any device work, with QW_ERR_ARG and a message naming the call."""
    L = qwlib.load()
    fake = C.c_void_p(16)
    out = C.c_void_p()
    for n_in, hidden, classes in ((0, 8, 4), (8, 0, 4), (8, 8, 1), (70000, 8, 4), (8, 8, 2000)):
        assert L.qw_mlp_create(n_in, hidden, classes, C.byref(out)) == qwlib.QW_ERR_ARG
        assert b"qw_mlp" in L.qw_last_error()
    assert L.qw_mlp_create(8, 8, 4, None) == qwlib.QW_ERR_ARG
    assert L.qw_mlp_param_count(None) == -1
    assert L.qw_mlp_set_params(None, fake, 1) == qwlib.QW_ERR_ARG
    assert L.qw_mlp_get_params(None, fake, 1) == qwlib.QW_ERR_ARG
    assert L.qw_mlp_loss_grad(None, fake, fake, 1, None, None, None) == qwlib.QW_ERR_ARG
    assert L.qw_mlp_train(None, fake, fake, 1, 1, 1, C.c_float(0.01), None, None) == qwlib.QW_ERR_ARG
    assert L.qw_mlp_predict(None, fake, 1, fake, None) == qwlib.QW_ERR_ARG
    assert L.qw_query_features(None, fake, 1, fake, None) == qwlib.QW_ERR_ARG
    assert b"qw_query_features" in L.qw_last_error()
    assert L.qw_index_set_start_model(None, None, C.c_float(0.5)) == qwlib.QW_ERR_ARG
    gbs = C.c_double()
    assert L.qw_measure_read_bandwidth(8, 1, C.byref(gbs), None) == qwlib.QW_ERR_ARG
    assert L.qw_measure_read_bandwidth(1 << 20, 0, C.byref(gbs), None) == qwlib.QW_ERR_ARG
    assert L.qw_measure_read_bandwidth(1 << 20, 1, None, None) == qwlib.QW_ERR_ARG
    L.qw_mlp_free(None)  # no-op


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
    assert qp.projection == qwlib.QW_PROJ_FP32


def test_host_bitmaps_need_bitmaps_without_device(qwlib):
    """The argument check runs before any device work."""
    L = qwlib.load()
    h = C.c_void_p()
    fake = C.c_void_p(16)
    p = qwlib.qw_index_params(m=8, w=4.0, c=2, v=10, host_bitmaps=1)
    assert L.qw_build_index(fake, 10, 4, fake, fake, C.byref(p), 0, None, C.byref(h)) == qwlib.QW_ERR_ARG
    assert b"host_bitmaps" in L.qw_last_error()


# ---------------------------------------------------------------- seeded projections
_GAMMA = 0x9E3779B97F4A7C15
_M64 = (1 << 64) - 1


def _splitmix64(seed, k):
    """SplitMix64's output for counter k (Steele, Lea and Flood, OOPSLA 2014):
    the state after k + 1 steps of adding the golden-ratio increment, mixed."""
    z = (seed + (k + 1) * _GAMMA) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def _draw_reference(seed, m, d, w):
    """The documented draw restated: uniforms from the top 53 bits, normals by
    the Box-Muller transform in pairs, offsets from the following counters."""
    import numpy as np
    u = lambda k: (_splitmix64(seed, k) >> 11) * 2.0 ** -53  # noqa: E731
    na = m * d
    A = np.empty(na, np.float32)
    for e in range(0, na, 2):
        r = math.sqrt(-2.0 * math.log(1.0 - u(e)))
        t = 2.0 * math.pi * u(e + 1)
        A[e] = np.float32(r * math.cos(t))
        if e + 1 < na:
            A[e + 1] = np.float32(r * math.sin(t))
    k0 = (na + 1) // 2 * 2
    wf = float(np.float32(w))  # the bucket width as the float the library takes
    b = np.array([np.float32(u(k0 + i) * wf) for i in range(m)], np.float32)
    b = np.where(b < np.float32(w), b, np.nextafter(np.float32(w), np.float32(0)))
    return A.reshape(m, d), b


@pytest.mark.parametrize("seed,m,d,w", [(0, 16, 32, 4.0), (12345, 7, 5, 2.719),
                                        (2 ** 63 + 11, 3, 3, 1.0)])
def test_draw_projections_is_the_documented_generator(qwlib, seed, m, d, w):
    import numpy as np
    A, b = qwlib.qw_draw_projections(seed, m, d, w)
    wantA, wantb = _draw_reference(seed, m, d, w)
    assert np.array_equal(A, wantA)
    assert np.array_equal(b, wantb)


def test_draw_projections_distribution(qwlib):
    """a ~ N(0, I): mean 0, variance 1, no correlation between neighbouring
    entries; b ~ U[0, w): inside the interval, mean w / 2; seeds differ."""
    import numpy as np
    A, b = qwlib.qw_draw_projections(7, 200, 500, 4.0)
    x = A.astype(np.float64).ravel()
    assert abs(x.mean()) < 0.01 and abs(x.var() - 1.0) < 0.01
    assert abs(np.corrcoef(x[:-1], x[1:])[0, 1]) < 0.01
    assert abs((x ** 4).mean() / x.var() ** 2 - 3.0) < 0.05  # Gaussian kurtosis
    assert np.all((b >= 0) & (b < 4.0)) and abs(b.mean() - 2.0) < 0.25
    A2, _ = qwlib.qw_draw_projections(8, 200, 500, 4.0)
    assert not np.array_equal(A, A2)
    A3, b3 = qwlib.qw_draw_projections(7, 200, 500, 4.0)
    assert np.array_equal(A, A3) and np.array_equal(b, b3)
