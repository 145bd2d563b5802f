"""The persisting-L2 cost model (qw_l2_split_model): the workload cache split
of Section 4 (Eq. 4: minimise index IO + data IO subject to size(C_I) +
size(C_D) = size(C)), restated for the GPU's L2.  Host code only: these run
without a GPU.

A region of U bytes read A bytes in total costs U + (A - U)(1 - min(1, S/U))
DRAM bytes with S persisting bytes: convex and decreasing in S with slope
-(A - U)/U until S = U.  So the optimum gives the set-aside first to the
region with more re-reads per byte, until that region fits, then the rest to
the other -- a greedy rule checked here against the library's grid search."""
import math

import numpy as np
import pytest

MB = float(1 << 20)


def _traffic(U, A, S):
    if U <= 0:
        return 0.0
    return U + max(A - U, 0.0) * (1.0 - min(1.0, S / U))


def _cost(S, UI, AI, UD, AD, p):
    SI = S * p / 1000.0
    return _traffic(UI, AI, SI) + _traffic(UD, AD, S - SI)


def _greedy(S, UI, AI, UD, AD):
    """Continuous optimum of the index share by the re-reads-per-byte rule."""
    rho_i = (AI - UI) / UI if UI > 0 else 0.0
    rho_d = (AD - UD) / UD if UD > 0 else 0.0
    if UI + UD <= S:
        return UI  # both fit: every share in [U_I, S - U_D] is optimal; the smallest
    if rho_i > rho_d:
        return min(S, UI)
    if rho_d > rho_i:
        return max(0.0, S - min(S, UD))
    return None  # equal densities: every split in a range is optimal


def test_index_denser_fits_gets_exactly_its_bytes(qwlib):
    # 16 MB of summaries read 40x, 512 MB of rows read 8x; 80 MB set-aside
    p = qwlib.qw_l2_split_model(80 * MB, 16 * MB, 640 * MB, 512 * MB, 4096 * MB)
    assert p == 200


def test_data_denser_takes_everything(qwlib):
    # index read twice per byte, data ten times: the data region alone is
    # larger than the set-aside, so the index gets nothing
    p = qwlib.qw_l2_split_model(64 * MB, 128 * MB, 256 * MB, 256 * MB, 2560 * MB)
    assert p == 0


def test_data_denser_but_fits_leaves_rest_to_index(qwlib):
    # data 24 MB read 100x fits; the index (read 3x) takes the other 40 MB
    p = qwlib.qw_l2_split_model(64 * MB, 128 * MB, 384 * MB, 24 * MB, 2400 * MB)
    assert p == 625


def test_no_rereads_every_split_equal_smallest_wins(qwlib):
    assert qwlib.qw_l2_split_model(64 * MB, 10 * MB, 10 * MB, 30 * MB, 30 * MB) == 0


def test_both_fit_index_gets_its_bytes_first(qwlib):
    # U_I + U_D <= S: the smallest split that holds the whole index is optimal
    p = qwlib.qw_l2_split_model(100 * MB, 25 * MB, 500 * MB, 50 * MB, 100 * MB)
    assert p == 250
    assert _cost(100 * MB, 25 * MB, 500 * MB, 50 * MB, 100 * MB, p) == pytest.approx(75 * MB)


def test_empty_regions(qwlib):
    assert qwlib.qw_l2_split_model(64 * MB, 0.0, 0.0, 10 * MB, 50 * MB) == 0
    assert qwlib.qw_l2_split_model(64 * MB, 10 * MB, 50 * MB, 0.0, 0.0) == 157  # ceil(10/64 * 1000)


@pytest.mark.parametrize("args", [(0.0, 1.0, 1.0, 1.0, 1.0), (-1.0, 1.0, 1.0, 1.0, 1.0),
                                  (1.0, -1.0, 1.0, 1.0, 1.0), (1.0, 1.0, math.nan, 1.0, 1.0),
                                  (1.0, 1.0, 1.0, math.inf, 1.0)])
def test_rejects_bad_arguments(qwlib, args):
    assert qwlib.qw_l2_split_model(*args) == -1


def test_random_cases_grid_optimum_and_greedy(qwlib):
    rng = np.random.default_rng(5)
    for _ in range(300):
        S = float(rng.uniform(1, 128)) * MB
        UI, UD = (float(x) * MB for x in rng.uniform(0.5, 300, 2))
        AI = UI * float(rng.uniform(1, 60))
        AD = UD * float(rng.uniform(1, 60))
        p = qwlib.qw_l2_split_model(S, UI, AI, UD, AD)
        assert 0 <= p <= 1000
        costs = [_cost(S, UI, AI, UD, AD, q) for q in range(1001)]
        best = min(costs)
        # the returned split is a grid minimum, and the first one
        assert costs[p] <= best * (1 + 1e-12)
        assert all(c > best * (1 + 1e-12) for c in costs[:p]) or p == 0
        g = _greedy(S, UI, AI, UD, AD)
        if g is not None:
            # the grid optimum is within one grid step of the greedy optimum
            assert abs(p * S / 1000.0 - g) <= S / 1000.0 + 1e-6 * S
