"""Host logic of bench.py that needs no GPU: the reference arm's schedule of
levels measures every level for any number of warm-up and timed steps, and
the workload's pair rate follows from per-level solve times."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("W,K", [(1, 1), (3, 3), (1, 4), (2, 5), (4, 1), (3, 10)])
def test_reference_arm_measures_every_level(bench, W, K):
    warm, timed, extra = bench.reference_levels(W, K)
    assert len(warm) == W and len(timed) == K
    assert set(warm) | set(timed) | set(extra) == set(bench.LEVELS)
    assert not set(extra) & (set(warm) | set(timed))
    # with the defaults the steps themselves reach every level
    if W + K >= 4:
        assert extra == []


def test_pair_rate_is_pairs_over_busy_core_seconds(bench):
    solve_s = {0: 1.0, 1: 2.0, 2: 4.0, 3: 8.0}
    value, pair = bench.pair_rate(solve_s, cores=2)
    # a pair at level l = a fine solve at l plus a coarse solve at l - 1
    assert pair == {0: 1.0, 1: 3.0, 2: 6.0, 3: 12.0}
    busy = (1024 * 1.0 + 256 * 3.0 + 64 * 6.0 + 16 * 12.0) / 2
    assert value == pytest.approx((1024 + 256 + 64 + 16) / busy)
