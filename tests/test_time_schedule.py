"""The library's host-side time split of a V-cycle (nmf_time_schedule) against the oracle's
(time_schedule), which its own pins tie to Algorithm V-cycle and Table 1.  Host code only:
no GPU needed."""
import numpy as np
import pytest

from oracle import nmf_oracle as o


@pytest.fixture(scope="module")
def native():
    from paper_1009_0881_gb300 import build, native as nat
    build.build()
    return nat


def test_time_split_matches_oracle(native):
    rng = np.random.default_rng(0)
    for L in range(1, 8):
        for _ in range(200):
            costs = list(rng.uniform(0.05, 40.0, L))
            T = float(rng.uniform(0.0, 5000.0))
            assert native.time_schedule(T, costs) == tuple(o.time_schedule(T, costs)), (L, T, costs)


def test_time_split_with_quarter_costs_is_table1(native):
    for L, K in ((2, 8), (3, 500), (4, 100)):
        costs = [0.25 ** l for l in range(L)]
        assert native.time_schedule(K * costs[0], costs) == ([K // 4] * (L - 1), K, [K // 2] * (L - 1))


def test_time_split_rejects_bad_costs(native):
    for costs in ([1.0, 0.0], [1.0, -2.0], []):
        with pytest.raises(native.NMFError):
            native.time_schedule(10.0, costs)


def test_level_sweeps_run_order(native):
    # (pre, coarse, post) with pre[l] / post[l] for level l + 1 -> the run order of
    # nmf_options.level_sweeps: pre_1 .. pre_{L-1}, coarse, post_{L-1} .. post_1
    flat = native._flat_level_sweeps(([11, 12, 13], 40, [21, 22, 23]), 4)
    assert flat.tolist() == [11, 12, 13, 40, 23, 22, 21]
    assert native._flat_level_sweeps(([], 7, []), 1).tolist() == [7]
    with pytest.raises(ValueError):
        native._flat_level_sweeps(([1], 2, [1, 2]), 2)
    # the library's split comes back in the same (pre, coarse, post) form
    pre, coarse, post = native.time_schedule(1000.0, [10.0, 8.0, 5.0])
    assert native._flat_level_sweeps((pre, coarse, post), 3).tolist() == [25, 7, 12, 15, 50]
