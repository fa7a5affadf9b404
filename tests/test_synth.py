"""The seeded generator: deterministic, documented SplitMix64, workload structure."""
import numpy as np

from paper_1009_0881_gb300 import synth


def test_splitmix64_known_values():
    # SplitMix64 finaliser of Steele, Lea and Flood applied to 0x9E3779B97F4A7C15 * (i+1) + key
    key = synth._stream_key(0, 0)
    z = np.array([key + np.uint64(0x9E3779B97F4A7C15)], dtype=np.uint64)
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    z = z ^ (z >> np.uint64(31))
    assert synth.splitmix64(0, 0, 1)[0] == z[0]
    # the reference sequence of SplitMix64 seeded with state 0: first output 0xE220A8397B1DCDAF
    s = np.array([0], dtype=np.uint64) + np.uint64(0x9E3779B97F4A7C15)
    assert synth._mix64(s)[0] == np.uint64(0xE220A8397B1DCDAF)


def test_distributions():
    u = synth.uniform(5, 1, 200000)
    assert 0.0 <= u.min() and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.005
    g = synth.gaussian(5, 2, 200000)
    assert abs(g.mean()) < 0.01 and abs(g.std() - 1.0) < 0.01
    e = synth.exponential(5, 3, 200000)
    assert abs(e.mean() - 1.0) < 0.01


def test_problem_structure_and_determinism():
    a = synth.make_problem(19, 19, 100, 7, data_seed=3)
    b = synth.make_problem(19, 19, 100, 7, data_seed=3)
    np.testing.assert_array_equal(a.M, b.M)
    assert a.M.dtype == np.float32 and a.M.shape == (361, 100)
    assert (a.M >= 0).all() and a.V.shape == (361, 7) and a.W.shape == (7, 100)
    assert ((a.V >= 0) & (a.V < 1)).all()
    # about half of W0 is zero
    assert 0.4 < (a.W0 == 0).mean() < 0.6
    c = synth.make_problem(19, 19, 100, 7, data_seed=4)
    assert not np.array_equal(a.M, c.M)
    # the initial iterate depends on init_seed only
    np.testing.assert_array_equal(a.V, c.V)


def test_batched_sizes_in_range():
    sizes = synth.batched_sizes(64)
    assert len(sizes) == 64
    for side, n, r in sizes:
        assert side in (16, 19, 32, 64, 92, 128) and 200 <= n <= 4000 and 5 <= r <= 64
