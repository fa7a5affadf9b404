"""Pins for the oracle's multigrid cycles (Section 4.3, Table 1, Section 4.1 bound)."""
import numpy as np
import pytest

from conftest import ROOT
from oracle import nmf_oracle as o
from paper_1009_0881_gb300 import synth


def _table1_rows():
    rows = []
    with open(f"{ROOT}/tests/golden/sweep_allocation_table1.txt") as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(t) for t in line.split()])
    return rows


def _count_sweeps(cycle, L, K, h=16, w=16):
    """Sweeps per level of a cycle, counted by replacing the inner algorithm with a counter."""
    counts = [0] * L
    p = synth.make_problem(h, w, 4, 2, data_seed=1)
    trace = []
    orig = dict(o.SWEEPS)
    o.SWEEPS["count"] = lambda M, V, W: (V, W)
    try:
        o.solve(p.M, h, w, p.V, p.W, algo="count", levels=L, K=K, cycle=cycle, trace=trace)
    finally:
        o.SWEEPS.clear()
        o.SWEEPS.update(orig)
    for level, _ in trace:
        counts[level - 1] += 1
    return counts


@pytest.mark.parametrize("row", _table1_rows())
def test_vcycle_sweep_allocation_matches_table1(row):
    L, k = row[0], row[1]
    assert _count_sweeps("vcycle", L, 4 * k) == row[2:]


@pytest.mark.parametrize("row", _table1_rows())
def test_nested_iteration_sweep_allocation_matches_table1(row):
    L, k = row[0], row[1]
    assert _count_sweeps("ni", L, 4 * k) == row[2:]


def _level_sequence(cycle, L, K, h=16, w=16):
    """Levels of the sweeps in the order a cycle runs them."""
    p = synth.make_problem(h, w, 4, 2, data_seed=1)
    trace = []
    orig = dict(o.SWEEPS)
    o.SWEEPS["count"] = lambda M, V, W: (V, W)
    try:
        o.solve(p.M, h, w, p.V, p.W, algo="count", levels=L, K=K, cycle=cycle, trace=trace)
    finally:
        o.SWEEPS.clear()
        o.SWEEPS.update(orig)
    return [level for level, _ in trace]


def test_vcycle_order_follows_algorithm():
    # Algorithm V-cycle: pre-smoothing at the fine level, the coarse cycle, then post-smoothing
    K = 8
    assert _level_sequence("vcycle", 2, K) == [1] * (K // 4) + [2] * K + [1] * (K // 2)
    assert _level_sequence("vcycle", 3, K) == ([1] * (K // 4) + [2] * (K // 4) + [3] * K + [2] * (K // 2)
                                               + [1] * (K // 2))


def test_fmg_allocation():
    # FMG(L, K) = FMG(L-1, K) on the coarser level, then V-cycle(L, 3K/4)
    K = 400
    assert _count_sweeps("fmg", 1, K) == [K]
    # L = 2: coarse gets K (the recursive FMG) + 3K/4 (inside the V-cycle); fine gets 3/4 * 3K/4
    Kv = 3 * K // 4
    assert _count_sweeps("fmg", 2, K) == [Kv // 4 + Kv // 2, K + Kv]


def test_single_level_cycles_equal_plain_algorithm():
    p = synth.make_problem(8, 8, 20, 3, data_seed=2)
    M = p.M.astype(np.float64)
    Vp, Wp = o.smooth(M, p.V.astype(np.float64), p.W.astype(np.float64), "hals", 7)
    for cyc in ("vcycle", "ni", "fmg"):
        V, W = o.solve(p.M, 8, 8, p.V, p.W, "hals", levels=1, K=7, cycle=cyc)
        np.testing.assert_array_equal(V, Vp)
        np.testing.assert_array_equal(W, Wp)


def test_w_passes_through_transfers_unchanged():
    # Only V is restricted and prolonged; W leaves the coarse level as it entered the prolongation
    p = synth.make_problem(9, 9, 30, 4, data_seed=3)
    hooks = []
    Ms = o.restrict_hierarchy(p.M, 9, 9, 2)
    grids = o.grid_hierarchy(9, 9, 2)
    o.vcycle(Ms, grids, p.V.astype(np.float64), p.W.astype(np.float64), "hals", 2, 8, hooks=hooks)
    (_, level, Vc, V, W), = hooks
    np.testing.assert_allclose(V, o.prolong(Vc, *grids[1], *grids[0]))


@pytest.mark.parametrize("algo", ["hals", "mu"])
def test_transfer_error_bound_at_every_prolongation(algo):
    # Section 4.1: ||M - P(V')W|| <= s_M ||M|| + ||P||_F ||R(M) - V'W||
    p = synth.make_problem(19, 19, 60, 6, data_seed=4)
    Ms = o.restrict_hierarchy(p.M, 19, 19, 3)
    grids = o.grid_hierarchy(19, 19, 3)
    hooks = []
    o.vcycle(Ms, grids, p.V.astype(np.float64), p.W.astype(np.float64), algo, 3, 8, hooks=hooks)
    assert len(hooks) == 2
    for _, level, Vc, V, W in hooks:
        M = Ms[level]
        h, w = grids[level]
        hc, wc = grids[level + 1]
        P = o.prolongation_matrix(hc, wc, h, w)
        lhs = np.linalg.norm(M - V @ W)
        sM = o.smoothness(M, h, w)
        rhs = sM * np.linalg.norm(M) + np.linalg.norm(P) * np.linalg.norm(Ms[level + 1] - Vc @ W)
        assert lhs <= rhs * (1 + 1e-12)


def test_multilevel_beats_single_level_on_smooth_data_mu():
    # Sections 4.4 and 5.1 (qualitative): at equal fine-level-equivalent work, MU gains most
    p = synth.make_problem(19, 19, 120, 8, data_seed=5)
    M = p.M.astype(np.float64)
    K = 40
    V1, W1 = o.solve(p.M, 19, 19, p.V, p.W, "mu", levels=1, K=K)
    V3, W3 = o.solve(p.M, 19, 19, p.V, p.W, "mu", levels=3, K=K)
    assert o.objective(M, V3, W3) < o.objective(M, V1, W1)


def test_anls_vcycle_independent_of_v_transfers():
    # Remark after Algorithm NI: ANLS only needs W, so V's transfers do not change its result
    p = synth.make_problem(8, 8, 15, 3, data_seed=6)
    Va, Wa = o.solve(p.M, 8, 8, p.V, p.W, "anls", levels=2, K=8)
    Vb, Wb = o.solve(p.M, 8, 8, np.zeros_like(p.V), p.W, "anls", levels=2, K=8)
    np.testing.assert_array_equal(Va, Vb)
    np.testing.assert_array_equal(Wa, Wb)


def _bottom_up_problem():
    p = synth.make_problem(9, 9, 30, 4, data_seed=11)
    Ms = o.restrict_hierarchy(p.M, 9, 9, 3)
    grids = o.grid_hierarchy(9, 9, 3)
    return Ms, grids, p.V.astype(np.float64), p.W.astype(np.float64)


@pytest.mark.parametrize("algo", ["hals", "mu"])
def test_nested_iteration_data_flow(algo):
    # Algorithm NI, rebuilt from the pinned pieces: the coarsest level solves from the
    # restricted initial V, each finer level starts its floor(3K/4) sweeps from the
    # prolongation of the coarser result, with the W that came out of it
    Ms, grids, V0, W0 = _bottom_up_problem()
    K = 8
    hooks = []
    V, W = o.nested_iteration(Ms, grids, V0, W0, algo, 3, K, hooks=hooks)
    Vc2, Wc2 = o.smooth(Ms[2], o.restrict(o.restrict(V0, *grids[0]), *grids[1]), W0, algo, K)
    V1, W1 = o.smooth(Ms[1], o.prolong(Vc2, *grids[2], *grids[1]), Wc2, algo, (3 * K) // 4)
    Vf, Wf = o.smooth(Ms[0], o.prolong(V1, *grids[1], *grids[0]), W1, algo, (3 * K) // 4)
    assert [(k, lvl) for k, lvl, _, _ in hooks] == [("ni", 1), ("ni", 0)]
    np.testing.assert_array_equal(hooks[0][2], Vc2)
    np.testing.assert_array_equal(hooks[0][3], Wc2)
    np.testing.assert_array_equal(hooks[1][2], V1)
    np.testing.assert_array_equal(hooks[1][3], W1)
    np.testing.assert_array_equal(V, Vf)
    np.testing.assert_array_equal(W, Wf)


@pytest.mark.parametrize("algo", ["hals", "mu"])
def test_fmg_data_flow(algo):
    # Algorithm FMG, rebuilt from the pinned pieces: FMG on the coarser level from the
    # restricted initial V (budget K), then a V-cycle over this level and the ones below
    # with budget floor(3K/4), started from the prolongation of the coarse result
    Ms, grids, V0, W0 = _bottom_up_problem()
    K = 8
    hooks = []
    V, W = o.full_multigrid(Ms, grids, V0, W0, algo, 3, K, hooks=hooks)
    Vc2, Wc2 = o.smooth(Ms[2], o.restrict(o.restrict(V0, *grids[0]), *grids[1]), W0, algo, K)
    V1, W1 = o.vcycle(Ms, grids, o.prolong(Vc2, *grids[2], *grids[1]), Wc2, algo, 2, (3 * K) // 4, level=1)
    Vf, Wf = o.vcycle(Ms, grids, o.prolong(V1, *grids[1], *grids[0]), W1, algo, 3, (3 * K) // 4, level=0)
    assert [(k, lvl) for k, lvl, _, _ in hooks] == [("fmg", 1), ("fmg", 0)]
    np.testing.assert_array_equal(hooks[0][2], Vc2)
    np.testing.assert_array_equal(hooks[0][3], Wc2)
    np.testing.assert_array_equal(hooks[1][2], V1)
    np.testing.assert_array_equal(hooks[1][3], W1)
    np.testing.assert_array_equal(V, Vf)
    np.testing.assert_array_equal(W, Wf)


def test_wcycle_with_two_levels_is_the_vcycle():
    # two visits of K/2 coarse sweeps in a row are one run of K sweeps (even K)
    p = synth.make_problem(9, 9, 30, 4, data_seed=12)
    for algo in ("hals", "mu"):
        a = o.solve(p.M, 9, 9, p.V, p.W, algo, levels=2, K=8, cycle="wcycle")
        b = o.solve(p.M, 9, 9, p.V, p.W, algo, levels=2, K=8, cycle="vcycle")
        np.testing.assert_array_equal(a[0], b[0])
        np.testing.assert_array_equal(a[1], b[1])


def test_wcycle_order_visits_the_coarser_level_twice():
    K = 8
    one = [2] * (K // 8) + [3] * (K // 4) * 2 + [2] * (K // 4)   # a visit of level 2 with budget K/2
    assert _level_sequence("wcycle", 3, K) == [1] * (K // 4) + one + one + [1] * (K // 2)


def test_wcycle_data_flow():
    # rebuilt from the pinned pieces: pre-smoothing, restriction, two coarse W-cycles with
    # budget K/2 that pass V and W on to each other, prolongation, post-smoothing
    Ms, grids, V0, W0 = _bottom_up_problem()
    K = 8
    V, W = o.wcycle(Ms, grids, V0, W0, "hals", 3, K)
    Vp, Wp = o.smooth(Ms[0], V0, W0, "hals", K // 4)
    Vc = o.restrict(Vp, *grids[0])
    Wc = Wp
    for _ in range(2):
        # a level-2 visit with budget K/2: its own two level-3 visits with budget K/4
        Va, Wa = o.smooth(Ms[1], Vc, Wc, "hals", (K // 2) // 4)
        Vcc = o.restrict(Va, *grids[1])
        Vcc, Wa = o.smooth(Ms[2], Vcc, Wa, "hals", 2 * ((K // 2) // 2))
        Va = o.prolong(Vcc, *grids[2], *grids[1])
        Vc, Wc = o.smooth(Ms[1], Va, Wa, "hals", (K // 2) // 2)
    Vf, Wf = o.smooth(Ms[0], o.prolong(Vc, *grids[1], *grids[0]), Wc, "hals", K // 2)
    np.testing.assert_array_equal(V, Vf)
    np.testing.assert_array_equal(W, Wf)


# ---------------------------------------------------------------- time budgets
# Algorithm V-cycle gives its levels shares of a time T (T/4 before, T/4 to the coarser
# cycle, T/2 after); Table 1 is that split when a sweep on a level costs a quarter of one
# on the level above.

@pytest.mark.parametrize("L,K", [(2, 8), (3, 100), (3, 500), (4, 40), (5, 12)])
def test_time_split_with_quarter_costs_is_table1(L, K):
    costs = [0.25 ** l for l in range(L)]
    pre, coarse, post = o.time_schedule(K * costs[0], costs)
    assert pre == [K // 4] * (L - 1) and post == [K // 2] * (L - 1) and coarse == K


def test_time_split_by_hand():
    # T = 1000, costs 10 / 8 / 5: level 1 gets 1000 (250 before, 500 after: 25 and 50
    # sweeps), level 2 gets 250 (62.5 / 8 -> 7 before, 125 / 8 -> 15 after), level 3 gets
    # 62.5 (62.5 / 5 -> 12 sweeps)
    assert o.time_schedule(1000.0, [10.0, 8.0, 5.0]) == ([25, 7], 12, [50, 15])
    # one level: all of T
    assert o.time_schedule(90.0, [7.0]) == ([], 12, [])


def test_explicit_counts_with_table1_counts_are_the_vcycle():
    p = synth.make_problem(9, 9, 30, 4, data_seed=13)
    for algo in ("hals", "mu"):
        a = o.solve(p.M, 9, 9, p.V, p.W, algo, levels=3, K=8)
        b = o.solve(p.M, 9, 9, p.V, p.W, algo, levels=3, level_sweeps=([2, 2], 8, [4, 4]))
        np.testing.assert_array_equal(a[0], b[0])
        np.testing.assert_array_equal(a[1], b[1])


def test_explicit_counts_order():
    # level of every sweep in the order the cycle runs them, with distinct counts
    p = synth.make_problem(16, 16, 4, 2, data_seed=1)
    trace = []
    orig = dict(o.SWEEPS)
    o.SWEEPS["count"] = lambda M, V, W: (V, W)
    try:
        o.solve(p.M, 16, 16, p.V, p.W, algo="count", levels=3, level_sweeps=([1, 2], 3, [5, 4]), trace=trace)
    finally:
        o.SWEEPS.clear()
        o.SWEEPS.update(orig)
    assert [lvl for lvl, _ in trace] == [1] + [2] * 2 + [3] * 3 + [2] * 4 + [1] * 5
