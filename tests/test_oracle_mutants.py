"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in the oracle (monkeypatching a function of
oracle/nmf_oracle.py, on the CPU) and runs the pin tests that should notice it;
at least one of them must fail.  The unpatched oracle passes all of them
(the same tests run unpatched in the other test modules).
"""
import numpy as np
import pytest

import test_oracle_columns as tcol
import test_oracle_cycles as tc
import test_oracle_sweeps as ts
import test_oracle_transfer as tt
from oracle import nmf_oracle as o


def _fails(*checks):
    """True if at least one check raises AssertionError."""
    for chk in checks:
        try:
            chk()
        except AssertionError:
            return True
    return False


def _hals_col_drop_term(V, A, B, k):
    # dropped term: forgets the coupling to the other columns
    if B[k, k] <= 0.0:
        return
    V[:, k] = np.maximum(0.0, A[:, k] / B[k, k])


def _hals_col_wrong_sign(V, A, B, k):
    if B[k, k] <= 0.0:
        return
    others = [l for l in range(V.shape[1]) if l != k]
    V[:, k] = np.maximum(0.0, (A[:, k] + V[:, others] @ B[others, k]) / B[k, k])


def _hals_row_wrong_index(W, C, D, k):
    # wrong index: divides by the first diagonal entry of D instead of D_kk
    if D[k, k] <= 0.0:
        return
    others = [l for l in range(W.shape[0]) if l != k]
    W[k, :] = np.maximum(0.0, (C[k, :] - D[k, others] @ W[others, :]) / D[0, 0])


def _hals_no_clamp(V, A, B, k):
    if B[k, k] <= 0.0:
        return
    others = [l for l in range(V.shape[1]) if l != k]
    V[:, k] = (A[:, k] - V[:, others] @ B[others, k]) / B[k, k]


def _mu_old_v(M, V, W):
    # W-step with the old V (Jacobi instead of the algorithm's order)
    V = np.array(V, dtype=np.float64)
    W = np.array(W, dtype=np.float64)
    Vn = V * (M @ W.T) / np.maximum(V @ (W @ W.T), o.EPS_MU)
    Wn = W * (V.T @ M) / np.maximum((V.T @ V) @ W, o.EPS_MU)
    return Vn, Wn


def _mu_transposed(M, V, W):
    V = np.array(V, dtype=np.float64)
    W = np.array(W, dtype=np.float64)
    V = V * (M @ W.T) / np.maximum(V @ (W @ W.T), o.EPS_MU)
    W = W * (V.T @ M) / np.maximum((V @ V.T)[: V.shape[1], : V.shape[1]] @ W, o.EPS_MU)
    return V, W


def _nnls_clip(G, b, max_outer=None):
    # projection of the unconstrained solution instead of the active-set method
    return np.maximum(0.0, np.linalg.solve(G + 1e-12 * np.eye(len(b)), b))


def _objective_squared(M, V, W):
    R = np.asarray(M, dtype=np.float64) - np.asarray(V, dtype=np.float64) @ np.asarray(W, dtype=np.float64)
    return float((R * R).sum())


def _rd_half_floor(k):
    return (k // 2,)


def _weight_corner_2(dy, dx):
    return 2.0 if (dy and dx) else float((2 - abs(dy)) * (2 - abs(dx)))


def _weight_flat(dy, dx):
    return 1.0


def _vcycle_swapped_budget(Ms, grids, V, W, algo, L, K, level=0, hooks=None, trace=None):
    M = Ms[level]
    if L == 1:
        return o.smooth(M, V, W, algo, K, trace, level + 1)
    V, W = o.smooth(M, V, W, algo, K // 2, trace, level + 1)
    Vc = o.restrict(V, *grids[level])
    Vc, W = _vcycle_swapped_budget(Ms, grids, Vc, W, algo, L - 1, K, level + 1, hooks, trace)
    V = o.prolong(Vc, *grids[level + 1], *grids[level])
    return o.smooth(M, V, W, algo, K // 4, trace, level + 1)


def _vcycle_coarsest_half(Ms, grids, V, W, algo, L, K, level=0, hooks=None, trace=None):
    M = Ms[level]
    if L == 1:
        return o.smooth(M, V, W, algo, K // 2, trace, level + 1)
    V, W = o.smooth(M, V, W, algo, K // 4, trace, level + 1)
    Vc = o.restrict(V, *grids[level])
    Vc, W = _vcycle_coarsest_half(Ms, grids, Vc, W, algo, L - 1, K, level + 1, hooks, trace)
    V = o.prolong(Vc, *grids[level + 1], *grids[level])
    return o.smooth(M, V, W, algo, K // 2, trace, level + 1)


def _ni_fine_from_v0(Ms, grids, V0, W0, algo, L, K, level=0, trace=None, hooks=None):
    # fine-level sweeps start from the initial V instead of the prolonged coarse result
    M = Ms[level]
    if L == 1:
        return o.smooth(M, V0, W0, algo, K, trace, level + 1)
    Vc0 = o.restrict(V0, *grids[level])
    Vc, W = _ni_fine_from_v0(Ms, grids, Vc0, W0, algo, L - 1, K, level + 1, trace, hooks)
    if hooks is not None:
        hooks.append(("ni", level, Vc.copy(), W.copy()))
    o.prolong(Vc, *grids[level + 1], *grids[level])
    return o.smooth(M, V0, W, algo, (3 * K) // 4, trace, level + 1)


def _fmg_vcycle_from_v0(Ms, grids, V0, W0, algo, L, K, level=0, trace=None, hooks=None):
    # the V-cycle after the coarse FMG starts from the initial V instead of P(V')
    M = Ms[level]
    if L == 1:
        return o.smooth(M, V0, W0, algo, K, trace, level + 1)
    Vc0 = o.restrict(V0, *grids[level])
    Vc, W = _fmg_vcycle_from_v0(Ms, grids, Vc0, W0, algo, L - 1, K, level + 1, trace, hooks)
    if hooks is not None:
        hooks.append(("fmg", level, Vc.copy(), W.copy()))
    return o.vcycle(Ms, grids, V0, W, algo, L, (3 * K) // 4, level, None, trace)


def _fmg_coarse_w0(Ms, grids, V0, W0, algo, L, K, level=0, trace=None, hooks=None):
    # the V-cycle gets the initial W instead of the W that left the coarse FMG
    M = Ms[level]
    if L == 1:
        return o.smooth(M, V0, W0, algo, K, trace, level + 1)
    Vc0 = o.restrict(V0, *grids[level])
    Vc, W = _fmg_coarse_w0(Ms, grids, Vc0, W0, algo, L - 1, K, level + 1, trace, hooks)
    if hooks is not None:
        hooks.append(("fmg", level, Vc.copy(), W.copy()))
    V = o.prolong(Vc, *grids[level + 1], *grids[level])
    return o.vcycle(Ms, grids, V, W0, algo, L, (3 * K) // 4, level, None, trace)


def _wcycle_single_visit(Ms, grids, V, W, algo, L, K, level=0, trace=None):
    # the coarser level visited once (a V-cycle with half the coarse budget)
    M = Ms[level]
    if L == 1:
        return o.smooth(M, V, W, algo, K, trace, level + 1)
    V, W = o.smooth(M, V, W, algo, K // 4, trace, level + 1)
    Vc = o.restrict(V, *grids[level])
    Vc, W = _wcycle_single_visit(Ms, grids, Vc, W, algo, L - 1, K // 2, level + 1, trace)
    V = o.prolong(Vc, *grids[level + 1], *grids[level])
    return o.smooth(M, V, W, algo, K // 2, trace, level + 1)


def _bpp_variant(G, b, max_iter=None, info=None, flip_y=False, no_backup=False):
    G = np.asarray(G, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    r = b.shape[0]
    max_iter = 5 * r if max_iter is None else max_iter
    tol = 1e-12 * max(1.0, float(np.max(np.abs(b))))
    F = np.zeros(r, dtype=bool)
    x = np.zeros(r)
    y = -b.copy()
    if info is not None:
        info.update(method="bpp", iterations=0)
    for it in range(max_iter):
        yy = -y if flip_y else y
        bad = np.flatnonzero((F & (x < 0.0)) | (~F & (yy < -tol)))
        if bad.size == 0:
            return np.where(F, x, 0.0)
        if no_backup:
            F[bad] = ~F[bad]
        else:
            F[bad] = ~F[bad]
        P = np.flatnonzero(F)
        x = np.zeros(r)
        if P.size:
            x[P] = np.linalg.lstsq(G[np.ix_(P, P)], b[P], rcond=None)[0]
        y = G @ x - b
        y[F] = 0.0
    if info is not None:
        info["method"] = "active set"
    return o.nnls_active_set(G, b)


def _bpp_wrong_gradient_sign(G, b, max_iter=None, info=None):
    # the gradient off the passive set taken with the wrong sign
    return _bpp_variant(G, b, max_iter, info, flip_y=True)


def _restrict_columns_zero_padded(X, n):
    # the ends not renormalised: the missing neighbour counted as a zero
    X = np.asarray(X, dtype=np.float64)
    Xp = np.concatenate([np.zeros((X.shape[0], 1)), X, np.zeros((X.shape[0], 1))], axis=1)
    return np.stack([(Xp[:, 2 * j] + 2 * Xp[:, 2 * j + 1] + Xp[:, 2 * j + 2]) / 4
                     for j in range((n + 1) // 2)], axis=1)


_vcycle_both = o.vcycle_both


def _vcycle_both_w_injected(Ms, grids, ns, V, W, algo, L, K, level=0, trace=None, hooks=None):
    # W prolonged by injection (odd columns copied from the left neighbour) instead of Eq. (4.2)
    saved = o.prolong_columns
    try:
        o.prolong_columns = lambda Y, nc, n: np.asarray(Y, np.float64)[:, np.arange(n) // 2]
        return _vcycle_both(Ms, grids, ns, V, W, algo, L, K, level, trace, hooks)
    finally:
        o.prolong_columns = saved


def _time_schedule_half_to_coarse(T, costs):
    # the coarser cycle given T/2 instead of T/4 of each level's time
    L = len(costs)
    pre, post = [], []
    for l in range(L - 1):
        Tl = T / 2.0 ** l
        pre.append(int(np.floor(Tl / (4.0 * costs[l]) + 1e-9)))
        post.append(int(np.floor(Tl / (2.0 * costs[l]) + 1e-9)))
    return pre, int(np.floor(T / 2.0 ** (L - 1) / costs[L - 1] + 1e-9)), post


def _table1_checks():
    return [lambda row=row: tc.test_vcycle_sweep_allocation_matches_table1(row) for row in tc._table1_rows()]


MUTANTS = {
    "restriction corner weight 2": ("restriction_weight", _weight_corner_2,
                                    [tt.test_restriction_matches_printed_3x3_example,
                                     tt.test_interior_restriction_is_eq_4_1]),
    "restriction unweighted": ("restriction_weight", _weight_flat,
                               [tt.test_restriction_matches_printed_3x3_example]),
    "prolongation drops odd neighbour": ("rd_half", _rd_half_floor,
                                         [tt.test_prolongation_matches_printed_2x2_example]),
    "HALS dropped coupling term": ("hals_update_V_column", _hals_col_drop_term,
                                   [lambda: ts.test_hals_column_update_is_exact_1d_minimiser(0)]),
    "HALS wrong sign": ("hals_update_V_column", _hals_col_wrong_sign,
                        [lambda: ts.test_hals_column_update_is_exact_1d_minimiser(0)]),
    "HALS missing clamp": ("hals_update_V_column", _hals_no_clamp,
                           [ts.test_hals_clamp_produces_zeros,
                            lambda: ts.test_hals_column_update_is_exact_1d_minimiser(0)]),
    "HALS W-row wrong diagonal index": ("hals_update_W_row", _hals_row_wrong_index,
                                        [lambda: ts.test_hals_row_update_is_exact_1d_minimiser(0)]),
    "MU W-step with old V": ("mu_sweep", _mu_old_v, [ts.test_mu_elementwise_formula_by_loops]),
    "MU transposed Gram": ("mu_sweep", _mu_transposed, [ts.test_mu_elementwise_formula_by_loops]),
    "NNLS clipped least squares": ("nnls_active_set", _nnls_clip,
                                   [lambda: ts.test_nnls_equals_support_enumeration(s) for s in range(8)]),
    "objective squared": ("objective", _objective_squared, [ts.test_objective_is_frobenius_norm_by_loops]),
    "V-cycle pre/post budgets swapped": ("vcycle", _vcycle_swapped_budget, [tc.test_vcycle_order_follows_algorithm]),
    "V-cycle coarsest level short": ("vcycle", _vcycle_coarsest_half, _table1_checks()),
    "NI fine sweeps from V0": ("nested_iteration", _ni_fine_from_v0,
                               [lambda: tc.test_nested_iteration_data_flow("hals")]),
    "FMG V-cycle from V0": ("full_multigrid", _fmg_vcycle_from_v0, [lambda: tc.test_fmg_data_flow("hals")]),
    "FMG V-cycle with the initial W": ("full_multigrid", _fmg_coarse_w0, [lambda: tc.test_fmg_data_flow("hals")]),
    "BPP gradient with the wrong sign": ("nnls_bpp", _bpp_wrong_gradient_sign,
                                         [lambda s=s: ts.test_bpp_equals_support_enumeration(s) for s in range(8)]),
    "column restriction with zero-padded ends": ("restrict_columns", _restrict_columns_zero_padded,
                                                 [lambda: tcol.test_column_restriction_closed_form(5),
                                                  lambda: tcol.test_pixel_operators_are_tensor_products_of_the_column_operators(4, 5)]),
    "column V-cycle prolongs W by injection": ("vcycle_both", _vcycle_both_w_injected,
                                               [lambda: tcol.test_column_vcycle_data_flow("hals")]),
    "time split gives the coarser cycle half": ("time_schedule", _time_schedule_half_to_coarse,
                                                [tc.test_time_split_by_hand,
                                                 lambda: tc.test_time_split_with_quarter_costs_is_table1(3, 100)]),
    "W-cycle visits the coarser level once": ("wcycle", _wcycle_single_visit,
                                              [tc.test_wcycle_order_visits_the_coarser_level_twice,
                                               tc.test_wcycle_data_flow]),
}


@pytest.mark.parametrize("name", list(MUTANTS))
def test_pins_catch_planted_mistake(name, monkeypatch):
    attr, bad, checks = MUTANTS[name]
    monkeypatch.setattr(o, attr, bad)
    if attr == "wcycle":
        monkeypatch.setitem(o.CYCLES, "wcycle", bad)
    if attr == "mu_sweep":
        monkeypatch.setitem(o.SWEEPS, "mu", bad)
    assert _fails(*checks), f"no pin noticed: {name}"
