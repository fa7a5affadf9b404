"""Pins for the oracle's inner NMF algorithms (Section 2, Appendix A)."""
import itertools

import numpy as np
import pytest

from oracle import nmf_oracle as o
from paper_1009_0881_gb300 import synth


def _tiny(seed=0, m=7, n=6, r=3):
    rng = np.random.default_rng(seed)
    M = rng.random((m, n))
    V = rng.random((m, r))
    W = rng.random((r, n))
    return M, V, W


def _f2(M, V, W):
    E = M - V @ W
    return float(np.sum(E * E))


# --------------------------- objective ---------------------------------------

def test_objective_is_frobenius_norm_by_loops():
    M, V, W = _tiny(1)
    s = 0.0
    for i in range(M.shape[0]):
        for j in range(M.shape[1]):
            vw = sum(V[i, k] * W[k, j] for k in range(V.shape[1]))
            s += (M[i, j] - vw) ** 2
    assert abs(o.objective(M, V, W) - np.sqrt(s)) < 1e-13


def test_column_expansion_identity_eq_6_1():
    # Eq. (6.1) equals the direct squared error
    for seed in range(3):
        M, V, W = _tiny(seed, 20, 15, 4)
        assert abs(o.objective_sq_expanded(M, V, W) - o.objective(M, V, W) ** 2) <= 1e-10 * _f2(M, V, W)


# --------------------------- HALS --------------------------------------------

def _brute_min_1d(fun, hi):
    """min over t in [0, hi] of a convex quadratic by dense scan + exact parabola through 3 points."""
    ts = np.linspace(0.0, hi, 2001)
    vals = np.array([fun(t) for t in ts])
    t0 = ts[int(np.argmin(vals))]
    # parabola through t = 0, 1, 2 gives the exact quadratic coefficients
    f0, f1, f2 = fun(0.0), fun(1.0), fun(2.0)
    a = (f2 - 2 * f1 + f0) / 2.0
    b = f1 - f0 - a
    vertex = max(0.0, -b / (2 * a)) if a > 0 else t0
    assert abs(vertex - t0) <= hi / 2000 + 1e-12  # scan and parabola agree
    return vertex


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_hals_column_update_is_exact_1d_minimiser(seed):
    # Section 2.3: each entry V_ik is the minimiser over V_ik >= 0 with all else fixed
    M, V, W = _tiny(seed)
    V = V.copy()
    A, B = M @ W.T, W @ W.T
    for k in range(V.shape[1]):
        before = V.copy()
        o.hals_update_V_column(V, A, B, k)
        for i in range(V.shape[0]):
            def fun(t, i=i):
                X = before.copy()
                X[i, k] = t
                return _f2(M, X, W)
            assert abs(V[i, k] - _brute_min_1d(fun, 5.0)) < 1e-9
        # entries of other columns untouched
        np.testing.assert_array_equal(np.delete(V, k, 1), np.delete(before, k, 1))


@pytest.mark.parametrize("seed", [0, 1])
def test_hals_row_update_is_exact_1d_minimiser(seed):
    M, V, W = _tiny(seed + 10)
    W = W.copy()
    C, D = V.T @ M, V.T @ V
    for k in range(W.shape[0]):
        before = W.copy()
        o.hals_update_W_row(W, C, D, k)
        for j in range(W.shape[1]):
            def fun(t, j=j):
                X = before.copy()
                X[k, j] = t
                return _f2(M, V, X)
            assert abs(W[k, j] - _brute_min_1d(fun, 5.0)) < 1e-9


def test_hals_clamp_produces_zeros():
    # a data matrix that wants a negative coefficient: the update clamps at exactly 0
    M = np.array([[0.0, 1.0], [1.0, 0.0]])
    V = np.array([[1.0, 1.0], [1.0, 0.0]])
    W = np.array([[1.0, 0.0], [0.0, 1.0]])
    V2 = V.copy()
    o.hals_update_V_column(V2, M @ W.T, W @ W.T, 0)
    assert V2[0, 0] == 0.0 and V2[1, 0] == 1.0


def test_hals_objective_nonincreasing_per_column():
    M, V, W = _tiny(4, 12, 9, 4)
    V, W = V.copy(), W.copy()
    f = _f2(M, V, W)
    for _ in range(5):
        A, B = M @ W.T, W @ W.T
        for k in range(4):
            o.hals_update_V_column(V, A, B, k)
            g = _f2(M, V, W)
            assert g <= f * (1 + 1e-14)
            f = g
        C, D = V.T @ M, V.T @ V
        for k in range(4):
            o.hals_update_W_row(W, C, D, k)
            g = _f2(M, V, W)
            assert g <= f * (1 + 1e-14)
            f = g


def test_hals_zero_diagonal_skips_update():
    M, V, W = _tiny(5)
    W = W.copy()
    W[1] = 0.0
    V2 = V.copy()
    o.hals_update_V_column(V2, M @ W.T, W @ W.T, 1)
    np.testing.assert_array_equal(V2, V)


def test_hals_drives_planted_exact_factorisation_to_zero():
    # M = V0 W0 exactly (no noise): HALS from U[0,1] reaches relative error < 1e-6
    p = synth.make_problem(16, 16, 80, 4, sigma=1.0, data_seed=2, noise=0.0)
    M = p.V0.astype(np.float64) @ p.W0.astype(np.float64)  # exact rank 4
    V, W = p.V.astype(np.float64), p.W.astype(np.float64)
    for _ in range(400):
        V, W = o.hals_sweep(M, V, W)
    assert o.objective(M, V, W) / np.linalg.norm(M) < 1e-6


def test_hals_planted_is_fixed_point():
    p = synth.make_problem(6, 6, 20, 3, data_seed=2, noise=0.0)
    V0, W0 = p.V0.astype(np.float64), p.W0.astype(np.float64)
    M = V0 @ W0
    V, W = o.hals_sweep(M, V0, W0)
    np.testing.assert_allclose(V @ W, M, rtol=1e-10, atol=1e-12)


def test_hals_sweep_order_v_then_w():
    # The W-step uses the new V: compare against composing the two half-steps
    M, V, W = _tiny(7)
    V1, W1 = o.hals_sweep(M, V, W)
    Vb = V.copy()
    A, B = M @ W.T, W @ W.T
    for k in range(3):
        o.hals_update_V_column(Vb, A, B, k)
    Wb = W.copy()
    C, D = Vb.T @ M, Vb.T @ Vb
    for k in range(3):
        o.hals_update_W_row(Wb, C, D, k)
    np.testing.assert_array_equal(V1, Vb)
    np.testing.assert_array_equal(W1, Wb)


# --------------------------- MU ----------------------------------------------

def test_mu_objective_nonincreasing():
    # Section 2.2: MU guarantees a nonincreasing objective
    p = synth.make_problem(8, 8, 30, 4, data_seed=5)
    M = p.M.astype(np.float64)
    V, W = p.V.astype(np.float64), p.W.astype(np.float64)
    f = o.objective(M, V, W)
    for _ in range(50):
        V, W = o.mu_sweep(M, V, W)
        g = o.objective(M, V, W)
        assert g <= f * (1 + 1e-13)
        f = g


def test_mu_planted_is_fixed_point_and_zeros_stay_zero():
    p = synth.make_problem(6, 6, 20, 3, data_seed=4, noise=0.0)
    V0, W0 = p.V0.astype(np.float64), p.W0.astype(np.float64)
    M = V0 @ W0
    V, W = o.mu_sweep(M, V0, W0)
    np.testing.assert_allclose(V, V0, rtol=1e-12, atol=1e-300)
    np.testing.assert_allclose(W, W0, rtol=1e-12, atol=1e-300)
    assert (W[W0 == 0] == 0).all()


def test_mu_elementwise_formula_by_loops():
    M, V, W = _tiny(8, 5, 4, 2)
    V1, W1 = o.mu_sweep(M, V, W)
    m, r = V.shape
    n = W.shape[1]
    Vx = np.zeros_like(V)
    for i in range(m):
        for k in range(r):
            num = sum(M[i, j] * W[k, j] for j in range(n))
            den = sum(V[i, l] * sum(W[l, j] * W[k, j] for j in range(n)) for l in range(r))
            Vx[i, k] = V[i, k] * num / den
    np.testing.assert_allclose(V1, Vx, rtol=1e-13)
    Wx = np.zeros_like(W)
    for k in range(r):
        for j in range(n):
            num = sum(Vx[i, k] * M[i, j] for i in range(m))
            den = sum(sum(Vx[i, k] * Vx[i, l] for i in range(m)) * W[l, j] for l in range(r))
            Wx[k, j] = W[k, j] * num / den
    np.testing.assert_allclose(W1, Wx, rtol=1e-13)


# --------------------------- NNLS / ANLS -------------------------------------

def _nnls_brute(G, b):
    """Enumerate all supports: solve the unconstrained problem on each, keep feasible, take the best."""
    r = len(b)
    best, bestx = 0.0, np.zeros(r)
    for size in range(1, r + 1):
        for S in itertools.combinations(range(r), size):
            S = list(S)
            try:
                xs = np.linalg.solve(G[np.ix_(S, S)], b[S])
            except np.linalg.LinAlgError:
                continue
            if (xs < 0).any():
                continue
            x = np.zeros(r)
            x[S] = xs
            val = 0.5 * x @ G @ x - b @ x
            if val < best - 1e-14:
                best, bestx = val, x
    return bestx


@pytest.mark.parametrize("seed", range(8))
def test_nnls_equals_support_enumeration(seed):
    rng = np.random.default_rng(seed)
    r = 3 + seed % 6  # up to 8 (2^8 supports)
    F = rng.standard_normal((r + 4, r))
    y = rng.standard_normal(r + 4)
    G, b = F.T @ F, F.T @ y
    x = o.nnls_active_set(G, b)
    np.testing.assert_allclose(x, _nnls_brute(G, b), atol=1e-10)


@pytest.mark.parametrize("seed", range(5))
def test_nnls_kkt(seed):
    rng = np.random.default_rng(100 + seed)
    r = 10
    F = rng.random((30, r))
    y = rng.standard_normal(30)
    G, b = F.T @ F, F.T @ y
    x = o.nnls_active_set(G, b)
    grad = G @ x - b
    scale = np.abs(b).max()
    assert (x >= 0).all()
    assert (grad >= -1e-10 * scale).all()
    assert np.abs(x * grad).max() <= 1e-10 * scale * max(1.0, x.max())


def test_nnls_matches_scipy_on_least_squares_form():
    scipy_opt = pytest.importorskip("scipy.optimize")
    rng = np.random.default_rng(3)
    F = rng.random((40, 12))
    y = rng.random(40) - 0.3
    x_ref, _ = scipy_opt.nnls(F, y)
    x = o.nnls_active_set(F.T @ F, F.T @ y)
    np.testing.assert_allclose(x, x_ref, atol=1e-9)


def test_nnls_singular_gram_gives_optimal_objective():
    # fewer observations than variables (m_l < r at a coarse level): x not unique, value unique
    rng = np.random.default_rng(9)
    F = rng.random((4, 7))
    y = rng.random(4)
    G, b = F.T @ F, F.T @ y
    x = o.nnls_active_set(G, b)
    assert (x >= 0).all()
    val = 0.5 * x @ G @ x - b @ x
    scipy_opt = pytest.importorskip("scipy.optimize")
    xs, _ = scipy_opt.nnls(F, y)
    assert abs(val - (0.5 * xs @ G @ xs - b @ xs)) < 1e-10


def test_anls_sweep_is_blockwise_optimal_and_ignores_v():
    p = synth.make_problem(6, 6, 25, 4, data_seed=6)
    M = p.M.astype(np.float64)
    V, W = p.V.astype(np.float64), p.W.astype(np.float64)
    V1, W1 = o.anls_sweep(M, V, W)
    V2, W2 = o.anls_sweep(M, np.zeros_like(V), W)  # V input unused (ANLS needs only W)
    np.testing.assert_array_equal(V1, V2)
    np.testing.assert_array_equal(W1, W2)
    # KKT of the V-step with the incoming W, and of the W-step with the new V
    gV = (V1 @ W - M) @ W.T
    gW = V1.T @ (V1 @ W1 - M)
    s = np.abs(M).max() * 10
    assert (gV >= -1e-9 * s).all() and np.abs(V1 * gV).max() < 1e-9 * s
    assert (gW >= -1e-9 * s).all() and np.abs(W1 * gW).max() < 1e-9 * s
    assert o.objective(M, V1, W1) <= o.objective(M, V, W)


def _at(precision, fn):
    saved = o.PRECISION
    try:
        o.PRECISION = precision
        return fn()
    finally:
        o.PRECISION = saved


def test_float32_products_exact_on_small_integers():
    # products of small integers are exact in float32, so the rounded variant equals FP64
    rng = np.random.default_rng(21)
    X = rng.integers(0, 9, (7, 30)).astype(np.float64)
    Y = rng.integers(0, 9, (30, 5)).astype(np.float64)
    np.testing.assert_array_equal(_at("fp32", lambda: o.product(X, Y)), X @ Y)
    np.testing.assert_array_equal(_at("bf16", lambda: o.product(X, Y, True)), X @ Y)


def test_float32_products_within_rounding_bound():
    # |fl32(X Y) - X Y| <= (K + 2) u |X| |Y| entrywise (operand rounding plus a K-term sum),
    # and the rounding does change the result
    rng = np.random.default_rng(22)
    X, Y = rng.random((20, 300)), rng.random((300, 9))
    P = _at("fp32", lambda: o.product(X, Y))
    exact = X @ Y
    u = 2.0 ** -24
    assert np.all(np.abs(P - exact) <= (300 + 2) * u * (np.abs(X) @ np.abs(Y)))
    assert np.any(P != exact)
    assert o.PRECISION is None


def test_bfloat16_rounding_definition():
    # 8 significant bits: exact for short mantissas, nearest otherwise, ties to even
    e = 2.0 ** -8
    x = np.array([1.5, 3.0, 0.25, -6.5, 1 + e, 1 + 3 * e, 1 + e + 2.0 ** -12, 0.0])
    want = np.array([1.5, 3.0, 0.25, -6.5, 1.0, 1 + 2 * 2 * e, 1 + 2 * e, 0.0])
    np.testing.assert_array_equal(o.round_bf16(x), want)
    rng = np.random.default_rng(5)
    y = rng.standard_normal(10000) * 10.0 ** rng.integers(-5, 5, 10000)
    assert np.all(np.abs(o.round_bf16(y) - y) <= e * np.abs(y))
    torch = pytest.importorskip("torch")
    ref = torch.from_numpy(y.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(o.round_bf16(y), ref)


def test_bf16_mode_rounds_only_the_products_with_M():
    rng = np.random.default_rng(23)
    M, W = rng.random((30, 50)), rng.random((4, 50))
    A = _at("bf16", lambda: o.product(M, W.T, True))
    B = _at("bf16", lambda: o.product(W, W.T))
    # float32 accumulation of 50 terms: within 50 u of the exact product of the rounded operands
    np.testing.assert_allclose(A, o.round_bf16(M) @ o.round_bf16(W).T, rtol=50 * 2.0 ** -24)
    np.testing.assert_allclose(B, W.astype(np.float32).astype(np.float64) @ W.astype(np.float32).astype(np.float64).T,
                               rtol=50 * 2.0 ** -24)
    assert np.abs(A - M @ W.T).max() > 1e-4 * np.abs(M @ W.T).max()


def test_solve_precision_option_restores_fp64():
    p = synth.make_problem(8, 8, 20, 3, data_seed=2)
    a = o.solve(p.M, 8, 8, p.V, p.W, "hals", levels=2, K=4, precision="fp32")
    assert o.PRECISION is None
    b = o.solve(p.M, 8, 8, p.V, p.W, "hals", levels=2, K=4)
    assert not np.array_equal(a[0], b[0])
    # float32 storage of the iterates
    np.testing.assert_array_equal(a[0], a[0].astype(np.float32).astype(np.float64))


# ---- block principal pivoting (the ANLS footnote of Section 2.1) --------------------------

@pytest.mark.parametrize("seed", range(8))
def test_bpp_equals_support_enumeration(seed):
    rng = np.random.default_rng(200 + seed)
    r = 3 + seed % 6
    F = rng.standard_normal((r + 4, r))
    y = rng.standard_normal(r + 4)
    G, b = F.T @ F, F.T @ y
    info = {}
    x = o.nnls_bpp(G, b, info=info)
    assert info["method"] == "bpp"
    np.testing.assert_allclose(x, _nnls_brute(G, b), atol=1e-10)


@pytest.mark.parametrize("r", [12, 30, 49, 64])
def test_bpp_converges_by_itself_and_meets_kkt(r):
    # positive definite Gram matrices of the ANLS shapes: block pivoting ends on its own
    # (no fallback) at the point the active-set method finds, where the KKT conditions hold
    rng = np.random.default_rng(r)
    F = rng.random((3 * r, r))
    y = rng.standard_normal(3 * r) + F @ np.maximum(0.0, rng.standard_normal(r))
    G, b = F.T @ F, F.T @ y
    info = {}
    x = o.nnls_bpp(G, b, info=info)
    assert info["method"] == "bpp" and info["iterations"] <= 5 * r
    np.testing.assert_allclose(x, o.nnls_active_set(G, b), atol=1e-9 * max(1.0, np.abs(x).max()))
    grad = G @ x - b
    scale = np.abs(b).max()
    assert (x >= 0).all() and (grad >= -1e-9 * scale).all()
    assert np.abs(x * grad).max() <= 1e-9 * scale * max(1.0, x.max())


def test_bpp_exchanges_many_variables_per_iteration():
    # the point of the method: far fewer iterations than variables it has to move
    rng = np.random.default_rng(77)
    r = 49
    F = rng.random((200, r))
    y = F @ np.where(rng.random(r) < 0.6, rng.random(r), 0.0)
    G, b = F.T @ F, F.T @ y
    info = {}
    x = o.nnls_bpp(G, b, info=info)
    assert info["method"] == "bpp"
    assert info["iterations"] < np.count_nonzero(x)


def test_bpp_singular_gram_falls_back_to_active_set():
    rng = np.random.default_rng(9)
    F = rng.random((4, 7))
    y = rng.random(4)
    G, b = F.T @ F, F.T @ y
    info = {}
    x = o.nnls_bpp(G, b, info=info)
    assert info["method"] == "active set"
    np.testing.assert_array_equal(x, o.nnls_active_set(G, b))


def test_anls_bpp_sweep_equals_active_set_sweep():
    p = synth.make_problem(8, 8, 60, 6, data_seed=8)
    M = p.M.astype(np.float64)
    V1, W1 = o.anls_sweep(M, p.V.astype(np.float64), p.W.astype(np.float64))
    V2, W2 = o.anls_bpp_sweep(M, p.V.astype(np.float64), p.W.astype(np.float64))
    np.testing.assert_allclose(V2, V1, atol=1e-10)
    np.testing.assert_allclose(W2, W1, atol=1e-10)
