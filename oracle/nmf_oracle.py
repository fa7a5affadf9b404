"""FP64 CPU oracle for the multilevel NMF of Gillis & Glineur,
"A Multilevel Approach for Nonnegative Matrix Factorization" (arXiv:1009.0881).

TEST INFRASTRUCTURE ONLY.  This module is the plain, slow, obviously correct
statement of what the GPU library computes.  Only the test suite, the smoke check
in ``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import it.
The CUDA library never calls it, shares no code with it and must fail loudly
when its extension is missing instead of falling back here.

Conventions (paper notation): M is m x n (column j = vectorised image j, pixel
(y, x) of an H x W grid at row y*W + x), V is m x r, W is r x n.  Everything is
float64.  Matrix products are numpy library calls; no step is blocked, fused or
reordered beyond what the paper states.

Readings of points the paper leaves open (each marked READING below):
  * grid sides that are not 2^a + 1: coarse side = ceil(side / 2), coarse (i, j)
    sits on fine (2i, 2j); border stencil weights are the in-bounds subset,
    renormalised to sum 1 (this reproduces the printed 3x3 -> 2x2 example);
  * prolongation at an even-size border averages over the in-bounds coarse
    neighbours only;
  * HALS with B_kk = 0 (resp. D_kk = 0) leaves that column of V (row of W)
    unchanged;
  * MU denominators are floored at EPS_MU = 1e-30;
  * the time budget T of the cycles becomes a sweep budget K: a level gets
    floor(K/4) pre-sweeps and floor(K/2) post-sweeps, the coarsest K sweeps
    (Table 1: 3k, ..., 3k, 4k sweeps with K = 4k);
  * NNLS (Appendix A.2) is Lawson-Hanson started from x = 0, with dual
    tolerance 1e-12 * max(1, max |b|) and an outer-iteration cap of 3r.

Pins: every function here is checked in tests/test_oracle_*.py against the
printed operator examples of Section 4.2, closed forms, invariants (row sums,
nonnegativity, monotone objective), brute-force minimisation on tiny inputs and
the transfer-error bound of Section 4.1.  The paper's dataset tables (Tables
3-5) cannot be reproduced without the datasets: parity unpinned for those
numbers, which the oracle does not claim to match.
"""
from __future__ import annotations

import numpy as np

EPS_MU = 1e-30


# ---------------------------------------------------------------------------
# Section 4.2: coarse grids
# ---------------------------------------------------------------------------

def coarse_grid(h: int, w: int) -> tuple[int, int]:
    """Keep one point out of two in each direction (Section 4.2, Figure 2).

    For a side 2^a + 1 this gives 2^(a-1) + 1.  READING for other sides:
    ceil(side / 2), i.e. the points 0, 2, 4, ... of the finer grid.
    """
    return (h + 1) // 2, (w + 1) // 2


def grid_hierarchy(h: int, w: int, levels: int) -> list[tuple[int, int]]:
    """Grids of levels 1 (finest, the input) .. L (coarsest)."""
    grids = [(h, w)]
    for _ in range(levels - 1):
        grids.append(coarse_grid(*grids[-1]))
    return grids


# ---------------------------------------------------------------------------
# Section 4.2, Eq. (4.1): full-weighting restriction
# ---------------------------------------------------------------------------

def restriction_weight(dy: int, dx: int) -> float:
    """Eq. (4.1): weight 4 at the centre, 2 on the edges, 1 at the corners (/16)."""
    return float((2 - abs(dy)) * (2 - abs(dx)))


def restrict(X: np.ndarray, h: int, w: int) -> np.ndarray:
    """Column-wise restriction R X of an (h*w) x c matrix (Section 4.1, Eq. (4.1)).

    Coarse pixel (i, j) is the weighted mean of the fine pixels (2i+dy, 2j+dx),
    dy, dx in {-1, 0, 1}.  On the border only in-bounds fine pixels are kept and
    the weights are divided by their sum ("weights adapted correspondingly").
    """
    X = np.asarray(X, dtype=np.float64)
    assert X.shape[0] == h * w
    hc, wc = coarse_grid(h, w)
    out = np.zeros((hc * wc,) + X.shape[1:])
    for i in range(hc):
        for j in range(wc):
            acc = np.zeros(X.shape[1:])
            total = 0.0
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    y, x = 2 * i + dy, 2 * j + dx
                    if 0 <= y < h and 0 <= x < w:
                        wt = restriction_weight(dy, dx)
                        acc = acc + wt * X[y * w + x]
                        total += wt
            out[i * wc + j] = acc / total
    return out


def restriction_matrix(h: int, w: int) -> np.ndarray:
    """The matrix R in R_+^{m' x m} of the restriction (Section 4.1)."""
    return restrict(np.eye(h * w), h, w)


# ---------------------------------------------------------------------------
# Section 4.2, Eq. (4.2): prolongation by the mean of coarse neighbours
# ---------------------------------------------------------------------------

def rd_half(k: int) -> tuple[int, ...]:
    """rd(k/2) of Eq. (4.2): {k/2} for even k, {(k-1)/2, (k+1)/2} for odd k."""
    if k % 2 == 0:
        return (k // 2,)
    return ((k - 1) // 2, (k + 1) // 2)


def prolong(Y: np.ndarray, hc: int, wc: int, h: int, w: int) -> np.ndarray:
    """Column-wise prolongation P Y of an (hc*wc) x c matrix to the h x w grid (Eq. (4.2)).

    Fine pixel (i, j) is the mean of the coarse pixels (i', j') with
    i' in rd(i/2), j' in rd(j/2).  READING: neighbours outside the coarse grid
    (only possible at an even-size border) are dropped from the mean.
    """
    Y = np.asarray(Y, dtype=np.float64)
    assert Y.shape[0] == hc * wc
    out = np.zeros((h * w,) + Y.shape[1:])
    for i in range(h):
        for j in range(w):
            nbrs = [(a, b) for a in rd_half(i) if a < hc for b in rd_half(j) if b < wc]
            acc = np.zeros(Y.shape[1:])
            for a, b in nbrs:
                acc = acc + Y[a * wc + b]
            out[i * w + j] = acc / len(nbrs)
    return out


def prolongation_matrix(hc: int, wc: int, h: int, w: int) -> np.ndarray:
    """The matrix P in R_+^{m x m'} of the prolongation (Section 4.1)."""
    return prolong(np.eye(hc * wc), hc, wc, h, w)


def smoothness(M: np.ndarray, h: int, w: int) -> float:
    """s_M = ||M - P(R(M))||_F / ||M||_F (Section 4.1)."""
    hc, wc = coarse_grid(h, w)
    PRM = prolong(restrict(M, h, w), hc, wc, h, w)
    return float(np.linalg.norm(M - PRM) / np.linalg.norm(M))


# ---------------------------------------------------------------------------
# Objective, problem (NMF) of Section 2
# ---------------------------------------------------------------------------

def objective(M: np.ndarray, V: np.ndarray, W: np.ndarray) -> float:
    """||M - VW||_F (the square root of the objective of problem (NMF))."""
    E = np.asarray(M, np.float64) - np.asarray(V, np.float64) @ np.asarray(W, np.float64)
    return float(np.sqrt(np.sum(E * E)))


def objective_sq_expanded(M: np.ndarray, V: np.ndarray, W: np.ndarray) -> float:
    """||M - VW||_F^2 by the column expansion of Eq. (6.1):
    sum_j ||M_:j||^2 - 2 (M_:j^T V) W_:j + W_:j^T (V^T V) W_:j."""
    total = 0.0
    VtV = V.T @ V
    for j in range(M.shape[1]):
        mj = M[:, j]
        wj = W[:, j]
        total += mj @ mj - 2.0 * (mj @ V) @ wj + wj @ VtV @ wj
    return float(total)


# ---------------------------------------------------------------------------
# The four products of a sweep (Appendix A.1): A = M W^T, B = W W^T, C = V^T M,
# D = V^T V, and the precision they are taken in.  FP64 by default (PRECISION None).
# READING: the paper computes in double and is silent on rounding; two settings
# state the arithmetic of reduced-precision implementations, step by step:
#   "fp32": the four products are float32 matrix products (float32 operands,
#           float32 accumulation, a library matmul), and V and W are stored in
#           float32 after each half of a sweep (V before C and D are formed);
#   "bf16": the precision form of this library: A and C have bfloat16 operands
#           (M and the factor, rounded to nearest, ties to even) accumulated in
#           float32, B and D are float32 products, V, W stored in float32.
# Cycles that start on a level with fewer pixels than the rank (nested iteration
# and full multigrid on the 19 x 19 grid with three levels: 25 pixels, r = 49) and
# short sweep budgets are sensitive to these roundings; solve(..., precision=...)
# sets the mode for one solve.
# ---------------------------------------------------------------------------
PRECISION = None


def round_bf16(X: np.ndarray) -> np.ndarray:
    """X rounded to bfloat16 (8 significant bits), returned as float64.

    From the format's definition: a bfloat16 is the upper 16 bits of a float32;
    rounding to nearest with ties to even adds 0x7FFF plus the lowest kept bit to
    the float32 bit pattern, then clears the low 16 bits."""
    x = np.ascontiguousarray(X, dtype=np.float32)
    bits = x.view(np.uint32).astype(np.uint64)
    bits = (bits + 0x7FFF + ((bits >> 16) & 1)) & 0xFFFF0000
    return bits.astype(np.uint32).view(np.float32).astype(np.float64)


def product(X: np.ndarray, Y: np.ndarray, factor_with_M: bool = False) -> np.ndarray:
    """X @ Y at the current PRECISION; factor_with_M marks A = M W^T and C = V^T M."""
    if PRECISION is None:
        return X @ Y
    if PRECISION == "bf16" and factor_with_M:
        X, Y = round_bf16(X), round_bf16(Y)
    return (np.asarray(X, np.float32) @ np.asarray(Y, np.float32)).astype(np.float64)


def store(X: np.ndarray) -> np.ndarray:
    """An iterate as stored between sweeps at the current PRECISION."""
    return X if PRECISION is None else np.asarray(X, np.float32).astype(np.float64)


# ---------------------------------------------------------------------------
# Section 2.3, Algorithm HALS
# ---------------------------------------------------------------------------

def hals_update_V_column(V: np.ndarray, A: np.ndarray, B: np.ndarray, k: int) -> None:
    """Column k of V set to the exact minimiser of ||M - VW||_F over V_:k >= 0, the other
    columns fixed (Section 2.3), in place.

    With the residual R_k = M - sum_{l != k} V_:l W_l: the objective is
    ||R_k - V_:k W_k:||^2, a separable quadratic in the entries of V_:k with curvature
    ||W_k:||^2 = B_kk and minimiser R_k W_k:^T / B_kk; clipping it at 0 is exact
    entrywise.  R_k W_k:^T expands to A_:k - sum_{l != k} V_:l B_lk with A = M W^T,
    B = W W^T, so the residual is never formed.
    READING: B_kk = 0 (row k of W is zero) leaves V_:k unchanged.
    """
    if B[k, k] <= 0.0:
        return
    others = [l for l in range(V.shape[1]) if l != k]
    V[:, k] = np.maximum(0.0, (A[:, k] - V[:, others] @ B[others, k]) / B[k, k])


def hals_update_W_row(W: np.ndarray, C: np.ndarray, D: np.ndarray, k: int) -> None:
    """Row k of W set to the exact minimiser of ||M - VW||_F over W_k: >= 0, the other rows
    fixed (Section 2.3), in place: by the same argument as for a column of V, the
    minimiser is V_:k^T R_k / ||V_:k||^2 clipped at 0, with V_:k^T R_k = C_k: -
    sum_{l != k} D_kl W_l:, C = V^T M, D = V^T V.
    READING: D_kk = 0 (column k of V is zero) leaves W_k: unchanged.
    """
    if D[k, k] <= 0.0:
        return
    others = [l for l in range(W.shape[0]) if l != k]
    W[k, :] = np.maximum(0.0, (C[k, :] - D[k, others] @ W[others, :]) / D[k, k])


def hals_sweep(M, V, W):
    """One HALS sweep (Section 2.3): block coordinate descent on ||M - VW||_F over the
    columns of V in order 1..r (each with the columns already updated), then over the rows
    of W in order with the new V."""
    V = np.array(V, dtype=np.float64)
    W = np.array(W, dtype=np.float64)
    A = product(M, W.T, True)
    B = product(W, W.T)
    for k in range(V.shape[1]):
        hals_update_V_column(V, A, B, k)
    V = store(V)
    C = product(V.T, M, True)
    D = product(V.T, V)
    for k in range(W.shape[0]):
        hals_update_W_row(W, C, D, k)
    return V, W


# ---------------------------------------------------------------------------
# Section 2.2, Algorithm MU (Lee and Seung)
# ---------------------------------------------------------------------------

def mu_sweep(M, V, W):
    """V <- V o [M W^T] / [V (W W^T)], then W <- W o [V^T M] / [(V^T V) W] (new V).

    READING: denominators are floored at EPS_MU (0/0 -> 0).
    """
    V = np.array(V, dtype=np.float64)
    W = np.array(W, dtype=np.float64)
    V = store(V * product(M, W.T, True) / np.maximum(V @ product(W, W.T), EPS_MU))
    W = W * product(V.T, M, True) / np.maximum(product(V.T, V) @ W, EPS_MU)
    return V, W


# ---------------------------------------------------------------------------
# Section 2.1 / Appendix A.2: ANLS with active-set NNLS
# ---------------------------------------------------------------------------

class NNLSNotConverged(RuntimeError):
    pass


def nnls_active_set(G: np.ndarray, b: np.ndarray, max_outer: int | None = None) -> np.ndarray:
    """argmin_{x >= 0} 1/2 x^T G x - b^T x, G = F^T F symmetric PSD.

    Lawson-Hanson active-set method (Appendix A.2, steps 0-3): variables are
    split into active (held at zero) and passive sets; the unconstrained least
    squares problem on the passive set is solved through its normal equations
    G_PP z_P = b_P; optimality is checked through the dual w = b - G x; an
    infeasible passive solution is interpolated back towards the previous x,
    so the objective decreases at every exchange.
    """
    G = np.asarray(G, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    r = b.shape[0]
    if max_outer is None:
        max_outer = 3 * r
    tol = 1e-12 * max(1.0, float(np.max(np.abs(b))) if r else 1.0)
    x = np.zeros(r)
    passive = np.zeros(r, dtype=bool)
    outer = 0
    while True:
        w = b - G @ x  # minus the gradient
        candidates = (~passive) & (w > tol)
        if not candidates.any():
            return x
        if outer >= max_outer:
            raise NNLSNotConverged(f"no convergence after {outer} exchanges")
        outer += 1
        j = int(np.argmax(np.where(candidates, w, -np.inf)))
        passive[j] = True
        while True:
            P = np.flatnonzero(passive)
            z = np.zeros(r)
            z[P] = np.linalg.solve(G[np.ix_(P, P)], b[P])
            if np.all(z[P] > 0.0):
                x = z
                break
            bad = P[z[P] <= 0.0]
            ratios = x[bad] / (x[bad] - z[bad])
            alpha = np.min(ratios)
            x = x + alpha * (z - x)
            x[bad[ratios <= alpha]] = 0.0  # the blocking variables land exactly on 0
            passive = passive & (x > 0.0)
            x[~passive] = 0.0


def nnls_bpp(G: np.ndarray, b: np.ndarray, max_iter: int | None = None, info: dict | None = None) -> np.ndarray:
    """argmin_{x >= 0} 1/2 x^T G x - b^T x by block principal pivoting.

    The ANLS footnote of Section 2.1 names this method (Kim and Park) as an
    alternative NNLS solver inside ANLS.  Variables are split into a passive set F
    (free) and its complement (held at zero).  Each iteration solves the
    unconstrained problem on F, x_F = G_FF^{-1} b_F, and forms the gradient
    y = G x - b on the complement.  The pair is optimal when x_F >= 0 and y >= 0 off
    F.  Otherwise the infeasible variables (x_k < 0 in F, y_k < -tol off F) change
    sides all at once while their number keeps decreasing; after three exchanges
    without a decrease only the infeasible variable of largest index changes side
    (the backup rule that makes the method finite).  READING: tol is the dual
    tolerance of the active-set method (1e-12 max(1, max |b|)), the iteration cap is
    5r, and when G_FF is singular (G only semidefinite) or the cap is reached the
    solution is taken from the active-set method.  ``info`` (optional dict) receives
    "method" ("bpp" or "active set") and "iterations".
    """
    G = np.asarray(G, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    r = b.shape[0]
    if max_iter is None:
        max_iter = 5 * r
    tol = 1e-12 * max(1.0, float(np.max(np.abs(b))) if r else 1.0)
    F = np.zeros(r, dtype=bool)
    x = np.zeros(r)
    y = -b.copy()
    nmin, backup = r + 1, 3
    if info is not None:
        info.update(method="bpp", iterations=0)
    for it in range(max_iter):
        infeasible = np.flatnonzero((F & (x < 0.0)) | (~F & (y < -tol)))
        if infeasible.size == 0:
            if info is not None:
                info["iterations"] = it
            return np.where(F, x, 0.0)
        if infeasible.size < nmin:
            nmin, backup = infeasible.size, 3
            F[infeasible] = ~F[infeasible]
        elif backup > 0:
            backup -= 1
            F[infeasible] = ~F[infeasible]
        else:
            k = infeasible[-1]
            F[k] = not F[k]
        P = np.flatnonzero(F)
        x = np.zeros(r)
        if P.size:
            GPP = G[np.ix_(P, P)]
            if np.linalg.matrix_rank(GPP) < P.size:
                if info is not None:
                    info["method"] = "active set"
                return nnls_active_set(G, b)
            x[P] = np.linalg.solve(GPP, b[P])
        y = G @ x - b
        y[F] = 0.0
    if info is not None:
        info["method"] = "active set"
    return nnls_active_set(G, b)


def anls_sweep(M, V, W):
    """One pass of Algorithm ANLS: V <- argmin_{V>=0} ||M-VW||, then W likewise.

    The V-step splits into m NNLS problems in r variables sharing G = W W^T with
    right-hand sides the rows of M W^T (Appendix A.2); the W-step into n problems
    sharing V^T V with right-hand sides the columns of V^T M.  The incoming V is
    not used (ANLS needs only W, Remark after Algorithm NI).
    """
    W = np.array(W, dtype=np.float64)
    m = M.shape[0]
    n = M.shape[1]
    G = product(W, W.T)
    A = product(M, W.T, True)
    V = store(np.stack([nnls_active_set(G, A[i]) for i in range(m)]))
    D = product(V.T, V)
    C = product(V.T, M, True)
    W = np.stack([nnls_active_set(D, C[:, j]) for j in range(n)], axis=1)
    return V, W


def anls_bpp_sweep(M, V, W):
    """Algorithm ANLS with its NNLS problems solved by block principal pivoting (nnls_bpp)."""
    W = np.array(W, dtype=np.float64)
    G = product(W, W.T)
    A = product(M, W.T, True)
    V = store(np.stack([nnls_bpp(G, A[i]) for i in range(M.shape[0])]))
    D = product(V.T, V)
    C = product(V.T, M, True)
    W = np.stack([nnls_bpp(D, C[:, j]) for j in range(M.shape[1])], axis=1)
    return V, W


SWEEPS = {"hals": hals_sweep, "mu": mu_sweep, "anls": anls_sweep, "anls_bpp": anls_bpp_sweep}


def smooth(M, V, W, algo: str, sweeps: int, trace=None, level: int = 1):
    """Run ``sweeps`` iterations of the chosen NMF algorithm ("NMF algorithm(M, V, W, T)")."""
    step = SWEEPS[algo]
    for _ in range(sweeps):
        V, W = step(M, V, W)
        V, W = store(V), store(W)
        if trace is not None:
            trace.append((level, objective(M, V, W)))
    return V, W


# ---------------------------------------------------------------------------
# Section 4.3: multigrid cycles
# ---------------------------------------------------------------------------

def restrict_hierarchy(M: np.ndarray, h: int, w: int, levels: int) -> list[np.ndarray]:
    """M at levels 1..L, each restricted once (footnote of Algorithm FMG)."""
    Ms = [np.asarray(M, dtype=np.float64)]
    grids = grid_hierarchy(h, w, levels)
    for l in range(levels - 1):
        Ms.append(restrict(Ms[-1], *grids[l]))
    return Ms


def vcycle(Ms, grids, V, W, algo: str, L: int, K: int, level: int = 0, hooks=None, trace=None):
    """Algorithm V-cycle with the sweep reading of Table 1.

    L = 1: K sweeps.  Otherwise: floor(K/4) sweeps; restrict V; V-cycle on the
    next coarser level with the same K (a quarter of the time at a level four
    times cheaper); prolong V; floor(K/2) sweeps.  W is never transferred.
    """
    M = Ms[level]
    if L == 1:
        return smooth(M, V, W, algo, K, trace, level + 1)
    V, W = smooth(M, V, W, algo, K // 4, trace, level + 1)
    Vc = restrict(V, *grids[level])
    Vc, W = vcycle(Ms, grids, Vc, W, algo, L - 1, K, level + 1, hooks, trace)
    V = prolong(Vc, *grids[level + 1], *grids[level])
    if hooks is not None:
        hooks.append(("prolong", level, Vc.copy(), V.copy(), W.copy()))
    return smooth(M, V, W, algo, K // 2, trace, level + 1)


# Algorithm V-cycle states its budgets as time: T/4 of smoothing before the restriction, T/4
# for the coarser V-cycle, T/2 of smoothing after the prolongation, all of T on the coarsest
# level.  READING: with per-sweep costs c_l of levels l = 1 (finest) .. L, level l < L receives
# T_l = T / 4^(l-1) and runs floor(T_l / (4 c_l)) sweeps before and floor(T_l / (2 c_l)) after,
# the coarsest floor(T_L / c_L).  Table 1's sweep counts are this split for c_l = c_1 / 4^(l-1)
# with T = K c_1; other costs (the measured ones of a machine) give other counts.

def time_schedule(T: float, costs) -> tuple[list[int], int, list[int]]:
    """(pre, coarse, post): sweeps of levels 1..L-1 before and after the coarser cycle, and of
    level L, for a V-cycle of total time T with per-sweep costs costs[l-1] (any common unit)."""
    L = len(costs)
    pre, post = [], []
    for l in range(L - 1):
        Tl = T / 4.0 ** l
        pre.append(int(np.floor(Tl / (4.0 * costs[l]) + 1e-9)))
        post.append(int(np.floor(Tl / (2.0 * costs[l]) + 1e-9)))
    coarse = int(np.floor(T / 4.0 ** (L - 1) / costs[L - 1] + 1e-9))
    return pre, coarse, post


def vcycle_counts(Ms, grids, V, W, algo: str, pre, coarse: int, post, level: int = 0, trace=None):
    """Algorithm V-cycle with explicit sweep counts per level (time_schedule): pre[level]
    sweeps, restriction of V, the coarser cycle, prolongation of V, post[level] sweeps; the
    coarsest level (level == len(pre)) runs `coarse` sweeps."""
    M = Ms[level]
    if level == len(pre):
        return smooth(M, V, W, algo, coarse, trace, level + 1)
    V, W = smooth(M, V, W, algo, pre[level], trace, level + 1)
    Vc = restrict(V, *grids[level])
    Vc, W = vcycle_counts(Ms, grids, Vc, W, algo, pre, coarse, post, level + 1, trace)
    V = prolong(Vc, *grids[level + 1], *grids[level])
    return smooth(M, V, W, algo, post[level], trace, level + 1)


def nested_iteration(Ms, grids, V0, W0, algo: str, L: int, K: int, level: int = 0, trace=None, hooks=None):
    """Algorithm NI: solve on the coarser level (K coarse sweeps), prolong, then floor(3K/4) sweeps.

    ``hooks`` (optional list) receives ("ni", level, Vc, W) with the coarse result that the
    prolongation and the fine-level sweeps start from.
    """
    M = Ms[level]
    if L == 1:
        return smooth(M, V0, W0, algo, K, trace, level + 1)
    Vc0 = restrict(V0, *grids[level])
    Vc, W = nested_iteration(Ms, grids, Vc0, W0, algo, L - 1, K, level + 1, trace, hooks)
    if hooks is not None:
        hooks.append(("ni", level, Vc.copy(), W.copy()))
    V = prolong(Vc, *grids[level + 1], *grids[level])
    return smooth(M, V, W, algo, (3 * K) // 4, trace, level + 1)


def full_multigrid(Ms, grids, V0, W0, algo: str, L: int, K: int, level: int = 0, trace=None, hooks=None):
    """Algorithm FMG: FMG on the coarser level (budget K), prolong, then a V-cycle with budget floor(3K/4).

    ``hooks`` (optional list) receives ("fmg", level, Vc, W) with the coarse result that the
    prolongation and the V-cycle start from.
    """
    M = Ms[level]
    if L == 1:
        return smooth(M, V0, W0, algo, K, trace, level + 1)
    Vc0 = restrict(V0, *grids[level])
    Vc, W = full_multigrid(Ms, grids, Vc0, W0, algo, L - 1, K, level + 1, trace, hooks)
    if hooks is not None:
        hooks.append(("fmg", level, Vc.copy(), W.copy()))
    V = prolong(Vc, *grids[level + 1], *grids[level])
    return vcycle(Ms, grids, V, W, algo, L, (3 * K) // 4, level, None, trace)


def wcycle(Ms, grids, V, W, algo: str, L: int, K: int, level: int = 0, trace=None):
    """W-cycle, one of the other grid cycles Section 7 names as an extension.

    As Algorithm V-cycle, except that the coarser level is visited twice in a row
    before the prolongation.  READING (sweep budget, as for the V-cycle): each visit
    gets half the coarse budget, K // 2, so the coarse share of the time matches the
    V-cycle's; with two levels the W-cycle is the V-cycle.
    """
    M = Ms[level]
    if L == 1:
        return smooth(M, V, W, algo, K, trace, level + 1)
    V, W = smooth(M, V, W, algo, K // 4, trace, level + 1)
    Vc = restrict(V, *grids[level])
    for _ in range(2):
        Vc, W = wcycle(Ms, grids, Vc, W, algo, L - 1, K // 2, level + 1, trace)
    V = prolong(Vc, *grids[level + 1], *grids[level])
    return smooth(M, V, W, algo, K // 2, trace, level + 1)


CYCLES = {"vcycle": vcycle, "ni": nested_iteration, "fmg": full_multigrid, "wcycle": wcycle}


# ---------------------------------------------------------------------------
# Section 6.1: the columns of M coarsened as well (image sequences)
# ---------------------------------------------------------------------------
# Section 6.1 notes that when the columns of M form a smooth sequence (video frames,
# hyperspectral bands) the multilevel strategy also applies to them.  READING: the
# sequence is a 1-D grid of n points and is coarsened like one side of the pixel grid
# (coarse point j on fine point 2j, ceil(n / 2) points): the restriction along it is
# Eq. (4.1) on an n x 1 grid (weights 1, 2, 1 renormalised at the ends) and the
# prolongation Eq. (4.2) on it.  M_{l+1} = R M_l R_n^T, W_{l+1} = W_l R_n^T and
# W_l = W_{l+1} P_n^T, next to the pixel transfers of V; the V-cycle otherwise as
# Algorithm V-cycle with the sweep reading of Table 1.

def restrict_columns(X: np.ndarray, n: int) -> np.ndarray:
    """X R_n^T: the columns of X (a sequence of n) restricted along the sequence."""
    return restrict(np.asarray(X, np.float64).T, n, 1).T


def prolong_columns(Y: np.ndarray, nc: int, n: int) -> np.ndarray:
    """Y P_n^T: a coarse sequence of nc columns prolonged to n columns."""
    return prolong(np.asarray(Y, np.float64).T, nc, 1, n, 1).T


def sequence_lengths(n: int, levels: int) -> list[int]:
    """n at levels 1 (finest) .. L."""
    ns = [n]
    for _ in range(levels - 1):
        ns.append((ns[-1] + 1) // 2)
    return ns


def restrict_hierarchy_both(M: np.ndarray, h: int, w: int, levels: int) -> list[np.ndarray]:
    """M at levels 1..L, restricted over the pixel grid and along the sequence."""
    Ms = [np.asarray(M, dtype=np.float64)]
    grids = grid_hierarchy(h, w, levels)
    ns = sequence_lengths(M.shape[1], levels)
    for l in range(levels - 1):
        Ms.append(restrict_columns(restrict(Ms[-1], *grids[l]), ns[l]))
    return Ms


def vcycle_both(Ms, grids, ns, V, W, algo: str, L: int, K: int, level: int = 0, trace=None, hooks=None):
    """V-cycle with V restricted over the pixel grid and W along the sequence."""
    M = Ms[level]
    if L == 1:
        return smooth(M, V, W, algo, K, trace, level + 1)
    V, W = smooth(M, V, W, algo, K // 4, trace, level + 1)
    Vc = restrict(V, *grids[level])
    Wc = restrict_columns(W, ns[level])
    Vc, Wc = vcycle_both(Ms, grids, ns, Vc, Wc, algo, L - 1, K, level + 1, trace, hooks)
    if hooks is not None:
        hooks.append(("both", level, Vc.copy(), Wc.copy()))
    V = prolong(Vc, *grids[level + 1], *grids[level])
    W = prolong_columns(Wc, ns[level + 1], ns[level])
    return smooth(M, V, W, algo, K // 2, trace, level + 1)


def solve(M, grid_h: int, grid_w: int, V0, W0, algo: str = "hals", levels: int = 1, K: int = 100,
          cycle: str = "vcycle", trace=None, precision: str = "fp64", coarsen_columns: bool = False,
          level_sweeps=None):
    """Multilevel NMF of M (m = grid_h * grid_w rows) from (V0, W0); returns (V, W).

    precision: "fp64" (default), "fp32" or "bf16" (see PRECISION).  coarsen_columns: the
    V-cycle coarsens the columns of M as a sequence too (vcycle_both).  level_sweeps: a
    V-cycle with explicit counts (pre, coarse, post) as time_schedule returns them (K unused)."""
    global PRECISION
    M = np.asarray(M, dtype=np.float64)
    Ms = restrict_hierarchy(M, grid_h, grid_w, levels)
    grids = grid_hierarchy(grid_h, grid_w, levels)
    V = np.asarray(V0, dtype=np.float64)
    W = np.asarray(W0, dtype=np.float64)
    saved = PRECISION
    PRECISION = {"fp64": None, "fp32": "fp32", "bf16": "bf16"}[precision]
    try:
        if level_sweeps is not None:
            pre, coarse, post = level_sweeps
            assert cycle == "vcycle" and len(pre) == len(post) == levels - 1
            return vcycle_counts(Ms, grids, V, W, algo, list(pre), int(coarse), list(post), trace=trace)
        if coarsen_columns:
            assert cycle == "vcycle", "column coarsening is defined for the V-cycle"
            Ms = restrict_hierarchy_both(M, grid_h, grid_w, levels)
            return vcycle_both(Ms, grids, sequence_lengths(M.shape[1], levels), V, W, algo, levels, K, trace=trace)
        if cycle == "vcycle":
            return vcycle(Ms, grids, V, W, algo, levels, K, trace=trace)
        return CYCLES[cycle](Ms, grids, V, W, algo, levels, K, trace=trace)
    finally:
        PRECISION = saved
