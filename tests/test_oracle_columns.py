"""Pins of the oracle's V-cycle that coarsens the columns of M too (Section 6.1: image
sequences, whose columns vary smoothly along the sequence).

The sequence of n columns is coarsened like one side of the pixel grid: the 1-D
full-weighting restriction (weights 1, 2, 1, renormalised at the ends) and the 1-D
mean-of-neighbours prolongation.  The pins: both written out as closed forms by loops,
the 2-D pixel operators as their tensor products (separability), the hierarchy
M_{l+1} = R M_l R_n^T, and the cycle's data flow rebuilt from those pieces.
"""
import numpy as np
import pytest

from oracle import nmf_oracle as o
from paper_1009_0881_gb300 import synth


def _restrict_1d_loops(x):
    """1-D full weighting by hand: coarse j from fine 2j-1, 2j, 2j+1, weights 1/4, 1/2, 1/4;
    at an end the missing neighbour is left out and the rest renormalised (2/3, 1/3)."""
    n = len(x)
    out = []
    for j in range((n + 1) // 2):
        c = 2 * j
        num, den = 2.0 * x[c], 2.0
        if c - 1 >= 0:
            num, den = num + x[c - 1], den + 1.0
        if c + 1 < n:
            num, den = num + x[c + 1], den + 1.0
        out.append(num / den)
    return np.array(out)


def _prolong_1d_loops(y, n):
    """1-D prolongation by hand: even fine i takes coarse i/2; odd i the mean of coarse
    (i-1)/2 and (i+1)/2, or coarse (i-1)/2 alone when (i+1)/2 is past the end."""
    out = []
    for i in range(n):
        if i % 2 == 0:
            out.append(y[i // 2])
        elif (i + 1) // 2 < len(y):
            out.append(0.5 * (y[(i - 1) // 2] + y[(i + 1) // 2]))
        else:
            out.append(y[(i - 1) // 2])
    return np.array(out)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 8, 9, 16, 33])
def test_column_restriction_closed_form(n):
    rng = np.random.default_rng(n)
    X = rng.random((3, n))
    got = o.restrict_columns(X, n)
    assert got.shape == (3, (n + 1) // 2)
    for row in range(3):
        np.testing.assert_allclose(got[row], _restrict_1d_loops(X[row]), rtol=1e-15, atol=0)


@pytest.mark.parametrize("n", [2, 3, 4, 5, 8, 9, 16, 33])
def test_column_prolongation_closed_form(n):
    rng = np.random.default_rng(100 + n)
    nc = (n + 1) // 2
    Y = rng.random((3, nc))
    got = o.prolong_columns(Y, nc, n)
    assert got.shape == (3, n)
    for row in range(3):
        np.testing.assert_allclose(got[row], _prolong_1d_loops(Y[row], n), rtol=1e-15, atol=0)


@pytest.mark.parametrize("h,w", [(3, 3), (4, 5), (7, 6), (9, 9)])
def test_pixel_operators_are_tensor_products_of_the_column_operators(h, w):
    # separability: the 2-D restriction (Eq. (4.1)) and prolongation (Eq. (4.2)) on an
    # h x w grid are the Kronecker products of the 1-D operators along y and along x,
    # so the column transfers are the same operators on a grid with one side
    R1 = lambda k: o.restrict_columns(np.eye(k), k).T                        # noqa: E731
    P1 = lambda k: o.prolong_columns(np.eye((k + 1) // 2), (k + 1) // 2, k).T  # noqa: E731
    np.testing.assert_allclose(np.kron(R1(h), R1(w)), o.restriction_matrix(h, w), rtol=1e-14, atol=1e-16)
    hc, wc = o.coarse_grid(h, w)
    np.testing.assert_allclose(np.kron(P1(h), P1(w)), o.prolongation_matrix(hc, wc, h, w),
                               rtol=1e-14, atol=1e-16)


def test_sequence_lengths():
    assert o.sequence_lengths(1024, 4) == [1024, 512, 256, 128]
    assert o.sequence_lengths(9, 4) == [9, 5, 3, 2]
    assert o.sequence_lengths(7, 1) == [7]


def test_hierarchy_restricts_rows_and_columns():
    p = synth.make_problem(9, 7, 23, 3, data_seed=5, sequence=True)
    Ms = o.restrict_hierarchy_both(p.M, 9, 7, 3)
    grids = o.grid_hierarchy(9, 7, 3)
    ns = o.sequence_lengths(23, 3)
    for l in range(2):
        R = o.restriction_matrix(*grids[l])
        Rn = o.restrict_columns(np.eye(ns[l]), ns[l]).T
        np.testing.assert_allclose(Ms[l + 1], R @ Ms[l] @ Rn.T, rtol=1e-12, atol=1e-15)
        assert Ms[l + 1].shape == (grids[l + 1][0] * grids[l + 1][1], ns[l + 1])


def test_columns_constant_along_the_sequence_are_fixed():
    # a sequence that does not change is its own restriction and prolongation
    X = np.outer(np.arange(1.0, 5.0), np.ones(11))
    np.testing.assert_allclose(o.restrict_columns(X, 11), X[:, :6], rtol=1e-15)
    np.testing.assert_allclose(o.prolong_columns(X[:, :6], 6, 11), X, rtol=1e-15)


def test_single_level_is_the_plain_algorithm():
    p = synth.make_problem(8, 8, 20, 3, data_seed=6, sequence=True)
    for algo in ("hals", "mu"):
        a = o.solve(p.M, 8, 8, p.V, p.W, algo, levels=1, K=6, coarsen_columns=True)
        b = o.smooth(p.M.astype(np.float64), p.V.astype(np.float64), p.W.astype(np.float64), algo, 6)
        np.testing.assert_array_equal(a[0], b[0])
        np.testing.assert_array_equal(a[1], b[1])


@pytest.mark.parametrize("algo", ["hals", "mu", "anls"])
def test_column_vcycle_data_flow(algo):
    # rebuilt from the pinned pieces: pre-smoothing on level 1, restriction of V over the
    # pixels and of W along the sequence, the same on level 2, K sweeps on level 3,
    # prolongation of both, post-smoothing on the way up
    p = synth.make_problem(9, 9, 30, 4, data_seed=11, sequence=True)
    grids = o.grid_hierarchy(9, 9, 3)
    ns = o.sequence_lengths(30, 3)
    Ms = o.restrict_hierarchy_both(p.M, 9, 9, 3)
    V0, W0 = p.V.astype(np.float64), p.W.astype(np.float64)
    K = 8
    hooks = []
    V, W = o.vcycle_both(Ms, grids, ns, V0, W0, algo, 3, K, hooks=hooks)
    V1, W1 = o.smooth(Ms[0], V0, W0, algo, K // 4)
    V2, W2 = o.smooth(Ms[1], o.restrict(V1, *grids[0]), o.restrict_columns(W1, ns[0]), algo, K // 4)
    V3, W3 = o.smooth(Ms[2], o.restrict(V2, *grids[1]), o.restrict_columns(W2, ns[1]), algo, K)
    V2, W2 = o.smooth(Ms[1], o.prolong(V3, *grids[2], *grids[1]), o.prolong_columns(W3, ns[2], ns[1]), algo, K // 2)
    Vf, Wf = o.smooth(Ms[0], o.prolong(V2, *grids[1], *grids[0]), o.prolong_columns(W2, ns[1], ns[0]), algo, K // 2)
    assert [(k, lvl) for k, lvl, _, _ in hooks] == [("both", 1), ("both", 0)]
    np.testing.assert_array_equal(hooks[0][2], V3)
    np.testing.assert_array_equal(hooks[0][3], W3)
    np.testing.assert_array_equal(V, Vf)
    np.testing.assert_array_equal(W, Wf)
    assert W.shape == (4, 30) and V.shape == (81, 4)


def test_planted_sequence_is_smooth_along_the_columns():
    # the input recipe: the rows of the planted W vary slowly along the sequence, so the
    # columns of M do too (what makes coarsening them pay off)
    p = synth.make_problem(16, 16, 256, 6, data_seed=3, sequence=True)
    M = p.M.astype(np.float64)
    step = np.linalg.norm(np.diff(M, axis=1)) / np.linalg.norm(M)
    shuffled = np.random.default_rng(0).permutation(M.shape[1])
    step_shuffled = np.linalg.norm(np.diff(M[:, shuffled], axis=1)) / np.linalg.norm(M)
    assert step < 0.25 * step_shuffled
