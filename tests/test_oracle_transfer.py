"""Pins for the oracle's grid hierarchy and transfer operators (Section 4.2)."""
import numpy as np
import pytest

from conftest import load_golden
from oracle import nmf_oracle as o


def test_restriction_matches_printed_3x3_example():
    # Section 4.2: R for a 3x3 -> 2x2 restriction, printed entry by entry
    R = o.restriction_matrix(3, 3)
    np.testing.assert_array_equal(R * 9, load_golden("restriction_3x3_to_2x2.txt") * 9)


def test_prolongation_matches_printed_2x2_example():
    # Section 4.2: P^T for a 2x2 -> 3x3 prolongation, printed entry by entry
    P = o.prolongation_matrix(2, 2, 3, 3)
    np.testing.assert_array_equal(P.T * 4, load_golden("prolongation_2x2_to_3x3_transposed.txt") * 4)


def test_interior_restriction_is_eq_4_1():
    # Eq. (4.1) at an interior coarse pixel of a 9x9 grid: (1/16) [1 2 1; 2 4 2; 1 2 1]
    R = o.restriction_matrix(9, 9)
    i, j = 2, 2  # coarse (2,2) sits on fine (4,4)
    row = R[i * 5 + j].reshape(9, 9)
    expect = np.zeros((9, 9))
    expect[3:6, 3:6] = np.array([[1, 2, 1], [2, 4, 2], [1, 2, 1]]) / 16.0
    np.testing.assert_allclose(row, expect, atol=0, rtol=0)


@pytest.mark.parametrize("h,w", [(3, 3), (5, 5), (9, 9), (16, 16), (19, 19), (7, 4), (12, 5)])
def test_rows_sum_to_one_and_nonnegative(h, w):
    R = o.restriction_matrix(h, w)
    hc, wc = o.coarse_grid(h, w)
    P = o.prolongation_matrix(hc, wc, h, w)
    assert R.shape == (hc * wc, h * w) and P.shape == (h * w, hc * wc)
    assert (R >= 0).all() and (P >= 0).all()
    np.testing.assert_allclose(R.sum(1), 1.0, rtol=1e-15)
    np.testing.assert_allclose(P.sum(1), 1.0, rtol=1e-15)


@pytest.mark.parametrize("h,w", [(5, 5), (16, 16), (19, 19), (10, 7)])
def test_grid_constant_image_is_fixed(h, w):
    # P(R(c 1)) = c 1: both operators average with weights summing to one
    c = 3.25
    X = np.full((h * w, 2), c)
    hc, wc = o.coarse_grid(h, w)
    Y = o.prolong(o.restrict(X, h, w), hc, wc, h, w)
    np.testing.assert_allclose(Y, c, rtol=1e-15)


def test_interior_full_weighting_is_quarter_bilinear_transpose():
    # In 2-D the interior rows of full weighting are 1/4 of the columns of bilinear prolongation
    h = w = 17
    hc, wc = o.coarse_grid(h, w)
    R = o.restriction_matrix(h, w)
    P = o.prolongation_matrix(hc, wc, h, w)
    for i in range(1, hc - 1):
        for j in range(1, wc - 1):
            np.testing.assert_allclose(R[i * wc + j], P[:, i * wc + j] / 4.0, rtol=0, atol=1e-16)


def test_stencil_application_equals_matrix_product():
    rng = np.random.default_rng(0)
    for h, w in [(16, 16), (19, 19), (6, 9)]:
        X = rng.random((h * w, 5))
        hc, wc = o.coarse_grid(h, w)
        np.testing.assert_allclose(o.restrict(X, h, w), o.restriction_matrix(h, w) @ X, rtol=1e-14)
        Y = rng.random((hc * wc, 4))
        np.testing.assert_allclose(o.prolong(Y, hc, wc, h, w), o.prolongation_matrix(hc, wc, h, w) @ Y, rtol=1e-14)


def test_grid_hierarchy_sizes():
    # Section 4.2: (2^a+1) x (2^b+1) -> (2^(a-1)+1) x (2^(b-1)+1)
    assert o.grid_hierarchy(17, 33, 3) == [(17, 33), (9, 17), (5, 9)]
    # other sides: ceil(side/2)
    assert o.grid_hierarchy(19, 19, 3) == [(19, 19), (10, 10), (5, 5)]
    assert o.grid_hierarchy(16, 16, 3) == [(16, 16), (8, 8), (4, 4)]
    assert o.grid_hierarchy(112, 92, 3) == [(112, 92), (56, 46), (28, 23)]


def test_even_border_prolongation_uses_existing_neighbour():
    # 4x4 fine from 2x2 coarse: fine row 3 (odd) has rd = {1, 2}; only coarse row 1 exists
    Y = np.arange(4.0).reshape(4, 1)
    F = o.prolong(Y, 2, 2, 4, 4).reshape(4, 4)
    assert F[3, 0] == Y[2, 0]  # coarse (1,0)
    assert F[3, 3] == Y[3, 0]
    assert F[1, 1] == Y.mean()


def test_smoothness_small_for_smooth_data_and_zero_for_constants():
    from paper_1009_0881_gb300 import synth
    p = synth.make_problem(19, 19, 50, 5, data_seed=3)
    s = o.smoothness(p.M.astype(np.float64), 19, 19)
    assert 0.0 < s < 0.2
    assert o.smoothness(np.ones((25, 3)), 5, 5) < 1e-15
