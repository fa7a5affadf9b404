"""Edge shapes through the C ABI against the FP64 oracle: one pixel, one image,
rank 1 and the maximum rank 64, odd and even grid sides, more levels than the
grid can halve (1 x 1 coarse grids), partial tiles, and rejected empty inputs.
Each case runs a few sweeps of a V-cycle and compares the final objective and
the iterates with the oracle's."""
import numpy as np
import pytest

from oracle import nmf_oracle as o
from paper_1009_0881_gb300 import native, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1009_0881_gb300 import build
    build.build()
    with native.Handle(0) as hd:
        yield hd


CASES = [  # (grid_h, grid_w, n, r, levels, K, algo)
    (1, 1, 5, 1, 1, 3, "hals"),
    (3, 3, 1, 1, 2, 4, "hals"),
    (5, 4, 7, 3, 3, 4, "hals"),
    (2, 2, 9, 2, 4, 4, "hals"),
    (16, 16, 33, 64, 2, 3, "hals"),
    (7, 9, 65, 17, 3, 4, "mu"),
    (13, 11, 130, 33, 2, 4, "hals"),
    (6, 6, 20, 5, 2, 3, "anls"),
    (1, 37, 70, 6, 3, 4, "hals"),
]


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}x{c[1]}_n{c[2]}_r{c[3]}_L{c[4]}_{c[6]}" for c in CASES])
def test_edge_shape_matches_oracle(h, case):
    gh, gw, n, r, L, K, algo = case
    p = synth.make_problem(gh, gw, n, r, sigma=1.0, data_seed=11)
    V, W = p.V.copy(), p.W.copy()
    h.solve(p.M, gh, gw, V, W, algo, levels=L, iters=K)
    assert np.isfinite(V).all() and np.isfinite(W).all()
    assert (V >= 0).all() and (W >= 0).all()
    Vo, Wo = o.solve(p.M, gh, gw, p.V, p.W, algo, levels=L, K=K)
    f, fo = o.objective(p.M, V, W), o.objective(p.M, Vo, Wo)
    # exact fits (one pixel, one image) end at zero up to FP32 rounding of M: the bar is
    # 1e-4 of the oracle's objective, or 1e-6 of ||M||_F when that is larger
    mnorm = float(np.linalg.norm(p.M.astype(np.float64)))
    assert abs(f - fo) <= max(1e-4 * fo, 1e-6 * mnorm), (f, fo)
    e = h.error(p.M, V, W)
    assert abs(e - f) <= max(1e-5 * f, 1e-6 * mnorm), (e, f)


def test_empty_inputs_rejected(h):
    for m_shape, gh, gw in (((0, 4), 0, 1), ((4, 0), 2, 2)):
        M = np.zeros(m_shape, np.float32)
        V = np.zeros((m_shape[0], 2), np.float32)
        W = np.zeros((2, m_shape[1]), np.float32)
        with pytest.raises(native.NMFError, match="EINVAL"):
            h.solve(M, gh, gw, V, W, "hals", levels=1, iters=2)
    # the handle stays usable
    p = synth.make_problem(4, 4, 8, 2, data_seed=1)
    h.solve(p.M, 4, 4, p.V.copy(), p.W.copy(), "hals", levels=2, iters=2)


def _edge_check(h, p, V, W, Vo, Wo):
    assert np.isfinite(V).all() and np.isfinite(W).all()
    assert (V >= 0).all() and (W >= 0).all()
    f, fo = o.objective(p.M, V, W), o.objective(p.M, Vo, Wo)
    mnorm = float(np.linalg.norm(p.M.astype(np.float64)))
    assert abs(f - fo) <= max(1e-4 * fo, 1e-6 * mnorm), (f, fo)


@pytest.mark.parametrize("L,K", [(1, 3), (3, 4)])
def test_edge_shapes_in_one_group(h, L, K):
    # the HALS / MU edge shapes as one grouped solve (one pixel, one image, r = 1 and 64,
    # grids too small to halve, a 1 x 37 strip)
    cases = [c for c in CASES if c[6] != "anls"]
    probs, batch = [], []
    for gh, gw, n, r, _, _, algo in cases:
        p = synth.make_problem(gh, gw, n, r, sigma=1.0, data_seed=11)
        probs.append((p, algo))
        batch.append(dict(M=p.M, grid_h=gh, grid_w=gw, V=p.V.copy(), W=p.W.copy(), algo=algo, levels=L, iters=K))
    res = h.solve_batch(batch, grouped=True)
    for (p, algo), d, (st, sweeps, obj) in zip(probs, batch, res):
        assert st == 0
        Vo, Wo = o.solve(p.M, p.grid_h, p.grid_w, p.V, p.W, algo, levels=L, K=K)
        _edge_check(h, p, d["V"], d["W"], Vo, Wo)


COLUMN_CASES = [  # (grid_h, grid_w, n, r, levels, K, algo): one image, two images, a strip, 4 levels
    (1, 1, 1, 1, 3, 4, "hals"),
    (3, 3, 2, 2, 3, 4, "hals"),
    (1, 37, 70, 6, 3, 4, "mu"),
    (5, 4, 7, 3, 4, 4, "anls"),
]


@pytest.mark.parametrize("case", COLUMN_CASES, ids=[f"{c[0]}x{c[1]}_n{c[2]}_r{c[3]}_L{c[4]}_{c[6]}" for c in COLUMN_CASES])
def test_edge_column_vcycle_matches_oracle(h, case):
    gh, gw, n, r, L, K, algo = case
    p = synth.make_problem(gh, gw, n, r, sigma=1.0, data_seed=11, sequence=True)
    V, W = p.V.copy(), p.W.copy()
    h.solve(p.M, gh, gw, V, W, algo, levels=L, iters=K, coarsen_columns=True)
    Vo, Wo = o.solve(p.M, gh, gw, p.V, p.W, algo, levels=L, K=K, coarsen_columns=True)
    _edge_check(h, p, V, W, Vo, Wo)


def test_empty_group_rejected(h):
    with pytest.raises(native.NMFError, match="EINVAL"):
        h.solve_batch([], grouped=True)
