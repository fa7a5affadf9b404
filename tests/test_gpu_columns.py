"""GPU parity of the V-cycle that coarsens the columns of M too (image sequences,
Section 6.1) against the FP64 oracle (oracle.solve(..., coarsen_columns=True)).

Bars (FP32 path), as for the pixel-only cycles: transfers within rtol 2e-6 (weighted
means of at most 3 float32 values along the sequence); a short cycle from identical
iterates within 1e-3 norm-wise for V and W and 1e-4 for the objective (ANLS: four times
the oracle's own float32 movement, objective 1e-3); whole cycles on the stored workloads
within 1e-3 of the oracle's final objective.
"""
import json
import os

import numpy as np
import pytest

from conftest import ROOT
from oracle import nmf_oracle as o
from paper_1009_0881_gb300 import native, synth

pytestmark = pytest.mark.gpu

GOLDEN = json.load(open(os.path.join(ROOT, "tests", "golden", "objectives.json")))


@pytest.fixture(scope="module")
def h():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1009_0881_gb300 import build
    build.build()
    with native.Handle(0) as hd:
        yield hd


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("n,r", [(1, 3), (2, 4), (7, 5), (1024, 10), (4095, 16)])
def test_sequence_transfers_match_oracle(h, n, r):
    # the library's transfers on an n x 1 grid, applied to W^T, are the oracle's column
    # transfers of W
    rng = np.random.default_rng(n)
    W = rng.random((r, n))
    Wt = np.ascontiguousarray(W.T, dtype=np.float32)
    nc = (n + 1) // 2
    Yt = np.zeros((nc, r), np.float32)
    h.restrict(Wt, n, 1, Yt)
    np.testing.assert_allclose(Yt.T, o.restrict_columns(Wt.T, n), rtol=2e-6, atol=1e-7)
    Ct = np.ascontiguousarray(rng.random((nc, r)), dtype=np.float32)
    Xt = np.zeros((n, r), np.float32)
    h.prolong(Ct, n, 1, Xt)
    np.testing.assert_allclose(Xt.T, o.prolong_columns(Ct.T, nc, n), rtol=2e-6, atol=1e-7)


# ragged sizes: odd grid sides, n not a multiple of any tile, coarsest level 3 x 2 pixels
@pytest.mark.parametrize("algo,K", [("hals", 12), ("mu", 12), ("anls", 4)])
def test_short_column_vcycle_matches_oracle(h, algo, K):
    gh, gw, n, r = 9, 7, 77, 5
    p = synth.make_problem(gh, gw, n, r, data_seed=21, sequence=True)
    V, W = p.V.copy(), p.W.copy()
    h.solve(p.M, gh, gw, V, W, algo, levels=3, iters=K, coarsen_columns=True)
    Vo, Wo = o.solve(p.M, gh, gw, p.V, p.W, algo, levels=3, K=K, coarsen_columns=True)
    bar_v = bar_w = 1e-3
    if algo == "anls":
        # ANLS solves with the Gram matrices of the 5 x 4 and 3 x 2 levels amplify rounding
        # by their condition numbers: the oracle itself at float32 precision (reading of the
        # precision modes) moves V and W by 3.4e-3 and 2.5e-3 here; the GPU must stay within
        # four times the oracle's own float32 movement
        V32, W32 = o.solve(p.M, gh, gw, p.V, p.W, algo, levels=3, K=K, coarsen_columns=True, precision="fp32")
        bar_v = max(bar_v, 4 * rel(V32, Vo))
        bar_w = max(bar_w, 4 * rel(W32, Wo))
    assert rel(V, Vo) <= bar_v and rel(W, Wo) <= bar_w, (rel(V, Vo), bar_v, rel(W, Wo), bar_w)
    fo = o.objective(p.M, Vo, Wo)
    assert abs(o.objective(p.M, V, W) - fo) <= (1e-3 if algo == "anls" else 1e-4) * fo
    assert (V >= 0).all() and (W >= 0).all()


def test_single_level_with_column_option_is_the_plain_solve(h):
    # one level has no transfers: the same kernels on the same plan shapes
    p = synth.make_problem(16, 16, 300, 6, data_seed=4, sequence=True)
    V1, W1 = p.V.copy(), p.W.copy()
    V2, W2 = p.V.copy(), p.W.copy()
    h.solve(p.M, 16, 16, V1, W1, "hals", levels=1, iters=10, coarsen_columns=True)
    h.solve(p.M, 16, 16, V2, W2, "hals", levels=1, iters=10)
    np.testing.assert_array_equal(V1, V2)
    np.testing.assert_array_equal(W1, W2)


SEQ_CASES = sorted(k for k in GOLDEN if k.startswith("seq"))


@pytest.mark.parametrize("name", SEQ_CASES)
def test_sequence_workloads_match_oracle(h, name):
    g = GOLDEN[name]
    gh, gw, n, r, sigma = synth.SEQUENCE_WORKLOADS[g["workload"]]
    p = synth.make_problem(gh, gw, n, r, sigma=sigma, sequence=True)
    V, W = p.V.copy(), p.W.copy()
    cols = g["cycle"] == "vcycle_cols"
    h.solve(p.M, gh, gw, V, W, g["algo"], levels=g["levels"], iters=g["K"],
            cycle="vcycle", coarsen_columns=cols)
    f = o.objective(p.M, V, W)
    print(f"{name}: GPU {f:.8g}, oracle {g['objective']:.8g}")
    assert abs(f - g["objective"]) <= 1e-3 * g["objective"], (f, g["objective"])


def test_block_pivoting_column_vcycle_matches_active_set_oracle(h):
    # ANLS by block principal pivoting on the sequence hierarchy (coarsest 4 x 4 grid, r = 10:
    # every NNLS problem has a unique solution) against the active-set oracle run
    g = GOLDEN["seq16_anls_cols_L3_K8"]
    gh, gw, n, r, sigma = synth.SEQUENCE_WORKLOADS[g["workload"]]
    p = synth.make_problem(gh, gw, n, r, sigma=sigma, sequence=True)
    V, W = p.V.copy(), p.W.copy()
    h.solve(p.M, gh, gw, V, W, "anls_bpp", levels=3, iters=8, coarsen_columns=True)
    f = o.objective(p.M, V, W)
    assert abs(f - g["objective"]) <= 1e-3 * g["objective"], (f, g["objective"])


def test_column_vcycle_trace_and_stop_after(h):
    p = synth.make_problem(16, 16, 1024, 10, sigma=2.0, sequence=True)
    K = 20
    V, W = p.V.copy(), p.W.copy()
    tr = h.solve(p.M, 16, 16, V, W, "hals", levels=3, iters=K, trace_len=1000, coarsen_columns=True)
    assert len(tr) == K // 4 + K // 2
    assert abs(tr[-1] - h.error(p.M, V, W)) <= 1e-6 * tr[-1]
    # a run stopped after the K/4 fine pre-sweeps skips the rest of the schedule (the
    # transfers too): its iterate is that of K/4 plain sweeps
    V2, W2 = p.V.copy(), p.W.copy()
    h.solve(p.M, 16, 16, V2, W2, "hals", levels=3, iters=K, stop_after=K // 4, coarsen_columns=True)
    Vo, Wo = o.smooth(p.M.astype(np.float64), p.V.astype(np.float64), p.W.astype(np.float64), "hals", K // 4)
    assert rel(V2, Vo) <= 1e-4 and rel(W2, Wo) <= 1e-4


def test_column_option_outside_its_scope_is_rejected(h):
    p = synth.make_problem(8, 8, 40, 3, data_seed=2, sequence=True)
    V, W = p.V.copy(), p.W.copy()
    with pytest.raises(native.NMFError) as ei:
        h.solve(p.M, 8, 8, V, W, "hals", levels=2, iters=4, cycle="fmg", coarsen_columns=True)
    assert ei.value.code == native.NMF_EINVAL
    with native.Handle(0, precision=native.NMF_BF16) as hb:
        with pytest.raises(native.NMFError) as ei:
            hb.solve(p.M, 8, 8, V, W, "hals", levels=2, iters=4, coarsen_columns=True)
        assert ei.value.code == native.NMF_EINVAL
    # the handle stays usable
    h.solve(p.M, 8, 8, V, W, "hals", levels=2, iters=4, coarsen_columns=True)
