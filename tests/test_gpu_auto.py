"""GPU tests of the per-problem precision choice (NMF_AUTO): HALS and MU problems on grids of
4096 pixels or more take the BF16 form with float32 finishing, everything else the float32
form.  A problem solved under NMF_AUTO must give exactly the bits of the form it maps to,
alone and in a batch (the forms themselves are checked against the oracle elsewhere)."""
import numpy as np
import pytest

from paper_1009_0881_gb300 import native, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def handles():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1009_0881_gb300 import build
    build.build()
    with native.Handle(0, precision=native.NMF_AUTO) as ha, native.Handle(0) as h32, \
            native.Handle(0, precision=native.NMF_BF16_FP32) as hbf:
        yield ha, h32, hbf


CASES = [  # (side, n, r, algo, form the choice maps it to)
    (32, 300, 12, "hals", "fp32"),     # 1024 pixels: float32
    (64, 400, 20, "hals", "bf16f"),    # 4096 pixels: BF16 with float32 finishing
    (64, 350, 16, "mu", "bf16f"),
    (92, 250, 24, "anls", "fp32"),     # ANLS: float32 at every size
]


def _problem(i, side, n, r):
    return synth.make_problem(side, side, n, r, sigma=0.04 * side, data_seed=40 + i)


def _solve(h, p, side, algo, L=3, K=12):
    V, W = p.V.copy(), p.W.copy()
    h.solve(p.M, side, side, V, W, algo, levels=L, iters=K)
    return V, W


@pytest.mark.parametrize("i", range(len(CASES)))
def test_auto_takes_the_form_it_maps_to(handles, i):
    ha, h32, hbf = handles
    side, n, r, algo, form = CASES[i]
    p = _problem(i, side, n, r)
    Va, Wa = _solve(ha, p, side, algo)
    Vf, Wf = _solve(h32 if form == "fp32" else hbf, p, side, algo)
    np.testing.assert_array_equal(Va, Vf)
    np.testing.assert_array_equal(Wa, Wf)


def test_auto_batch_equals_alone(handles):
    ha, h32, hbf = handles
    batch, alone = [], []
    for i, (side, n, r, algo, form) in enumerate(CASES):
        p = _problem(i, side, n, r)
        batch.append(dict(M=p.M, grid_h=side, grid_w=side, V=p.V.copy(), W=p.W.copy(), algo=algo, levels=3, iters=12))
        alone.append(_solve(ha, p, side, algo))
    res = ha.solve_batch(batch)
    for d, (V, W), (st, sweeps, obj) in zip(batch, alone, res):
        assert st == 0
        np.testing.assert_array_equal(d["V"], V)
        np.testing.assert_array_equal(d["W"], W)


def test_auto_workspace_sits_between_the_forms(handles):
    ha, h32, hbf = handles
    ds = []
    for i, (side, n, r, algo, form) in enumerate(CASES):
        p = _problem(i, side, n, r)
        ds.append(dict(M=p.M, grid_h=side, grid_w=side, V=p.V, W=p.W, algo=algo, levels=3, iters=12))
    b32, bbf, bauto = h32.workspace_bytes(ds), hbf.workspace_bytes(ds), ha.workspace_bytes(ds)
    assert b32 < bauto < bbf, (b32, bauto, bbf)
