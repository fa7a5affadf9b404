"""Documented failure paths of the C ABI, driven from the host without a GPU fault.

* NMF_ENOCONV: the ANLS active-set solve (Appendix A.2) stops at an exchange cap
  set through nmf_set_limits; the call reports the cap and leaves a feasible
  (nonnegative, finite) iterate.
* NMF_ETIMEOUT: the grid barriers of the persistent kernels get a spin budget of
  zero polls, so every CTA that is not the last to arrive gives up at once; the
  kernel leaves without touching anything in flight, the call reports the
  timeout, and the same handle then solves normally with the default budget.
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


def test_nnls_exchange_cap_returns_enoconv_with_a_feasible_iterate(h):
    p = synth.make_problem(16, 16, 300, 10, data_seed=3)
    # V0 = 0: every V-row solve starts from an empty passive set, so a row whose solution
    # has two or more positive entries needs at least two exchanges
    V = np.zeros_like(p.V)
    W = p.W.copy()
    h.set_limits(nnls_max_exchanges=1)
    try:
        with pytest.raises(native.NMFError) as ei:
            h.solve(p.M, 16, 16, V, W, "anls", levels=1, iters=1)
        assert ei.value.code == native.NMF_ENOCONV
        assert np.isfinite(V).all() and np.isfinite(W).all()
        assert (V >= 0).all() and (W >= 0).all()
    finally:
        h.set_limits()
    # the default cap (3r) solves the same problem
    V = np.zeros_like(p.V)
    W = p.W.copy()
    h.solve(p.M, 16, 16, V, W, "anls", levels=1, iters=1)
    Vo, Wo = o.anls_sweep(p.M.astype(np.float64), np.zeros(p.V.shape), p.W.astype(np.float64))
    f, fo = o.objective(p.M, V, W), o.objective(p.M, Vo, Wo)
    assert abs(f - fo) <= 1e-4 * fo, (f, fo)


def test_grid_barrier_timeout_returns_etimeout_and_handle_recovers(h):
    g = GOLDEN["grid19_hals_L3_K500"]
    gh, gw, n, r, sigma = synth.WORKLOADS[g["workload"]]
    p = synth.make_problem(gh, gw, n, r, sigma=sigma)
    V, W = p.V.copy(), p.W.copy()
    h.set_limits(barrier_spins=0)
    try:
        with pytest.raises(native.NMFError) as ei:
            h.solve(p.M, gh, gw, V, W, "hals", levels=3, iters=8)
        assert ei.value.code == native.NMF_ETIMEOUT
    finally:
        h.set_limits()
    # same handle, default budget: the full golden solve
    V, W = p.V.copy(), p.W.copy()
    h.solve(p.M, gh, gw, V, W, "hals", levels=3, iters=g["K"])
    f = o.objective(p.M, V, W)
    assert abs(f - g["objective"]) <= 1e-3 * g["objective"], (f, g["objective"])
