"""GPU tests of the batched form (nmf_solve_batch): many uneven problems in one
CUDA graph of concurrent branches.

Required property: a problem's result is the same alone and in the batch.  The
batch runs the same kernels with the same launch shapes and summation orders
as nmf_solve, so the comparison is bitwise.  The stopping rule (relative
objective change of consecutive finest-level post-smoothing sweeps) is checked
against the per-sweep objective trace of the standalone solve.
"""
import numpy as np
import pytest

from oracle import nmf_oracle as o
from paper_1009_0881_gb300 import native, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=[native.NMF_FP32, native.NMF_BF16], ids=["fp32", "bf16"])
def h(request):
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1009_0881_gb300 import build
    build.build()
    with native.Handle(0, precision=request.param) as hd:
        hd.precision = request.param
        yield hd


MIX = [  # (side_h, side_w, n, r, algo, levels, iters)
    (16, 16, 700, 10, "hals", 3, 40),
    (19, 19, 2429, 49, "hals", 3, 20),
    (32, 32, 300, 5, "mu", 3, 40),
    (64, 64, 1200, 64, "hals", 2, 12),
    (92, 92, 250, 23, "hals", 3, 16),
    (16, 16, 900, 7, "mu", 1, 30),
    (128, 128, 400, 33, "hals", 3, 8),
]


def _problems(seed0=0):
    out = []
    for i, (gh, gw, n, r, algo, L, K) in enumerate(MIX):
        p = synth.make_problem(gh, gw, n, r, sigma=0.04 * gw if gw > 19 else 2.0, data_seed=seed0 + i)
        out.append((p, algo, L, K))
    return out


def test_batch_equals_alone(h):
    probs = _problems()
    batch = []
    for p, algo, L, K in probs:
        batch.append(dict(M=p.M, grid_h=p.grid_h, grid_w=p.grid_w, V=p.V.copy(), W=p.W.copy(), algo=algo,
                          levels=L, iters=K))
    res = h.solve_batch(batch)
    for (p, algo, L, K), d, (st, sweeps, obj) in zip(probs, batch, res):
        assert st == 0
        assert sweeps == sum(native.schedule("vcycle", L, K))
        V, W = p.V.copy(), p.W.copy()
        h.solve(p.M, p.grid_h, p.grid_w, V, W, algo, levels=L, iters=K)
        np.testing.assert_array_equal(d["V"], V)
        np.testing.assert_array_equal(d["W"], W)
        assert abs(obj - h.error(p.M, V, W)) <= 1e-9 * obj


def test_batch_repeat_and_order_independence(h):
    probs = _problems(seed0=10)
    def run(order):
        batch = [dict(M=probs[i][0].M, grid_h=probs[i][0].grid_h, grid_w=probs[i][0].grid_w, V=probs[i][0].V.copy(),
                      W=probs[i][0].W.copy(), algo=probs[i][1], levels=probs[i][2], iters=probs[i][3]) for i in order]
        h.solve_batch(batch)
        return {i: (d["V"], d["W"]) for i, d in zip(order, batch)}
    a = run(list(range(len(probs))))
    b = run(list(reversed(range(len(probs)))))
    for i in a:
        np.testing.assert_array_equal(a[i][0], b[i][0])
        np.testing.assert_array_equal(a[i][1], b[i][1])


@pytest.mark.parametrize("algo,tol", [("hals", 1e-3), ("hals", 1e-2), ("anls", 1e-2)])
def test_stopping_rule_matches_standalone_trace(h, algo, tol):
    # the batched run stops after the first post-smoothing sweep t with |f_{t-1} - f_t| <= tol f_t
    p = synth.make_problem(19, 19, 2429, 49, data_seed=3)
    L, K = 3, (200 if algo == "hals" else 24)
    V, W = p.V.copy(), p.W.copy()
    n_fine = native.schedule("vcycle", L, K)[0]
    tr = h.solve(p.M, 19, 19, V, W, algo, levels=L, iters=K, trace_len=n_fine)
    post = tr[K // 4:]
    stop = len(post)
    for t in range(1, len(post)):
        if abs(post[t - 1] - post[t]) <= tol * post[t]:
            stop = t + 1
            break
    d = dict(M=p.M, grid_h=19, grid_w=19, V=p.V.copy(), W=p.W.copy(), algo=algo, levels=L, iters=K, rel_tol=tol)
    (st, sweeps, obj), = h.solve_batch([d])
    total = sum(native.schedule("vcycle", L, K))
    assert st == 0
    assert sweeps == total - len(post) + stop
    # the iterate is the standalone one after the same number of sweeps
    V2, W2 = p.V.copy(), p.W.copy()
    h.solve(p.M, 19, 19, V2, W2, algo, levels=L, iters=K, stop_after=sweeps)
    np.testing.assert_array_equal(d["V"], V2)
    np.testing.assert_array_equal(d["W"], W2)
    assert abs(obj - post[stop - 1]) <= 1e-12 * obj


def test_batch_of_uneven_sizes_against_oracle(h):
    # the 64 requests of the uneven-size pool (sides 16 .. 128, n 200 .. 4000, r 5 .. 64, HALS /
    # MU / ANLS in turn, three levels, short fixed budgets) in one batch, each result against the
    # oracle's objective for the same request (tests/golden/served_sample.json): float32 against
    # FP64, BF16 against the oracle's bf16 mode, with the bars of test_gpu_serve.sample_bar
    import json
    import os
    from conftest import ROOT
    from test_gpu_serve import BF16_SAMPLE_MEDIAN, sample_reference
    G = json.load(open(os.path.join(ROOT, "tests", "golden", "served_sample.json")))
    key = "objective" if h.precision == native.NMF_FP32 else "objective_bf16"
    batch, rows = [], []
    for row in G["requests"]:
        p = synth.make_problem(row["side"], row["side"], row["n"], row["r"], row["sigma"], row["index"])
        batch.append(dict(M=p.M, grid_h=row["side"], grid_w=row["side"], V=p.V.copy(), W=p.W.copy(),
                          algo=row["algo"], levels=row["levels"], iters=row["iters"]))
        rows.append((row, p))
    res = h.solve_batch(batch)
    errs = []
    for (st, sweeps, obj), (row, p), d in zip(res, rows, batch):
        assert st == 0
        ref_f, bar = sample_reference(row, key)
        err = abs(obj - ref_f) / ref_f
        errs.append(err)
        assert err <= bar, (row, obj)
        assert abs(obj - o.objective(p.M, d["V"], d["W"])) <= 1e-6 * obj
    if key == "objective_bf16":
        assert float(np.median(errs)) <= BF16_SAMPLE_MEDIAN
    print(f"batch of 64 against the oracle: max rel. error {max(errs):.2e}, median {float(np.median(errs)):.2e}")


def test_batch_with_explicit_counts_equals_alone(h):
    # problems carrying explicit V-cycle counts (nmf_problem.level_sweeps) get the bits of a
    # standalone solve with the same counts; a problem without them keeps its iters schedule
    probs = _problems()[:4]
    counts = [([2, 1], 5, [4, 3]), None, ([1, 0], 7, [2, 2]), ([3], 4, [5])]
    batch = []
    for (p, algo, L, K), ls in zip(probs, counts):
        if ls is not None and len(ls[0]) != L - 1:
            ls = ([1] * (L - 1), 3, [2] * (L - 1))
        batch.append(dict(M=p.M, grid_h=p.grid_h, grid_w=p.grid_w, V=p.V.copy(), W=p.W.copy(), algo=algo,
                          levels=L, iters=K, level_sweeps=ls))
    res = h.solve_batch(batch)
    for (p, algo, L, K), d, (st, sweeps, obj) in zip(probs, batch, res):
        assert st == 0
        ls = d["level_sweeps"]
        if ls is not None:
            assert sweeps == sum(ls[0]) + ls[1] + sum(ls[2])
        V, W = p.V.copy(), p.W.copy()
        h.solve(p.M, p.grid_h, p.grid_w, V, W, algo, levels=L, iters=K, level_sweeps=ls)
        np.testing.assert_array_equal(d["V"], V)
        np.testing.assert_array_equal(d["W"], W)
