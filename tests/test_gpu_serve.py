"""GPU tests of the serving form (nmf_server_*): requests of uneven size arrive
while others run; native worker threads, one stream and workspace per slot,
admit them in arrival order under an HBM budget.

Required properties: a request's result is bitwise the one nmf_solve_batch
gives it alone (same plan, same kernels, same summation orders); the memory the
slots hold never exceeds the budget; a request larger than the budget is
refused at submission with NMF_ENOMEM.
"""
import threading
import time

import numpy as np
import pytest

from paper_1009_0881_gb300 import native, synth

pytestmark = pytest.mark.gpu

REQS = [  # (side_h, side_w, n, r, algo, levels, iters)
    (16, 16, 700, 10, "hals", 3, 40),
    (32, 32, 300, 5, "mu", 3, 40),
    (19, 19, 2429, 49, "anls", 2, 4),
    (64, 64, 1200, 64, "hals", 2, 12),
    (92, 92, 250, 23, "mu", 3, 16),
    (16, 16, 900, 7, "hals", 1, 30),
    (128, 128, 400, 33, "hals", 3, 8),
    (24, 24, 500, 12, "anls", 3, 6),
]


@pytest.fixture(scope="module", params=[native.NMF_FP32, native.NMF_BF16], ids=["fp32", "bf16"])
def ref(request):
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1009_0881_gb300 import build
    build.build()
    with native.Handle(0, precision=request.param) as hd:
        hd.precision = request.param
        yield hd


def _requests(seed0):
    out = []
    for i, (gh, gw, n, r, algo, L, K) in enumerate(REQS):
        p = synth.make_problem(gh, gw, n, r, sigma=0.04 * gw if gw > 19 else 2.0, data_seed=seed0 + i)
        out.append(dict(M=p.M, grid_h=gh, grid_w=gw, V=p.V.copy(), W=p.W.copy(), algo=algo, levels=L, iters=K))
    return out


def _alone(ref, reqs):
    res = []
    for d in reqs:
        e = dict(d, V=d["V"].copy(), W=d["W"].copy())
        (st, sweeps, obj), = ref.solve_batch([e])
        assert st == 0
        res.append((e["V"], e["W"], sweeps, obj))
    return res


def _serve(srv, reqs, gap_s=0.0):
    tickets = []
    for d in reqs:
        tickets.append(srv.submit(d))
        if gap_s:
            time.sleep(gap_s)
    return [srv.poll(t, -1) for t in tickets]


def test_served_equals_alone(ref):
    reqs = _requests(200)
    want = _alone(ref, reqs)
    with native.Server(0, slots=3, precision=ref.precision) as srv:
        got = _serve(srv, reqs, gap_s=0.002)
        assert srv.stats()["completed"] == len(reqs)
    for d, (V, W, sweeps, obj), (st, sw, ob, lat) in zip(reqs, want, got):
        assert st == 0 and lat > 0
        assert sw == sweeps
        np.testing.assert_array_equal(d["V"], V)
        np.testing.assert_array_equal(d["W"], W)
        assert ob == obj


def test_budget_admission(ref):
    reqs = _requests(300)
    want = _alone(ref, reqs)
    need = [ref.workspace_bytes(d) for d in reqs]
    # room for the largest request and a little more: slots must give memory back
    budget = max(need) + min(need)
    seen = []
    stop = threading.Event()
    with native.Server(0, hbm_budget_bytes=budget, slots=4, precision=ref.precision) as srv:
        def watch():
            while not stop.is_set():
                seen.append(srv.stats()["bytes_held"])
                time.sleep(0.0005)
        th = threading.Thread(target=watch)
        th.start()
        try:
            got = _serve(srv, reqs)
        finally:
            stop.set()
            th.join()
        # a request larger than the budget is refused up front
        big = synth.make_problem(128, 128, 4000, 64, data_seed=1)
        d = dict(M=big.M, grid_h=128, grid_w=128, V=big.V.copy(), W=big.W.copy(), levels=3, iters=4)
        assert ref.workspace_bytes(d) > budget
        with pytest.raises(native.NMFError) as ei:
            srv.submit(d)
        assert ei.value.code == -2
    assert max(seen) <= budget
    for d, (V, W, sweeps, obj), (st, sw, ob, lat) in zip(reqs, want, got):
        assert st == 0
        np.testing.assert_array_equal(d["V"], V)
        np.testing.assert_array_equal(d["W"], W)


def test_bad_request_fails_alone(ref):
    reqs = _requests(400)[:3]
    bad = dict(reqs[1], levels=0)
    with native.Server(0, slots=2, precision=ref.precision) as srv:
        with pytest.raises(native.NMFError):
            srv.submit(bad)
        got = _serve(srv, reqs)
    assert all(g[0] == 0 for g in got)


def _sample_problem(row):
    p = synth.make_problem(row["side"], row["side"], row["n"], row["r"], row["sigma"], row["index"])
    return p, dict(M=p.M, grid_h=row["side"], grid_w=row["side"], V=p.V.copy(), W=p.W.copy(), algo=row["algo"],
                   levels=row["levels"], iters=row["iters"])


def sample_bar(row):
    """Bar of one sampled request against the oracle run at the same precision: 1e-3, except
    ANLS on a hierarchy whose coarsest grid has fewer pixels than r, where the NNLS solutions
    of that level are not unique and each side's choice carries into the finer levels (the
    objective alone is compared there, at 1e-2; the largest difference measured is 5.7e-3)."""
    if row["algo"] == "anls" and row["coarsest_pixels"] < row["r"]:
        return 1e-2
    return 1e-3


# BF16 requests against the oracle's bf16 mode: the median within 1e-3 (measured 7.8e-5), each
# request within 5e-2 (measured 4.3e-2).  With budgets of 2-4 sweeps from a random start the first
# sweeps move the iterates far, and a bfloat16 rounding of V that flips between the GPU's float32
# and the oracle's values moves C by ~2^-8 of that entry: short runs drift apart by percents, where
# the converged precision-form workloads agree (test_gpu_bf16).
BF16_SAMPLE_BAR = 5e-2
BF16_SAMPLE_MEDIAN = 1e-3


def sample_reference(row, key):
    """(oracle objective, bar) of one sampled request for the form whose oracle value is
    row[key].  Where the oracle's bf16 mode has no value (its active-set NNLS cycled on a
    rounded singular Gram matrix) the FP64 value stands in."""
    if key == "objective_bf16":
        return (row["objective"] if row.get(key) is None else row[key]), BF16_SAMPLE_BAR
    return row[key], sample_bar(row)


def test_served_sample_against_fp64_oracle(ref):
    # a seeded, size-stratified sample of 64 requests of the serving workload (every size of the
    # uneven pool, HALS / MU / ANLS in turn, three levels, short fixed budgets), all in flight in
    # one server at once; each result against the oracle's objective for the same request
    # (tests/golden/served_sample.json, written by tests/golden/make_served_sample.py): the
    # float32 form against the FP64 oracle, the BF16 form against the oracle in its bf16 mode
    # (the same bfloat16 operands); the BF16 form's distance to FP64 is printed, not gated.
    import json
    import os
    from conftest import ROOT
    G = json.load(open(os.path.join(ROOT, "tests", "golden", "served_sample.json")))
    assert len(G["requests"]) >= 64
    key = "objective" if ref.precision == native.NMF_FP32 else "objective_bf16"
    errs, to64 = [], []
    with native.Server(0, hbm_budget_bytes=40 * 10**9, slots=8, precision=ref.precision) as srv:
        pending = []
        for row in G["requests"]:
            p, d = _sample_problem(row)
            pending.append((srv.submit(d), d, row))
        for t, d, row in pending:
            st, sweeps, obj, lat = srv.poll(t, -1)
            assert st == 0, (row, st)
            ref_f, bar = sample_reference(row, key)
            e = abs(obj - ref_f) / ref_f
            errs.append((e / bar, e, row["algo"], row["side"], row["r"]))
            to64.append(abs(obj - row["objective"]) / row["objective"])
            assert (d["V"] >= 0).all() and (d["W"] >= 0).all()
    worst = max(errs)
    print(f"served sample ({'fp32' if ref.precision == native.NMF_FP32 else 'bf16'}): max rel. error "
          f"{max(e[1] for e in errs):.2e}, median {float(np.median([e[1] for e in errs])):.2e}; "
          f"against FP64: max {max(to64):.2e}, median {float(np.median(to64)):.2e}")
    assert worst[0] <= 1.0, worst
    if key == "objective_bf16":
        assert float(np.median([e[1] for e in errs])) <= BF16_SAMPLE_MEDIAN
