"""GPU tests of the grouped form (nmf_solve_grouped): every half-sweep of many problems'
common schedule in one persistent launch over all their tiles.

Bars (FP32): a single sweep from identical iterates within 1e-5 of the FP64 oracle
(norm-wise, V and W); whole cycles within 1e-3 of the oracle's objective (the 64-request
sample's HALS and MU requests, tests/golden/served_sample.json).  A problem's result
does not depend on the rest of the group (bitwise), and the stopping rule stops where
the per-sweep objective says it should.
"""
import json
import os

import numpy as np
import pytest

from conftest import ROOT
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


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


# ragged shapes: grids that are not multiples of the 64-row tile, n not a multiple of the
# 32-row stage, ranks in every padded-width class (16, 32, 48, 64 columns)
SHAPES = [(9, 7, 77, 5), (19, 19, 2429, 49), (64, 64, 500, 33), (16, 16, 1000, 10), (13, 17, 131, 64),
          (128, 92, 203, 40)]


# shapes whose three-level hierarchy keeps at least r pixels on the coarsest grid: there the
# iterates are unique and float32 sums in another order stay within rounding of each other
# (on a coarsest grid with fewer pixels than r the objective is flat and the order of the
# sums can decide where a run settles, as on the 19 x 19 grid at three levels)
WELL_POSED = [SHAPES[0], SHAPES[2], SHAPES[3], SHAPES[5]]


def _group(shapes, algo, L, K, rel_tol=0.0, seed0=0):
    out = []
    for i, (gh, gw, n, r) in enumerate(shapes):
        p = synth.make_problem(gh, gw, n, r, sigma=0.04 * gw if gw > 19 else 2.0, data_seed=seed0 + i)
        out.append((p, dict(M=p.M, grid_h=gh, grid_w=gw, V=p.V.copy(), W=p.W.copy(), algo=algo, levels=L,
                            iters=K, rel_tol=rel_tol)))
    return out


@pytest.mark.parametrize("algo", ["hals", "mu"])
def test_single_sweep_matches_oracle(h, algo):
    g = _group(SHAPES, algo, 1, 1)
    res = h.solve_batch([d for _, d in g], grouped=True)
    for (p, d), (st, sweeps, obj) in zip(g, res):
        assert st == 0 and sweeps == 1
        Vo, Wo = o.smooth(p.M.astype(np.float64), p.V.astype(np.float64), p.W.astype(np.float64), algo, 1)
        # a HALS V-step from a random start zeroes whole columns of V (D_kk = 0: the row of W
        # is left as it is) or leaves them at rounding level, where the float32 D_kk is a few
        # ulps of noise and the W-step divides by it: those rows of W are not determined by
        # the data.  W is compared on the rows whose column of V is above 1e-3 of the largest,
        # and VW (which the undetermined rows do not touch) as a whole
        cn = np.linalg.norm(Vo, axis=0)
        kept = cn > 1e-3 * cn.max()
        ew = rel(d["W"][kept], Wo[kept])
        evw = rel(d["V"].astype(np.float64) @ d["W"], Vo @ Wo)
        print(f"grouped {algo} sweep {p.M.shape} r={p.V.shape[1]}: V {rel(d['V'], Vo):.2e}, W {ew:.2e} "
              f"({kept.sum()} rows), VW {evw:.2e}")
        assert rel(d["V"], Vo) <= 1e-5 and ew <= 1e-5 and evw <= 1e-5, (p.M.shape, rel(d["V"], Vo), ew, evw)
        assert abs(obj - o.objective(p.M, Vo, Wo)) <= 1e-5 * obj


@pytest.mark.parametrize("algo,L,K", [("hals", 3, 12), ("mu", 2, 10)])
def test_result_does_not_depend_on_the_group(h, algo, L, K):
    g = _group(SHAPES, algo, L, K)
    res = h.solve_batch([d for _, d in g], grouped=True)
    again = _group(SHAPES, algo, L, K)
    res2 = h.solve_batch([d for _, d in again], grouped=True)
    for i, ((p, d), (_, d2)) in enumerate(zip(g, again)):
        # run to run
        np.testing.assert_array_equal(d["V"], d2["V"])
        np.testing.assert_array_equal(d["W"], d2["W"])
        assert res[i] == res2[i]
    for i in (0, 1, 4):
        alone = _group(SHAPES, algo, L, K)[i][1]
        r1 = h.solve_batch([alone], grouped=True)[0]
        np.testing.assert_array_equal(alone["V"], g[i][1]["V"])
        np.testing.assert_array_equal(alone["W"], g[i][1]["W"])
        assert r1 == res[i]


def test_cycles_close_to_plain_solve(h):
    # the grouped form and nmf_solve differ only in the order of float32 sums
    g = _group(WELL_POSED, "hals", 3, 20)
    res = h.solve_batch([d for _, d in g], grouped=True)
    for (p, d), (st, sweeps, obj) in zip(g, res):
        V, W = p.V.copy(), p.W.copy()
        h.solve(p.M, d["grid_h"], d["grid_w"], V, W, "hals", levels=3, iters=20)
        f = o.objective(p.M, V, W)
        assert st == 0 and abs(obj - f) <= 1e-4 * f, (p.M.shape, obj, f)
        assert abs(obj - o.objective(p.M, d["V"], d["W"])) <= 1e-6 * obj


def test_sample_against_fp64_oracle(h):
    # the 64-request sample's HALS and MU requests (three levels, K = 4), each algorithm as
    # one grouped solve, against the FP64 oracle's stored objectives at 1e-3
    G = json.load(open(os.path.join(ROOT, "tests", "golden", "served_sample.json")))
    worst = 0.0
    for algo in ("hals", "mu"):
        rows = [row for row in G["requests"] if row["algo"] == algo]
        assert len(rows) >= 20
        batch = []
        for row in rows:
            p = synth.make_problem(row["side"], row["side"], row["n"], row["r"], row["sigma"], row["index"])
            batch.append(dict(M=p.M, grid_h=row["side"], grid_w=row["side"], V=p.V.copy(), W=p.W.copy(), algo=algo,
                              levels=row["levels"], iters=row["iters"]))
        res = h.solve_batch(batch, grouped=True)
        for row, d, (st, sweeps, obj) in zip(rows, batch, res):
            assert st == 0
            e = abs(obj - row["objective"]) / row["objective"]
            worst = max(worst, e)
            assert e <= 1e-3, (row, obj)
            assert (d["V"] >= 0).all() and (d["W"] >= 0).all()
    print(f"grouped sample: max rel. error {worst:.2e}")


def test_hals_and_mu_in_one_group(h):
    # the update rule is a per-problem choice: a group mixing HALS and MU problems gives each
    # the bits it gets in a group of its own algorithm
    mixed = _group(WELL_POSED, "hals", 2, 6)
    for i in (1, 3):
        mixed[i][1]["algo"] = "mu"
    res = h.solve_batch([d for _, d in mixed], grouped=True)
    for i, (p, d) in enumerate(mixed):
        alone = _group(WELL_POSED, d["algo"], 2, 6)[i][1]
        r1 = h.solve_batch([alone], grouped=True)[0]
        np.testing.assert_array_equal(alone["V"], d["V"])
        np.testing.assert_array_equal(alone["W"], d["W"])
        assert r1 == res[i]


def test_stopping_rule(h):
    # each problem stops after the first watched sweep whose objective changed by at most
    # 1e-3 relative; the sweeps counted agree with the problem's own objective trace
    K = 40
    g = _group(WELL_POSED, "hals", 3, K, rel_tol=1e-3)
    res = h.solve_batch([d for _, d in g], grouped=True)
    full = sum(native.schedule("vcycle", 3, K))
    post = K // 2
    for (p, d), (st, sweeps, obj) in zip(g, res):
        assert st == 0 and full - post < sweeps <= full
        # the plain solve's trace of the last fine run gives where the rule fires (within one
        # sweep: the two forms' float32 sums differ)
        V, W = p.V.copy(), p.W.copy()
        tr = h.solve(p.M, d["grid_h"], d["grid_w"], V, W, "hals", levels=3, iters=K, trace_len=1000)[-post:]
        stop = next((t + 1 for t in range(1, post) if abs(tr[t - 1] - tr[t]) <= 1e-3 * tr[t]), post)
        assert abs((sweeps - (full - post)) - stop) <= 1, (sweeps - (full - post), stop)
        assert abs(obj - o.objective(p.M, d["V"], d["W"])) <= 1e-6 * obj


def test_outside_its_scope_is_rejected(h):
    g = _group(SHAPES[:2], "hals", 2, 4)
    g[1][1]["algo"] = "anls"
    with pytest.raises(native.NMFError) as ei:
        h.solve_batch([d for _, d in g], grouped=True)
    assert ei.value.code == native.NMF_EINVAL
    g = _group(SHAPES[:2], "hals", 2, 4)
    g[1][1]["levels"] = 3
    with pytest.raises(native.NMFError):
        h.solve_batch([d for _, d in g], grouped=True)
    with native.Handle(0, precision=native.NMF_BF16) as hb:
        with pytest.raises(native.NMFError):
            hb.solve_batch([d for _, d in _group(SHAPES[:2], "hals", 2, 4)], grouped=True)
    # the handle stays usable
    res = h.solve_batch([d for _, d in _group(SHAPES[:2], "hals", 2, 4)], grouped=True)
    assert all(st == 0 for st, _, _ in res)


@pytest.mark.parametrize("cycle", ["ni", "fmg", "wcycle"])
def test_other_cycles_against_oracle(h, cycle):
    # every cycle the schedule builder knows runs grouped: the result within 1e-3 of the FP64
    # oracle's objective for the same cycle (shapes whose coarsest grid keeps r pixels)
    g = _group(WELL_POSED[:3], "hals", 3, 12)
    for _, d in g:
        d["cycle"] = cycle
    res = h.solve_batch([d for _, d in g], grouped=True)
    for (p, d), (st, sweeps, obj) in zip(g, res):
        assert st == 0
        Vo, Wo = o.solve(p.M, d["grid_h"], d["grid_w"], p.V, p.W, "hals", levels=3, K=12, cycle=cycle)
        fo = o.objective(p.M, Vo, Wo)
        assert abs(obj - fo) <= 1e-3 * fo, (cycle, p.M.shape, obj, fo)
        assert sweeps == sum(native.schedule(cycle, 3, 12))
