"""Write tests/golden/objectives.json: final ||M - VW||_F of the FP64 oracle for the
seeded workloads (calls only oracle/ and the input generator).

Usage: python tests/golden/make_objectives.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

from oracle import nmf_oracle as o  # noqa: E402
from paper_1009_0881_gb300 import synth  # noqa: E402

CASES = [
    # name, workload, algo, levels, K, cycle
    ("grid16_hals_L3_K100", "grid16_n1000_r10", "hals", 3, 100, "vcycle"),
    ("grid16_hals_L1_K100", "grid16_n1000_r10", "hals", 1, 100, "vcycle"),
    ("grid19_hals_L3_K500", "grid19_n2429_r49", "hals", 3, 500, "vcycle"),
    ("grid19_hals_L1_K500", "grid19_n2429_r49", "hals", 1, 500, "vcycle"),
    ("grid19_mu_L3_K500", "grid19_n2429_r49", "mu", 3, 500, "vcycle"),
    ("grid19_mu_L1_K500", "grid19_n2429_r49", "mu", 1, 500, "vcycle"),
    ("grid19_anls_L2_K8", "grid19_n2429_r49", "anls", 2, 8, "vcycle"),
    # the headline workload's ANLS, NI and FMG at three levels (the 5 x 5 level has m_l = 25 < r:
    # its iterates are not unique, only the objective is compared)
    ("grid19_anls_L3_K8", "grid19_n2429_r49", "anls", 3, 8, "vcycle"),
    ("grid19_anls_L3_K500", "grid19_n2429_r49", "anls", 3, 500, "vcycle"),
    ("grid19_anls_L1_K500", "grid19_n2429_r49", "anls", 1, 500, "vcycle"),
    ("grid19_hals_fmg_L3_K100", "grid19_n2429_r49", "hals", 3, 100, "fmg"),
    ("grid19_hals_ni_L3_K100", "grid19_n2429_r49", "hals", 3, 100, "ni"),
    ("grid19_mu_fmg_L3_K100", "grid19_n2429_r49", "mu", 3, 100, "fmg"),
    ("grid19_anls_fmg_L3_K8", "grid19_n2429_r49", "anls", 3, 8, "fmg"),
    # W-cycle (Section 7 extension)
    ("grid19_hals_wcycle_L3_K100", "grid19_n2429_r49", "hals", 3, 100, "wcycle"),
    ("grid16_mu_wcycle_L3_K100", "grid16_n1000_r10", "mu", 3, 100, "wcycle"),
    # full multigrid and nested iteration start on the coarsest level: keep m_l >= r there
    ("grid19_hals_fmg_L2_K100", "grid19_n2429_r49", "hals", 2, 100, "fmg"),
    ("grid19_hals_ni_L2_K100", "grid19_n2429_r49", "hals", 2, 100, "ni"),
    ("grid16_hals_fmg_L3_K100", "grid16_n1000_r10", "hals", 3, 100, "fmg"),
    ("grid16_hals_ni_L3_K100", "grid16_n1000_r10", "hals", 3, 100, "ni"),
    ("grid16_mu_fmg_L3_K100", "grid16_n1000_r10", "mu", 3, 100, "fmg"),
    # precision-form workloads (ORL shape; 256 x 256 grid)
    ("grid112x92_hals_L3_K100", "grid112x92_n400_r40", "hals", 3, 100, "vcycle"),
    ("grid256_hals_L3_K20", "grid256_n2000_r64", "hals", 3, 20, "vcycle"),
    ("grid256_hals_L3_K100", "grid256_n2000_r64", "hals", 3, 100, "vcycle"),
    # image sequences (Section 6.1): V-cycles that coarsen the columns too ("vcycle_cols"),
    # beside the pixel-only V-cycle and the single-level run on the same data
    ("seq16_hals_cols_L3_K100", "seq16_n1024_r10", "hals", 3, 100, "vcycle_cols"),
    ("seq16_mu_cols_L3_K100", "seq16_n1024_r10", "mu", 3, 100, "vcycle_cols"),
    ("seq16_anls_cols_L3_K8", "seq16_n1024_r10", "anls", 3, 8, "vcycle_cols"),
    ("seq16_hals_L3_K100", "seq16_n1024_r10", "hals", 3, 100, "vcycle"),
    ("seq32_hals_cols_L3_K100", "seq32_n4096_r16", "hals", 3, 100, "vcycle_cols"),
    ("seq32_hals_cols_L4_K100", "seq32_n4096_r16", "hals", 4, 100, "vcycle_cols"),
    ("seq32_hals_L3_K100", "seq32_n4096_r16", "hals", 3, 100, "vcycle"),
    ("seq32_hals_L1_K100", "seq32_n4096_r16", "hals", 1, 100, "vcycle"),
    # V-cycles with explicit per-level counts (the time split of Algorithm V-cycle with
    # measured per-sweep costs): see LEVEL_SWEEPS
    ("grid19_hals_timed_L3", "grid19_n2429_r49", "hals", 3, 0, "vcycle_counts"),
    ("grid19_mu_timed_L3", "grid19_n2429_r49", "mu", 3, 0, "vcycle_counts"),
    # ANLS on the sequence: the W-step's n rows shrink with the columns (Section 6.1)
    ("seq32_anls_L1_K20", "seq32_n4096_r16", "anls", 1, 20, "vcycle"),
    ("seq32_anls_L3_K20", "seq32_n4096_r16", "anls", 3, 20, "vcycle"),
    ("seq32_anls_cols_L3_K20", "seq32_n4096_r16", "anls", 3, 20, "vcycle_cols"),
]


# (pre, coarse, post) of the explicit-count cases: the split of T = 500 finest-sweep times with
# per-sweep costs 28.0 / 22.4 / 16.3 us (19x19 / 10x10 / 5x5 levels, as measured on the GPU)
LEVEL_SWEEPS = {"grid19_hals_timed_L3": ([125, 39], 53, [250, 78]),
                "grid19_mu_timed_L3": ([125, 39], 53, [250, 78])}


def _problem(wl):
    """(grid_h, grid_w, Problem) of a named workload."""
    if wl in synth.SEQUENCE_WORKLOADS:
        h, w, n, r, sigma = synth.SEQUENCE_WORKLOADS[wl]
        return h, w, synth.make_problem(h, w, n, r, sigma=sigma, sequence=True)
    h, w, n, r, sigma = synth.WORKLOADS[wl]
    return h, w, synth.make_problem(h, w, n, r, sigma=sigma)


def _solve(p, h, w, algo, L, K, cyc, name=None, **kw):
    if cyc == "vcycle_counts":
        return o.solve(p.M, h, w, p.V, p.W, algo, levels=L, level_sweeps=LEVEL_SWEEPS[name], **kw)
    if cyc == "vcycle_cols":
        return o.solve(p.M, h, w, p.V, p.W, algo, levels=L, K=K, coarsen_columns=True, **kw)
    return o.solve(p.M, h, w, p.V, p.W, algo, levels=L, K=K, cycle=cyc, **kw)


# Cycles that start on a level with fewer pixels than the rank: their result depends on
# rounding (oracle reading PRECISION), so the values at float32 precision are stored beside the
# FP64 one.
FP32_PRODUCT_CASES = {"grid19_hals_fmg_L3_K100", "grid19_hals_ni_L3_K100", "grid19_mu_fmg_L3_K100",
                      "grid19_anls_fmg_L3_K8", "grid19_anls_L3_K500"}


def _fp32_value(name, threads):
    """Final objective of case `name` with the oracle at float32 precision, run in a child
    process whose float32 matrix products use `threads` threads (None if its active-set NNLS
    cycled on a rounded singular Gram matrix)."""
    import subprocess
    env = dict(os.environ, OPENBLAS_NUM_THREADS=str(threads), OMP_NUM_THREADS=str(threads),
               MKL_NUM_THREADS=str(threads))
    out = subprocess.run([sys.executable, os.path.abspath(__file__), "--fp32", name], env=env, check=True,
                         capture_output=True, text=True).stdout.strip().splitlines()[-1]
    return None if out == "None" else float(out)


def _fp32_child(name):
    for nm, wl, algo, L, K, cyc in CASES:
        if nm == name:
            h, w, p = _problem(wl)
            try:
                V, W = _solve(p, h, w, algo, L, K, cyc, name=nm, precision="fp32")
                print(repr(o.objective(p.M.astype(np.float64), V, W)))
            except o.NNLSNotConverged:
                print("None")
            return


def _store(path, name, entry):
    """Merge one entry into the JSON file (several writers may run at once)."""
    import fcntl
    with open(path + ".lock", "w") as lk:
        fcntl.flock(lk, fcntl.LOCK_EX)
        out = json.load(open(path)) if os.path.exists(path) else {}
        out[name] = entry
        with open(path, "w") as f:
            json.dump(out, f, indent=1, sort_keys=True)
            f.write("\n")


def main(only=None):
    path = os.path.join(HERE, "objectives.json")
    for name, wl, algo, L, K, cyc in CASES:
        if only and name not in only:
            continue
        h, w, p = _problem(wl)
        t = time.time()
        V, W = _solve(p, h, w, algo, L, K, cyc, name=name)
        f = o.objective(p.M.astype(np.float64), V, W)
        entry = {"workload": wl, "algo": algo, "levels": L, "K": K, "cycle": cyc, "objective": f,
                 "norm_M": float(np.linalg.norm(p.M.astype(np.float64)))}
        if cyc == "vcycle_counts":
            entry["level_sweeps"] = LEVEL_SWEEPS[name]
        if name in FP32_PRODUCT_CASES:
            # the oracle at float32 precision with two summation orders of its float32 matrix
            # products (the library matmul on one thread and on four): on these cycles the two
            # orders end in different places, so both are kept
            entry["objective_fp32"] = [_fp32_value(name, threads) for threads in (1, 4)]
        _store(path, name, entry)
        print(f"{name}: {f:.10g} ({time.time() - t:.1f} s)", flush=True)


def add_fp32(name):
    """Add the float32 values to a stored entry, the two summation orders run side by side
    (for cases whose FP64 run takes hours)."""
    from concurrent.futures import ThreadPoolExecutor
    path = os.path.join(HERE, "objectives.json")
    entry = json.load(open(path))[name]
    with ThreadPoolExecutor(2) as ex:
        entry["objective_fp32"] = list(ex.map(lambda t: _fp32_value(name, t), (1, 4)))
    _store(path, name, entry)
    print(f"{name}: float32 {entry['objective_fp32']}", flush=True)


if __name__ == "__main__":
    if len(sys.argv) == 3 and sys.argv[1] == "--fp32":
        _fp32_child(sys.argv[2])
    elif len(sys.argv) == 3 and sys.argv[1] == "--add-fp32":
        add_fp32(sys.argv[2])
    else:
        main(sys.argv[1:] or None)
