"""Write tests/golden/served_sample.json: the FP64 oracle's final ||M - VW||_F for a
seeded sample of 64 requests of the serving workload (calls only oracle/ and the
input generator).

The sample: problem i (i = 0..63) of the uneven-size pool (side in {16, 19, 32, 64,
92, 128}, n ~ U[200, 4000], r ~ U[5, 64], data seed i, as the batched and served
forms draw it), its algorithm cycling through HALS, MU, ANLS so that every size
stratum meets every algorithm, three levels and a short fixed sweep budget (the
oracle's cost on the largest sizes is the limit): K = 4 for HALS and MU, K = 2
for ANLS.  A served request with the same (problem, algorithm, L, K) and no
stopping rule must reach the stored objective: "objective" at FP64, and
"objective_bf16" with the oracle in its bf16 mode (the library's precision form).

Usage: python tests/golden/make_served_sample.py [workers]
"""
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

from oracle import nmf_oracle as o  # noqa: E402
from paper_1009_0881_gb300 import synth  # noqa: E402

COUNT = 64
LEVELS = 3
ITERS = {"hals": 4, "mu": 4, "anls": 2}
ALGOS = ("hals", "mu", "anls")


def sample():
    """(index, side, n, r, sigma, algo, levels, iters) of every sampled request."""
    out = []
    for i, (side, n, r) in enumerate(synth.batched_sizes(COUNT)):
        algo = ALGOS[i % 3]
        out.append((i, side, n, r, 0.04 * side if side > 19 else 2.0, algo, LEVELS, ITERS[algo]))
    return out


def _one(item):
    i, side, n, r, sigma, algo, L, K = item
    p = synth.make_problem(side, side, n, r, sigma, i)
    t = time.time()
    V, W = o.solve(p.M, side, side, p.V, p.W, algo, levels=L, K=K)
    f = o.objective(p.M.astype(np.float64), V, W)
    try:
        V, W = o.solve(p.M, side, side, p.V, p.W, algo, levels=L, K=K, precision="bf16")
        fb = o.objective(p.M.astype(np.float64), V, W)
    except o.NNLSNotConverged:
        # the active-set method can cycle on a rounded singular Gram matrix: no bf16 value
        fb = None
    # coarsest grid of the hierarchy: ANLS there is not unique when it has fewer pixels than r
    cs = side
    for _ in range(L - 1):
        cs = (cs + 1) // 2
    return {"index": i, "side": side, "n": n, "r": r, "sigma": sigma, "algo": algo, "levels": L, "iters": K,
            "objective": f, "objective_bf16": fb, "coarsest_pixels": cs * cs, "seconds": time.time() - t}


def main(workers):
    with mp.get_context("spawn").Pool(workers) as pool:
        rows = pool.map(_one, sample(), chunksize=1)
    path = os.path.join(HERE, "served_sample.json")
    with open(path, "w") as f:
        json.dump({"count": COUNT, "levels": LEVELS, "iters": ITERS, "requests": rows}, f, indent=1)
        f.write("\n")
    print(f"{len(rows)} requests, oracle time {sum(r['seconds'] for r in rows):.0f} s")


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else max(1, (os.cpu_count() or 2) - 1))
