"""Iterations the oracle's textbook CG needs on the benchmark workload.

Test infrastructure (see oracle/__init__.py).  Writes
tests/golden/cg_iters_32x4.json: the number of CG iterations (Sec. 7.1
baseline) to a true relative residual <= tol for one source of the 32^4,
m = 0.01 workload, with the seeded inputs of hisq_inputs (links drawn with the
CPU torch generator, seed 1001; sources seed 2100).  The benchmark's CPU
baseline multiplies the oracle's measured time per CG iteration by this count
to report a time to solution per right-hand side.

Usage: python -m oracle.cg_iteration_count [column ...]
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import hisq_inputs as hi  # noqa: E402
from oracle import hisq  # noqa: E402

DIMS = (32, 32, 32, 32)
MASS = 0.01
LINK_SEED = 1001
SRC_SEED = 2100
N_SRC = 16
TOL = 1e-10
OUT = os.path.join(ROOT, "tests", "golden", "cg_iters_32x4.json")


def main(columns):
    fat, lng = hi.random_links_torch(DIMS, LINK_SEED, "cpu")
    fat, lng = fat.numpy(), lng.numpy()
    b = hi.gaussian_sources(DIMS, N_SRC, SRC_SEED)
    rows = []
    for j in columns:
        t = time.time()
        x, it, res = hisq.cg(DIMS, fat, lng, MASS, b[j:j + 1], tol=TOL, max_iter=20000)
        rows.append({"column": int(j), "iterations": int(it[0]), "true_rel_res": float(res[0]),
                     "seconds": round(time.time() - t, 1)})
        print(rows[-1], flush=True)
    doc = {"dims": list(DIMS), "mass": MASS, "link_seed": LINK_SEED, "link_generator": "torch-cpu",
           "source_seed": SRC_SEED, "n_sources": N_SRC, "tol": TOL, "solver": "oracle textbook CG",
           "results": rows,
           "iterations_mean": float(np.mean([r["iterations"] for r in rows]))}
    with open(OUT, "w") as f:
        json.dump(doc, f, indent=1)
    print(OUT)


if __name__ == "__main__":
    cols = [int(c) for c in sys.argv[1:]] or [0]
    main(cols)
