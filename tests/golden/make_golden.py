"""Writes the stored expected values of tests/golden/ by calling the FP64 oracle only.

Run from the repository root:  python tests/golden/make_golden.py [name ...]
Each output is a small JSON file named for the workload, holding the oracle's efficiency,
uniformity, weights and trap fields after the full GSW run of that workload, plus the
command and oracle thread count that produced it.  Only workloads whose full oracle run is
too slow for a test (minutes on a few cores) are stored; the others are recomputed live.
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_0907_4027_gb300 import workloads as wl  # noqa: E402

STORED = ["rand1000_1920"]


def run(name: str) -> str:
    w = wl.NAMED[name]()
    t0 = time.time()
    r = oracle.gsw(w.geom, w.xyz, w.iters, w.phi0, w.w0)
    out = {
        "workload": name, "W": w.W, "H": w.H, "M": w.M, "iters": w.iters,
        "source": "oracle.gsw (FP64, tests/golden/make_golden.py)",
        "oracle_threads": oracle.set_threads(), "seconds": round(time.time() - t0, 1),
        "e": r["e"], "u": r["u"],
        "w": r["w"].tolist(), "V_re": r["V"].real.tolist(), "V_im": r["V"].imag.tolist(),
    }
    path = os.path.join(HERE, f"{name}_gsw.json")
    with open(path, "w") as f:
        json.dump(out, f)
    return path


if __name__ == "__main__":
    for n in (sys.argv[1:] or STORED):
        print(run(n))
