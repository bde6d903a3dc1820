"""Writes ``objectives.json``: the float64 oracle's objective trajectory
(Eq. (3.1), ||V - WH||_F^2) on the measured workloads, from Algorithm 1's
seeded start, H-first order, eps = 1e-10.

The values come only from ``oracle/nmf_oracle.py`` (the MM updates of
Eqs. (3.3)-(3.4), Section 3.1) run on the seeded inputs of
``paper_1003_3272_gb300/synth.py``.  The benchmark and the GPU tests compare
the GPU's objective after the same number of iterations against them.

Run from the repository root (several minutes; the large workload needs
about 40 GB of host memory):

    python tests/golden/make_objectives.py [workload ...]
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import nmf_oracle as orc  # noqa: E402
from paper_1003_3272_gb300 import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "objectives.json")


def objective_blocks(V, W, H, block=4096):
    """The oracle's direct residual summed over row blocks (bounded memory)."""
    return float(sum(orc.objective(V[i:i + block], W[i:i + block], H)
                     for i in range(0, V.shape[0], block)))


def trajectory(pr, checkpoints):
    W = pr.W0.astype(np.float64)
    H = pr.H0.astype(np.float64)
    out = {"0": objective_blocks(pr.V, W, H)}
    for k in range(1, max(checkpoints) + 1):
        W, H = orc.step(pr.V, W, H, pr.eps, "h_first")
        if k in checkpoints:
            out[str(k)] = objective_blocks(pr.V, W, H)
    return out


def workloads():
    return {
        "faces_361x2429_r10": (synth.faces, [10, 50]),
        "planted_1024x1024_r50": (lambda: synth.planted(p=1024, n=1024, r=50, iters=10), [10]),
        "planted_8192x8192_r50": (synth.planted, [10, 200]),
        "tall_65536x4096_r16": (lambda: synth.tall(16), [10, 20]),
        "tall_65536x4096_r32": (lambda: synth.tall(32), [10, 20]),
        "tall_65536x4096_r64": (lambda: synth.tall(64), [10, 20]),
        "tall_65536x4096_r128": (lambda: synth.tall(128), [10, 20]),
        "large_131072x16384_r64": (synth.large, [20]),
    }


def main(names):
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as fh:
            data = json.load(fh)
    data.setdefault("_about", {
        "what": "float64 oracle objective ||V - WH||_F^2 after k MM iterations "
                "(H first, eps 1e-10) from the seeded uniform(0,1) start",
        "writer": "tests/golden/make_objectives.py (oracle/nmf_oracle.py only)"})
    todo = workloads()
    for name in names or list(todo):
        make, cps = todo[name]
        t0 = time.time()
        pr = make()
        data[name] = {"p": pr.p, "n": pr.n, "r": pr.r, "seed": pr.seed,
                      "objective": trajectory(pr, cps)}
        del pr
        print(f"{name}: {data[name]['objective']} ({time.time() - t0:.0f} s)", flush=True)
        with open(OUT, "w") as fh:
            json.dump(data, fh, indent=1, sort_keys=True)
            fh.write("\n")


if __name__ == "__main__":
    main(sys.argv[1:])
