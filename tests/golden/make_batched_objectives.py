"""Writes ``batched_objectives.json``: the float64 oracle's objective
||V - WH||_F^2 (Eq. (3.1)) after 100 MM iterations (Eqs. (3.3)-(3.4), H
first, eps 1e-10) from the seeded start, for a fixed sample of the batched
workload's 512 instances (every 32nd).

The values come only from ``oracle/nmf_oracle.py`` run on the seeded inputs
of ``paper_1003_3272_gb300/synth.py``; the benchmark compares the batched
kernels' objectives after the same iterations against them.  Run from the
repository root (under a minute):

    python tests/golden/make_batched_objectives.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import nmf_oracle as orc  # noqa: E402
from paper_1003_3272_gb300 import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "batched_objectives.json")
ITERS = 100
SAMPLE = list(range(0, 512, 32))


def main():
    probs = synth.batch(iters=ITERS)
    out = {"_about": {"what": f"float64 oracle objective after {ITERS} MM iterations (H first, "
                              "eps 1e-10) of sampled instances of synth.batch()",
                      "writer": "tests/golden/make_batched_objectives.py (oracle/nmf_oracle.py only)"},
           "iters": ITERS, "objective": {}}
    for b in SAMPLE:
        pr = probs[b]
        W, H, _, _ = orc.run(pr.V, pr.W0, pr.H0, ITERS, eps=pr.eps)
        out["objective"][str(b)] = orc.objective(pr.V, W, H)
        print(b, pr.name, out["objective"][str(b)], flush=True)
    with open(OUT, "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
