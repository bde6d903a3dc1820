"""Writes ``pet_objectives.json``: the float64 oracle's penalised PET
objective (Eq. (PET-objpen)) after k iterations of Algorithm 2 from
lambda = 1, for each penalty constant of the PET workloads.

The values come only from ``oracle/pet_oracle.py`` (Section 3.2, Algorithm
2) run on the seeded inputs of ``paper_1003_3272_gb300/synth.py``; the
benchmark compares the GPU's objectives after the same number of iterations
against them.  Run from the repository root (a few minutes):

    python tests/golden/make_pet_objectives.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import pet_oracle as po  # noqa: E402
from paper_1003_3272_gb300 import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "pet_objectives.json")


def main():
    out = {"_about": {"what": "float64 oracle objective f(lambda) of Eq. (PET-objpen) after k "
                              "iterations of Algorithm 2 from lambda = 1, per penalty constant",
                      "writer": "tests/golden/make_pet_objectives.py (oracle/pet_oracle.py only)"}}
    for build in (synth.pet, synth.pet_large):
        pr = build()
        ent = {"d": pr.d, "p": pr.p, "iters": pr.iters, "mu": list(pr.mu), "objective": {}}
        for mu in pr.mu:
            _, fs, _ = po.run(pr.E, pr.y, mu, pr.nbr_ptr, pr.nbr_idx, pr.iters)
            ent["objective"][repr(mu)] = {"0": fs[0], str(pr.iters): fs[-1]}
            print(pr.name, mu, fs[0], fs[-1], flush=True)
        out[pr.name] = ent
    with open(OUT, "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
