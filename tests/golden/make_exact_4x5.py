"""Writes ``exact_4x5.txt``: one MM iteration of a 4 x 5, rank-2 problem with
small integer entries, in exact rational arithmetic.

The values come only from ``oracle/exact.py`` (the paper's elementwise
Eqs. (3.3)-(3.4), Section 3.1, evaluated with Fractions).  Run from the
repository root:  python tests/golden/make_exact_4x5.py
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import exact  # noqa: E402

# data (build V, paper X), left factor (build W, paper V), right (build H, paper W)
V = [[3, 1, 4, 1, 5],
     [9, 2, 6, 5, 3],
     [5, 8, 9, 7, 9],
     [3, 2, 3, 8, 4]]
W = [[1, 2],
     [3, 1],
     [2, 2],
     [1, 3]]
H = [[2, 1, 1, 3, 1],
     [1, 2, 3, 1, 2]]


def fmt(M):
    return "\n".join(" ".join(f"{x.numerator}/{x.denominator}" for x in row) for row in M)


def main():
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "exact_4x5.txt")
    lines = ["# One MM iteration, exact rationals (oracle/exact.py).",
             "# Source: Section 3.1, Eqs. (3.3) and (3.4); objective Eq. (3.1).",
             "# Build letters: V (4x5 data), W (4x2 left), H (2x5 right); eps = 0.",
             "[V]", fmt([[__import__('fractions').Fraction(x) for x in r] for r in V]),
             "[W0]", fmt([[__import__('fractions').Fraction(x) for x in r] for r in W]),
             "[H0]", fmt([[__import__('fractions').Fraction(x) for x in r] for r in H])]
    f0 = exact.objective(V, W, H)
    lines += ["[f0]", f"{f0.numerator}/{f0.denominator}"]
    for order in ("h_first", "w_first"):
        W1, H1 = exact.iteration(V, W, H, order=order)
        f1 = exact.objective(V, W1, H1)
        lines += [f"[W1 {order}]", fmt(W1), f"[H1 {order}]", fmt(H1),
                  f"[f1 {order}]", f"{f1.numerator}/{f1.denominator}"]
    with open(out, "w") as fh:
        fh.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
