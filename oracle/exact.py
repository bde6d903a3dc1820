"""Exact rational arithmetic form of one MM iteration, for tiny inputs.

TEST INFRASTRUCTURE ONLY (same rule as ``nmf_oracle``).

This is the paper's *elementwise* statement of the updates, Section 3.1,
Eqs. (3.3)-(3.4), evaluated with ``fractions.Fraction`` so that there is no
rounding at all.  In the paper's letters (X data, V left, W right factor):

    v_{n+1,ik} = v_{nik} * sum_j x_ij w_nkj / sum_j b_nij w_nkj,
                 b_nij = sum_k v_nik w_nkj
    w_{n+1,kj} = w_nkj * sum_i x_ij v_{n+1,ik} / sum_i c_nij v_{n+1,ik},
                 c_nij = sum_k v_{n+1,ik} w_nkj

It is deliberately a different formulation from the float64 oracle (which
groups the denominators through the r x r Gram matrix), so that agreement
between the two pins the grouping, the transposes and the indices.
Pure-Python loops: use it only on inputs of a few dozen entries.
"""
from __future__ import annotations

from fractions import Fraction


def _F(a):
    return [[Fraction(x) for x in row] for row in a]


def left_update(X, V, W, eps=Fraction(0)):
    """Eq. (3.3): new left factor (paper V, build W) from X, V_n, W_n."""
    X, V, W = _F(X), _F(V), _F(W)
    p, q, r = len(X), len(X[0]), len(W)
    b = [[sum(V[i][k] * W[k][j] for k in range(r)) for j in range(q)]
         for i in range(p)]
    out = []
    for i in range(p):
        row = []
        for k in range(r):
            num = sum(X[i][j] * W[k][j] for j in range(q))
            den = sum(b[i][j] * W[k][j] for j in range(q)) + eps
            row.append(V[i][k] * num / den)
        out.append(row)
    return out


def right_update(X, V1, W, eps=Fraction(0)):
    """Eq. (3.4): new right factor (paper W, build H) from X, V_{n+1}, W_n."""
    X, V1, W = _F(X), _F(V1), _F(W)
    p, q, r = len(X), len(X[0]), len(W)
    c = [[sum(V1[i][k] * W[k][j] for k in range(r)) for j in range(q)]
         for i in range(p)]
    out = []
    for k in range(r):
        row = []
        for j in range(q):
            num = sum(X[i][j] * V1[i][k] for i in range(p))
            den = sum(c[i][j] * V1[i][k] for i in range(p)) + eps
            row.append(W[k][j] * num / den)
        out.append(row)
    return out


def iteration(X, V, W, eps=Fraction(0), order="w_first"):
    """One full iteration.  ``w_first`` is Algorithm 1's order (paper V, i.e.
    the build's left factor W, first); ``h_first`` updates the right factor
    first.  Returns (left, right) as lists of Fractions."""
    if order == "w_first":
        V1 = left_update(X, V, W, eps)
        W1 = right_update(X, V1, W, eps)
    else:
        # right factor first: Eq. (3.4) with the *current* left factor, then
        # Eq. (3.3) with the new right factor.
        W1 = right_update(X, V, W, eps)
        V1 = left_update(X, V, W1, eps)
    return V1, W1


def objective(X, V, W):
    """Eq. (3.1) exactly: sum_ij (x_ij - sum_k v_ik w_kj)^2."""
    X, V, W = _F(X), _F(V), _F(W)
    p, q, r = len(X), len(X[0]), len(W)
    return sum((X[i][j] - sum(V[i][k] * W[k][j] for k in range(r))) ** 2
               for i in range(p) for j in range(q))
