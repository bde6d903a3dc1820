"""FP64 CPU oracle for the multiplicative-update (MM) NMF iteration.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference arm may import this module.  The CUDA
library never calls it, and it never calls the CUDA library: the two share no
code.  Inputs come from ``paper_1003_3272_gb300.synth`` (seeded draws only).

Source: Zhou, Lange & Suchard, "Graphics Processing Units and High-Dimensional
Optimization", Section 3.1 (NNMF).  The paper's letters are mapped as

    paper X (p x q)  ->  V (p x n)   data
    paper V (p x r)  ->  W (p x r)   left factor
    paper W (r x q)  ->  H (r x n)   right factor

Everything is computed in float64 from the float32 inputs widened exactly.
Matrix products use numpy's float64 matmul (a library primitive standing for
the sums the paper writes out); there is no blocking, fusion or reordering
beyond that.

Readings of the paper taken here (each listed in the design notes):
  * update order: ``"h_first"`` (right factor, then left factor) is the
    default; ``"w_first"`` is Algorithm 1's own order (left factor first).
  * eps is added to the denominator only:  x <- x * num / (den + eps).
  * the denominators are associated as (W^T W) H and W (H H^T), the products
    the paper names after Eq. (3.4) (V_n W_n W_n^t and V^t V W_n in its
    letters), grouped so that the r x r Gram matrix is formed first.
  * the objective is ||V - WH||_F^2 (Eq. (3.1)), evaluated as a direct
    residual (not through the trace identity).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "wtv", "vht", "gram_w", "gram_h", "update_h", "update_w", "step", "run",
    "objective", "relative_change", "converged", "surrogate",
    "update_h_columns", "update_w_rows",
]


def _f64(a):
    return np.asarray(a, dtype=np.float64)


# --- products named in Section 3.1 (after Eq. (3.4)) ---------------------------

def wtv(W, V):
    """W^T V (r x n): numerator of the right-factor update, Eq. (3.4)
    (the paper's V_{n+1}^t X)."""
    return _f64(W).T @ _f64(V)


def vht(V, H):
    """V H^T (p x r): numerator of the left-factor update, Eq. (3.3)
    (the paper's X W_n^t)."""
    return _f64(V) @ _f64(H).T


def gram_w(W):
    """W^T W (r x r), the Gram matrix inside the right-factor denominator."""
    W = _f64(W)
    return W.T @ W


def gram_h(H):
    """H H^T (r x r), the Gram matrix inside the left-factor denominator."""
    H = _f64(H)
    return H @ H.T


# --- the two block updates ------------------------------------------------------

def update_h(V, W, H, eps=1e-10):
    """Right-factor MM update, Eq. (3.4) in build letters:

        H_kj <- H_kj * (W^T V)_kj / ((W^T W H)_kj + eps)

    with W the *current* (already updated, in the paper's order) left factor.
    Returns the new H (float64)."""
    H = _f64(H)
    num = wtv(W, V)
    den = gram_w(W) @ H + eps
    return (H * num) / den


def update_w(V, W, H, eps=1e-10):
    """Left-factor MM update, Eq. (3.3) in build letters:

        W_ik <- W_ik * (V H^T)_ik / ((W H H^T)_ik + eps)

    Returns the new W (float64)."""
    W = _f64(W)
    num = vht(V, H)
    den = W @ gram_h(H) + eps
    return (W * num) / den


def update_h_columns(V, W, H, cols, eps=1e-10):
    """Columns ``cols`` of the right-factor update of Eq. (3.4), for checking
    samples of a problem too large to update whole.  Column j of the new H
    depends only on column j of V and of H (and on all of W):

        H_kj <- H_kj * (W^T V_:j)_k / ((W^T W) H_:j + eps)_k

    Returns the new columns, r x len(cols) (float64)."""
    cols = np.asarray(cols)
    Vc = _f64(np.asarray(V)[:, cols])
    Hc = _f64(np.asarray(H)[:, cols])
    return update_h(Vc, W, Hc, eps)


def update_w_rows(V, W, H, rows, eps=1e-10):
    """Rows ``rows`` of the left-factor update of Eq. (3.3).  Row i of the new
    W depends only on row i of V and of W (and on all of H):

        W_ik <- W_ik * (V_i: H^T)_k / (W_i: (H H^T) + eps)_k

    Returns the new rows, len(rows) x r (float64)."""
    rows = np.asarray(rows)
    Vr = _f64(np.asarray(V)[rows, :])
    Wr = _f64(np.asarray(W)[rows, :])
    return update_w(Vr, Wr, H, eps)


def step(V, W, H, eps=1e-10, order="h_first"):
    """One MM iteration (one pass of Algorithm 1's loop body).

    ``order="h_first"``: H from (W, H), then W from (W, new H).
    ``order="w_first"``: Algorithm 1's order -- W first, then H with new W."""
    if order == "h_first":
        H = update_h(V, W, H, eps)
        W = update_w(V, W, H, eps)
    elif order == "w_first":
        W = update_w(V, W, H, eps)
        H = update_h(V, W, H, eps)
    else:
        raise ValueError(f"unknown order {order!r}")
    return _f64(W), _f64(H)


def objective(V, W, H):
    """f(W, H) = ||V - W H||_F^2, Eq. (3.1), as a direct float64 residual
    summed by numpy's pairwise summation."""
    R = _f64(V) - _f64(W) @ _f64(H)
    return float(np.sum(R * R))


def relative_change(f_prev, f):
    """The stopping statistic of Section 3's introduction:
    |f_n - f_{n-1}| / (|f_{n-1}| + 1)."""
    return abs(f - f_prev) / (abs(f_prev) + 1.0)


def converged(f_prev, f, tol=1e-9):
    """True when the relative change falls below ``tol`` (the paper uses 1e-9)."""
    return relative_change(f_prev, f) < tol


def run(V, W0, H0, iters, eps=1e-10, order="h_first", tol=0.0,
        track_objective=False):
    """Algorithm 1 from given starting factors.

    Runs ``iters`` iterations, stopping early when ``tol > 0`` and the
    relative change of the objective drops below ``tol`` (Section 3's rule;
    the objective is then evaluated after every iteration).  Returns
    ``(W, H, fs, n_done)`` where ``fs`` is the list of objective values after
    each iteration when tracked (empty otherwise)."""
    W, H = _f64(W0), _f64(H0)
    fs = []
    f_prev = objective(V, W, H) if (tol > 0 or track_objective) else None
    n_done = 0
    for _ in range(iters):
        W, H = step(V, W, H, eps, order)
        n_done += 1
        if tol > 0 or track_objective:
            f = objective(V, W, H)
            fs.append(f)
            if tol > 0 and converged(f_prev, f, tol):
                break
            f_prev = f
    return W, H, fs, n_done


def surrogate(V, W, H, Wn, Hn):
    """The majorising surrogate g(W, H | W_n, H_n) of Eq. (3.2), written out
    elementwise (slow: small inputs only).

        g = sum_ijk (a_ikj / b_ij) (v_ij - (b_ij / a_ikj) w_ik h_kj)^2
        a_ikj = Wn_ik Hn_kj,   b_ij = sum_k a_ikj

    Terms with a_ikj = 0 are omitted (they carry zero weight)."""
    V, W, H, Wn, Hn = map(_f64, (V, W, H, Wn, Hn))
    p, n = V.shape
    r = W.shape[1]
    g = 0.0
    for i in range(p):
        for j in range(n):
            a = [Wn[i, k] * Hn[k, j] for k in range(r)]
            b = sum(a)
            for k in range(r):
                if a[k] == 0.0:
                    continue
                t = V[i, j] - (b / a[k]) * W[i, k] * H[k, j]
                g += (a[k] / b) * t * t
    return g
