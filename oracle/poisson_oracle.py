"""FP64 CPU oracle for the Poisson variant of the MM NMF iteration.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference arm may import this module.  The CUDA
library never calls it, and it never calls the CUDA library.

Source: Zhou, Lange & Suchard, Section 3.1, the closing paragraph on the
Poisson model for the counts: instead of Eq. (3.1) maximise the
loglikelihood

    L(W, H) = sum_ij [ v_ij ln(sum_k w_ik h_kj) - sum_k w_ik h_kj ]

by the "pure MM" update the paper prints after it (letters mapped as in
``nmf_oracle``: paper X, V, W -> V, W, H here).  With b_ij = (W H)_ij from
the *current* factors, both factors move at once:

    w_ik <- w_ik * sqrt( (sum_j v_ij h_kj / b_ij) / (sum_j h_kj) )
    h_kj <- h_kj * sqrt( (sum_i v_ij w_ik / b_ij) / (sum_i w_ik) )

Readings taken here (each listed in the design notes):
  * the printed left-hand side "w_{n+1,ij}" of the second update is
    w_{n+1,kj} (its right-hand side and the first update fix the indices),
    and b_nij = sum_k v_nik w_nkj in the paper's letters;
  * both updates use the factors of iteration n (a simultaneous update,
    as the derivation through one minorising function gives; see
    ``surrogate``), not the alternating order of Algorithm 1;
  * eps (1e-10) guards the two divisions as in the Gaussian form:
    v_ij / (b_ij + eps) and num / (den + eps); it only matters when b_ij
    or a factor's row or column sum is zero;
  * 0 ln 0 = 0: an entry with v_ij = 0 adds -b_ij to L whatever b_ij is.

Matrix products use numpy's float64 matmul; there is no blocking, fusion or
reordering beyond that.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = ["product", "loglik", "step", "run", "surrogate"]


def _f64(a):
    return np.asarray(a, dtype=np.float64)


def product(W, H):
    """b = W H (p x n), the Poisson means of the model."""
    return _f64(W) @ _f64(H)


def loglik(V, W, H):
    """L(W, H) = sum_ij [v_ij ln b_ij - b_ij] (the Poisson loglikelihood up
    to the constant -sum ln v_ij!), with 0 ln 0 = 0, summed in float64."""
    V = _f64(V)
    B = product(W, H)
    pos = V > 0
    t = -B
    t[pos] += V[pos] * np.log(B[pos])
    return float(np.sum(t))


def step(V, W, H, eps=1e-10):
    """One Poisson MM iteration: both factors from (W, H) of this iteration.
    Returns (W', H') in float64."""
    V, W, H = _f64(V), _f64(W), _f64(H)
    B = W @ H
    Q = np.divide(V, B + eps, out=np.zeros_like(V), where=V > 0)   # v_ij / b_ij, 0 if v_ij = 0
    num_w = Q @ H.T                       # sum_j v_ij h_kj / b_ij   (p x r)
    num_h = W.T @ Q                       # sum_i v_ij w_ik / b_ij   (r x n)
    den_w = H.sum(axis=1)                 # sum_j h_kj               (r)
    den_h = W.sum(axis=0)                 # sum_i w_ik               (r)
    W1 = W * np.sqrt(num_w / (den_w[None, :] + eps))
    H1 = H * np.sqrt(num_h / (den_h[:, None] + eps))
    return W1, H1


def run(V, W0, H0, iters, eps=1e-10, tol=0.0, track=False):
    """Iterate ``step``; with ``tol > 0`` stop once
    |L_n - L_{n-1}| / (|L_{n-1}| + 1) < tol (Section 3's rule applied to L).
    Returns (W, H, Ls, n_done), Ls the loglikelihood after each iteration
    when tracked or tested."""
    W, H = _f64(W0), _f64(H0)
    Ls = []
    want = tol > 0 or track
    L_prev = loglik(V, W, H) if want else None
    n = 0
    for _ in range(iters):
        W, H = step(V, W, H, eps)
        n += 1
        if want:
            L = loglik(V, W, H)
            Ls.append(L)
            if tol > 0 and abs(L - L_prev) / (abs(L_prev) + 1.0) < tol:
                break
            L_prev = L
    return W, H, Ls, n


def surrogate(V, W, H, Wn, Hn):
    """The minorising function behind the update, written out elementwise
    (pure Python loops: small inputs only).  With a_ikj = wn_ik hn_kj and
    b_ij = sum_k a_ikj, concavity of ln (Jensen over the weights a/b) and
    2xy <= x^2 c/d + y^2 d/c give

      g(W, H | Wn, Hn) = sum_ij v_ij sum_k (a_ikj/b_ij) ln(b_ij w_ik h_kj / a_ikj)
                       - 1/2 sum_ijk [ w_ik^2 hn_kj / wn_ik + h_kj^2 wn_ik / hn_kj ]

    with g <= L everywhere and g = L at (Wn, Hn); its maximiser over (W, H)
    separates per entry and is the update in ``step`` (eps = 0)."""
    V, W, H, Wn, Hn = map(_f64, (V, W, H, Wn, Hn))
    p, n = V.shape
    r = W.shape[1]
    g = 0.0
    for i in range(p):
        for j in range(n):
            a = [Wn[i, k] * Hn[k, j] for k in range(r)]
            b = sum(a)
            for k in range(r):
                if V[i, j] != 0.0 and a[k] != 0.0:
                    g += V[i, j] * (a[k] / b) * math.log(b * W[i, k] * H[k, j] / a[k])
                g -= 0.5 * (W[i, k] ** 2 * Hn[k, j] / Wn[i, k] + H[k, j] ** 2 * Wn[i, k] / Hn[k, j])
    return g
