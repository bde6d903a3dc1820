"""Float64 oracle of penalised PET image reconstruction by MM (Section 3.2,
Algorithm 2).  Test infrastructure: only tests/, __graft_entry__.smoke()
and bench.py's CPU-baseline / reference leg import it; nothing on the
library's compute path does.

Problem (Section 3.2).  Pixel intensities lambda (p), counts y (d) along d
lines of flight, geometry constants e_ij >= 0 (E, d x p).  Loglikelihood

    L(lambda) = sum_i [ y_i ln(sum_j e_ij lambda_j) - sum_j e_ij lambda_j ]

and the penalised objective (maximised), N the pairs of adjacent pixels,

    f(lambda) = L(lambda) - mu/2 sum_{{j,k} in N} (lambda_j - lambda_k)^2 .

Algorithm 2: scale E to unit column sums; |N_j| and a_j = -2 mu |N_j|;
lambda_0 = 1; repeat:

    z_ij    = y_i e_ij lambda_nj / sum_k e_ik lambda_nk
    b_nj    = mu (|N_j| lambda_nj + sum_{k in N_j} lambda_nk) - 1
    c_nj    = sum_i z_ij
    lambda_{n+1,j} = the positive root of a_j x^2 + b_nj x + c_nj = 0 .

Readings where the paper is silent or at odds with itself:
  * b_nj: the display after the stationarity condition omits mu; the
    algorithm listing and the stationarity condition itself both carry it.
    The listing's form is used (it is the one the derivation gives).
  * The root.  The paper writes (-b - sqrt(b^2 - 4ac)) / (2a).  With a < 0
    and c >= 0 that numerator cancels when b < 0 (the usual case: b is near
    -1 for small mu), so the same root is evaluated as
    2c / (-b + sqrt(b^2 - 4ac)) there (multiplying through by the conjugate),
    and by the paper's form when b > 0.  With mu = 0 (a = 0) the quadratic is
    the linear equation b x + c = 0 with b = -1, and the conjugate form gives
    x = c: the EM update of Eq. (PET_algorithm) with unit column sums.  With
    c = 0 and b = 0 the root is 0.
  * A line with y_i = 0 adds nothing to c (0 ln 0 = 0 in L), even where
    sum_k e_ik lambda_k = 0 (lines that cross no pixel, or see only zeros).
  * N is given as CSR arrays (ptr, idx) of each pixel's neighbours; the
    penalty's sum over pairs counts each pair once.
Test-only checks and the sampled update for large problems follow the
same steps.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = ["normalise_columns", "neighbour_counts", "neighbour_sums", "pairs",
           "loglik", "penalty", "objective", "positive_root", "quadratic_coefficients",
           "update", "update_pixels", "run", "surrogate", "relative_change"]


def _f64(a):
    return np.asarray(a, dtype=np.float64)


def normalise_columns(E):
    """Algorithm 2, first step: E scaled to unit l1 column norms
    (sum_i e_ij = 1 for every j).  Every column must have a positive sum."""
    E = _f64(E)
    s = E.sum(axis=0)
    if np.any(s <= 0):
        raise ValueError("every pixel must be crossed by some line (column sum > 0)")
    return E / s[None, :]


def neighbour_counts(ptr):
    """|N_j| = number of neighbours of pixel j."""
    ptr = np.asarray(ptr, dtype=np.int64)
    return (ptr[1:] - ptr[:-1]).astype(np.float64)


def neighbour_sums(lam, ptr, idx):
    """sum_{k in N_j} lam_k for every pixel j (a plain loop over the CSR)."""
    lam = _f64(lam)
    ptr = np.asarray(ptr, dtype=np.int64)
    idx = np.asarray(idx, dtype=np.int64)
    out = np.zeros(len(ptr) - 1)
    for j in range(len(ptr) - 1):
        out[j] = lam[idx[ptr[j]:ptr[j + 1]]].sum()
    return out


def pairs(ptr, idx):
    """The unordered neighbour pairs {j, k} (j < k), each once."""
    ptr = np.asarray(ptr, dtype=np.int64)
    idx = np.asarray(idx, dtype=np.int64)
    out = []
    for j in range(len(ptr) - 1):
        for k in idx[ptr[j]:ptr[j + 1]]:
            if j < k:
                out.append((j, int(k)))
    return np.asarray(out, dtype=np.int64).reshape(-1, 2)


def loglik(E, y, lam):
    """L(lambda) = sum_i [y_i ln (E lambda)_i - (E lambda)_i], a term with
    y_i = 0 contributing -(E lambda)_i only (0 ln 0 = 0)."""
    E, y, lam = _f64(E), _f64(y), _f64(lam)
    s = E @ lam
    pos = y > 0
    return float(np.sum(y[pos] * np.log(s[pos])) - np.sum(s))


def penalty(lam, pr):
    """sum over pairs {j, k} of (lambda_j - lambda_k)^2 (pr: pairs())."""
    lam = _f64(lam)
    if len(pr) == 0:
        return 0.0
    dlt = lam[pr[:, 0]] - lam[pr[:, 1]]
    return float(np.sum(dlt * dlt))


def objective(E, y, lam, mu, pr):
    """f(lambda) = L(lambda) - mu/2 * penalty (Eq. (PET-objpen)); E here is
    the matrix the iteration uses (scaled to unit column sums)."""
    return loglik(E, y, lam) - 0.5 * float(mu) * penalty(lam, pr)


def positive_root(a, b, c):
    """The positive root of a x^2 + b x + c = 0 for a <= 0, c >= 0 (the
    quadratic of Algorithm 2's last step), elementwise; see the module
    docstring for the form used on each sign of b and for a = 0."""
    a, b, c = np.broadcast_arrays(_f64(a), _f64(b), _f64(c))
    disc = np.sqrt(b * b - 4.0 * a * c)
    out = np.empty(a.shape)
    neg = b <= 0
    den = -b + disc
    with np.errstate(divide="ignore", invalid="ignore"):
        out[neg] = np.where(den[neg] > 0, 2.0 * c[neg] / den[neg], 0.0)
        out[~neg] = (-b[~neg] - disc[~neg]) / (2.0 * a[~neg])
    return out


def quadratic_coefficients(En, y, lam, mu, ptr, idx):
    """(a_j, b_nj, c_nj) of Algorithm 2 at lambda_n = lam, with z_ij formed
    for every line and pixel as the listing does (En: unit column sums)."""
    En, y, lam = _f64(En), _f64(y), _f64(lam)
    s = En @ lam                                   # sum_k e_ik lambda_nk
    with np.errstate(divide="ignore", invalid="ignore"):
        ratio = np.where(y > 0, y / s, 0.0)        # y_i / sum_k e_ik lambda_nk
    z = ratio[:, None] * En * lam[None, :]         # z_ij
    c = z.sum(axis=0)
    Nj = neighbour_counts(ptr)
    a = -2.0 * float(mu) * Nj
    b = float(mu) * (Nj * lam + neighbour_sums(lam, ptr, idx)) - 1.0
    return a, b, c


def update(En, y, lam, mu, ptr, idx):
    """One MM iteration of Algorithm 2 (En already has unit column sums)."""
    a, b, c = quadratic_coefficients(En, y, lam, mu, ptr, idx)
    return positive_root(a, b, c)


def update_pixels(En, y, lam, mu, ptr, idx, cols):
    """Pixels `cols` of one iteration, for checking problems too large to
    form z for every pixel: c_nj needs column j of E and the projections
    sum_k e_ik lambda_nk of every line."""
    En, y, lam = _f64(En), _f64(y), _f64(lam)
    cols = np.asarray(cols)
    s = En @ lam
    with np.errstate(divide="ignore", invalid="ignore"):
        ratio = np.where(y > 0, y / s, 0.0)
    z = ratio[:, None] * En[:, cols] * lam[None, cols]
    c = z.sum(axis=0)
    Nj = neighbour_counts(ptr)[cols]
    a = -2.0 * float(mu) * Nj
    b = float(mu) * (Nj * lam[cols] + neighbour_sums(lam, ptr, idx)[cols]) - 1.0
    return positive_root(a, b, c)


def relative_change(f_prev, f):
    """Section 3's stopping statistic |f_n - f_{n-1}| / (|f_{n-1}| + 1)."""
    return abs(f - f_prev) / (abs(f_prev) + 1.0)


def run(E, y, mu, ptr, idx, iters, tol=0.0, lam0=None):
    """Algorithm 2 from lambda_0 = 1 (or lam0) on the raw geometry E:
    scale E, iterate `iters` times or until the relative change of f drops
    below tol (tol > 0).  Returns (lambda, objective trajectory, iterations)."""
    En = normalise_columns(E)
    pr = pairs(ptr, idx)
    lam = np.ones(En.shape[1]) if lam0 is None else _f64(lam0).copy()
    fs = [objective(En, y, lam, mu, pr)]
    done = 0
    for _ in range(iters):
        lam = update(En, y, lam, mu, ptr, idx)
        done += 1
        fs.append(objective(En, y, lam, mu, pr))
        if tol > 0 and relative_change(fs[-2], fs[-1]) < tol:
            break
    return lam, fs, done


def surrogate(En, y, lam, lam_n, mu, pr):
    """The minorising function g(lambda | lambda_n) of Section 3.2, written
    out term by term: Jensen's minoriser of L,

        Q = sum_i y_i sum_j w_ij ln(e_ij lambda_j / w_ij) - sum_ij e_ij lambda_j,
        w_ij = e_ij lambda_nj / sum_k e_ik lambda_nk   (terms with w_ij = 0 vanish),

    minus mu/4 sum_pairs [(2 lambda_j - lambda_nj - lambda_nk)^2
                          + (2 lambda_k - lambda_nj - lambda_nk)^2]."""
    En, y, lam, lam_n = _f64(En), _f64(y), _f64(lam), _f64(lam_n)
    d, p = En.shape
    Q = 0.0
    for i in range(d):
        s_n = float(np.dot(En[i], lam_n))
        for j in range(p):
            e = En[i, j]
            if e == 0.0:
                continue
            Q -= e * lam[j]
            if y[i] > 0 and lam_n[j] > 0:
                w = e * lam_n[j] / s_n
                Q += y[i] * w * math.log(e * lam[j] / w)
    pen = 0.0
    for j, k in pr:
        m = lam_n[j] + lam_n[k]
        pen += (2.0 * lam[j] - m) ** 2 + (2.0 * lam[k] - m) ** 2
    return Q - 0.25 * float(mu) * pen
