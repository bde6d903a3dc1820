"""Pins of the PET oracle (oracle/pet_oracle.py; Section 3.2, Algorithm 2)
against what the mathematics fixes, not against its own formulas: L on hand
cases, the EM update of Eq. (PET_algorithm) written out with w_nij for
mu = 0, the positive root as a root, the update as the maximiser of the
minorising function g (stationarity by central differences, and no nearby
point beating it), minorisation and tangency of g, ascent of f at every
iteration, the noise-free fixed point, exact power-of-two equivariance,
permutation equivariance, the KKT conditions at a converged point, and
planted mistakes each failing a pin.  CPU only."""
import math

import numpy as np
import pytest

from oracle import pet_oracle as po
from paper_1003_3272_gb300 import synth


def tiny(grid=4, ndet=8, seed=3, mean=6.0):
    return synth.pet_problem(grid, ndet, seed, mean_count=mean, iters=10)


def rand_lam(p, seed):
    return np.random.default_rng(seed).uniform(0.2, 3.0, p)


# --- the objective -------------------------------------------------------------

def test_loglik_hand_case():
    E = np.array([[1.0, 0.5], [0.0, 2.0], [0.0, 0.0]])
    y = np.array([3.0, 0.0, 0.0])
    lam = np.array([2.0, 1.0])
    # s = (2.5, 2, 0); the zero-count lines add -s_i, the empty line adds 0
    assert po.loglik(E, y, lam) == pytest.approx(3 * math.log(2.5) - 2.5 - 2.0, rel=1e-15)


def test_penalty_counts_each_pair_once():
    ptr, idx = synth.grid_neighbours(2)            # 2 x 2: pairs 01, 02, 13, 23
    pr = po.pairs(ptr, idx)
    assert sorted(map(tuple, pr)) == [(0, 1), (0, 2), (1, 3), (2, 3)]
    lam = np.array([1.0, 2.0, 4.0, 8.0])
    assert po.penalty(lam, pr) == 1 + 9 + 36 + 16
    E = np.eye(4)
    y = np.ones(4)
    f = po.objective(E, y, lam, 0.5, pr)
    assert f == pytest.approx(po.loglik(E, y, lam) - 0.25 * 62.0, rel=1e-15)


def test_normalise_columns():
    pr = tiny()
    En = po.normalise_columns(pr.E)
    np.testing.assert_allclose(En.sum(axis=0), 1.0, rtol=1e-14)
    E = pr.E.astype(np.float64).copy()
    E[:, 3] = 0.0
    with pytest.raises(ValueError):
        po.normalise_columns(E)


def test_neighbour_counts_on_the_grid():
    ptr, idx = synth.grid_neighbours(5)
    Nj = po.neighbour_counts(ptr).reshape(5, 5)
    assert Nj[0, 0] == 2 and Nj[0, 2] == 3 and Nj[2, 2] == 4
    # symmetric system
    pairs = {(j, int(k)) for j in range(25) for k in idx[ptr[j]:ptr[j + 1]]}
    assert all((k, j) in pairs for j, k in pairs)


# --- the root ------------------------------------------------------------------

def test_positive_root_is_the_positive_root():
    rng = np.random.default_rng(0)
    a = -rng.uniform(1e-6, 10.0, 2000)
    b = rng.uniform(-5.0, 5.0, 2000)
    c = rng.uniform(0.0, 50.0, 2000)
    x = po.positive_root(a, b, c)
    assert np.all(x >= 0)
    scale = np.abs(a) * x * x + np.abs(b) * x + c
    assert np.max(np.abs(a * x * x + b * x + c) / scale) < 1e-14
    # the other root, c / (a x), is not positive (product of the roots c/a <= 0)
    other = np.where(x > 0, c / (a * np.where(x > 0, x, 1.0)), 0.0)
    assert np.all(other <= 0)
    # library routine on a few cases, and the paper's printed form where it
    # does not cancel (b > 0)
    for i in range(20):
        r = np.roots([a[i], b[i], c[i]]).real
        assert x[i] == pytest.approx(r.max(), rel=1e-10)
    pos = b > 0
    paper = (-b[pos] - np.sqrt(b[pos] ** 2 - 4 * a[pos] * c[pos])) / (2 * a[pos])
    np.testing.assert_allclose(x[pos], paper, rtol=1e-13)


def test_root_special_cases():
    # mu = 0: the linear equation -x + c = 0
    assert po.positive_root(0.0, -1.0, 2.5) == 2.5
    # c = 0: the maximiser of b x + a x^2 on x >= 0 is max(0, -b / a)
    assert po.positive_root(-2.0, 3.0, 0.0) == pytest.approx(1.5, rel=1e-15)
    assert po.positive_root(-2.0, -3.0, 0.0) == 0.0
    assert po.positive_root(-2.0, 0.0, 0.0) == 0.0
    # continuity as a -> 0 from below
    assert po.positive_root(-1e-12, -1.0, 2.0) == pytest.approx(2.0, rel=1e-10)


# --- the update ----------------------------------------------------------------

def test_mu0_is_the_em_update_written_out():
    """mu = 0: lambda_{n+1,j} = sum_i y_i w_nij / sum_i e_ij with
    w_nij = e_ij lambda_nj / sum_k e_ik lambda_nk (Eq. (PET_algorithm)),
    by loops on the raw geometry in raw units; the oracle works on the
    scaled E, whose intensities are sigma_j lambda_j."""
    pr = tiny()
    E = pr.E.astype(np.float64)
    d, p = E.shape
    lam_raw = rand_lam(p, 1)
    em = np.zeros(p)
    for j in range(p):
        num = 0.0
        for i in range(d):
            s = sum(E[i, k] * lam_raw[k] for k in range(p))
            if E[i, j] > 0 and pr.y[i] > 0:
                num += pr.y[i] * E[i, j] * lam_raw[j] / s
        em[j] = num / sum(E[i, j] for i in range(d))
    sigma = E.sum(axis=0)
    En = po.normalise_columns(E)
    new = po.update(En, pr.y, sigma * lam_raw, 0.0, pr.nbr_ptr, pr.nbr_idx)
    np.testing.assert_allclose(new, sigma * em, rtol=1e-12)


@pytest.mark.parametrize("mu", [0.0, 0.05, 3.0])
def test_update_maximises_the_surrogate(mu):
    """The new point is a stationary point of g(. | lambda_n) (central
    differences of g written out term by term), and no nearby point has a
    larger g."""
    pr = tiny()
    En = po.normalise_columns(pr.E)
    prs = po.pairs(pr.nbr_ptr, pr.nbr_idx)
    lam_n = rand_lam(pr.p, 2)
    new = po.update(En, pr.y, lam_n, mu, pr.nbr_ptr, pr.nbr_idx)
    assert np.all(new > 0)
    g = lambda lam: po.surrogate(En, pr.y, lam, lam_n, mu, prs)
    g0 = g(new)
    h = 1e-6
    grad = np.zeros(pr.p)
    for j in range(pr.p):
        e = np.zeros(pr.p)
        e[j] = h * new[j]
        grad[j] = (g(new + e) - g(new - e)) / (2 * e[j])
    # the gradient's scale at the anchor: sum_i e_ij = 1, so O(1) per pixel
    assert np.max(np.abs(grad)) < 1e-6
    rng = np.random.default_rng(4)
    for _ in range(20):
        trial = new * (1 + 0.05 * rng.standard_normal(pr.p))
        assert g(np.abs(trial)) <= g0 + 1e-12 * abs(g0)


@pytest.mark.parametrize("mu", [0.0, 0.05, 3.0])
def test_surrogate_minorises_and_touches(mu):
    pr = tiny()
    En = po.normalise_columns(pr.E)
    prs = po.pairs(pr.nbr_ptr, pr.nbr_idx)
    lam_n = rand_lam(pr.p, 5)
    fn = po.objective(En, pr.y, lam_n, mu, prs)
    assert po.surrogate(En, pr.y, lam_n, lam_n, mu, prs) == pytest.approx(fn, rel=1e-13)
    rng = np.random.default_rng(6)
    for _ in range(30):
        lam = rng.uniform(0.05, 5.0, pr.p)
        assert po.surrogate(En, pr.y, lam, lam_n, mu, prs) <= \
            po.objective(En, pr.y, lam, mu, prs) + 1e-12 * abs(fn)


@pytest.mark.parametrize("mu", [0.0, 1e-4, 1e-2, 1.0])
def test_ascent_every_iteration(mu):
    pr = synth.pet_problem(16, 24, 7, mean_count=15.0)
    lam, fs, done = po.run(pr.E, pr.y, mu, pr.nbr_ptr, pr.nbr_idx, 60)
    assert done == 60
    assert np.all(np.diff(fs) >= -1e-12 * np.abs(fs[1:]))
    assert np.all(lam >= 0) and np.all(np.isfinite(lam))


def test_noise_free_counts_are_a_fixed_point():
    """y = E lambda* exactly (real-valued, no noise) and mu = 0: lambda* is
    a fixed point of the EM map (every y_i / (E lambda*)_i = 1)."""
    pr = synth.pet_problem(8, 16, 1)
    En = po.normalise_columns(pr.E)
    lam = rand_lam(pr.p, 8)
    y = En @ lam
    new = po.update(En, y, lam, 0.0, pr.nbr_ptr, pr.nbr_idx)
    np.testing.assert_allclose(new, lam, rtol=1e-13)


def test_power_of_two_equivariance_is_exact():
    """lambda -> 4 lambda, y -> 4 y, mu -> mu / 4 scales the update by 4
    exactly: f(4 lambda; 4 y, mu / 4) = 4 f(lambda; y, mu) + const, and every
    step of the update scales by a power of two."""
    pr = synth.pet_problem(8, 16, 2)
    En = po.normalise_columns(pr.E)
    lam = rand_lam(pr.p, 9)
    for mu in (0.0, 1e-3, 0.7):
        a = po.update(En, pr.y, lam, mu, pr.nbr_ptr, pr.nbr_idx)
        b = po.update(En, 4.0 * pr.y, 4.0 * lam, mu / 4.0, pr.nbr_ptr, pr.nbr_idx)
        assert np.array_equal(b, 4.0 * a)


def test_permutation_equivariance():
    pr = synth.pet_problem(8, 16, 4)
    En = po.normalise_columns(pr.E)
    lam = rand_lam(pr.p, 10)
    rng = np.random.default_rng(11)
    pp = rng.permutation(pr.p)               # new pixel q is old pixel pp[q]
    dp = rng.permutation(pr.d)
    inv = np.argsort(pp)
    ptr, idx = pr.nbr_ptr, pr.nbr_idx
    nptr, nidx = [0], []
    for q in range(pr.p):
        j = pp[q]
        nidx.extend(inv[idx[ptr[j]:ptr[j + 1]]].tolist())
        nptr.append(len(nidx))
    for mu in (0.0, 0.01):
        a = po.update(En, pr.y, lam, mu, ptr, idx)
        b = po.update(En[dp][:, pp], pr.y[dp], lam[pp], mu, np.array(nptr), np.array(nidx))
        np.testing.assert_allclose(b, a[pp], rtol=1e-12)


def test_kkt_at_a_converged_point():
    """After convergence, the gradient of f (central differences of the
    objective itself) vanishes on pixels with positive intensity and is not
    positive where the iteration drove the intensity to zero."""
    pr = synth.pet_problem(8, 16, 5, mean_count=30.0)
    mu = 1e-2
    lam, fs, done = po.run(pr.E, pr.y, mu, pr.nbr_ptr, pr.nbr_idx, 20000, tol=1e-15)
    En = po.normalise_columns(pr.E)
    prs = po.pairs(pr.nbr_ptr, pr.nbr_idx)
    f = lambda x: po.objective(En, pr.y, x, mu, prs)
    grad = np.zeros(pr.p)
    for j in range(pr.p):
        h = 1e-6 * max(lam[j], 1e-3)
        e = np.zeros(pr.p)
        e[j] = h
        lo = np.maximum(lam - e, 0.0)
        grad[j] = (f(lam + e) - f(lo)) / (h + (lam[j] - lo[j]))
    pos = lam > 1e-3 * lam.max()
    assert pos.sum() > pr.p // 2
    assert np.max(np.abs(grad[pos])) < 1e-5
    assert np.all(grad[~pos] <= 1e-5)


def test_sampled_update_matches_the_full_update():
    pr = synth.pet_problem(16, 24, 6)
    En = po.normalise_columns(pr.E)
    lam = rand_lam(pr.p, 12)
    cols = np.array([0, 5, 17, 100, 255, 3, 3])
    full = po.update(En, pr.y, lam, 1e-3, pr.nbr_ptr, pr.nbr_idx)
    np.testing.assert_allclose(po.update_pixels(En, pr.y, lam, 1e-3, pr.nbr_ptr, pr.nbr_idx,
                                                cols), full[cols], rtol=1e-14)


def test_stopping_rule():
    assert po.relative_change(-100.0, -100.0) == 0.0
    assert po.relative_change(-99.0, -100.0) == pytest.approx(1.0 / 100.0)
    pr = synth.pet_problem(8, 16, 5)
    _, fs, done = po.run(pr.E, pr.y, 1e-2, pr.nbr_ptr, pr.nbr_idx, 100000, tol=1e-9)
    assert done < 100000
    assert po.relative_change(fs[-2], fs[-1]) < 1e-9
    assert all(po.relative_change(fs[i], fs[i + 1]) >= 1e-9 for i in range(len(fs) - 2))


# --- planted mistakes ----------------------------------------------------------

def _mistaken_update(kind):
    def upd(En, y, lam, mu, ptr, idx):
        s = En @ lam
        with np.errstate(divide="ignore", invalid="ignore"):
            ratio = np.where(y > 0, s / y if kind == "inverted_ratio" else y / s, 0.0)
        z = ratio[:, None] * En * (1.0 if kind == "no_lambda_in_c" else lam[None, :])
        c = z.sum(axis=0)
        Nj = po.neighbour_counts(ptr)
        a = (-1.0 if kind == "a_without_2" else -2.0) * mu * Nj
        nb = po.neighbour_sums(lam, ptr, idx)
        if kind == "b_without_mu":
            b = (Nj * lam + nb) - 1.0
        elif kind == "b_without_minus_one":
            b = mu * (Nj * lam + nb)
        else:
            b = mu * (Nj * lam + nb) - 1.0
        if kind == "other_root":
            return (-b + np.sqrt(b * b - 4 * a * c)) / (2 * a)
        return po.positive_root(a, b, c)
    return upd


@pytest.mark.parametrize("kind", ["inverted_ratio", "no_lambda_in_c", "a_without_2",
                                  "b_without_mu", "b_without_minus_one", "other_root"])
def test_planted_mistakes_fail_a_pin(kind):
    """Each mistake, planted in a copy of the update, fails the stationarity
    pin or the fixed-point pin (and so would the oracle if it carried it)."""
    upd = _mistaken_update(kind)
    pr = tiny()
    En = po.normalise_columns(pr.E)
    prs = po.pairs(pr.nbr_ptr, pr.nbr_idx)
    lam_n = rand_lam(pr.p, 2)
    failed = False
    # fixed point at mu = 0
    y = En @ lam_n
    with np.errstate(all="ignore"):
        fp = upd(En, y, lam_n, 0.0, pr.nbr_ptr, pr.nbr_idx)
    if not np.allclose(fp, lam_n, rtol=1e-10):
        failed = True
    # stationarity of the surrogate at mu = 0.05
    mu = 0.05
    with np.errstate(all="ignore"):
        new = upd(En, pr.y, lam_n, mu, pr.nbr_ptr, pr.nbr_idx)
    if not np.all(np.isfinite(new)) or np.any(new <= 0):
        failed = True
    else:
        g = lambda lam: po.surrogate(En, pr.y, lam, lam_n, mu, prs)
        for j in range(pr.p):
            e = np.zeros(pr.p)
            e[j] = 1e-6 * new[j]
            if abs((g(new + e) - g(new - e)) / (2 * e[j])) > 1e-6:
                failed = True
                break
    assert failed, kind
    # the correct update passes both
    good = po.update(En, y, lam_n, 0.0, pr.nbr_ptr, pr.nbr_idx)
    assert np.allclose(good, lam_n, rtol=1e-10)


# --- the generator (inputs, not the method) ------------------------------------

def test_geometry_rows_are_chord_lengths_inside_the_grid():
    """Each row of E sums to the length of its line inside [0, G]^2, which
    is found here by clipping the line to the square analytically."""
    G, nd = 8, 12
    E = synth.pet_system_matrix(G, nd).astype(np.float64)
    c = G / 2.0
    R = 0.5 * math.sqrt(2.0) * G + 1.0
    ang = 2.0 * math.pi * (np.arange(nd) + 0.5) / nd
    det = np.stack([c + R * np.cos(ang), c + R * np.sin(ang)], axis=1)
    ia, ib = np.triu_indices(nd, 1)
    for i, (a, b) in enumerate(zip(ia, ib)):
        P, D = det[a], det[b] - det[a]
        t0, t1 = 0.0, 1.0
        for k in range(2):
            if D[k] != 0:
                u, v = (0 - P[k]) / D[k], (G - P[k]) / D[k]
                t0, t1 = max(t0, min(u, v)), min(t1, max(u, v))
            elif not 0 <= P[k] <= G:          # parallel to this axis, outside
                t1 = t0
        chord = max(0.0, t1 - t0) * math.hypot(*D)
        assert E[i].sum() == pytest.approx(chord, rel=1e-5, abs=1e-5)
    assert np.all(E.sum(axis=0) > 0)


def test_workload_columns_are_all_crossed():
    pr = synth.pet()
    assert pr.d == 2016 and pr.p == 4096
    assert np.all(pr.E.astype(np.float64).sum(axis=0) > 0)
    assert np.all(pr.y >= 0) and np.all(pr.y == np.round(pr.y))
