"""Pins of the Poisson-variant oracle (Section 3.1, the Poisson model for the
counts) to facts that do not come from the update formula itself: the
loglikelihood's definition, the MM properties the paper claims (ascent,
minorisation, tangency), the derivation it leaves to the reader (the update
is the stationary point of the minorising function), exact symmetries and
fixed points.  CPU only."""
import math

import numpy as np
import pytest

from oracle import poisson_oracle as po


def _problem(p, n, r, seed, zeros=0.0):
    rng = np.random.default_rng(seed)
    V = rng.poisson(3.0, size=(p, n)).astype(np.float64)
    if zeros:
        V[rng.random((p, n)) < zeros] = 0.0
    W = rng.uniform(0.1, 1.0, size=(p, r))
    H = rng.uniform(0.1, 1.0, size=(r, n))
    return V, W, H


def test_loglik_definition_small_cases():
    """L = sum v ln b - b; an entry with v = 0 adds -b (0 ln 0 = 0)."""
    assert po.loglik([[2.0]], [[1.0]], [[3.0]]) == pytest.approx(2 * math.log(3.0) - 3.0, rel=1e-15)
    assert po.loglik([[0.0]], [[0.5]], [[4.0]]) == -2.0
    assert po.loglik([[0.0]], [[0.0]], [[4.0]]) == 0.0
    # 2 x 2 by hand: b = [[1, 2], [3, 6]]
    V = [[1.0, 0.0], [2.0, 5.0]]
    W = [[1.0], [3.0]]
    H = [[1.0, 2.0]]
    want = (1 * math.log(1) - 1) + (0 - 2) + (2 * math.log(3) - 3) + (5 * math.log(6) - 6)
    assert po.loglik(V, W, H) == pytest.approx(want, rel=1e-15)


@pytest.mark.parametrize("zeros", [0.0, 0.4])
def test_ascent_every_iteration(zeros):
    """The MM property: L never decreases."""
    V, W, H = _problem(23, 17, 4, seed=1, zeros=zeros)
    L = po.loglik(V, W, H)
    for _ in range(60):
        W, H = po.step(V, W, H)
        L1 = po.loglik(V, W, H)
        assert L1 >= L - 1e-12 * abs(L)
        L = L1


def test_tangency_and_minorisation():
    """g(Wn, Hn | Wn, Hn) = L(Wn, Hn) and g <= L at other points."""
    V, Wn, Hn = _problem(5, 6, 3, seed=2, zeros=0.2)
    assert po.surrogate(V, Wn, Hn, Wn, Hn) == pytest.approx(po.loglik(V, Wn, Hn), rel=1e-13)
    rng = np.random.default_rng(3)
    for _ in range(20):
        W = Wn * rng.uniform(0.3, 3.0, size=Wn.shape)
        H = Hn * rng.uniform(0.3, 3.0, size=Hn.shape)
        assert po.surrogate(V, W, H, Wn, Hn) <= po.loglik(V, W, H) + 1e-12


def test_update_is_the_stationary_point_of_the_minoriser():
    """The derivation the paper leaves to the reader: with eps = 0 the update
    zeroes the gradient of g(. | Wn, Hn) (central differences, every entry)
    and beats every nearby point.  A dropped term, a wrong index or a
    transposed operand in the update moves it off the stationary point."""
    V, Wn, Hn = _problem(4, 5, 2, seed=4, zeros=0.25)
    W1, H1 = po.step(V, Wn, Hn, eps=0.0)
    g0 = po.surrogate(V, W1, H1, Wn, Hn)
    h = 1e-6
    for M in (W1, H1):
        for idx in np.ndindex(M.shape):
            old = M[idx]
            M[idx] = old * (1 + h)
            gp = po.surrogate(V, W1, H1, Wn, Hn)
            M[idx] = old * (1 - h)
            gm = po.surrogate(V, W1, H1, Wn, Hn)
            M[idx] = old
            grad = (gp - gm) / (2 * h * old)
            assert abs(grad) < 1e-6 * max(1.0, abs(g0)), (idx, grad)
    rng = np.random.default_rng(5)
    for _ in range(10):
        W = W1 * (1 + 1e-3 * rng.standard_normal(W1.shape))
        H = H1 * (1 + 1e-3 * rng.standard_normal(H1.shape))
        assert po.surrogate(V, W, H, Wn, Hn) <= g0 + 1e-12


def test_exact_data_is_a_fixed_point():
    """V = W0 H0 maximises L over b, and the update leaves W0, H0 as they are."""
    rng = np.random.default_rng(6)
    W0 = rng.uniform(0.5, 2.0, size=(30, 3))
    H0 = rng.uniform(0.5, 2.0, size=(3, 40))
    V = W0 @ H0
    W1, H1 = po.step(V, W0, H0, eps=0.0)
    np.testing.assert_allclose(W1, W0, rtol=1e-14)
    np.testing.assert_allclose(H1, H0, rtol=1e-14)


def test_power_of_two_rescaling_is_exact():
    """(W D, D^-1 H) with D a diagonal of powers of two: b is unchanged and
    the update maps to (W' D, D^-1 H'), bit for bit (eps = 0)."""
    V, W, H = _problem(13, 11, 4, seed=7, zeros=0.3)
    d = 2.0 ** np.array([-3, 0, 2, 5])
    W1, H1 = po.step(V, W, H, eps=0.0)
    W2, H2 = po.step(V, W * d[None, :], H / d[:, None], eps=0.0)
    assert np.array_equal(W2, W1 * d[None, :])
    assert np.array_equal(H2, H1 / d[:, None])


def test_permutations_commute_with_the_update():
    """Permuting rows of (V, W), columns of (V, H) and the ranks permutes the
    updated factors the same way."""
    V, W, H = _problem(9, 12, 3, seed=8, zeros=0.2)
    rng = np.random.default_rng(9)
    pi, pj, pk = rng.permutation(9), rng.permutation(12), rng.permutation(3)
    W1, H1 = po.step(V, W, H)
    W2, H2 = po.step(V[pi][:, pj], W[pi][:, pk], H[pk][:, pj])
    np.testing.assert_allclose(W2, W1[pi][:, pk], rtol=1e-14)
    np.testing.assert_allclose(H2, H1[pk][:, pj], rtol=1e-14)


def test_kkt_conditions_at_convergence():
    """At a limit the update's ratio is 1 wherever the entry is positive,
    which is dL/dw_ik = 0 (dL/dh_kj = 0); entries driven to zero sit on the
    boundary with dL <= 0.  These are the Karush-Kuhn-Tucker conditions of
    maximising L over nonnegative factors."""
    V, W, H = _problem(15, 10, 2, seed=10)
    W, H, _, _ = po.run(V, W, H, 3000)
    B = W @ H
    gW = (V / B) @ H.T - H.sum(axis=1)[None, :]
    gH = W.T @ (V / B) - W.sum(axis=0)[:, None]
    scale = np.abs(V).sum() / V.size
    for F, g in ((W, gW), (H, gH)):
        interior = F > 1e-3 * F.max()
        assert interior.sum() > F.size // 2
        assert np.max(np.abs(g[interior])) < 1e-6 * scale
        assert np.all(g[~interior] < 1e-6 * scale)


def test_stopping_rule():
    V, W, H = _problem(20, 25, 3, seed=11)
    _, _, Ls, n = po.run(V, W, H, 100000, tol=1e-8)
    assert n < 100000
    assert abs(Ls[-1] - Ls[-2]) / (abs(Ls[-2]) + 1) < 1e-8
    assert all(abs(Ls[i] - Ls[i - 1]) / (abs(Ls[i - 1]) + 1) >= 1e-8 for i in range(1, len(Ls) - 1))
