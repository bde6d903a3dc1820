"""Pins of the FP64 oracle to facts the paper and the mathematics fix.

Each test is chosen so that a plausible slip in the oracle (a dropped term, a
wrong sign, a transposed operand, a wrong index, the wrong update order)
fails at least one of them.  No GPU, no CUDA library.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import exact
from oracle import nmf_oracle as orc
from paper_1003_3272_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_problem(p, n, r, seed, zero_frac=0.0):
    rng = np.random.default_rng(seed)
    V = rng.random((p, n))
    if zero_frac:
        V[rng.random((p, n)) < zero_frac] = 0.0
    W = rng.random((p, r)) + 0.05
    H = rng.random((r, n)) + 0.05
    return V, W, H


# --- brute-force products on tiny integer inputs -----------------------------------

def _brute_matmul(A, B):
    n, m, k = len(A), len(B[0]), len(B)
    return [[sum(A[i][t] * B[t][j] for t in range(k)) for j in range(m)] for i in range(n)]


def _T(A):
    return [list(c) for c in zip(*A)]


def test_products_match_triple_sums_4x5():
    V = [[3, 1, 4, 1, 5], [9, 2, 6, 5, 3], [5, 8, 9, 7, 9], [3, 2, 3, 8, 4]]
    W = [[1, 2], [3, 1], [2, 2], [1, 3]]
    H = [[2, 1, 1, 3, 1], [1, 2, 3, 1, 2]]
    assert np.array_equal(orc.wtv(W, V), np.array(_brute_matmul(_T(W), V), float))
    assert np.array_equal(orc.vht(V, H), np.array(_brute_matmul(V, _T(H)), float))
    assert np.array_equal(orc.gram_w(W), np.array(_brute_matmul(_T(W), W), float))
    assert np.array_equal(orc.gram_h(H), np.array(_brute_matmul(H, _T(H)), float))
    # shapes: numerators are r x n and p x r, Grams r x r
    assert orc.wtv(W, V).shape == (2, 5)
    assert orc.vht(V, H).shape == (4, 2)


def _read_golden(path):
    blocks, cur = {}, None
    with open(path) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("["):
                cur = line[1:-1]
                blocks[cur] = []
            else:
                blocks[cur].append([Fraction(x) for x in line.split()])
    return blocks


@pytest.mark.parametrize("order", ["h_first", "w_first"])
def test_one_iteration_matches_exact_rational_golden(order):
    """Float64 oracle (Gram-grouped matrix form) vs the paper's elementwise
    updates in exact rationals, stored in tests/golden/exact_4x5.txt."""
    g = _read_golden(os.path.join(GOLDEN, "exact_4x5.txt"))
    V = np.array(g["V"], float)
    W0 = np.array(g["W0"], float)
    H0 = np.array(g["H0"], float)
    W1, H1 = orc.step(V, W0, H0, eps=0.0, order=order)
    W1x = np.array([[float(x) for x in row] for row in g[f"W1 {order}"]])
    H1x = np.array([[float(x) for x in row] for row in g[f"H1 {order}"]])
    np.testing.assert_allclose(W1, W1x, rtol=1e-14, atol=0)
    np.testing.assert_allclose(H1, H1x, rtol=1e-14, atol=0)
    f0 = float(g["f0"][0][0])
    f1 = float(g[f"f1 {order}"][0][0])
    assert orc.objective(V, W0, H0) == pytest.approx(f0, rel=1e-15)
    assert orc.objective(V, W1, H1) == pytest.approx(f1, rel=1e-12)
    assert f1 <= f0  # the MM descent property


def test_orders_differ():
    """The two update orders are different block-relaxation maps."""
    g = _read_golden(os.path.join(GOLDEN, "exact_4x5.txt"))
    assert g["W1 h_first"] != g["W1 w_first"]


def test_exact_form_reproduces_on_random_rationals():
    rng = np.random.default_rng(7)
    V = rng.integers(0, 7, (3, 4)).tolist()
    W = rng.integers(1, 4, (3, 2)).tolist()
    H = rng.integers(1, 4, (2, 4)).tolist()
    for order in ("h_first", "w_first"):
        Wx, Hx = exact.iteration(V, W, H, order=order)
        Wf, Hf = orc.step(np.array(V, float), np.array(W, float), np.array(H, float),
                          eps=0.0, order=order)
        np.testing.assert_allclose(Wf, np.array(Wx, dtype=float), rtol=1e-14)
        np.testing.assert_allclose(Hf, np.array(Hx, dtype=float), rtol=1e-14)


def test_sampled_updates_match_exact_elementwise_forms():
    """The column / row sampled updates (used to check problems too large to
    update whole) equal the paper's elementwise updates in exact rationals on
    the sampled columns / rows, including unsorted and repeated indices."""
    rng = np.random.default_rng(11)
    V = rng.integers(0, 7, (5, 6)).tolist()
    W = rng.integers(1, 4, (5, 3)).tolist()
    H = rng.integers(1, 4, (3, 6)).tolist()
    Va, Wa, Ha = (np.array(a, float) for a in (V, W, H))
    cols = [4, 0, 4, 2]
    rows = [3, 1, 1]
    Hx = np.array(exact.right_update(V, W, H), dtype=float)
    np.testing.assert_allclose(orc.update_h_columns(Va, Wa, Ha, cols, eps=0.0),
                               Hx[:, cols], rtol=1e-14)
    Wx = np.array(exact.left_update(V, W, H), dtype=float)
    np.testing.assert_allclose(orc.update_w_rows(Va, Wa, Ha, rows, eps=0.0),
                               Wx[rows], rtol=1e-14)


def test_objective_matches_exact_sum():
    rng = np.random.default_rng(3)
    V = rng.integers(0, 9, (4, 6))
    W = rng.integers(0, 4, (4, 3))
    H = rng.integers(0, 4, (3, 6))
    fx = exact.objective(V.tolist(), W.tolist(), H.tolist())
    assert orc.objective(V, W, H) == float(fx)


# --- MM invariants -----------------------------------------------------------------

@pytest.mark.parametrize("order", ["h_first", "w_first"])
@pytest.mark.parametrize("zero_frac", [0.0, 0.3])
def test_descent_every_iteration_and_half_step(order, zero_frac):
    """The MM descent property (Section 2 and Eq. (3.2)): f never increases,
    also after each block (half) update."""
    V, W, H = _rand_problem(23, 31, 4, 11, zero_frac)
    f = orc.objective(V, W, H)
    for _ in range(60):
        if order == "h_first":
            H = orc.update_h(V, W, H, 0.0)
            f1 = orc.objective(V, W, H)
            W = orc.update_w(V, W, H, 0.0)
        else:
            W = orc.update_w(V, W, H, 0.0)
            f1 = orc.objective(V, W, H)
            H = orc.update_h(V, W, H, 0.0)
        f2 = orc.objective(V, W, H)
        assert f1 <= f * (1 + 1e-13)
        assert f2 <= f1 * (1 + 1e-13)
        f = f2


def test_nonnegativity_and_absorbing_zeros():
    V, W, H = _rand_problem(17, 19, 3, 5, zero_frac=0.5)
    H[1, 3] = 0.0
    W[4, 2] = 0.0
    for _ in range(20):
        W, H = orc.step(V, W, H, eps=1e-10)
        assert W.min() >= 0 and H.min() >= 0
        assert H[1, 3] == 0.0 and W[4, 2] == 0.0


def test_zero_row_with_eps_stays_finite():
    """A zero row of V drives its W row to 0; eps keeps 0/0 out."""
    V, W, H = _rand_problem(9, 8, 2, 6)
    V[2, :] = 0.0
    for _ in range(3):
        W, H = orc.step(V, W, H, eps=1e-10)
    assert np.all(np.isfinite(W)) and np.all(np.isfinite(H))
    assert np.all(W[2] == 0.0)


def test_planted_factors_are_a_fixed_point():
    """V = W0 H0 exactly: the MM map leaves (W0, H0) unchanged (fixed point,
    Section 2 condition (d)); eps = 0."""
    pr = synth.exact_planted(24, 20, 3, seed=1)
    W, H = orc.step(pr.V, pr.W0, pr.H0, eps=0.0)
    np.testing.assert_allclose(W, pr.W0, rtol=1e-14)
    np.testing.assert_allclose(H, pr.H0, rtol=1e-14)
    assert orc.objective(pr.V, W, H) < 1e-20


def test_rank_one_closed_form():
    a = np.array([1.0, 2.0, 0.5, 4.0])
    b = np.array([3.0, 0.25, 1.0, 2.0, 8.0])
    V = np.outer(a, b)
    W, H = a[:, None].copy(), b[None, :].copy()
    assert orc.objective(V, W, H) == 0.0
    W1, H1 = orc.step(V, W, H, eps=0.0)
    np.testing.assert_allclose(W1, W, rtol=1e-15)
    np.testing.assert_allclose(H1, H, rtol=1e-15)


def test_numerators_and_denominators_are_the_gradient():
    """den - num are half the gradient of f (Eq. (3.1)):
    d f / d H = 2 (W^T W H - W^T V),  d f / d W = 2 (W H H^T - V H^T).
    Central differences of the objective pin every product's operands and
    transposes."""
    V, W, H = _rand_problem(7, 9, 3, 21)
    gH = 2 * (orc.gram_w(W) @ H - orc.wtv(W, V))
    gW = 2 * (W @ orc.gram_h(H) - orc.vht(V, H))
    h = 1e-6
    for (k, j) in [(0, 0), (2, 5), (1, 8)]:
        Hp, Hm = H.copy(), H.copy()
        Hp[k, j] += h
        Hm[k, j] -= h
        fd = (orc.objective(V, W, Hp) - orc.objective(V, W, Hm)) / (2 * h)
        assert fd == pytest.approx(gH[k, j], rel=1e-6, abs=1e-8)
    for (i, k) in [(0, 0), (6, 2), (3, 1)]:
        Wp, Wm = W.copy(), W.copy()
        Wp[i, k] += h
        Wm[i, k] -= h
        fd = (orc.objective(V, Wp, H) - orc.objective(V, Wm, H)) / (2 * h)
        assert fd == pytest.approx(gW[i, k], rel=1e-6, abs=1e-8)


def test_surrogate_majorises_and_touches():
    """Eq. (3.2): g(theta | theta_n) >= f(theta), with equality at theta_n."""
    V, Wn, Hn = _rand_problem(4, 5, 2, 31)
    fn = orc.objective(V, Wn, Hn)
    assert orc.surrogate(V, Wn, Hn, Wn, Hn) == pytest.approx(fn, rel=1e-13)
    rng = np.random.default_rng(1)
    for _ in range(5):
        W = Wn * rng.uniform(0.5, 1.5, Wn.shape)
        H = Hn * rng.uniform(0.5, 1.5, Hn.shape)
        assert orc.surrogate(V, W, H, Wn, Hn) >= orc.objective(V, W, H) * (1 - 1e-13)


def test_updates_minimise_the_surrogate_blockwise():
    """The H update is the exact minimiser of g(Wn, H | Wn, Hn) over H, and the
    W update of g(W, H1 | Wn, H1) over W (block relaxation, Section 3.1):
    the surrogate's partial derivatives vanish there."""
    V, Wn, Hn = _rand_problem(4, 5, 2, 41)
    H1 = orc.update_h(V, Wn, Hn, 0.0)
    h = 1e-5
    for (k, j) in [(0, 0), (1, 3), (0, 4)]:
        Hp, Hm = H1.copy(), H1.copy()
        Hp[k, j] += h
        Hm[k, j] -= h
        d = (orc.surrogate(V, Wn, Hp, Wn, Hn) - orc.surrogate(V, Wn, Hm, Wn, Hn)) / (2 * h)
        assert abs(d) < 1e-6
    W1 = orc.update_w(V, Wn, H1, 0.0)
    for (i, k) in [(0, 0), (3, 1), (2, 0)]:
        Wp, Wm = W1.copy(), W1.copy()
        Wp[i, k] += h
        Wm[i, k] -= h
        d = (orc.surrogate(V, Wp, H1, Wn, H1) - orc.surrogate(V, Wm, H1, Wn, H1)) / (2 * h)
        assert abs(d) < 1e-6


def test_power_of_two_rescaling_is_exactly_equivariant():
    """W -> W D, H -> D^-1 H (D a power-of-two diagonal) maps the iterates the
    same way, bit for bit, when eps = 0."""
    V, W, H = _rand_problem(12, 10, 3, 8)
    D = np.array([2.0, 0.25, 8.0])
    W1, H1 = orc.step(V, W, H, eps=0.0)
    W2, H2 = orc.step(V, W * D, H / D[:, None], eps=0.0)
    assert np.array_equal(W2, W1 * D)
    assert np.array_equal(H2, H1 / D[:, None])


def test_permutation_equivariance():
    V, W, H = _rand_problem(11, 13, 3, 9)
    rp = np.random.default_rng(0).permutation(11)
    cp = np.random.default_rng(1).permutation(13)
    W1, H1 = orc.step(V, W, H)
    W2, H2 = orc.step(V[rp][:, cp], W[rp], H[:, cp])
    np.testing.assert_allclose(W2, W1[rp], rtol=1e-13)
    np.testing.assert_allclose(H2, H1[:, cp], rtol=1e-13)


def test_trace_identity_agrees_when_well_conditioned():
    """f = ||V||^2 - 2<W, V H^T> + <W^T W, H H^T> (same value as the direct
    residual when ||V||^2 / f is small)."""
    V, W, H = _rand_problem(30, 40, 5, 2)
    f_direct = orc.objective(V, W, H)
    f_trace = (np.sum(V * V) - 2 * np.sum(W * orc.vht(V, H))
               + np.sum(orc.gram_w(W) * orc.gram_h(H)))
    assert f_trace == pytest.approx(f_direct, rel=1e-12)


def test_stopping_rule():
    assert orc.relative_change(10.0, 9.0) == pytest.approx(1.0 / 11.0)
    assert orc.relative_change(-3.0, -3.5) == pytest.approx(0.5 / 4.0)
    assert orc.converged(1e6, 1e6 - 1e-4, 1e-9)
    assert not orc.converged(1e6, 1e6 - 1e-2, 1e-9)
    V, W, H = _rand_problem(10, 12, 2, 4)
    W1, H1, fs, nd = orc.run(V, W, H, 100000, eps=0.0, tol=1e-6)
    assert nd < 100000
    assert orc.relative_change(fs[-2], fs[-1]) < 1e-6
    assert all(orc.relative_change(a, b) >= 1e-6 for a, b in zip(fs[:-2], fs[1:-1]))


def test_run_matches_repeated_step():
    V, W, H = _rand_problem(8, 9, 2, 14)
    Wr, Hr, _, nd = orc.run(V, W, H, 5)
    assert nd == 5
    for _ in range(5):
        W, H = orc.step(V, W, H)
    assert np.array_equal(Wr, W) and np.array_equal(Hr, H)


# --- the seeded generators -------------------------------------------------------

def test_splitmix64_published_outputs():
    """SplitMix64 from state 0 yields 0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4
    (the generator's published first outputs)."""
    g = synth.GAMMA
    with np.errstate(over="ignore"):
        z = synth._mix64(np.array([g, g * np.uint64(2)], dtype=np.uint64))
    assert int(z[0]) == 0xE220A8397B1DCDAF
    assert int(z[1]) == 0x6E789E6AA1B965F4


def test_distributions():
    u = synth.uniform_open(5, 1, (200000,))
    assert u.dtype == np.float32 and u.min() > 0 and u.max() < 1
    assert abs(u.mean() - 0.5) < 0.005
    u0 = synth.uniform_closed_open(5, 2, (200000,))
    assert u0.min() >= 0 and u0.max() < 1
    e = synth.exponential(5, 3, (200000,))
    assert e.min() > 0 and abs(e.mean() - 1.0) < 0.01
    z = synth.abs_normal(5, 4, (200000,), 0.01)
    assert z.min() >= 0 and abs(z.mean() - 0.01 * np.sqrt(2 / np.pi)) < 1e-4
    ks = synth.uniform_int(5, 6, 100000, 4, 32)
    assert ks.min() == 4 and ks.max() == 32
    # chunk boundaries do not change the stream
    a = synth.uniform_open(9, 1, (5000000,))
    b = synth.words(9, 1, 4194300, 10)
    assert np.array_equal(a[4194300:4194310],
                          (((b >> np.uint64(41)).astype(np.float64) + 0.5) * 2.0 ** -23).astype(np.float32))
    # the extreme words map strictly inside (0, 1), exactly
    top = np.array([np.uint64(2**64 - 1), np.uint64(0)])
    ext = (((top >> np.uint64(41)).astype(np.float64) + 0.5) * 2.0 ** -23).astype(np.float32)
    assert ext[0] < 1.0 and ext[1] > 0.0
    assert float(ext[0]) == 1.0 - 2.0 ** -24 and float(ext[1]) == 2.0 ** -24


# --- planted mistakes: each plausible slip in the oracle fails a pin ------------------

def _golden_check(step_fn, order="h_first"):
    g = _read_golden(os.path.join(GOLDEN, "exact_4x5.txt"))
    V = np.array(g["V"], float)
    W0 = np.array(g["W0"], float)
    H0 = np.array(g["H0"], float)
    W1, H1 = step_fn(V, W0, H0)
    W1x = np.array([[float(x) for x in row] for row in g[f"W1 {order}"]])
    H1x = np.array([[float(x) for x in row] for row in g[f"H1 {order}"]])
    return np.allclose(W1, W1x, rtol=1e-12) and np.allclose(H1, H1x, rtol=1e-12)


def _mutant_steps():
    f64 = lambda a: np.asarray(a, float)

    def wrong_gram(V, W, H):          # W-update denominator with W^T W instead of H H^T
        H = orc.update_h(V, W, H, 0.0)
        W = f64(W) * orc.vht(V, H) / (f64(W) @ orc.gram_w(W))
        return W, H

    def stale_h(V, W, H):             # W update uses the old H (no block relaxation)
        H1 = orc.update_h(V, W, H, 0.0)
        return orc.update_w(V, W, H, 0.0), H1

    def swapped(V, W, H):             # numerator / denominator swapped
        H = f64(H) * (orc.gram_w(W) @ f64(H)) / orc.wtv(W, V)
        W = f64(W) * (f64(W) @ orc.gram_h(H)) / orc.vht(V, H)
        return W, H

    def dropped_factor(V, W, H):      # forgot to multiply by the old iterate
        H = orc.wtv(W, V) / (orc.gram_w(W) @ f64(H))
        W = orc.vht(V, H) / (f64(W) @ orc.gram_h(H))
        return W, H

    def transposed_gram(V, W, H):     # den = H^T-side product (G H)^T misuse: H G
        H = f64(H)
        G = orc.gram_w(W)
        Gs = G + np.triu(np.ones_like(G))     # non-symmetric stand-in for a wrong Gram index
        H = H * orc.wtv(W, V) / (Gs @ H)
        W = orc.update_w(V, W, H, 0.0)
        return W, H

    return [wrong_gram, stale_h, swapped, dropped_factor, transposed_gram]


@pytest.mark.parametrize("mutant", _mutant_steps(), ids=lambda f: f.__name__)
def test_planted_mistakes_fail_the_exact_pin(mutant):
    assert _golden_check(lambda V, W, H: orc.step(V, W, H, 0.0))      # the oracle passes
    assert not _golden_check(mutant)                                   # the mutant does not


def test_stored_objective_trajectories():
    """tests/golden/objectives.json (the oracle's trajectories on the measured
    workloads): every stored trajectory descends (the MM property), and the
    small workloads' entries reproduce from the oracle here."""
    import json
    with open(os.path.join(GOLDEN, "objectives.json")) as fh:
        d = json.load(fh)
    for name, e in d.items():
        if name.startswith("_"):
            continue
        ks = sorted(int(k) for k in e["objective"])
        fs = [e["objective"][str(k)] for k in ks]
        assert all(b <= a for a, b in zip(fs, fs[1:])), name
    pr = synth.faces()
    W, H, _, _ = orc.run(pr.V, pr.W0, pr.H0, 10, eps=pr.eps)
    assert orc.objective(pr.V, W, H) == pytest.approx(
        d["faces_361x2429_r10"]["objective"]["10"], rel=1e-12)
    pr = synth.planted(p=1024, n=1024, r=50, iters=10)
    assert orc.objective(pr.V, pr.W0, pr.H0) == pytest.approx(
        d["planted_1024x1024_r50"]["objective"]["0"], rel=1e-12)
