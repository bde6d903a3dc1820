"""Pins of the quasi-Newton oracle (the acceleration the paper names in
Section 4) to facts outside its own formula: on an affine contraction the
secant conditions determine the Jacobian exactly once the memory spans the
space, so the scheme lands on the fixed point; in one dimension after a
single iteration; the safeguard keeps the MM descent on NMF and never loses
to the plain MM iterates it is built from.  CPU only."""
import numpy as np
import pytest

from oracle import nmf_oracle as orc
from oracle import qn_oracle as qn
from paper_1003_3272_gb300 import synth


def _affine(N, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((N, N)))
    lam = rng.uniform(0.5, 0.95, N)
    A = Q @ np.diag(lam) @ Q.T
    xs = rng.uniform(5.0, 10.0, N)             # the fixed point, well inside x >= 0
    b = xs - A @ xs
    return (lambda x: A @ x + b), xs


def test_scalar_map_one_iteration():
    F = lambda x: 0.8 * x + 1.0                # fixed point 5
    x, gs, acc = qn.qn_run(F, lambda x: float((x[0] - 5.0) ** 2), np.array([4.0]), 1, 1)
    assert acc == 1 and abs(x[0] - 5.0) < 1e-12


@pytest.mark.parametrize("N", [3, 6])
def test_affine_contraction_exact_once_the_memory_spans(N):
    F, xs = _affine(N, seed=N)
    g = lambda x: float(np.sum((x - xs) ** 2))
    x0 = xs + np.random.default_rng(1).uniform(-0.5, 0.5, N)
    x, gs, acc = qn.qn_run(F, g, x0, N, N)
    assert np.max(np.abs(x - xs)) < 1e-9 * np.max(xs)
    # plain iteration of the same map is nowhere near after 2N evaluations
    y = x0.copy()
    for _ in range(2 * N):
        y = F(y)
    assert np.max(np.abs(y - xs)) > 1e-3


def test_singular_system_falls_back():
    U = np.ones((4, 2))
    assert qn.qn_step_point(np.zeros(4), U, U, U[:, 0]) is None


def test_nmf_safeguard_descent_and_gain():
    pr = synth.uniform_problem(40, 60, 4, seed=9)
    p, n, r = pr.p, pr.n, pr.r
    pack = lambda W, H: np.concatenate([np.ravel(W), np.ravel(H)])
    unpack = lambda x: (x[:p * r].reshape(p, r), x[p * r:].reshape(r, n))
    F = lambda x: pack(*orc.step(pr.V, *unpack(x), pr.eps))
    g = lambda x: orc.objective(pr.V, *unpack(x))
    x0 = pack(pr.W0.astype(np.float64), pr.H0.astype(np.float64))
    K = 30
    x, gs, acc = qn.qn_run(F, g, x0, 5, K)
    assert np.all(x >= 0)
    assert all(b <= a * (1 + 1e-12) for a, b in zip(gs, gs[1:]))
    # never worse than the plain MM iterate of each step; here much better
    y = x0.copy()
    for _ in range(2 * K):
        y = F(y)
    assert gs[-1] <= g(y)
    assert acc > 0
