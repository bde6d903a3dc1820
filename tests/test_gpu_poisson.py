"""Parity of the Poisson model's CUDA path (through the C ABI) with the FP64
Poisson oracle (Section 3.1, the simultaneous square-root MM update).

Bars (float32 products, compensated sums, float64 update): per-entry
relative iterate error <= 2e-5 after one iteration and <= 2e-4 after 20;
the loglikelihood evaluated on the GPU's own factors within 1e-12 of the
oracle's value there (both in float64).
"""
import numpy as np
import pytest

from oracle import poisson_oracle as po
from paper_1003_3272_gb300 import synth
from gpu_util import entry_rel_err, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1003_3272_gb300 import build, nmf
    build.build()
    nmf.load()


def _ctx(pr, **kw):
    from paper_1003_3272_gb300 import nmf
    V, W, H = to_dev(pr.V), to_dev(pr.W0), to_dev(pr.H0)
    return nmf.NMF(V, W, H, eps=pr.eps, model="poisson", **kw), W, H


SHAPES = [(70, 90, 3, 5.0), (129, 200, 17, 5.0), (300, 257, 50, 2.0), (64, 64, 64, 8.0),
          (5, 333, 4, 0.5), (1000, 65, 33, 1.0), (200, 130, 1, 3.0)]


@pytest.mark.parametrize("p,n,r,mean", SHAPES)
def test_one_iteration_matches_oracle(p, n, r, mean):
    """Ragged shapes (several tiles and a ragged tail in both directions),
    ranks 1 .. 64, sparse and dense counts."""
    pr = synth.counts_problem(p, n, r, seed=p + 3 * n + r, mean=mean)
    m, W, H = _ctx(pr)
    with m:
        L0 = m.objective()
        m.step(1)
        L1 = m.objective()
        W1, H1 = to_host(W), to_host(H)
    W1o, H1o = po.step(pr.V, pr.W0, pr.H0, pr.eps)
    assert entry_rel_err(W1, W1o)[0] < 2e-5
    assert entry_rel_err(H1, H1o)[0] < 2e-5
    assert abs(L0 - po.loglik(pr.V, pr.W0, pr.H0)) <= 1e-12 * abs(L0)
    assert abs(L1 - po.loglik(pr.V, W1, H1)) <= 1e-12 * abs(L1)
    assert L1 >= L0


def test_twenty_iterations_trajectory_and_ascent():
    pr = synth.counts_problem(257, 390, 12, seed=21, mean=3.0)
    m, W, H = _ctx(pr)
    Ls = []
    with m:
        Ls.append(m.objective())
        for _ in range(20):
            m.step(1)
            Ls.append(m.objective())
        Wg, Hg = to_host(W), to_host(H)
    Wo, Ho, Lo, _ = po.run(pr.V, pr.W0, pr.H0, 20, eps=pr.eps, track=True)
    assert entry_rel_err(Wg, Wo)[0] < 2e-4
    assert entry_rel_err(Hg, Ho)[0] < 2e-4
    assert abs(Ls[-1] - Lo[-1]) <= 1e-6 * abs(Lo[-1])
    assert all(b >= a - 1e-12 * abs(a) for a, b in zip(Ls, Ls[1:]))


def test_deterministic():
    pr = synth.counts_problem(300, 300, 20, seed=5)
    outs = []
    for _ in range(2):
        m, W, H = _ctx(pr)
        with m:
            m.step(3)
            outs.append((to_host(W), to_host(H), m.objective()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    assert outs[0][2] == outs[1][2]


def test_exact_data_is_a_fixed_point():
    """V = W0 H0 exactly in float32 (small integers on a power-of-two grid):
    every ratio is 1 up to the float32 rounding of the sums, so the factors
    stay within a few ulps."""
    pr = synth.exact_planted(200, 300, 6, seed=4)
    m, W, H = _ctx(pr)
    with m:
        m.step(1)
        W1, H1 = to_host(W), to_host(H)
    assert entry_rel_err(W1, pr.W0.astype(np.float64))[0] < 1e-6
    assert entry_rel_err(H1, pr.H0.astype(np.float64))[0] < 1e-6


def test_full_size_sampled():
    """The 8192 x 8192, r = 50 counts workload in the benchmark's launch
    configuration: one iteration, sampled rows of W and columns of H against
    the oracle's formula evaluated one row / column at a time."""
    pr = synth.counts()
    m, W, H = _ctx(pr)
    with m:
        m.step(1)
        W1, H1 = to_host(W), to_host(H)
    rng = np.random.default_rng(0)
    rows = np.sort(rng.choice(pr.p, 24, replace=False))
    cols = np.sort(rng.choice(pr.n, 24, replace=False))
    V = pr.V.astype(np.float64)
    W0, H0 = pr.W0.astype(np.float64), pr.H0.astype(np.float64)
    hs, ws = H0.sum(axis=1), W0.sum(axis=0)
    for i in rows:
        q = V[i] / (W0[i] @ H0 + pr.eps)
        want = W0[i] * np.sqrt((H0 @ q) / (hs + pr.eps))
        assert entry_rel_err(W1[i], want)[0] < 2e-5
    for j in cols:
        q = V[:, j] / (W0 @ H0[:, j] + pr.eps)
        want = H0[:, j] * np.sqrt((W0.T @ q) / (ws + pr.eps))
        assert entry_rel_err(H1[:, j], want)[0] < 2e-5


def test_device_loop_and_stopping_rule():
    """nmf_converge and nmf_run stop after the same iteration with the same
    factors; the oracle's own run with the rule stops within a few iterations
    of it."""
    pr = synth.counts_problem(120, 150, 4, seed=9, mean=4.0)
    res = []
    for method in ("run", "converge"):
        m, W, H = _ctx(pr)
        with m:
            done, L = getattr(m, method)(100000, tol=1e-7, check_every=1)
            res.append((done, L, to_host(W), to_host(H)))
    assert res[0][0] == res[1][0] < 100000 and res[0][1] == res[1][1]
    assert np.array_equal(res[0][2], res[1][2]) and np.array_equal(res[0][3], res[1][3])
    _, _, Ls, nd = po.run(pr.V, pr.W0, pr.H0, 100000, eps=pr.eps, tol=1e-7)
    assert abs(res[0][0] - nd) <= max(3, nd // 50), (res[0][0], nd)
    assert abs(res[0][1] - Ls[-1]) <= 1e-7 * abs(Ls[-1])


def test_requests_the_model_does_not_serve():
    from paper_1003_3272_gb300 import nmf
    pr = synth.counts_problem(100, 120, 8, seed=1)
    with pytest.raises(nmf.NMFError) as ei:
        _ctx(pr, prec="tf32")
    assert ei.value.status == nmf.EUNSUPPORTED
    big = synth.counts_problem(100, 120, 65, seed=1)
    with pytest.raises(nmf.NMFError) as ei:
        _ctx(big)
    assert ei.value.status == nmf.EUNSUPPORTED
    m, _, _ = _ctx(pr)
    with m:
        with pytest.raises(nmf.NMFError) as ei:
            m.half_step(0)
        assert ei.value.status == nmf.EUNSUPPORTED
        with pytest.raises(nmf.NMFError) as ei:
            m.gram(0)
        assert ei.value.status == nmf.EUNSUPPORTED


def test_solve_with_host_buffers_and_restart():
    """The one-call solve (host V, W, H copied in and out) and a seeded
    restart serve the Poisson model: both equal the context's own steps."""
    import torch
    from paper_1003_3272_gb300 import nmf
    pr = synth.counts_problem(150, 170, 6, seed=13)
    Wh, Hh = pr.W0.copy(), pr.H0.copy()
    L = nmf.solve(pr.V, Wh, Hh, 4, eps=pr.eps, model="poisson")
    m, W, H = _ctx(pr)
    with m:
        m.step(4)
        assert L == m.objective()
        assert np.array_equal(Wh.astype(np.float64), to_host(W))
        assert np.array_equal(Hh.astype(np.float64), to_host(H))
        m.restart(77)
        torch.cuda.synchronize()
        W0, H0 = synth.starting_factors(77, pr.p, pr.n, pr.r)
        assert np.array_equal(to_host(W), W0.astype(np.float64))
        assert np.array_equal(to_host(H), H0.astype(np.float64))


@pytest.mark.parametrize("max_iters,k", [(17, 5), (3, 8)])
def test_device_loop_budget_poisson(max_iters, k):
    """tol = 0: exactly max_iters iterations (rounds of k on the device, the
    remainder on the host), equal to nmf_step."""
    pr = synth.counts_problem(90, 140, 5, seed=17)
    m, W, H = _ctx(pr)
    with m:
        done, L = m.converge(max_iters, tol=0.0, check_every=k)
        Wc, Hc = to_host(W), to_host(H)
    m2, W2, H2 = _ctx(pr)
    with m2:
        m2.step(max_iters)
        L2 = m2.objective()
    assert done == max_iters and L == L2
    assert np.array_equal(Wc, to_host(W2)) and np.array_equal(Hc, to_host(H2))
