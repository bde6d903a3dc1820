"""Parity of the Poisson model's split-BF16x3 tensor-core form (Section 3.1,
the simultaneous square-root MM update; NMF_BF16X3) with the FP64 Poisson
oracle, through the C ABI.

Bars.  Each factor entry is split x = hi + lo + d with |lo| <= 2^-9 |x| and
|d| <= 2^-18 |x|; a product keeps hi hi' + hi lo' + lo hi', so it drops
lo lo' and the two residuals: at most 3 * 2^-18 (1.1e-5) relative.  b = W H
and the numerator (q H^T or W^T q) each carry that bound (the float32
accumulation adds a few units of 2^-24 per term), the ratio twice it, and the
square root halves it again: about 1.2e-5 per entry in the worst case, which
sums of a handful of terms (p = 5 below) come close to (1.1e-5 observed).
One iteration: per-entry relative iterate error <= 2e-5 (the float32 form's
bar too).  After twenty iterations: relative loglikelihood error <= 1e-6
against the oracle's own trajectory (the headline criterion is 1e-5),
per-entry p99 <= 2e-5.  The loglikelihood evaluated on the GPU's own
factors: within 1e-12 of the oracle there (float64 on both sides).
"""
import numpy as np
import pytest

from oracle import poisson_oracle as po
from paper_1003_3272_gb300 import synth
from gpu_util import entry_rel_err, to_dev, to_host

pytestmark = pytest.mark.gpu

ONE_ITER_BAR = 2e-5
OBJ_BAR = 1e-6
P99_BAR_20 = 2e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1003_3272_gb300 import build, nmf
    build.build()
    nmf.load()


def _ctx(pr, prec="bf16x3", **kw):
    from paper_1003_3272_gb300 import nmf
    V, W, H = to_dev(pr.V), to_dev(pr.W0), to_dev(pr.H0)
    return nmf.NMF(V, W, H, eps=pr.eps, model="poisson", prec=prec, **kw), W, H


# Several 128-row panels and 64-wide tiles with ragged tails in both passes
# (n odd too: the blocked copy of V pads with zeros); ranks 1 .. 64 (rank
# padding 16, 32, 48, 64); sparse and dense counts.
SHAPES = [(70, 93, 3, 5.0), (129, 200, 17, 5.0), (300, 256, 50, 2.0), (64, 64, 64, 8.0),
          (5, 333, 4, 0.5), (1000, 67, 33, 1.0), (200, 131, 1, 3.0), (257, 1028, 48, 2.0),
          (384, 640, 16, 4.0), (130, 5, 2, 6.0)]


@pytest.mark.parametrize("p,n,r,mean", SHAPES)
def test_one_iteration_matches_oracle(p, n, r, mean):
    pr = synth.counts_problem(p, n, r, seed=p + 3 * n + r, mean=mean)
    m, W, H = _ctx(pr)
    with m:
        L0 = m.objective()
        m.step(1)
        L1 = m.objective()
        W1, H1 = to_host(W), to_host(H)
    W1o, H1o = po.step(pr.V, pr.W0, pr.H0, pr.eps)
    assert entry_rel_err(W1, W1o)[0] < ONE_ITER_BAR
    assert entry_rel_err(H1, H1o)[0] < ONE_ITER_BAR
    assert abs(L0 - po.loglik(pr.V, pr.W0, pr.H0)) <= 1e-12 * abs(L0)
    assert abs(L1 - po.loglik(pr.V, W1, H1)) <= 1e-12 * abs(L1)
    assert L1 >= L0


@pytest.mark.parametrize("p,n,r", [(1, 9, 1), (7, 1, 1), (2, 3, 2)])
def test_smallest_shapes(p, n, r):
    """A single row or column of V: one partial panel and tile per pass."""
    pr = synth.counts_problem(p, n, r, seed=40 + p + n, mean=6.0)
    m, W, H = _ctx(pr)
    with m:
        m.step(2)
        W2, H2 = to_host(W), to_host(H)
    W2o, H2o, _, _ = po.run(pr.V, pr.W0, pr.H0, 2, eps=pr.eps)
    assert entry_rel_err(W2, W2o)[0] < 2 * ONE_ITER_BAR
    assert entry_rel_err(H2, H2o)[0] < 2 * ONE_ITER_BAR


def test_misaligned_v_equals_aligned():
    """V as a view that starts 4 bytes into its allocation (not 16-byte
    aligned, the blocked copy's scalar path): the same iterates, bit for
    bit, as from an aligned copy."""
    import torch
    from paper_1003_3272_gb300 import nmf
    pr = synth.counts_problem(150, 203, 9, seed=12)
    base = torch.zeros(pr.p * pr.n + 1, dtype=torch.float32, device="cuda")
    Vm = base[1:].view(pr.p, pr.n)
    Vm.copy_(to_dev(pr.V))
    assert Vm.data_ptr() % 16 != 0
    outs = []
    for V in (Vm, to_dev(pr.V)):
        W, H = to_dev(pr.W0), to_dev(pr.H0)
        with nmf.NMF(V, W, H, eps=pr.eps, model="poisson", prec="bf16x3") as m:
            m.step(3)
            outs.append((to_host(W), to_host(H), m.objective()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    assert outs[0][2] == outs[1][2]


def test_twenty_iterations_objective_and_iterates():
    pr = synth.counts_problem(257, 392, 12, seed=21, mean=3.0)
    m, W, H = _ctx(pr)
    Ls = []
    with m:
        Ls.append(m.objective())
        for _ in range(20):
            m.step(1)
            Ls.append(m.objective())
        Wg, Hg = to_host(W), to_host(H)
    Wo, Ho, Lo, _ = po.run(pr.V, pr.W0, pr.H0, 20, eps=pr.eps, track=True)
    assert abs(Ls[-1] - Lo[-1]) <= OBJ_BAR * abs(Lo[-1])
    assert entry_rel_err(Wg, Wo)[1] <= P99_BAR_20
    assert entry_rel_err(Hg, Ho)[1] <= P99_BAR_20
    assert all(b >= a - 1e-9 * abs(a) for a, b in zip(Ls, Ls[1:]))


def test_agrees_with_the_float32_form():
    """The two precisions of the same model after five iterations: their
    loglikelihoods within the objective bar, their iterates within 1e-3."""
    pr = synth.counts_problem(333, 516, 24, seed=8, mean=4.0)
    out = {}
    for prec in ("fp32", "bf16x3"):
        m, W, H = _ctx(pr, prec=prec)
        with m:
            m.step(5)
            out[prec] = (m.objective(), to_host(W), to_host(H))
    assert abs(out["fp32"][0] - out["bf16x3"][0]) <= OBJ_BAR * abs(out["fp32"][0])
    assert entry_rel_err(out["bf16x3"][1], out["fp32"][1])[0] < 1e-3
    assert entry_rel_err(out["bf16x3"][2], out["fp32"][2])[0] < 1e-3


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
    """V = W0 H0 with W0, H0 on a coarse power-of-two grid: the bf16 split is
    exact (lo = 0), so every product and float32 partial sum is exact, every
    ratio is 1 and the factors stay put."""
    pr = synth.exact_planted(200, 300, 6, seed=4)
    m, W, H = _ctx(pr)
    with m:
        m.step(1)
        W1, H1 = to_host(W), to_host(H)
    assert entry_rel_err(W1, pr.W0.astype(np.float64))[0] < 1e-6
    assert entry_rel_err(H1, pr.H0.astype(np.float64))[0] < 1e-6


def test_full_size_sampled():
    """The 8192 x 8192, r = 50 counts workload in the benchmark's launch
    configuration: one iteration, sampled rows of W and columns of H (and the
    first and last of each) against the update formula evaluated one row /
    column at a time in float64."""
    pr = synth.counts()
    m, W, H = _ctx(pr)
    with m:
        m.step(1)
        W1, H1 = to_host(W), to_host(H)
    rng = np.random.default_rng(1)
    rows = np.sort(rng.choice(pr.p, 24, replace=False))
    cols = np.sort(rng.choice(pr.n, 24, replace=False))
    V = pr.V.astype(np.float64)
    W0, H0 = pr.W0.astype(np.float64), pr.H0.astype(np.float64)
    hs, ws = H0.sum(axis=1), W0.sum(axis=0)
    for i in list(rows) + [0, pr.p - 1]:
        q = V[i] / (W0[i] @ H0 + pr.eps)
        want = W0[i] * np.sqrt((H0 @ q) / (hs + pr.eps))
        assert entry_rel_err(W1[i], want)[0] < ONE_ITER_BAR
    for j in list(cols) + [0, pr.n - 1]:
        q = V[:, j] / (W0 @ H0[:, j] + pr.eps)
        want = H0[:, j] * np.sqrt((W0.T @ q) / (ws + pr.eps))
        assert entry_rel_err(H1[:, j], want)[0] < ONE_ITER_BAR


def test_device_loop_equals_steps():
    """nmf_converge (a CUDA graph of the three launches per iteration) equals
    nmf_step iteration for iteration."""
    pr = synth.counts_problem(90, 140, 5, seed=17)
    m, W, H = _ctx(pr)
    with m:
        done, L = m.converge(11, tol=0.0, check_every=4)
        Wc, Hc = to_host(W), to_host(H)
    m2, W2, H2 = _ctx(pr)
    with m2:
        m2.step(11)
        L2 = m2.objective()
    assert done == 11 and L == L2
    assert np.array_equal(Wc, to_host(W2)) and np.array_equal(Hc, to_host(H2))


def test_restart_rebuilds_the_planes():
    """A seeded restart gives the factor planes and denominators of the new
    start: the next iteration equals a fresh context's on the same start."""
    import torch
    pr = synth.counts_problem(150, 172, 6, seed=13)
    m, W, H = _ctx(pr)
    with m:
        m.step(2)
        m.restart(77)
        m.step(1)
        torch.cuda.synchronize()
        Wr, Hr = to_host(W), to_host(H)
    W0, H0 = synth.starting_factors(77, pr.p, pr.n, pr.r)
    pr2 = synth.Problem(pr.name, pr.V, W0, H0, pr.r, pr.iters, pr.eps, pr.seed)
    m2, W2, H2 = _ctx(pr2)
    with m2:
        m2.step(1)
        assert np.array_equal(Wr, to_host(W2)) and np.array_equal(Hr, to_host(H2))


def test_requests_the_form_does_not_serve():
    from paper_1003_3272_gb300 import nmf
    pr = synth.counts_problem(100, 122, 65, seed=1)
    with pytest.raises(nmf.NMFError) as ei:
        _ctx(pr)
    assert ei.value.status == nmf.EUNSUPPORTED
    pr = synth.counts_problem(100, 120, 8, seed=1)
    for prec in ("tf32", "bf16"):
        with pytest.raises(nmf.NMFError) as ei:
            _ctx(pr, prec=prec)
        assert ei.value.status == nmf.EUNSUPPORTED


def test_expired_waits_leave_the_factors():
    """Failure detection without a fault: the hook makes the first pass's
    first V stage wait for bytes that never come; every block gives up its
    bounded waits, the update leaves W and H as they were, the next
    objective reports NMF_ETIMEOUT, and the context then runs on exactly as
    one that never had the failed iteration."""
    import time
    from paper_1003_3272_gb300 import nmf
    pr = synth.counts_problem(300, 400, 10, seed=31)
    m, W, H = _ctx(pr)
    with m:
        m.step(1)
        W1, H1 = to_host(W), to_host(H)
        m.expire_next_wait()
        t0 = time.time()
        m.step(1)
        with pytest.raises(nmf.NMFError) as ei:
            m.objective()
        assert ei.value.status == nmf.ETIMEOUT
        assert time.time() - t0 < 60
        np.testing.assert_array_equal(to_host(W), W1)
        np.testing.assert_array_equal(to_host(H), H1)
        m.step(2)
        L = m.objective()
        Wf, Hf = to_host(W), to_host(H)
    m2, W2, H2 = _ctx(pr)
    with m2:
        m2.step(3)
        assert m2.objective() == L
        assert np.array_equal(to_host(W2), Wf) and np.array_equal(to_host(H2), Hf)
