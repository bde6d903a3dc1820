"""Section 3's stopping rule run on the device (nmf_converge): one CUDA graph
whose while-node repeats k iterations, the objective and the test.

The host-side loop (nmf_run) takes the same float64 test on the same
objective values, and every kernel is deterministic, so the two must agree
bit for bit: the same iteration count, the same objective, the same W and H.
The oracle's own run with the rule pins where it stops.
"""
import numpy as np
import pytest

from oracle import nmf_oracle as orc
from paper_1003_3272_gb300 import synth
from gpu_util import to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1003_3272_gb300 import build, nmf
    build.build()
    nmf.load()


def _both(pr, prec, order, max_iters, tol, k):
    """(iters, f, W, H) of the host loop and of the device loop from one start."""
    from paper_1003_3272_gb300 import nmf
    out = []
    for method in ("run", "converge"):
        V, W, H = to_dev(pr.V), to_dev(pr.W0), to_dev(pr.H0)
        with nmf.NMF(V, W, H, eps=pr.eps, prec=prec, order=order) as m:
            done, f = getattr(m, method)(max_iters, tol=tol, check_every=k)
        out.append((done, f, to_host(W), to_host(H)))
    return out


@pytest.mark.parametrize("prec", ["fp32", "tf32", "bf16x3", "bf16"])
@pytest.mark.parametrize("k", [1, 7])
def test_device_loop_equals_host_loop(prec, k):
    pr = synth.uniform_problem(361, 2429, 10, seed=synth.BASE_SEED)
    (d0, f0, W0, H0), (d1, f1, W1, H1) = _both(pr, prec, "h_first", 100000, 1e-6, k)
    assert d0 < 100000 and d0 % k == 0
    assert d1 == d0 and f1 == f0
    assert np.array_equal(W1, W0) and np.array_equal(H1, H0)


def test_device_loop_paper_order():
    """Algorithm 1's order (W first) through the device loop."""
    pr = synth.uniform_problem(257, 190, 9, seed=8)
    (d0, f0, W0, H0), (d1, f1, W1, H1) = _both(pr, "fp32", "w_first", 100000, 1e-7, 3)
    assert d1 == d0 < 100000 and f1 == f0
    assert np.array_equal(W1, W0) and np.array_equal(H1, H0)


@pytest.mark.parametrize("max_iters,k", [(23, 5), (3, 10), (0, 4), (20, 20)])
def test_device_loop_iteration_budget(max_iters, k):
    """tol = 0 never stops early: exactly max_iters iterations, the rounds of
    k on the device and the remainder on the host; equal to nmf_step."""
    from paper_1003_3272_gb300 import nmf
    pr = synth.uniform_problem(130, 300, 6, seed=3)
    (d1, f1, W1, H1) = _both(pr, "bf16x3", "h_first", max_iters, 0.0, k)[1]
    V, W, H = to_dev(pr.V), to_dev(pr.W0), to_dev(pr.H0)
    with nmf.NMF(V, W, H, eps=pr.eps, prec="bf16x3") as m:
        m.step(max_iters)
        f = m.objective()
    assert d1 == max_iters and f1 == f
    assert np.array_equal(W1, to_host(W)) and np.array_equal(H1, to_host(H))


def test_device_loop_graph_reuse_and_rebuild():
    """A second call reuses the graph (same k), a third builds another (new
    k); each continues from the factors the previous call left."""
    from paper_1003_3272_gb300 import nmf
    pr = synth.uniform_problem(200, 333, 5, seed=11)
    res = []
    for method in ("run", "converge"):
        V, W, H = to_dev(pr.V), to_dev(pr.W0), to_dev(pr.H0)
        with nmf.NMF(V, W, H, eps=pr.eps, prec="tf32") as m:
            a = getattr(m, method)(40, tol=0.0, check_every=4)
            b = getattr(m, method)(40, tol=0.0, check_every=4)
            c = getattr(m, method)(30, tol=1e-5, check_every=6)
        res.append((a, b, c, to_host(W), to_host(H)))
    assert res[0][:3] == res[1][:3]
    assert np.array_equal(res[0][3], res[1][3]) and np.array_equal(res[0][4], res[1][4])


def test_device_loop_stops_where_the_oracle_does():
    """Against the float64 oracle's own run with the rule (tol = 1e-6):
    the iteration count within a few iterations, the objective within 1e-5."""
    from paper_1003_3272_gb300 import nmf
    pr = synth.uniform_problem(60, 70, 3, seed=2)
    V, W, H = to_dev(pr.V), to_dev(pr.W0), to_dev(pr.H0)
    with nmf.NMF(V, W, H) as m:
        done, f = m.converge(100000, tol=1e-6, check_every=1)
    _, _, fs, nd = orc.run(pr.V, pr.W0, pr.H0, 100000, eps=pr.eps, tol=1e-6)
    assert done < 100000
    assert abs(done - nd) <= max(3, nd // 50), (done, nd)
    assert abs(f - fs[-1]) / fs[-1] < 1e-5


def test_device_loop_reports_an_expired_wait():
    """A bounded grid-wide wait that runs out inside an ordinary step is
    reported, and the context then runs the device loop normally."""
    from paper_1003_3272_gb300 import nmf
    pr = synth.uniform_problem(128, 256, 4, seed=5)
    V, W, H = to_dev(pr.V), to_dev(pr.W0), to_dev(pr.H0)
    with nmf.NMF(V, W, H, eps=pr.eps, prec="bf16x3") as m:
        m.converge(8, tol=0.0, check_every=4)      # builds the graph
        m.expire_next_wait()
        m.step(1)
        with pytest.raises(nmf.NMFError) as ei:
            m.objective()
        assert ei.value.status == nmf.ETIMEOUT
        done, f = m.converge(8, tol=0.0, check_every=4)
        assert done == 8 and np.isfinite(f)
