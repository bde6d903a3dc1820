"""Quasi-Newton acceleration of the MM map on the GPU (nmf_qn_run) against
the quasi-Newton oracle and the properties its safeguard guarantees."""
import numpy as np
import pytest

from oracle import nmf_oracle as orc
from oracle import poisson_oracle as po
from oracle import qn_oracle as qn
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
    return nmf.NMF(V, W, H, eps=pr.eps, **kw), W, H


def _oracle_maps(pr, model="gaussian"):
    p, n, r = pr.p, pr.n, pr.r
    pack = lambda W, H: np.concatenate([np.ravel(W), np.ravel(H)])
    unpack = lambda x: (x[:p * r].reshape(p, r), x[p * r:].reshape(r, n))
    if model == "gaussian":
        F = lambda x: pack(*orc.step(pr.V, *unpack(x), pr.eps))
        g = lambda x: orc.objective(pr.V, *unpack(x))
    else:
        F = lambda x: pack(*po.step(pr.V, *unpack(x), pr.eps))
        g = lambda x: -po.loglik(pr.V, *unpack(x))
    x0 = pack(pr.W0.astype(np.float64), pr.H0.astype(np.float64))
    return F, g, x0, unpack


@pytest.mark.parametrize("prec,bar", [("fp32", 1e-4), ("bf16x3", 2e-3)])
def test_first_iteration_matches_oracle(prec, bar):
    """One iteration with memory 1: the secant pair, the scalar system and
    the quasi-Newton point (or its fallback) as the oracle takes them; the
    float32 form at the FP32 iterate bar (1e-4 per entry), the split-bf16
    form at its own (the products carry 2^-17 relative operand error)."""
    pr = synth.uniform_problem(60, 80, 4, seed=21)
    m, W, H = _ctx(pr, prec=prec)
    with m:
        done, f, taken = m.qn_run(1, 1)
        Wg, Hg = to_host(W), to_host(H)
    F, g, x0, unpack = _oracle_maps(pr)
    x, gs, acc = qn.qn_run(F, g, x0, 1, 1)
    Wo, Ho = unpack(x)
    assert done == 1 and taken == acc
    assert entry_rel_err(Wg, Wo)[0] < bar and entry_rel_err(Hg, Ho)[0] < bar
    assert abs(f - gs[-1]) <= 1e-4 * gs[-1]


def test_safeguard_and_gain_over_plain_mm():
    """Nonnegative factors, an objective no worse than 2K plain MM iterations
    from the same start (the oracle's run on this problem is far below it),
    and quasi-Newton points taken."""
    pr = synth.uniform_problem(40, 60, 4, seed=9)
    m, W, H = _ctx(pr)
    with m:
        done, f, taken = m.qn_run(5, 30)
        assert to_host(W).min() >= 0 and to_host(H).min() >= 0
    m2, _, _ = _ctx(pr)
    with m2:
        m2.step(60)
        f_mm = m2.objective()
    F, g, x0, _ = _oracle_maps(pr)
    _, gs, acc = qn.qn_run(F, g, x0, 5, 30)
    assert done == 30 and taken > 0 and np.isfinite(f)
    assert f <= f_mm
    assert abs(f - gs[-1]) <= 2e-2 * gs[-1]


def test_stopping_rule_and_determinism():
    pr = synth.faces()
    res = []
    for _ in range(2):
        m, W, H = _ctx(pr, prec="bf16x3")
        with m:
            res.append(m.qn_run(8, 100000, tol=1e-7) + (to_host(W), to_host(H)))
    assert res[0][0] < 100000
    assert res[0][:3] == res[1][:3]
    assert np.array_equal(res[0][3], res[1][3]) and np.array_equal(res[0][4], res[1][4])


def test_poisson_model():
    pr = synth.counts_problem(80, 100, 4, seed=3)
    m, W, H = _ctx(pr, model="poisson")
    with m:
        L0 = m.objective()
        done, L, taken = m.qn_run(4, 15)
        assert to_host(W).min() >= 0 and to_host(H).min() >= 0
    F, g, x0, _ = _oracle_maps(pr, "poisson")
    _, gs, _ = qn.qn_run(F, g, x0, 4, 15)
    assert done == 15 and L >= L0
    assert abs(L - (-gs[-1])) <= 1e-3 * abs(gs[-1])


def test_workspace_is_sized_by_the_first_call():
    from paper_1003_3272_gb300 import nmf
    pr = synth.uniform_problem(50, 70, 3, seed=4)
    m, _, _ = _ctx(pr)
    with m:
        m.qn_run(4, 2)
        m.qn_run(2, 2)
        with pytest.raises(nmf.NMFError) as ei:
            m.qn_run(6, 2)
        assert ei.value.status == nmf.EINVAL
