"""nmf_converge_resident: every MM iteration of a small problem in one
persistent launch (Algorithm 1, Eqs. (3.3)-(3.4); Section 3's stopping rule
on Eq. (3.1)).

Its float32 sums run in another order than the streaming kernels', so it is
held to the float32 path's bars against the FP64 oracle: per-entry relative
iterate error <= 1e-4 after 10 updates, relative objective error <= 1e-6;
and it must stop where the oracle's own run with the rule stops.
"""
import numpy as np
import pytest

from oracle import nmf_oracle as orc
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


def _resident(V, W0, H0, iters, eps=1e-10, order="h_first", tol=0.0, k=None):
    """(done, f, W, H) of one nmf_converge_resident call from (W0, H0)."""
    from paper_1003_3272_gb300 import nmf
    Vd, W, H = to_dev(V), to_dev(W0), to_dev(H0)
    with nmf.NMF(Vd, W, H, eps=eps, order=order) as m:
        done, f = m.converge_resident(iters, tol=tol, check_every=k or max(iters, 1))
    return done, f, to_host(W), to_host(H)


@pytest.mark.parametrize("order", ["h_first", "w_first"])
def test_faces_ten_iterations(order):
    pr = synth.faces()
    done, fg, Wg, Hg = _resident(pr.V, pr.W0, pr.H0, 10, pr.eps, order)
    Wo, Ho, _, _ = orc.run(pr.V, pr.W0, pr.H0, 10, eps=pr.eps, order=order)
    fo = orc.objective(pr.V, Wo, Ho)
    assert done == 10
    ew, eh = entry_rel_err(Wg, Wo), entry_rel_err(Hg, Ho)
    assert ew[0] <= 1e-4 and eh[0] <= 1e-4, (ew, eh)
    assert abs(fg - fo) / fo <= 1e-6


# ragged slices (p or n not a multiple of the grid, fewer rows or columns
# than blocks, one row, one column) and every rank padding (4, 8, 12, 16)
SHAPES = [(1, 9, 1), (7, 1, 1), (60, 70, 3), (257, 190, 9), (153, 301, 5), (152, 152, 4),
          (500, 333, 16), (100, 2000, 12), (2000, 100, 8), (361, 2429, 12)]


@pytest.mark.parametrize("p,n,r", SHAPES)
def test_shapes_match_oracle(p, n, r):
    pr = synth.uniform_problem(p, n, r, seed=p * 3 + n + r)
    done, fg, Wg, Hg = _resident(pr.V, pr.W0, pr.H0, 10, pr.eps)
    Wo, Ho, _, _ = orc.run(pr.V, pr.W0, pr.H0, 10, eps=pr.eps)
    fo = orc.objective(pr.V, Wo, Ho)
    assert done == 10
    ew, eh = entry_rel_err(Wg, Wo), entry_rel_err(Hg, Ho)
    assert ew[0] <= 1e-4 and eh[0] <= 1e-4, (p, n, r, ew, eh)
    # an exact fit (r = min(p, n)) drives f to the float32 floor: residuals of
    # a few units in the last place of the entries, ~1e-14 of ||V||^2
    floor = 1e-13 * float(np.sum(pr.V.astype(np.float64) ** 2))
    assert abs(fg - fo) <= 1e-6 * fo + floor, (p, n, r, fg, fo)


def test_stops_where_the_oracle_does():
    """tol = 1e-6, testing every iteration: the iteration count within a few
    iterations of the float64 oracle's, the objective within 1e-5; and the
    same within the same margin as the graph-driven device loop."""
    from paper_1003_3272_gb300 import nmf
    pr = synth.uniform_problem(60, 70, 3, seed=2)
    done, f, _, _ = _resident(pr.V, pr.W0, pr.H0, 100000, pr.eps, tol=1e-6, k=1)
    _, _, fs, nd = orc.run(pr.V, pr.W0, pr.H0, 100000, eps=pr.eps, tol=1e-6)
    assert done < 100000
    assert abs(done - nd) <= max(3, nd // 50), (done, nd)
    assert abs(f - fs[-1]) / fs[-1] < 1e-5
    V, W, H = to_dev(pr.V), to_dev(pr.W0), to_dev(pr.H0)
    with nmf.NMF(V, W, H) as m:
        d2, f2 = m.converge(100000, tol=1e-6, check_every=1)
    assert abs(done - d2) <= max(3, d2 // 50), (done, d2)


@pytest.mark.parametrize("max_iters,k", [(23, 5), (3, 10), (0, 4), (20, 20)])
def test_iteration_budget(max_iters, k):
    """tol = 0 never stops early: exactly max_iters iterations (rounds of k,
    then the remainder), and *f_out is the objective of the final factors."""
    from paper_1003_3272_gb300 import nmf
    pr = synth.uniform_problem(130, 300, 6, seed=3)
    V, W, H = to_dev(pr.V), to_dev(pr.W0), to_dev(pr.H0)
    with nmf.NMF(V, W, H, eps=pr.eps) as m:
        done, f = m.converge_resident(max_iters, tol=0.0, check_every=k)
        f_api = m.objective()
    assert done == max_iters
    # the same float32 residuals: nmf_objective adds them 32 at a time in
    # float32 before float64 (evaluation error up to ~1e-8), this kernel
    # every square in float64
    assert abs(f - f_api) <= 1e-8 * f_api
    Wo, Ho, _, _ = orc.run(pr.V, pr.W0, pr.H0, max_iters, eps=pr.eps)
    assert entry_rel_err(to_host(W), Wo)[0] <= 1e-4
    assert entry_rel_err(to_host(H), Ho)[0] <= 1e-4


def test_other_entry_points_continue_from_the_new_factors():
    """After the resident run, nmf_step continues from its W and H (the
    operand planes and Grams are re-formed): 6 + 4 iterations against the
    oracle's 10, and the Gram read back is the new W's."""
    from paper_1003_3272_gb300 import nmf
    pr = synth.uniform_problem(257, 190, 9, seed=8)
    V, W, H = to_dev(pr.V), to_dev(pr.W0), to_dev(pr.H0)
    with nmf.NMF(V, W, H, eps=pr.eps) as m:
        m.converge_resident(6, tol=0.0, check_every=3)
        np.testing.assert_allclose(m.gram(0), orc.gram_w(to_host(W)), rtol=2e-6)
        m.step(4)
        f = m.objective()
    Wo, Ho, _, _ = orc.run(pr.V, pr.W0, pr.H0, 10, eps=pr.eps)
    assert entry_rel_err(to_host(W), Wo)[0] <= 1e-4
    assert entry_rel_err(to_host(H), Ho)[0] <= 1e-4
    assert abs(f - orc.objective(pr.V, Wo, Ho)) / f <= 1e-6


def test_descent_and_determinism():
    """f never increases from one call to the next (the MM property), and two
    runs from one start are bitwise equal."""
    from paper_1003_3272_gb300 import nmf
    pr = synth.faces()
    outs = []
    for _ in range(2):
        V, W, H = to_dev(pr.V), to_dev(pr.W0), to_dev(pr.H0)
        fs = []
        with nmf.NMF(V, W, H, eps=pr.eps) as m:
            for _ in range(15):
                fs.append(m.converge_resident(2, tol=0.0, check_every=2)[1])
        for a, b in zip(fs, fs[1:]):
            assert b <= a * (1 + 1e-6), (a, b)
        outs.append((fs, to_host(W), to_host(H)))
    assert outs[0][0] == outs[1][0]
    assert np.array_equal(outs[0][1], outs[1][1]) and np.array_equal(outs[0][2], outs[1][2])


def test_exact_planted_fixed_point():
    pr = synth.exact_planted(512, 384, 8, seed=3)
    done, fg, Wg, Hg = _resident(pr.V, pr.W0, pr.H0, 3, eps=0.0)
    np.testing.assert_allclose(Wg, pr.W0, rtol=2e-6)
    np.testing.assert_allclose(Hg, pr.H0, rtol=2e-6)
    assert fg <= 1e-12 * float(np.sum(pr.V.astype(np.float64) ** 2))


def test_unsupported_requests():
    """Other precisions, the Poisson model, r > 16 and problems whose slices
    do not fit one block's shared memory are refused; bad arguments are
    NMF_EINVAL."""
    from paper_1003_3272_gb300 import nmf
    pr = synth.uniform_problem(100, 120, 4, seed=1)
    for kw in ({"prec": "bf16x3"}, {"prec": "tf32"}, {"model": "poisson"}):
        V, W, H = to_dev(pr.V), to_dev(pr.W0), to_dev(pr.H0)
        with nmf.NMF(V, W, H, **kw) as m:
            with pytest.raises(nmf.NMFError) as ei:
                m.converge_resident(5)
            assert ei.value.status == nmf.EUNSUPPORTED
    pr = synth.uniform_problem(100, 120, 17, seed=1)
    V, W, H = to_dev(pr.V), to_dev(pr.W0), to_dev(pr.H0)
    with nmf.NMF(V, W, H) as m:
        with pytest.raises(nmf.NMFError) as ei:
            m.converge_resident(5)
        assert ei.value.status == nmf.EUNSUPPORTED
        with pytest.raises(nmf.NMFError) as ei:
            m.converge_resident(5, check_every=0)
        assert ei.value.status == nmf.EINVAL
    pr = synth.uniform_problem(6000, 6000, 4, seed=1, iters=1)
    V, W, H = to_dev(pr.V), to_dev(pr.W0), to_dev(pr.H0)
    with nmf.NMF(V, W, H) as m:
        with pytest.raises(nmf.NMFError) as ei:
            m.converge_resident(5)
        assert ei.value.status == nmf.EUNSUPPORTED
