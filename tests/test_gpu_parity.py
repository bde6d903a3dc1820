"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bars (float32 path): per-entry relative iterate error <= 1e-4 after 10
updates and relative objective error <= 1e-6; tensor-core forms have their
own bars in test_gpu_precisions.py.
"""
import numpy as np
import pytest

from oracle import nmf_oracle as orc
from paper_1003_3272_gb300 import synth
from gpu_util import entry_rel_err, oracle_run, run_gpu, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1003_3272_gb300 import build, nmf
    build.build()
    nmf.load()


def test_seeded_start_is_bitwise_the_generator():
    """Algorithm 1's uniform(0,1) start drawn on the device equals the
    generator module's draw bit for bit."""
    import torch
    from paper_1003_3272_gb300 import nmf
    p, n, r, seed = 300, 411, 7, 12345
    V = to_dev(synth.uniform_closed_open(1, 0, (p, n)))
    W = torch.zeros(p, r, device="cuda")
    H = torch.zeros(r, n, device="cuda")
    with nmf.NMF(V, W, H, seed=seed, init_from_seed=True):
        torch.cuda.synchronize()
    W0, H0 = synth.starting_factors(seed, p, n, r)
    assert np.array_equal(W.cpu().numpy(), W0)
    assert np.array_equal(H.cpu().numpy(), H0)


SHAPES = [(333, 517, 1), (333, 517, 3), (257, 131, 10), (129, 1030, 17), (700, 300, 50),
          (200, 260, 64), (150, 400, 100), (128, 128, 128), (1000, 77, 33)]


@pytest.mark.parametrize("p,n,r", SHAPES)
def test_half_steps_match_oracle(p, n, r):
    """One H update, then one W update, each from identical float32 inputs."""
    from paper_1003_3272_gb300 import nmf
    pr = synth.uniform_problem(p, n, r, seed=p * 7 + n + r)
    V, W, H = to_dev(pr.V), to_dev(pr.W0), to_dev(pr.H0)
    with nmf.NMF(V, W, H) as m:
        m.half_step(0)
        H1 = to_host(H)
        H1_ref = orc.update_h(pr.V, pr.W0, pr.H0, pr.eps)
        e = entry_rel_err(H1, H1_ref)
        assert e[0] < 2e-5, e
        m.half_step(1)
        W1 = to_host(W)
        # oracle W update from the GPU's own (float32) H: isolates this half step
        W1_ref = orc.update_w(pr.V, pr.W0, H1, pr.eps)
        e = entry_rel_err(W1, W1_ref)
        assert e[0] < 2e-5, e
        G = m.gram(0)
        np.testing.assert_allclose(G, orc.gram_w(W1), rtol=2e-6)
        GH = m.gram(1)
        np.testing.assert_allclose(GH, orc.gram_h(H1), rtol=2e-6)


@pytest.mark.parametrize("order", ["h_first", "w_first"])
def test_faces_ten_iterations(order):
    pr = synth.faces()
    Wg, Hg, fg = run_gpu(pr.V, pr.W0, pr.H0, 10, order=order)
    Wo, Ho, fo = oracle_run(pr.V, pr.W0, pr.H0, 10, order=order)
    ew, eh = entry_rel_err(Wg, Wo), entry_rel_err(Hg, Ho)
    assert ew[0] <= 1e-4 and eh[0] <= 1e-4, (ew, eh)
    assert abs(fg - fo) / fo <= 1e-6
    # evaluation error of the objective at the GPU's own iterate
    assert abs(fg - orc.objective(pr.V, Wg, Hg)) / fg <= 1e-9


def test_faces_full_run_and_descent():
    """The faces-shaped workload: 50 iterations; f never increases."""
    from paper_1003_3272_gb300 import nmf
    pr = synth.faces()
    V, W, H = to_dev(pr.V), to_dev(pr.W0), to_dev(pr.H0)
    fs = []
    with nmf.NMF(V, W, H) as m:
        fs.append(m.objective())
        for _ in range(pr.iters):
            m.step(1)
            fs.append(m.objective())
    for a, b in zip(fs, fs[1:]):
        assert b <= a * (1 + 1e-6)
    Wo, Ho, fo = oracle_run(pr.V, pr.W0, pr.H0, pr.iters)
    assert abs(fs[-1] - fo) / fo <= 1e-6
    ew, eh = entry_rel_err(to_host(W), Wo), entry_rel_err(to_host(H), Ho)
    assert ew[1] <= 1e-4 and eh[1] <= 1e-4, (ew, eh)


def test_planted_reduced_ten_iterations():
    """Planted low-rank workload at 1024 x 1024, r = 50 (large ||V||^2 / f)."""
    pr = synth.planted(p=1024, n=1024, r=50, iters=10)
    Wg, Hg, fg = run_gpu(pr.V, pr.W0, pr.H0, 10)
    Wo, Ho, fo = oracle_run(pr.V, pr.W0, pr.H0, 10)
    ew, eh = entry_rel_err(Wg, Wo), entry_rel_err(Hg, Ho)
    assert ew[0] <= 1e-4 and eh[0] <= 1e-4, (ew, eh)
    assert abs(fg - fo) / fo <= 1e-6
    assert abs(fg - orc.objective(pr.V, Wg, Hg)) / fg <= 1e-8


@pytest.mark.parametrize("split_k", [1, 2, 4, 8])
def test_split_k_variants(split_k):
    """Every cluster size (K-splits per tile) of the float32 kernel."""
    pr = synth.uniform_problem(520, 700, 20, seed=77)
    Wg, Hg, fg = run_gpu(pr.V, pr.W0, pr.H0, 5, split_k=split_k)
    Wo, Ho, fo = oracle_run(pr.V, pr.W0, pr.H0, 5)
    assert entry_rel_err(Wg, Wo)[0] <= 1e-4
    assert entry_rel_err(Hg, Ho)[0] <= 1e-4
    assert abs(fg - fo) / fo <= 1e-6


def test_deterministic_bitwise():
    pr = synth.uniform_problem(600, 900, 24, seed=5)
    a = run_gpu(pr.V, pr.W0, pr.H0, 6)
    b = run_gpu(pr.V, pr.W0, pr.H0, 6)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and a[2] == b[2]


def test_resume_matches_uninterrupted_run():
    """Checkpoint/resume: the MM state is (W, H); a fresh context from saved
    factors continues the trajectory bit for bit."""
    pr = synth.uniform_problem(300, 350, 12, seed=9)
    Wa, Ha, _ = run_gpu(pr.V, pr.W0, pr.H0, 6)
    W3, H3, _ = run_gpu(pr.V, pr.W0, pr.H0, 3)
    Wb, Hb, _ = run_gpu(pr.V, W3.astype(np.float32), H3.astype(np.float32), 3)
    assert np.array_equal(Wa, Wb) and np.array_equal(Ha, Hb)


def test_exact_planted_fixed_point():
    pr = synth.exact_planted(512, 384, 8, seed=3)
    Wg, Hg, fg = run_gpu(pr.V, pr.W0, pr.H0, 3, eps=0.0)
    np.testing.assert_allclose(Wg, pr.W0, rtol=2e-6)
    np.testing.assert_allclose(Hg, pr.H0, rtol=2e-6)
    assert fg <= 1e-12 * float(np.sum(pr.V.astype(np.float64) ** 2))


def test_zero_rows_and_columns_stay_finite():
    pr = synth.uniform_problem(200, 300, 6, seed=4)
    V = pr.V.copy()
    V[17, :] = 0
    V[:, 101] = 0
    Wg, Hg, fg = run_gpu(V, pr.W0, pr.H0, 4)
    assert np.all(np.isfinite(Wg)) and np.all(np.isfinite(Hg))
    assert np.all(Wg[17] == 0) and np.all(Hg[:, 101] == 0)
    Wo, Ho, fo = oracle_run(V, pr.W0, pr.H0, 4)
    assert entry_rel_err(Wg, Wo)[0] <= 1e-4 and abs(fg - fo) / fo <= 1e-6


def test_rank_equals_min_dimension_and_tiny_shapes():
    for (p, n, r) in [(5, 7, 5), (1, 1, 1), (3, 200, 2), (200, 3, 3)]:
        pr = synth.uniform_problem(p, n, r, seed=p + n)
        Wg, Hg, fg = run_gpu(pr.V, pr.W0, pr.H0, 3)
        Wo, Ho, fo = oracle_run(pr.V, pr.W0, pr.H0, 3)
        assert entry_rel_err(Wg, Wo)[0] <= 1e-4, (p, n, r)
        assert entry_rel_err(Hg, Ho)[0] <= 1e-4, (p, n, r)


def test_validate_rejects_negative_entries():
    import torch
    from paper_1003_3272_gb300 import nmf
    pr = synth.uniform_problem(64, 80, 4, seed=1)
    V = pr.V.copy()
    V[3, 5] = -1.0
    with pytest.raises(nmf.NMFError) as ei:
        nmf.NMF(to_dev(V), to_dev(pr.W0), to_dev(pr.H0), validate=True)
    assert ei.value.status == nmf.ENONFINITE
    V[3, 5] = float("nan")
    with pytest.raises(nmf.NMFError):
        nmf.NMF(to_dev(V), to_dev(pr.W0), to_dev(pr.H0), validate=True)
    torch.cuda.synchronize()


def test_solve_with_host_buffers_equals_device_path():
    from paper_1003_3272_gb300 import nmf
    pr = synth.uniform_problem(257, 190, 9, seed=8)
    Wh, Hh = pr.W0.copy(), pr.H0.copy()
    f = nmf.solve(pr.V, Wh, Hh, 5)
    Wg, Hg, fg = run_gpu(pr.V, pr.W0, pr.H0, 5)
    assert np.array_equal(Wh.astype(np.float64), Wg) and np.array_equal(Hh.astype(np.float64), Hg)
    assert f == fg


def test_stopping_rule_run():
    from paper_1003_3272_gb300 import nmf
    pr = synth.uniform_problem(60, 70, 3, seed=2)
    V, W, H = to_dev(pr.V), to_dev(pr.W0), to_dev(pr.H0)
    with nmf.NMF(V, W, H) as m:
        done, f = m.run(100000, tol=1e-6, check_every=1)
    _, _, fs, nd = orc.run(pr.V, pr.W0, pr.H0, 100000, eps=pr.eps, tol=1e-6)
    assert done < 100000
    assert abs(done - nd) <= max(3, nd // 50), (done, nd)
    assert abs(f - fs[-1]) / fs[-1] < 1e-5


def test_planted_full_size_sampled():
    """The planted workload at its full size (8192 x 8192, r = 50) in the
    benchmark's launch configuration: one H update then one W update,
    checked on sampled rows/columns against the oracle computed one by one."""
    from paper_1003_3272_gb300 import nmf
    pr = synth.planted()
    V, W, H = to_dev(pr.V), to_dev(pr.W0), to_dev(pr.H0)
    rng = np.random.default_rng(0)
    cols = np.sort(rng.choice(pr.n, 48, replace=False))
    rows = np.sort(rng.choice(pr.p, 48, replace=False))
    with nmf.NMF(V, W, H) as m:
        m.half_step(0)
        H1 = to_host(H)
        Hs = orc.update_h_columns(pr.V, pr.W0, pr.H0, cols, pr.eps)
        assert entry_rel_err(H1[:, cols], Hs)[0] < 5e-5
        m.half_step(1)
        W1 = to_host(W)
        Ws = orc.update_w_rows(pr.V, pr.W0, H1, rows, pr.eps)
        assert entry_rel_err(W1[rows], Ws)[0] < 5e-5


def test_update_division_is_the_ieee_division():
    """The update divides by Markstein's quotient correction where its
    conditions hold: every significand of the divisor against 64 dividends,
    plus random operand pairs over the whole float32 range, bit for bit
    against the IEEE division."""
    from paper_1003_3272_gb300 import nmf
    count = (64 << 23) + (1 << 29)
    mism, quick = nmf.selfcheck_div(count, seed=7)
    assert mism == 0
    assert quick > (64 << 23)          # the sweep and most random pairs took the quick form


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_expired_device_wait_is_reported_and_the_context_recovers(prec):
    """Failure detection without a fault: the next half step's grid-wide
    waits get a target the device counter never reaches; every block's
    bounded wait runs out, the launch skips its update and records
    NMF_ETIMEOUT, the next synchronising call reports it, and the context
    then works on (the skipped half step left the factors as they were)."""
    import time
    from paper_1003_3272_gb300 import nmf
    pr = synth.faces()
    V, W, H = to_dev(pr.V), to_dev(pr.W0), to_dev(pr.H0)
    with nmf.NMF(V, W, H, eps=pr.eps, prec=prec) as m:
        m.step(2)
        f2 = m.objective()
        W2, H2 = to_host(W), to_host(H)
        m.expire_next_wait()
        t0 = time.time()
        m.half_step(0)                     # H update: its waits run out
        with pytest.raises(nmf.NMFError) as ei:
            m.objective()
        assert ei.value.status == nmf.ETIMEOUT
        assert time.time() - t0 < 60
        np.testing.assert_array_equal(to_host(H), H2)   # the update was skipped
        assert m.objective() == f2                      # state as before, no error left
        m.step(2)
        f4 = m.objective()
        assert np.isfinite(f4) and f4 <= f2
    np.testing.assert_array_equal(to_host(W).shape, W2.shape)
