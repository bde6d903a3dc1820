"""Batched form: many independent problems in one grouped persistent launch
per half step (replayed from a CUDA graph), against the FP64 oracle."""
import numpy as np
import pytest

from oracle import nmf_oracle as orc
from paper_1003_3272_gb300 import synth
from gpu_util import entry_rel_err, to_dev, to_host

pytestmark = pytest.mark.gpu

OBJ_BAR = {"bf16x3": 1e-5, "tf32": 1e-3, "bf16": 1e-2}
ENTRY_P99_BAR = {"bf16x3": 2e-3, "tf32": 5e-2, "bf16": 3e-1}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1003_3272_gb300 import build, nmf
    build.build()
    nmf.load()


def _small_batch(count, seed, pmax=700):
    return synth.batch(count=count, seed=seed, iters=5, pmin=64, pmax=pmax, rmin=4, rmax=32)


def _run(probs, iters, prec):
    from paper_1003_3272_gb300 import nmf
    Vs = [to_dev(pr.V) for pr in probs]
    Ws = [to_dev(pr.W0) for pr in probs]
    Hs = [to_dev(pr.H0) for pr in probs]
    b = nmf.Batch(Vs, Ws, Hs, prec=prec)
    b.step(iters)
    f = b.objective()
    out = [(to_host(W), to_host(H)) for W, H in zip(Ws, Hs)]
    b.close()
    return out, f


@pytest.mark.parametrize("prec", ["bf16x3", "tf32", "bf16"])
def test_batched_matches_oracle(prec):
    probs = _small_batch(12, seed=11)
    out, f = _run(probs, 5, prec)
    for pr, (Wg, Hg), fg in zip(probs, out, f):
        Wo, Ho, _, _ = orc.run(pr.V, pr.W0, pr.H0, 5, eps=pr.eps)
        fo = orc.objective(pr.V, Wo, Ho)
        assert abs(fg - fo) / fo <= OBJ_BAR[prec], (pr.name, fg, fo)
        assert entry_rel_err(Wg, Wo)[1] <= ENTRY_P99_BAR[prec], pr.name
        assert entry_rel_err(Hg, Ho)[1] <= ENTRY_P99_BAR[prec], pr.name
        # the batched objective evaluates the GPU's own iterate to float64 accuracy
        assert abs(fg - orc.objective(pr.V, Wg, Hg)) / fg <= 1e-8


def test_batched_half_step_bound_bf16x3():
    """One iteration from identical float32 inputs: each instance's H and W
    updates are within the BF16x3 single-half-step bound of the oracle's."""
    probs = _small_batch(8, seed=5)
    out, _ = _run(probs, 1, "bf16x3")
    for pr, (Wg, Hg) in zip(probs, out):
        H1 = orc.update_h(pr.V, pr.W0, pr.H0, pr.eps)
        assert entry_rel_err(Hg, H1)[0] < 5e-5, pr.name
        W1 = orc.update_w(pr.V, pr.W0, Hg, pr.eps)
        assert entry_rel_err(Wg, W1)[0] < 5e-5, pr.name


def test_batched_equals_single_contexts_within_precision():
    from paper_1003_3272_gb300 import nmf
    probs = _small_batch(6, seed=7)
    out, f = _run(probs, 4, "bf16x3")
    for pr, (Wg, Hg), fg in zip(probs, out, f):
        V, W, H = to_dev(pr.V), to_dev(pr.W0), to_dev(pr.H0)
        with nmf.NMF(V, W, H, prec="bf16x3") as m:
            m.step(4)
            fs = m.objective()
        assert abs(fg - fs) / fs <= 2e-6
        assert entry_rel_err(Wg, to_host(W))[1] <= 1e-4


def test_batched_deterministic():
    probs = _small_batch(10, seed=3)
    a, fa = _run(probs, 3, "bf16x3")
    b, fb = _run(probs, 3, "bf16x3")
    assert np.array_equal(fa, fb)
    for (W1, H1), (W2, H2) in zip(a, b):
        assert np.array_equal(W1, W2) and np.array_equal(H1, H2)


def test_batched_descent_and_ragged_shapes():
    """Extremes of the workload's shape ranges, including rank 4 and 32 and
    sizes that are not multiples of a tile; the objective decreases."""
    from paper_1003_3272_gb300 import nmf
    shapes = [(64, 64, 4), (64, 2048, 32), (2048, 64, 17), (1000, 333, 32), (129, 257, 5)]
    probs = [synth.uniform_problem(p, n, r, seed=100 + i) for i, (p, n, r) in enumerate(shapes)]
    Vs = [to_dev(pr.V) for pr in probs]
    Ws = [to_dev(pr.W0) for pr in probs]
    Hs = [to_dev(pr.H0) for pr in probs]
    b = nmf.Batch(Vs, Ws, Hs, prec="bf16x3")
    f0 = b.objective()
    b.step(3)
    f3 = b.objective()
    b.close()
    for pr, a0, a3, W, H in zip(probs, f0, f3, Ws, Hs):
        assert a3 < a0
        Wo, Ho, _, _ = orc.run(pr.V, pr.W0, pr.H0, 3, eps=pr.eps)
        assert abs(a3 - orc.objective(pr.V, Wo, Ho)) / a3 <= 1e-5


def test_batched_workload_sample_full_size():
    """The batched workload's own instance shapes (512 problems, p, n in
    64..2048, r in 4..32): run the whole batch one iteration and check a
    sample of instances against the oracle one by one."""
    probs = synth.batch(count=512, iters=1)
    out, f = _run(probs, 1, "bf16x3")
    rng = np.random.default_rng(0)
    for b in rng.choice(len(probs), 12, replace=False):
        pr = probs[b]
        Wo, Ho, _, _ = orc.run(pr.V, pr.W0, pr.H0, 1, eps=pr.eps)
        fo = orc.objective(pr.V, Wo, Ho)
        assert abs(f[b] - fo) / fo <= 1e-5, pr.name
        assert entry_rel_err(out[b][1], Ho)[0] < 5e-5, pr.name


def _candidates():
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    return [f"{pol}/{g}" for pol in ("lpt", "glpt", "rr")
            for g in (sms, sms - sms // 8, sms - sms // 4)]


@pytest.mark.parametrize("which", range(9))
def test_every_tuner_candidate_matches_the_oracle(which, monkeypatch):
    """Each schedule the autotuner may choose (policy x grid), forced through
    NMF_BATCHED_SCHEDULE, gives the oracle's iterates within the BF16x3 bars;
    the batch reports the forced choice."""
    from paper_1003_3272_gb300 import nmf
    name = _candidates()[which]
    monkeypatch.setenv("NMF_BATCHED_SCHEDULE", name)
    probs = _small_batch(10, seed=40 + which)
    Vs = [to_dev(pr.V) for pr in probs]
    Ws = [to_dev(pr.W0) for pr in probs]
    Hs = [to_dev(pr.H0) for pr in probs]
    b = nmf.Batch(Vs, Ws, Hs, prec="bf16x3")
    assert b.schedule == name
    b.step(3)
    f = b.objective()
    b.close()
    for pr, W, H, fg in zip(probs, Ws, Hs, f):
        Wo, Ho, _, _ = orc.run(pr.V, pr.W0, pr.H0, 3, eps=pr.eps)
        fo = orc.objective(pr.V, Wo, Ho)
        assert abs(fg - fo) / fo <= OBJ_BAR["bf16x3"], (name, pr.name)
        assert entry_rel_err(to_host(W), Wo)[1] <= ENTRY_P99_BAR["bf16x3"], (name, pr.name)
        assert entry_rel_err(to_host(H), Ho)[1] <= ENTRY_P99_BAR["bf16x3"], (name, pr.name)


def test_unknown_forced_schedule_is_rejected(monkeypatch):
    from paper_1003_3272_gb300 import nmf
    monkeypatch.setenv("NMF_BATCHED_SCHEDULE", "nosuch/7")
    probs = _small_batch(2, seed=1)
    with pytest.raises(nmf.NMFError) as ei:
        nmf.Batch([to_dev(p.V) for p in probs], [to_dev(p.W0) for p in probs],
                  [to_dev(p.H0) for p in probs], prec="bf16x3")
    assert ei.value.status == nmf.EINVAL


def test_expired_waits_in_the_grouped_kernel():
    """Failure detection without a fault: the hook makes every bounded wait
    of the next iteration run out; no factor changes, the next objective
    reports NMF_ETIMEOUT, and the batch then runs on exactly as a batch that
    never had the failed iteration."""
    import time
    from paper_1003_3272_gb300 import nmf
    probs = _small_batch(6, seed=9)
    ref, fref = _run(probs, 3, "bf16x3")
    Vs = [to_dev(pr.V) for pr in probs]
    Ws = [to_dev(pr.W0) for pr in probs]
    Hs = [to_dev(pr.H0) for pr in probs]
    b = nmf.Batch(Vs, Ws, Hs, prec="bf16x3")
    b.step(1)
    W1, H1 = [to_host(W) for W in Ws], [to_host(H) for H in Hs]
    b.expire_next_wait()
    t0 = time.time()
    b.step(1)
    with pytest.raises(nmf.NMFError) as ei:
        b.objective()
    assert ei.value.status == nmf.ETIMEOUT
    assert time.time() - t0 < 60
    for W, H, w1, h1 in zip(Ws, Hs, W1, H1):
        np.testing.assert_array_equal(to_host(W), w1)
        np.testing.assert_array_equal(to_host(H), h1)
    b.step(2)
    f = b.objective()
    b.close()
    assert np.array_equal(f, fref)
    for (Wr, Hr), W, H in zip(ref, Ws, Hs):
        assert np.array_equal(to_host(W), Wr) and np.array_equal(to_host(H), Hr)
