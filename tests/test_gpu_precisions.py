"""Tensor-core precisions (TF32, split BF16x3, BF16) against the FP64 oracle.

Per-product error of each form (operands rounded once, float32 accumulate):
  BF16x3  x = hi + lo (bf16 each), dropped lo*lo term: <= ~2^-16 relative
  TF32    operands rounded to nearest TF32 (11 significant bits): <= ~2^-10
  BF16    operands rounded to nearest bf16 (8 significant bits):  <= ~2^-7
One MM half step inherits that bound (the update is a ratio of such products
to float32 denominators).  The objective is always evaluated from the float32
data and factors, so its evaluation error is that of the float32 path.
"""
import numpy as np
import pytest

from oracle import nmf_oracle as orc
from paper_1003_3272_gb300 import synth
from gpu_util import entry_rel_err, oracle_run, run_gpu, to_dev, to_host

pytestmark = pytest.mark.gpu

HALF_STEP_BAR = {"bf16x3": 5e-5, "tf32": 3e-3, "bf16": 2.5e-2}
# after 10 iterations on the faces-shaped workload
ITER_ENTRY_BAR = {"bf16x3": 2e-3, "tf32": 5e-2, "bf16": 3e-1}
ITER_OBJ_BAR = {"bf16x3": 1e-5, "tf32": 1e-3, "bf16": 1e-2}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1003_3272_gb300 import build, nmf
    build.build()
    nmf.load()


SHAPES = [(333, 517, 1), (257, 131, 10), (129, 1030, 17), (700, 300, 50), (200, 260, 64),
          (150, 400, 100), (128, 128, 128), (1000, 77, 33), (64, 700, 16)]


@pytest.mark.parametrize("prec", ["bf16x3", "tf32", "bf16"])
@pytest.mark.parametrize("p,n,r", SHAPES)
def test_half_steps(prec, p, n, r):
    from paper_1003_3272_gb300 import nmf
    pr = synth.uniform_problem(p, n, r, seed=p * 5 + n + r)
    V, W, H = to_dev(pr.V), to_dev(pr.W0), to_dev(pr.H0)
    with nmf.NMF(V, W, H, prec=prec) as m:
        m.half_step(0)
        H1 = to_host(H)
        e = entry_rel_err(H1, orc.update_h(pr.V, pr.W0, pr.H0, pr.eps))
        assert e[0] < HALF_STEP_BAR[prec], (prec, e)
        m.half_step(1)
        W1 = to_host(W)
        e = entry_rel_err(W1, orc.update_w(pr.V, pr.W0, H1, pr.eps))
        assert e[0] < HALF_STEP_BAR[prec], (prec, e)
        # Grams are formed from the float32 factors in every precision
        np.testing.assert_allclose(m.gram(0), orc.gram_w(W1), rtol=2e-6)
        np.testing.assert_allclose(m.gram(1), orc.gram_h(H1), rtol=2e-6)


@pytest.mark.parametrize("prec", ["bf16x3", "tf32", "bf16"])
def test_faces_ten_iterations(prec):
    pr = synth.faces()
    Wg, Hg, fg = run_gpu(pr.V, pr.W0, pr.H0, 10, prec=prec)
    Wo, Ho, fo = oracle_run(pr.V, pr.W0, pr.H0, 10)
    ew, eh = entry_rel_err(Wg, Wo), entry_rel_err(Hg, Ho)
    rel_f = abs(fg - fo) / fo
    print(f"{prec}: faces 10 it: W err max {ew[0]:.2e} p99 {ew[1]:.2e}; "
          f"H err max {eh[0]:.2e} p99 {eh[1]:.2e}; rel obj {rel_f:.2e}")
    assert max(ew[1], eh[1]) <= ITER_ENTRY_BAR[prec], (ew, eh)
    assert rel_f <= ITER_OBJ_BAR[prec], rel_f
    assert abs(fg - orc.objective(pr.V, Wg, Hg)) / fg <= 1e-9


@pytest.mark.parametrize("prec", ["bf16x3", "tf32", "bf16"])
def test_planted_reduced(prec):
    pr = synth.planted(p=1024, n=1024, r=50, iters=10)
    Wg, Hg, fg = run_gpu(pr.V, pr.W0, pr.H0, 10, prec=prec)
    Wo, Ho, fo = oracle_run(pr.V, pr.W0, pr.H0, 10)
    rel_f = abs(fg - fo) / fo
    print(f"{prec}: planted 1024 r50 10 it: rel obj {rel_f:.2e}")
    assert rel_f <= ITER_OBJ_BAR[prec]
    # descent within the precision's noise
    assert fg < orc.objective(pr.V, pr.W0, pr.H0)


@pytest.mark.parametrize("prec", ["bf16x3", "tf32", "bf16"])
def test_deterministic(prec):
    pr = synth.uniform_problem(700, 900, 40, seed=3)
    a = run_gpu(pr.V, pr.W0, pr.H0, 4, prec=prec)
    b = run_gpu(pr.V, pr.W0, pr.H0, 4, prec=prec)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("prec", ["bf16x3", "tf32"])
@pytest.mark.parametrize("split_k", [1, 2, 4, 8])
def test_cluster_split_variants(prec, split_k):
    """Every cluster size (K-splits per tile) gives the same answer within the
    precision's bar; results are deterministic for a given split."""
    pr = synth.uniform_problem(300, 1100, 24, seed=12)
    Wg, Hg, fg = run_gpu(pr.V, pr.W0, pr.H0, 3, prec=prec, split_k=split_k)
    Wo, Ho, fo = oracle_run(pr.V, pr.W0, pr.H0, 3)
    assert abs(fg - fo) / fo <= ITER_OBJ_BAR[prec]
    assert entry_rel_err(Wg, Wo)[1] <= ITER_ENTRY_BAR[prec]


def test_invalid_cluster_split_is_rejected():
    from paper_1003_3272_gb300 import nmf
    pr = synth.uniform_problem(300, 1100, 24, seed=12)
    with pytest.raises(nmf.NMFError) as ei:
        nmf.NMF(to_dev(pr.V), to_dev(pr.W0), to_dev(pr.H0), prec="bf16x3", split_k=5)
    assert ei.value.status == nmf.EINVAL


def test_many_tiles_persistent_loop():
    """More row tiles than co-resident clusters: the persistent grid walks
    several tiles per cluster (tall V)."""
    pr = synth.uniform_problem(40000, 300, 16, seed=21)
    Wg, Hg, fg = run_gpu(pr.V, pr.W0, pr.H0, 2, prec="bf16x3")
    Wo, Ho, fo = oracle_run(pr.V, pr.W0, pr.H0, 2)
    assert entry_rel_err(Wg, Wo)[0] <= 1e-3
    assert abs(fg - fo) / fo <= 1e-5


def test_exact_planted_fixed_point_bf16x3():
    """Small-integer planted factors are exact in bf16, so the split form is
    exact too: the planted point stays fixed."""
    pr = synth.exact_planted(512, 384, 8, seed=3)
    Wg, Hg, fg = run_gpu(pr.V, pr.W0, pr.H0, 3, eps=0.0, prec="bf16x3")
    np.testing.assert_allclose(Wg, pr.W0, rtol=2e-6)
    np.testing.assert_allclose(Hg, pr.H0, rtol=2e-6)


def test_planted_full_size_sampled_bf16x3():
    """Full-size planted workload (8192 x 8192, r = 50), benchmark launch
    configuration, sampled columns / rows checked one by one."""
    from paper_1003_3272_gb300 import nmf
    pr = synth.planted()
    V, W, H = to_dev(pr.V), to_dev(pr.W0), to_dev(pr.H0)
    rng = np.random.default_rng(1)
    cols = np.sort(rng.choice(pr.n, 48, replace=False))
    rows = np.sort(rng.choice(pr.p, 48, replace=False))
    with nmf.NMF(V, W, H, prec="bf16x3") as m:
        m.half_step(0)
        H1 = to_host(H)
        Hs = orc.update_h_columns(pr.V, pr.W0, pr.H0, cols, pr.eps)
        assert entry_rel_err(H1[:, cols], Hs)[0] < 5e-5
        m.half_step(1)
        W1 = to_host(W)
        Ws = orc.update_w_rows(pr.V, pr.W0, H1, rows, pr.eps)
        assert entry_rel_err(W1[rows], Ws)[0] < 5e-5
