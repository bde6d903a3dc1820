"""Penalised PET reconstruction on the GPU (include/pet.h; Section 3.2,
Algorithm 2) against the float64 oracle (oracle/pet_oracle.py) on the same
seeded inputs.

Bars (float32 projections and ratios, float64 update): per-pixel relative
error |x - x*| / max(|x*|, 1e-6 max|x*|) <= 2e-5 after one iteration and
<= 1e-4 after ten (the float32 iterate bar); the objective at the GPU's own
intensities within 1e-9 of the oracle's (both float64), and the objective
after k iterations within 1e-6 of the oracle's trajectory."""
import numpy as np
import pytest

from oracle import pet_oracle as po
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


def _gpu(E, y, ptr, idx, mu, iters, lam0=None):
    import torch
    from paper_1003_3272_gb300 import nmf
    Ed, yd = to_dev(E), to_dev(y)
    lam = None if lam0 is None else to_dev(lam0)
    with nmf.PET(Ed, yd, ptr, idx, mu, lam=lam, init_ones=lam0 is None) as m:
        f0 = m.objective()
        m.step(iters)
        f = m.objective()
        lam = to_host(m.lam)
    torch.cuda.synchronize()
    return lam, f0, f


def _check(pr_E, pr_y, ptr, idx, mu, iters, bar):
    lam, f0, f = _gpu(pr_E, pr_y, ptr, idx, mu, iters)
    En = po.normalise_columns(pr_E)
    prs = po.pairs(ptr, idx)
    for k, m in enumerate(mu):
        lo, fs, _ = po.run(pr_E, pr_y, m, ptr, idx, iters)
        err = entry_rel_err(lam[k], lo)[0]
        assert err <= bar, (k, m, err)
        assert abs(f0[k] - fs[0]) <= 1e-12 * abs(fs[0])
        # evaluation at the GPU's own intensities, and the trajectory
        fe = po.objective(En, pr_y, lam[k], m, prs)
        assert abs(f[k] - fe) <= 1e-9 * abs(fe), (k, f[k], fe)
        assert abs(f[k] - fs[-1]) <= 1e-6 * abs(fs[-1]), (k, f[k], fs[-1])
    return lam


MU = (0.0, 1e-4, 1e-3, 1e-2)


@pytest.mark.parametrize("grid,ndet,mu", [
    (16, 24, MU), (12, 20, (1e-2,)), (8, 16, (0.0, 0.3, 5.0)), (20, 28, MU + (0.1, 1.0, 3.0, 10.0)),
])
@pytest.mark.parametrize("iters,bar", [(1, 2e-5), (10, 1e-4)])
def test_iterations_match_the_oracle(grid, ndet, mu, iters, bar):
    pr = synth.pet_problem(grid, ndet, 11 + grid, mean_count=20.0)
    _check(pr.E, pr.y, pr.nbr_ptr, pr.nbr_idx, mu, iters, bar)


def test_ragged_columns_take_the_scalar_path():
    """p = 253 (not a multiple of 4: element loads, a partial last column
    block) with a chain neighbourhood, and d not a multiple of eight."""
    pr = synth.pet_problem(16, 24, 5)
    keep = np.arange(253)
    E = np.ascontiguousarray(pr.E[:, keep])
    ok = E.sum(axis=0) > 0
    assert ok.all()
    rows = np.arange(E.shape[0] - 3)
    E, y = np.ascontiguousarray(E[rows]), np.ascontiguousarray(pr.y[rows])
    p = E.shape[1]
    ptr = np.zeros(p + 1, np.int32)
    idx = []
    for j in range(p):
        for k in (j - 1, j + 1):
            if 0 <= k < p:
                idx.append(k)
        ptr[j + 1] = len(idx)
    _check(E, y, ptr, np.asarray(idx, np.int32), (0.0, 1e-3, 0.5), 10, 1e-4)


def test_tiny_problem():
    """d = 5 lines, p = 3 pixels, one isolated pixel (no neighbours)."""
    E = np.array([[1.0, 0.5, 0.0], [0.0, 1.0, 1.0], [0.3, 0.3, 0.3], [1.0, 0.0, 2.0],
                  [0.0, 0.0, 0.0]], np.float32)
    y = np.array([4.0, 7.0, 2.0, 0.0, 0.0], np.float32)
    ptr = np.array([0, 1, 2, 2], np.int32)
    idx = np.array([1, 0], np.int32)
    _check(E, y, ptr, idx, (0.0, 0.1, 2.0), 10, 1e-4)


def test_paper_size():
    """The paper's example shape (64 x 64 pixels, 2016 lines), the four
    penalty constants together, 20 iterations."""
    pr = synth.pet()
    _check(pr.E, pr.y, pr.nbr_ptr, pr.nbr_idx, pr.mu, 20, 1e-4)


def test_images_are_independent_and_deterministic():
    """Repeated runs are bitwise identical, and image k of a multi-image run
    is the single-image run with mu_k up to float32 rounding (the back
    projection splits the lines into as many segments as one wave of its
    blocks holds, and its register use, so that count, depends on the number
    of images: the float32 partial sums are grouped differently)."""
    pr = synth.pet_problem(16, 24, 3)
    lam, _, f = _gpu(pr.E, pr.y, pr.nbr_ptr, pr.nbr_idx, MU, 7)
    lam2, _, f2 = _gpu(pr.E, pr.y, pr.nbr_ptr, pr.nbr_idx, MU, 7)
    assert np.array_equal(lam, lam2) and np.array_equal(f, f2)
    for k, m in enumerate(MU):
        one, _, _ = _gpu(pr.E, pr.y, pr.nbr_ptr, pr.nbr_idx, (m,), 7)
        assert entry_rel_err(one[0], lam[k])[0] < 1e-5, k


def test_noise_free_counts_are_nearly_fixed():
    """y = E lambda* (no noise, in float64 then rounded to float32) and
    mu = 0: the EM map moves lambda* only by the rounding of y."""
    pr = synth.pet_problem(16, 24, 8)
    En = po.normalise_columns(pr.E)
    lam_star = np.random.default_rng(1).uniform(0.5, 4.0, pr.p)
    y = (En @ lam_star).astype(np.float32)
    lam, _, _ = _gpu(pr.E, y, pr.nbr_ptr, pr.nbr_idx, (0.0,), 5,
                     lam0=lam_star[None, :].astype(np.float32))
    assert entry_rel_err(lam[0], lam_star)[0] < 2e-5


def test_start_from_a_given_intensity():
    pr = synth.pet_problem(12, 20, 9)
    lam0 = np.random.default_rng(2).uniform(0.5, 2.0, (2, pr.p)).astype(np.float32)
    lam, _, _ = _gpu(pr.E, pr.y, pr.nbr_ptr, pr.nbr_idx, (0.0, 1e-2), 3, lam0=lam0)
    for k, m in enumerate((0.0, 1e-2)):
        lo, _, _ = po.run(pr.E, pr.y, m, pr.nbr_ptr, pr.nbr_idx, 3, lam0=lam0[k])
        assert entry_rel_err(lam[k], lo)[0] < 5e-5


def test_large_workload_sampled():
    """The 128 x 128, 8128-line workload (E 532 MB) in the benchmark's
    launch configuration: after 3 iterations, sampled pixels of the fourth
    against the oracle's update of the GPU's own third iterate, and the
    objective at the GPU's intensities against the oracle's."""
    import torch
    from paper_1003_3272_gb300 import nmf
    pr = synth.pet_large()
    Ed, yd = to_dev(pr.E), to_dev(pr.y)
    with nmf.PET(Ed, yd, pr.nbr_ptr, pr.nbr_idx, pr.mu) as m:
        m.step(3)
        lam3 = to_host(m.lam)
        m.step(1)
        lam4 = to_host(m.lam)
        f4 = m.objective()
    del Ed, yd
    torch.cuda.empty_cache()
    En = po.normalise_columns(pr.E)
    cols = np.sort(np.random.default_rng(0).choice(pr.p, 96, replace=False))
    prs = po.pairs(pr.nbr_ptr, pr.nbr_idx)
    for k, mu in enumerate(pr.mu):
        ref = po.update_pixels(En, pr.y, lam3[k], mu, pr.nbr_ptr, pr.nbr_idx, cols)
        assert entry_rel_err(lam4[k][cols], ref)[0] < 2e-5, k
        fe = po.objective(En, pr.y, lam4[k], mu, prs)
        assert abs(f4[k] - fe) <= 1e-9 * abs(fe), k


def test_run_stops_where_the_oracle_does():
    from paper_1003_3272_gb300 import nmf
    pr = synth.pet_problem(12, 20, 4)
    mu = (1e-2, 0.1)
    Ed, yd = to_dev(pr.E), to_dev(pr.y)
    with nmf.PET(Ed, yd, pr.nbr_ptr, pr.nbr_idx, mu) as m:
        done, f = m.run(100000, tol=1e-8, check_every=1)
    nds = []
    for k, mk in enumerate(mu):
        _, fs, nd = po.run(pr.E, pr.y, mk, pr.nbr_ptr, pr.nbr_idx, 100000, tol=1e-8)
        nds.append(nd)
        assert abs(f[k] - fs[-1]) <= 1e-6 * abs(fs[-1])
    assert abs(done - max(nds)) <= 2, (done, nds)


@pytest.mark.parametrize("what,status", [("E_negative", "ENONFINITE"), ("E_nan", "ENONFINITE"),
                                          ("zero_column", "EINVAL"), ("y_negative", "ENONFINITE"),
                                          ("lam_negative", "ENONFINITE")])
def test_bad_inputs_are_found_on_the_device(what, status):
    from paper_1003_3272_gb300 import nmf
    pr = synth.pet_problem(8, 16, 1)
    E, y = pr.E.copy(), pr.y.copy()
    lam0 = None
    if what == "E_negative":
        E[3, 5] = -1.0
    elif what == "E_nan":
        E[2, 7] = np.nan
    elif what == "zero_column":
        E[:, 9] = 0.0
    elif what == "y_negative":
        y[4] = -2.0
    else:
        lam0 = np.ones((1, pr.p), np.float32)
        lam0[0, 3] = -1.0
    lam = None if lam0 is None else to_dev(lam0)
    with pytest.raises(nmf.NMFError) as ei:
        nmf.PET(to_dev(E), to_dev(y), pr.nbr_ptr, pr.nbr_idx, (0.1,), lam=lam,
                init_ones=lam0 is None)
    assert ei.value.status == getattr(nmf, status)
