"""nmf_gram_noalloc: the Gram matrix of a factor without any allocation.

Callers that cannot call cudaMalloc (their device memory belongs to another
allocator, or cudaMalloc's possible device synchronisation is not allowed on
their path) use this entry point; its scratch is a static device array in
the library.  Expected values come from the float64 oracle alone.  This file
is collected last so that a run stopping at the first failure has run every
other test first; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from oracle import nmf_oracle as orc
from paper_1003_3272_gb300 import synth

pytestmark = pytest.mark.gpu

SCRATCH_FLOATS = 1 << 21     # the static scratch: ceil(M/128) r^2 + r^2 floats at most


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1003_3272_gb300 import build, nmf
    build.build()
    return nmf.load()


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _gram(lib, F, layout, M, ldf, r, out, stream):
    return lib.nmf_gram_noalloc(ctypes.c_void_p(F.data_ptr()), layout, M, ldf, r,
                                ctypes.c_void_p(out.data_ptr()), stream)


def test_gram_noalloc_matches_the_oracle_on_two_calls_in_a_row(lib):
    """W^T W, then H H^T, then W^T W again: each against the oracle's
    float64 Gram at the Gram tolerance of the parity tests (rtol 2e-6); the
    repeat gives the same bits (the scratch keeps the last call's contents,
    and every entry the kernels read is rewritten first)."""
    import torch
    from paper_1003_3272_gb300 import nmf
    pr = synth.uniform_problem(3000, 2000, 50, seed=31)
    W, H = _dev(pr.W0), _dev(pr.H0)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    gw = torch.full((50, 50), float("nan"), dtype=torch.float64, device="cuda")
    gh = torch.full((50, 50), float("nan"), dtype=torch.float64, device="cuda")
    gw2 = torch.full((50, 50), float("nan"), dtype=torch.float64, device="cuda")
    assert _gram(lib, W, 0, 3000, 50, 50, gw, st) == nmf.OK, lib.nmf_last_error(None)
    assert _gram(lib, H, 1, 2000, 2000, 50, gh, st) == nmf.OK, lib.nmf_last_error(None)
    assert _gram(lib, W, 0, 3000, 50, 50, gw2, st) == nmf.OK, lib.nmf_last_error(None)
    torch.cuda.synchronize()
    np.testing.assert_allclose(gw.cpu().numpy(), orc.gram_w(pr.W0), rtol=2e-6)
    np.testing.assert_allclose(gh.cpu().numpy(), orc.gram_h(pr.H0), rtol=2e-6)
    assert np.array_equal(gw2.cpu().numpy(), gw.cpu().numpy())


def test_gram_noalloc_at_the_scratch_limit(lib):
    """r = 128 and M = 127 * 128 need exactly 2^21 floats: the last tile's
    partial and the float32 Gram fill the end of the array.  One row more is
    rejected with NMF_EINVAL before anything is launched."""
    import torch
    from paper_1003_3272_gb300 import nmf
    r, M = 128, 127 * 128
    assert -(-M // 128) * r * r + r * r == SCRATCH_FLOATS
    rng = np.random.default_rng(5)
    W0 = rng.random((M + 1, r), dtype=np.float32)
    W = _dev(W0)
    out = torch.full((r, r), float("nan"), dtype=torch.float64, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert _gram(lib, W, 0, M, r, r, out, st) == nmf.OK, lib.nmf_last_error(None)
    torch.cuda.synchronize()
    np.testing.assert_allclose(out.cpu().numpy(), orc.gram_w(W0[:M]), rtol=2e-6)
    # layout 1 (H-like, r x M with a row pitch) at the same limit
    Ht = np.ascontiguousarray(W0[:M].T)
    Hd = _dev(Ht)
    out1 = torch.full((r, r), float("nan"), dtype=torch.float64, device="cuda")
    assert _gram(lib, Hd, 1, M, M, r, out1, st) == nmf.OK, lib.nmf_last_error(None)
    torch.cuda.synchronize()
    np.testing.assert_allclose(out1.cpu().numpy(), orc.gram_h(Ht), rtol=2e-6)
    assert _gram(lib, W, 0, M + 1, r, r, out, st) == nmf.EINVAL
    assert b"static scratch" in lib.nmf_last_error(None)


def test_gram_noalloc_rejects_bad_arguments(lib):
    import torch
    from paper_1003_3272_gb300 import nmf
    out = torch.zeros(128, 128, dtype=torch.float64, device="cuda")
    W = torch.zeros(200 * 128, 128, device="cuda")
    assert _gram(lib, W, 0, 200 * 128, 128, 128, out, None) == nmf.EINVAL
    assert lib.nmf_gram_noalloc(None, 0, 10, 4, 4, ctypes.c_void_p(out.data_ptr()),
                                None) == nmf.EINVAL
    assert _gram(lib, W, 0, 10, 5, 4, out, None) == nmf.EINVAL      # ldf != r
    assert _gram(lib, W, 2, 10, 4, 4, out, None) == nmf.EINVAL      # layout
