"""nmf_gram_noalloc: the Gram matrix of a factor without any allocation.

Callers that cannot call cudaMalloc (their device memory belongs to another
allocator, or cudaMalloc's possible device synchronisation is not allowed on
their path) use this entry point; its scratch is a static device array in
the library.  This file is collected last so that a run stopping at the
first failure has run every other test first; it also passes on its own in
a fresh process.
"""
import ctypes

import numpy as np
import pytest

from paper_1003_3272_gb300 import synth

pytestmark = pytest.mark.gpu


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


def test_gram_noalloc_matches_context_grams(lib):
    """Two calls in a row (W^T W, then H H^T) agree with the Grams the
    context entry point (nmf_init / nmf_read_gram) formed from the same
    factors, within the Gram tolerance of the parity tests (rtol 2e-6)."""
    import torch
    from paper_1003_3272_gb300 import nmf
    pr = synth.uniform_problem(3000, 2000, 50, seed=31)
    V, W, H = _dev(pr.V), _dev(pr.W0), _dev(pr.H0)
    stream = torch.cuda.current_stream()
    with nmf.NMF(V, W, H) as m:
        ref_w, ref_h = m.gram(0), m.gram(1)
    gw = torch.full((50, 50), float("nan"), dtype=torch.float64, device="cuda")
    gh = torch.full((50, 50), float("nan"), dtype=torch.float64, device="cuda")
    st = ctypes.c_void_p(stream.cuda_stream)
    s1 = lib.nmf_gram_noalloc(ctypes.c_void_p(W.data_ptr()), 0, 3000, 50, 50,
                              ctypes.c_void_p(gw.data_ptr()), st)
    s2 = lib.nmf_gram_noalloc(ctypes.c_void_p(H.data_ptr()), 1, 2000, 2000, 50,
                              ctypes.c_void_p(gh.data_ptr()), st)
    assert s1 == nmf.OK and s2 == nmf.OK, lib.nmf_last_error(None)
    torch.cuda.synchronize()
    np.testing.assert_allclose(gw.cpu().numpy(), ref_w, rtol=2e-6)
    np.testing.assert_allclose(gh.cpu().numpy(), ref_h, rtol=2e-6)
    # the scratch keeps the last call's contents: a repeat gives the same bits
    s3 = lib.nmf_gram_noalloc(ctypes.c_void_p(W.data_ptr()), 0, 3000, 50, 50,
                              ctypes.c_void_p(gh.data_ptr()), st)
    assert s3 == nmf.OK
    torch.cuda.synchronize()
    assert np.array_equal(gh.cpu().numpy(), gw.cpu().numpy())


def test_gram_noalloc_rejects_sizes_beyond_the_scratch(lib):
    import torch
    from paper_1003_3272_gb300 import nmf
    W = torch.zeros(200 * 128, 128, device="cuda")  # large enough even if launched
    out = torch.zeros(128, 128, dtype=torch.float64, device="cuda")
    # ceil(M/128) * 128^2 + 128^2 > 2^21 once M > 127 * 128
    st = lib.nmf_gram_noalloc(ctypes.c_void_p(W.data_ptr()), 0, 200 * 128, 128, 128,
                              ctypes.c_void_p(out.data_ptr()), None)
    assert st == nmf.EINVAL
    assert b"static scratch" in lib.nmf_last_error(None)
    st = lib.nmf_gram_noalloc(None, 0, 10, 4, 4, ctypes.c_void_p(out.data_ptr()), None)
    assert st == nmf.EINVAL
