"""Host-side checks of the C-ABI library: it loads, exports every symbol
include/nmf.h declares, and rejects bad arguments before touching a GPU."""
import ctypes
import os
import re

import pytest

from paper_1003_3272_gb300 import build as nbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    nbuild.build()
    from paper_1003_3272_gb300 import nmf
    return nmf.load()


def _declared():
    names = []
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not f.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"\b((?:nmf|pet)_\w+)\s*\(", src)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "nmf_init" in names and "nmf_batched_step" in names and "pet_init" in names
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_the_header():
    from paper_1003_3272_gb300 import nmf
    assert sorted(nmf.EXPORTS) == _declared()


def test_status_strings_and_version(lib):
    for s in range(7):
        assert lib.nmf_status_str(s).decode().startswith("NMF_")
    assert b"sm_103a" in lib.nmf_version()


def test_config_struct_layout(lib):
    from paper_1003_3272_gb300 import nmf
    cfg = nmf.Config()
    assert lib.nmf_config_default(ctypes.byref(cfg), 10, 20, 3) == nmf.OK
    assert (cfg.p, cfg.n, cfg.r) == (10, 20, 3)
    assert cfg.eps == pytest.approx(1e-10)
    assert cfg.prec == nmf.FP32 and cfg.order == nmf.H_FIRST
    assert cfg.model == nmf.GAUSSIAN
    assert ctypes.sizeof(nmf.Config) == 56
    assert nmf.Config.model.offset == 52   # the last int32 of the header's struct


@pytest.mark.parametrize("model,prec,r,want", [
    (5, "fp32", 10, "EINVAL"),             # no such model
    ("poisson", "bf16", 10, "EUNSUPPORTED"),     # fp32 and bf16x3 only
    ("poisson", "tf32", 10, "EUNSUPPORTED"),
    ("poisson", "bf16x3", 65, "EUNSUPPORTED"),   # the tensor-core form: ranks up to 64
    ("poisson", "fp32", 65, "EUNSUPPORTED"),     # ranks up to 64
])
def test_model_requests_checked_on_the_host(lib, model, prec, r, want):
    from paper_1003_3272_gb300 import nmf
    cfg = nmf.make_config(100, 120, r, prec=prec, model=model)
    ctx = ctypes.c_void_p(123)
    dummy = ctypes.c_void_p(16)
    st = lib.nmf_init(ctypes.byref(cfg), dummy, dummy, dummy, None, ctypes.byref(ctx))
    assert st == getattr(nmf, want)
    assert ctx.value is None


def test_device_loop_rejects_bad_arguments(lib):
    from paper_1003_3272_gb300 import nmf
    done, f = ctypes.c_int(), ctypes.c_double()
    assert lib.nmf_converge(None, 10, 1e-9, 1, ctypes.byref(done), ctypes.byref(f)) == nmf.EINVAL
    assert lib.nmf_run(None, 10, 1e-9, 1, ctypes.byref(done), ctypes.byref(f)) == nmf.EINVAL
    assert lib.nmf_converge_resident(None, 10, 1e-9, 1, ctypes.byref(done),
                                     ctypes.byref(f)) == nmf.EINVAL


@pytest.mark.parametrize("bad", [
    dict(r=0), dict(r=129), dict(r=30, p=20), dict(r=30, n=20), dict(eps=-1.0),
    dict(eps=float("nan")), dict(prec=7), dict(order=5), dict(split_k=-2), dict(p=0),
])
def test_invalid_configs_are_rejected_on_the_host(lib, bad):
    from paper_1003_3272_gb300 import nmf
    args = dict(p=100, n=120, r=10)
    args.update({k: v for k, v in bad.items() if k in ("p", "n", "r")})
    cfg = nmf.Config()
    lib.nmf_config_default(ctypes.byref(cfg), args["p"], args["n"], args["r"])
    for k in ("eps", "prec", "order", "split_k"):
        if k in bad:
            setattr(cfg, k, bad[k])
    ctx = ctypes.c_void_p(123)
    dummy = ctypes.c_void_p(16)
    st = lib.nmf_init(ctypes.byref(cfg), dummy, dummy, dummy, None, ctypes.byref(ctx))
    assert st == nmf.EINVAL
    assert ctx.value is None
    assert len(lib.nmf_last_error(None)) > 0


def test_null_pointers_rejected(lib):
    from paper_1003_3272_gb300 import nmf
    cfg = nmf.Config()
    lib.nmf_config_default(ctypes.byref(cfg), 10, 10, 2)
    ctx = ctypes.c_void_p()
    assert lib.nmf_init(ctypes.byref(cfg), None, None, None, None, ctypes.byref(ctx)) == nmf.EINVAL
    assert lib.nmf_init(None, None, None, None, None, ctypes.byref(ctx)) == nmf.EINVAL
    assert lib.nmf_step(None, 1) == nmf.EINVAL
    assert lib.nmf_objective(None, None) == nmf.EINVAL
    assert lib.nmf_half_step(None, 0) == nmf.EINVAL
    lib.nmf_destroy(None)  # no-op


def test_batched_rejections_on_the_host(lib):
    from paper_1003_3272_gb300 import nmf
    cfgs = (nmf.Config * 2)()
    for i in range(2):
        lib.nmf_config_default(ctypes.byref(cfgs[i]), 100, 120, 10)
        cfgs[i].prec = nmf.BF16X3
    ptrs = (ctypes.c_void_p * 2)(16, 16)
    out = ctypes.c_void_p(123)
    # a rank above the grouped kernel's 32
    cfgs[1].r = 40
    assert lib.nmf_batched_init(2, cfgs, ptrs, ptrs, ptrs, None, ctypes.byref(out)) == nmf.EINVAL
    assert out.value is None
    cfgs[1].r = 10
    # mixed precisions
    cfgs[1].prec = nmf.TF32
    assert lib.nmf_batched_init(2, cfgs, ptrs, ptrs, ptrs, None, ctypes.byref(out)) == nmf.EINVAL
    # the float32 form is not a grouped tensor-core launch
    for i in range(2):
        cfgs[i].prec = nmf.FP32
    assert lib.nmf_batched_init(2, cfgs, ptrs, ptrs, ptrs, None, ctypes.byref(out)) == nmf.EUNSUPPORTED
    assert lib.nmf_batched_init(0, cfgs, ptrs, ptrs, ptrs, None, ctypes.byref(out)) == nmf.EINVAL
    assert lib.nmf_batched_step(None, 1) == nmf.EINVAL


def _pet_init(lib, d=6, p=4, nimg=1, mu=(0.0,), ptr=None, idx=None):
    import numpy as np
    if ptr is None:   # a chain 0-1-2-3
        ptr = [0, 1, 3, 5, 6]
    if idx is None:
        idx = [1, 0, 2, 1, 3, 2]
    ptr = np.asarray(ptr, dtype=np.int32)
    idx = np.asarray(idx, dtype=np.int32)
    mu = np.asarray(mu, dtype=np.float64)
    ctx = ctypes.c_void_p(123)
    dummy = ctypes.c_void_p(16)
    st = lib.pet_init(d, p, dummy, dummy, ptr.ctypes.data_as(ctypes.c_void_p),
                      idx.ctypes.data_as(ctypes.c_void_p), nimg,
                      mu.ctypes.data_as(ctypes.c_void_p), dummy, 1, None, ctypes.byref(ctx))
    return st, ctx


@pytest.mark.parametrize("bad", [
    dict(d=0), dict(p=0), dict(nimg=0, mu=()), dict(nimg=9, mu=(0.0,) * 9),
    dict(mu=(-1.0,)), dict(mu=(float("nan"),)), dict(mu=(float("inf"),)),
    dict(ptr=[1, 1, 3, 5, 6]),                               # does not start at 0
    dict(ptr=[0, 2, 1, 5, 6]),                               # decreasing
    dict(ptr=[0, 1, 3, 5, 6], idx=[1, 0, 2, 1, 3, 4]),       # out of range
    dict(ptr=[0, 1, 3, 5, 6], idx=[1, 1, 2, 1, 3, 2]),       # pixel 1 its own neighbour
    dict(ptr=[0, 1, 2, 4, 5], idx=[1, 2, 1, 3, 2]),          # 0 -> 1 without 1 -> 0
])
def test_pet_init_rejects_bad_arguments_on_the_host(lib, bad):
    from paper_1003_3272_gb300 import nmf
    st, ctx = _pet_init(lib, **bad)
    assert st == nmf.EINVAL
    assert ctx.value is None
    assert len(lib.pet_last_error(None)) > 0


def test_pet_null_arguments(lib):
    from paper_1003_3272_gb300 import nmf
    ctx = ctypes.c_void_p()
    assert lib.pet_init(4, 4, None, None, None, None, 1, None, None, 1, None,
                        ctypes.byref(ctx)) == nmf.EINVAL
    assert lib.pet_step(None, 1) == nmf.EINVAL
    assert lib.pet_objective(None, None) == nmf.EINVAL
    done = ctypes.c_int()
    assert lib.pet_run(None, 10, 1e-9, 1, ctypes.byref(done), None) == nmf.EINVAL
    lib.pet_destroy(None)  # no-op
