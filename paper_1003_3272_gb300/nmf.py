"""Thin ctypes binding of ``libnmf.so`` (declared in ``include/nmf.h``).

Argument marshalling only: every step of the MM iteration runs in the
library's sm_103a kernels.  PyTorch supplies device memory and streams.  If
the library is missing or cannot be loaded this module raises -- there is no
fallback of any kind.
"""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libnmf.so")

# nmf_status
OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ENONFINITE, EUNSUPPORTED = range(7)
# nmf_precision
FP32, TF32, BF16X3, BF16 = range(4)
PRECISIONS = {"fp32": FP32, "tf32": TF32, "bf16x3": BF16X3, "bf16": BF16}
# nmf_order
H_FIRST, W_FIRST = 0, 1
ORDERS = {"h_first": H_FIRST, "w_first": W_FIRST}
# nmf_model
GAUSSIAN, POISSON = 0, 1
MODELS = {"gaussian": GAUSSIAN, "poisson": POISSON}


class Config(ctypes.Structure):
    _fields_ = [
        ("p", ctypes.c_int64),
        ("n", ctypes.c_int64),
        ("r", ctypes.c_int32),
        ("eps", ctypes.c_float),
        ("prec", ctypes.c_int),
        ("order", ctypes.c_int),
        ("seed", ctypes.c_uint64),
        ("init_from_seed", ctypes.c_int32),
        ("validate", ctypes.c_int32),
        ("split_k", ctypes.c_int32),
        ("model", ctypes.c_int32),
    ]


EXPORTS = [
    "nmf_config_default", "nmf_init", "nmf_step", "nmf_half_step", "nmf_objective",
    "nmf_run", "nmf_read_gram", "nmf_solve", "nmf_destroy", "nmf_batched_init",
    "nmf_batched_step", "nmf_batched_objective", "nmf_batched_destroy",
    "nmf_status_str", "nmf_last_error", "nmf_version", "nmf_restart",
    "nmf_kernel_launches", "nmf_profile_enable", "nmf_profile_read", "nmf_gram_noalloc",
    "nmf_selfcheck_div", "nmf_test_expire_next_wait", "nmf_converge", "nmf_qn_run",
    "nmf_converge_resident",
    "nmf_batched_schedule", "nmf_batched_test_expire_next_wait",
    # include/pet.h: penalised PET reconstruction (Section 3.2, Algorithm 2)
    "pet_init", "pet_step", "pet_restart", "pet_objective", "pet_run", "pet_profile_enable",
    "pet_profile_read", "pet_destroy", "pet_last_error",
]

_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load the library (once).  Raises if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            f"libnmf.so not found at {path}; build it with "
            "`python -m paper_1003_3272_gb300.build` (needs nvcc)")
    lib = ctypes.CDLL(path)
    c_p, i64, i32, f32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_float
    cfgp = ctypes.POINTER(Config)
    sig = {
        "nmf_config_default": ([cfgp, i64, i64, i32], ctypes.c_int),
        "nmf_init": ([cfgp, c_p, c_p, c_p, c_p, ctypes.POINTER(c_p)], ctypes.c_int),
        "nmf_step": ([c_p, ctypes.c_int], ctypes.c_int),
        "nmf_half_step": ([c_p, ctypes.c_int], ctypes.c_int),
        "nmf_objective": ([c_p, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
        "nmf_run": ([c_p, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                     ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
        "nmf_converge": ([c_p, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                          ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)],
                         ctypes.c_int),
        "nmf_converge_resident": ([c_p, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                   ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)],
                                  ctypes.c_int),
        "nmf_qn_run": ([c_p, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                        ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                        ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
        "nmf_read_gram": ([c_p, ctypes.c_int, c_p], ctypes.c_int),
        "nmf_solve": ([cfgp, c_p, c_p, c_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double), c_p],
                      ctypes.c_int),
        "nmf_destroy": ([c_p], None),
        "nmf_batched_init": ([ctypes.c_int, cfgp, c_p, c_p, c_p, c_p, ctypes.POINTER(c_p)],
                             ctypes.c_int),
        "nmf_batched_step": ([c_p, ctypes.c_int], ctypes.c_int),
        "nmf_batched_objective": ([c_p, c_p], ctypes.c_int),
        "nmf_batched_destroy": ([c_p], None),
        "nmf_batched_schedule": ([c_p], ctypes.c_char_p),
        "nmf_batched_test_expire_next_wait": ([c_p], ctypes.c_int),
        "nmf_status_str": ([ctypes.c_int], ctypes.c_char_p),
        "nmf_last_error": ([c_p], ctypes.c_char_p),
        "nmf_version": ([], ctypes.c_char_p),
        "nmf_restart": ([c_p, ctypes.c_uint64], ctypes.c_int),
        "nmf_kernel_launches": ([], ctypes.c_uint64),
        "nmf_gram_noalloc": ([c_p, i32, i64, i64, i32, c_p, c_p], ctypes.c_int),
        "nmf_selfcheck_div": ([i64, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64),
                               ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
        "nmf_test_expire_next_wait": ([c_p], ctypes.c_int),
        "nmf_profile_enable": ([c_p, ctypes.c_int], ctypes.c_int),
        "nmf_profile_read": ([c_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                              ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
        "pet_init": ([i64, i64, c_p, c_p, c_p, c_p, i32, c_p, c_p, i32, c_p,
                      ctypes.POINTER(c_p)], ctypes.c_int),
        "pet_step": ([c_p, ctypes.c_int], ctypes.c_int),
        "pet_restart": ([c_p], ctypes.c_int),
        "pet_objective": ([c_p, c_p], ctypes.c_int),
        "pet_run": ([c_p, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                     ctypes.POINTER(ctypes.c_int), c_p], ctypes.c_int),
        "pet_profile_enable": ([c_p, ctypes.c_int], ctypes.c_int),
        "pet_profile_read": ([c_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                              ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
        "pet_destroy": ([c_p], None),
        "pet_last_error": ([c_p], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def kernel_launches() -> int:
    """Kernels launched by the library so far in this process."""
    return int(load().nmf_kernel_launches())


def selfcheck_div(count: int, seed: int = 1):
    """(mismatches, quick) of the update's division against the IEEE
    division over `count` operand pairs on the current device."""
    lib = load()
    mm, q = ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib.nmf_selfcheck_div(count, seed, ctypes.byref(mm), ctypes.byref(q)))
    return mm.value, q.value


class NMFError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


def _check(status: int, ctx=None):
    if status != OK:
        lib = load()
        why = lib.nmf_last_error(ctx).decode()
        raise NMFError(status, f"{lib.nmf_status_str(status).decode()}: {why}")


def make_config(p, n, r, eps=1e-10, prec="fp32", order="h_first", seed=0,
                init_from_seed=False, validate=False, split_k=0, model="gaussian") -> Config:
    lib = load()
    cfg = Config()
    _check(lib.nmf_config_default(ctypes.byref(cfg), int(p), int(n), int(r)))
    cfg.eps = float(eps)
    cfg.prec = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
    cfg.order = ORDERS[order] if isinstance(order, str) else int(order)
    cfg.seed = int(seed)
    cfg.init_from_seed = int(bool(init_from_seed))
    cfg.validate = int(bool(validate))
    cfg.split_k = int(split_k)
    cfg.model = MODELS[model] if isinstance(model, str) else int(model)
    return cfg


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _stream_handle(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class NMF:
    """An MM NMF context over device tensors V (p x n), W (p x r), H (r x n),
    all float32, contiguous, on the current CUDA device.  W and H are
    updated in place."""

    def __init__(self, V, W, H, eps=1e-10, prec="fp32", order="h_first", seed=0,
                 init_from_seed=False, validate=False, split_k=0, stream=None,
                 model="gaussian"):
        import torch
        for name, t in (("V", V), ("W", W), ("H", H)):
            if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
                raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
        p, n = V.shape
        r = W.shape[1]
        if W.shape != (p, r) or H.shape != (r, n):
            raise ValueError("shapes must be V (p, n), W (p, r), H (r, n)")
        self.lib = load()
        self.V, self.W, self.H = V, W, H
        self.p, self.n, self.r = p, n, r
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.cfg = make_config(p, n, r, eps, prec, order, seed, init_from_seed, validate,
                               split_k, model)
        ctx = ctypes.c_void_p()
        _check(self.lib.nmf_init(ctypes.byref(self.cfg), _ptr(V), _ptr(W), _ptr(H),
                                 _stream_handle(self.stream), ctypes.byref(ctx)))
        self.ctx = ctx

    def step(self, iters: int = 1):
        _check(self.lib.nmf_step(self.ctx, int(iters)), self.ctx)

    def half_step(self, which: int):
        _check(self.lib.nmf_half_step(self.ctx, int(which)), self.ctx)

    def objective(self) -> float:
        f = ctypes.c_double()
        _check(self.lib.nmf_objective(self.ctx, ctypes.byref(f)), self.ctx)
        return f.value

    def run(self, max_iters: int, tol: float = 1e-9, check_every: int = 1):
        done, f = ctypes.c_int(), ctypes.c_double()
        _check(self.lib.nmf_run(self.ctx, int(max_iters), float(tol), int(check_every),
                                ctypes.byref(done), ctypes.byref(f)), self.ctx)
        return done.value, f.value

    def converge(self, max_iters: int, tol: float = 1e-9, check_every: int = 1):
        """run() with the loop on the device (one CUDA graph with a while-node;
        the stopping test sets its condition).  Same results as run()."""
        done, f = ctypes.c_int(), ctypes.c_double()
        _check(self.lib.nmf_converge(self.ctx, int(max_iters), float(tol), int(check_every),
                                     ctypes.byref(done), ctypes.byref(f)), self.ctx)
        return done.value, f.value

    def converge_resident(self, max_iters: int, tol: float = 1e-9, check_every: int = 1):
        """converge() with every iteration in one persistent launch (small
        problems, NMF_FP32, r <= 16; see nmf_converge_resident).  Same rule
        and return values; float32 rounding differs from converge()."""
        done, f = ctypes.c_int(), ctypes.c_double()
        _check(self.lib.nmf_converge_resident(self.ctx, int(max_iters), float(tol),
                                              int(check_every), ctypes.byref(done),
                                              ctypes.byref(f)), self.ctx)
        return done.value, f.value

    def qn_run(self, q: int, max_iters: int, tol: float = 0.0):
        """Quasi-Newton acceleration with memory q (see nmf_qn_run).
        Returns (iterations, objective, quasi-Newton points taken)."""
        done, f, taken = ctypes.c_int(), ctypes.c_double(), ctypes.c_int()
        _check(self.lib.nmf_qn_run(self.ctx, int(q), int(max_iters), float(tol),
                                   ctypes.byref(done), ctypes.byref(f), ctypes.byref(taken)),
               self.ctx)
        return done.value, f.value, taken.value

    def expire_next_wait(self):
        """Test hook: the next half step's grid-wide waits run out (about
        3 s); the next synchronising call raises NMFError(ETIMEOUT)."""
        _check(self.lib.nmf_test_expire_next_wait(self.ctx), self.ctx)

    def restart(self, seed: int):
        """Algorithm 1's seeded start on the same V (no allocation)."""
        _check(self.lib.nmf_restart(self.ctx, int(seed)), self.ctx)

    def profile(self, on: bool = True):
        _check(self.lib.nmf_profile_enable(self.ctx, int(bool(on))), self.ctx)

    def profile_read(self, kind: int):
        """(total ms, launches) of one kind: 0 streaming products, 1 Gram
        reductions, 2 objective, 3 operand copies / seeding."""
        ms, cnt = ctypes.c_double(), ctypes.c_int64()
        _check(self.lib.nmf_profile_read(self.ctx, int(kind), ctypes.byref(ms),
                                         ctypes.byref(cnt)), self.ctx)
        return ms.value, cnt.value

    def gram(self, which: int):
        import numpy as np
        out = np.empty((self.r, self.r), dtype=np.float64)
        _check(self.lib.nmf_read_gram(self.ctx, int(which), out.ctypes.data_as(ctypes.c_void_p)),
               self.ctx)
        return out

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.nmf_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def solve(V, W, H, iters, eps=1e-10, prec="fp32", order="h_first", stream=None,
          split_k=0, model="gaussian") -> float:
    """One-call solve through ``nmf_solve``.  V, W, H are numpy float32 arrays
    (host; copied in and out inside the call, W and H overwritten) or CUDA
    tensors.  Returns the final objective."""
    import numpy as np
    lib = load()

    def ptr(a):
        if isinstance(a, np.ndarray):
            if not (a.dtype == np.float32 and a.flags.c_contiguous):
                raise ValueError("host arrays must be C-contiguous float32")
            return a.ctypes.data_as(ctypes.c_void_p)
        return _ptr(a)

    p, n = V.shape
    r = W.shape[1]
    cfg = make_config(p, n, r, eps, prec, order, split_k=split_k, model=model)
    f = ctypes.c_double()
    st = ctypes.c_void_p(stream.cuda_stream) if stream is not None else ctypes.c_void_p()
    _check(lib.nmf_solve(ctypes.byref(cfg), ptr(V), ptr(W), ptr(H), int(iters),
                         ctypes.byref(f), st))
    return f.value


class Batch:
    """Many independent MM NMF problems updated together by the grouped
    persistent kernel (``nmf_batched_*``).  ``Vs``, ``Ws``, ``Hs``: lists of
    contiguous float32 CUDA tensors."""

    def __init__(self, Vs, Ws, Hs, eps=1e-10, prec="fp32", stream=None):
        import torch
        self.lib = load()
        count = len(Vs)
        if not (len(Ws) == count and len(Hs) == count and count > 0):
            raise ValueError("need the same positive number of V, W, H tensors")
        cfgs = (Config * count)()
        for b in range(count):
            p, n = Vs[b].shape
            r = Ws[b].shape[1]
            cfgs[b] = make_config(p, n, r, eps, prec)
        arr = lambda ts: (ctypes.c_void_p * count)(*[t.data_ptr() for t in ts])
        self._keep = (Vs, Ws, Hs, cfgs)
        self.count = count
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        ctx = ctypes.c_void_p()
        _check(self.lib.nmf_batched_init(count, cfgs, arr(Vs), arr(Ws), arr(Hs),
                                         _stream_handle(self.stream), ctypes.byref(ctx)))
        self.ctx = ctx

    def step(self, iters: int = 1):
        _check(self.lib.nmf_batched_step(self.ctx, int(iters)))

    def objective(self):
        import numpy as np
        out = np.empty(self.count, dtype=np.float64)
        _check(self.lib.nmf_batched_objective(self.ctx, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    @property
    def schedule(self) -> str:
        """The autotuner's choice, "policy/grid"."""
        return self.lib.nmf_batched_schedule(self.ctx).decode()

    def expire_next_wait(self):
        """Test hook: the next iteration's bounded waits run out; the next
        objective() raises NMFError(ETIMEOUT)."""
        _check(self.lib.nmf_batched_test_expire_next_wait(self.ctx))

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.nmf_batched_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _pet_check(status: int, ctx=None):
    if status != OK:
        lib = load()
        why = lib.pet_last_error(ctx).decode()
        raise NMFError(status, f"{lib.nmf_status_str(status).decode()}: {why}")


class PET:
    """Penalised PET reconstruction (Section 3.2, Algorithm 2) through
    ``pet_*``: E (d x p) and y (d) contiguous float32 CUDA tensors (raw
    geometry and counts), the neighbourhood system as host CSR arrays
    (int32), one image per penalty constant in ``mu``.  ``lam`` (nimg x p
    float32 CUDA tensor) is updated in place; when None it is allocated and
    set to Algorithm 2's start lambda = 1."""

    def __init__(self, E, y, nbr_ptr, nbr_idx, mu, lam=None, init_ones=True, stream=None):
        import numpy as np
        import torch
        for name, t in (("E", E), ("y", y)):
            if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
                raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
        d, p = E.shape
        if y.shape != (d,):
            raise ValueError("y must have shape (d,)")
        mu = np.ascontiguousarray(np.atleast_1d(np.asarray(mu, dtype=np.float64)))
        k = len(mu)
        if lam is None:
            lam = torch.ones(k, p, device=E.device, dtype=torch.float32)
            init_ones = True
        if not (lam.is_cuda and lam.dtype == torch.float32 and lam.is_contiguous()
                and tuple(lam.shape) == (k, p)):
            raise ValueError("lam must be a contiguous float32 CUDA tensor of shape (nimg, p)")
        self.lib = load()
        self.E, self.y, self.lam, self.mu = E, y, lam, mu
        self.d, self.p, self.nimg = d, p, k
        self._ptr = np.ascontiguousarray(nbr_ptr, dtype=np.int32)
        self._idx = np.ascontiguousarray(nbr_idx, dtype=np.int32)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        ctx = ctypes.c_void_p()
        _pet_check(self.lib.pet_init(
            d, p, _ptr(E), _ptr(y), self._ptr.ctypes.data_as(ctypes.c_void_p),
            self._idx.ctypes.data_as(ctypes.c_void_p), k, mu.ctypes.data_as(ctypes.c_void_p),
            _ptr(lam), int(bool(init_ones)), _stream_handle(self.stream), ctypes.byref(ctx)))
        self.ctx = ctx

    def step(self, iters: int = 1):
        _pet_check(self.lib.pet_step(self.ctx, int(iters)), self.ctx)

    def restart(self):
        """Algorithm 2's start (lambda = 1) on the same inputs."""
        _pet_check(self.lib.pet_restart(self.ctx), self.ctx)

    def objective(self):
        import numpy as np
        out = np.empty(self.nimg, dtype=np.float64)
        _pet_check(self.lib.pet_objective(self.ctx, out.ctypes.data_as(ctypes.c_void_p)),
                   self.ctx)
        return out

    def run(self, max_iters: int, tol: float = 1e-9, check_every: int = 1):
        import numpy as np
        done = ctypes.c_int()
        out = np.empty(self.nimg, dtype=np.float64)
        _pet_check(self.lib.pet_run(self.ctx, int(max_iters), float(tol), int(check_every),
                                    ctypes.byref(done), out.ctypes.data_as(ctypes.c_void_p)),
                   self.ctx)
        return done.value, out

    def profile(self, on: bool = True):
        _pet_check(self.lib.pet_profile_enable(self.ctx, int(bool(on))), self.ctx)

    def profile_read(self, kind: int):
        """(total ms, launches): 0 forward projection, 1 back projection with
        the update, 2 objective."""
        ms, cnt = ctypes.c_double(), ctypes.c_int64()
        _pet_check(self.lib.pet_profile_read(self.ctx, int(kind), ctypes.byref(ms),
                                             ctypes.byref(cnt)), self.ctx)
        return ms.value, cnt.value

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.pet_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
