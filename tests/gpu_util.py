"""Helpers shared by the GPU parity tests (test code, not product code)."""
import numpy as np

from oracle import nmf_oracle as orc


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def to_host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def entry_rel_err(x_gpu, x_ref):
    """max and p99 of |x - ref| / max(|ref|, 1e-6 * max|ref|), plus the strict
    max without the floor."""
    x_gpu = np.asarray(x_gpu, np.float64)
    x_ref = np.asarray(x_ref, np.float64)
    floor = 1e-6 * np.max(np.abs(x_ref)) if x_ref.size else 0.0
    e = np.abs(x_gpu - x_ref) / np.maximum(np.abs(x_ref), floor)
    strict = np.abs(x_gpu - x_ref) / np.maximum(np.abs(x_ref), 1e-300)
    strict = strict[np.abs(x_ref) > 0]
    return (float(e.max()) if e.size else 0.0,
            float(np.percentile(e, 99)) if e.size else 0.0,
            float(strict.max()) if strict.size else 0.0)


def run_gpu(prob_V, W0, H0, iters, prec="fp32", order="h_first", eps=1e-10, split_k=0):
    """Run `iters` iterations through the C-ABI; returns (W, H, f) on host."""
    from paper_1003_3272_gb300 import nmf
    V, W, H = to_dev(prob_V), to_dev(W0), to_dev(H0)
    with nmf.NMF(V, W, H, eps=eps, prec=prec, order=order, split_k=split_k) as m:
        m.step(iters)
        f = m.objective()
    return to_host(W), to_host(H), f


def oracle_run(V, W0, H0, iters, order="h_first", eps=1e-10):
    W, H, _, _ = orc.run(V, W0, H0, iters, eps=eps, order=order)
    return W, H, orc.objective(V, W, H)
