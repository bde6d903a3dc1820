"""Benchmark of the GB300 MM-NMF library on the planted low-rank workload.

Workload (one "step" = one full pass of the hot path): on V = W* H* + |N(0,
0.01^2)| (8192 x 8192, W*, H* iid Gamma(1,1), rank 50) the step restarts from
Algorithm 1's seeded uniform(0,1) start (operand copies of V, seeded W and H,
starting Grams), runs 200 MM iterations (each: W^T V stream + H update +
Gram, V H^T stream + W update + Gram), evaluates the objective ||V - WH||_F^2
and applies the relative-change stopping test.  Metric: MM updates (full
iterations) per second, aggregated over all GPUs; each GPU solves its own
replica (weak scaling, no collective in the data path).

The headline line is the split-BF16x3 tensor-core form (the form that meets
the 1e-5 relative objective bar); `by_precision` reports the plain FP32 form
and TF32 / BF16 on the same workload, `batched` the 512-instance batched
workload (grouped persistent launches), `accuracy` each form's objective
error against the FP64 oracle, `converge` Section 3's protocol (iterate to a
relative objective change below 1e-9, testing every iteration) on the
CBCL-shaped 361 x 2429, r = 10 workload with the loop on the host and on
the device (one CUDA graph), `poisson` the paper's Poisson variant (the
simultaneous square-root update) on an 8192 x 8192, r = 50 counts matrix.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU
oracle instead (the reference arm), on a bounded sample of the same workload.

`--workload` selects one of the other measured matrices instead of the
planted one (same step: restart + the workload's iterations + objective):
  faces   361 x 2429, V iid uniform [0,1), r = 10, 50 iterations
  tall    65536 x 4096, V iid uniform [0,1), r = --rank (16/32/64/128),
          20 iterations (the precision sweep)
  large   131072 x 16384, V iid Exponential(1), r = 64, 20 iterations
  batched 512 independent problems (p, n in 64..2048, r in 4..32),
          100 iterations per step through the grouped batched launches
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "NMF MM updates/s & % roofline: plain FP32 vs mixed-prec/batched @1e-5 rel obj"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                  "sm_max_mhz": 2070.0}
SMS = 152
FFMA_PER_SM_PER_CLK = 128


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        d["_source"] = "measured"
        return d
    d = dict(PEAKS_FALLBACK)
    d["_source"] = "fallback"
    return d


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region.

    nvidia-smi is started before the warm-up and its first sample awaited, so
    its start-up (which takes driver locks) does not fall inside the timed
    region; only samples taken inside the window given to stop() count."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self._t = None

    def start(self, wait_s=10.0):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except OSError:
            self.proc = None
            return
        t0 = time.perf_counter()
        while not self.lines and time.perf_counter() - t0 < wait_s and self.proc.poll() is None:
            time.sleep(0.02)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def stop(self, window=None):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self._t:
            self._t.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = self.lines
        if window is not None:
            inside = [x for x in lines if window[0] <= x[0] <= window[1] + 0.15]
            lines = inside if inside else lines[-1:]
        for _, ln in lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(n_gpus, backend=None):
    """One process per GPU (torchrun's RANK / LOCAL_RANK / WORLD_SIZE); NCCL
    on GPUs, gloo where there is none (the host-side logic's tests)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        if backend is None:
            backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, ws):
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, seconds, ws):
    """Whole-job throughput of `ws` replicas: the units all ranks processed
    over the slowest rank's time (the time is already the max over ranks)."""
    return units_per_rank * ws / seconds


def algorithmic(prec, p, n, r):
    """Algorithmic bytes and flops of one V-streaming launch (either half):
    the V operand once in the precision's format, the other factor's plane,
    the updated factor read and written (plus its operand plane), and
    2 p n r product flops + 2 M r^2 denominator flops (M = p or n; averaged)."""
    vb = {"fp32": 4, "tf32": 4, "bf16x3": 4, "bf16": 2}[prec]
    yb = vb
    m_avg = (p + n) / 2
    bytes_ = p * n * vb + m_avg * r * yb + m_avg * r * (4 + 4 + yb)
    flops = 2.0 * p * n * r + 2.0 * m_avg * r * r
    return bytes_, flops


# The device code of each kernel whose DRAM traffic is recorded: its own
# translation unit and the headers with device code it includes (host-only
# declarations, nmf_internal.cuh, are left out: they change no kernel).
KERNEL_SOURCES = {
    "k_stream_tc": ["k_stream_tc.cu", "tc_epi.cuh", "tc_ptx.cuh", "epilogue.cuh", "tc.cuh",
                    "nmf_device.cuh"],
    "k_stream_f32": ["k_stream_f32.cu", "tc_epi.cuh", "tc_ptx.cuh", "epilogue.cuh", "tc.cuh",
                     "nmf_device.cuh"],
}


def kernel_source_digest(kernel="k_stream_tc"):
    """sha256 over one kernel's device sources: a recorded ncu traffic figure
    is used only while the kernel is unchanged since its capture."""
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_1003_3272_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def read_traffic(kernel_key):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum)
    from the committed ncu summary, or None when absent or stale."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        with open(path) as fh:
            d = json.load(fh).get(kernel_key)
    except (OSError, ValueError):
        return None
    kernel = kernel_key.split("/")[0]
    if not d or kernel not in KERNEL_SOURCES or d.get("kernel_digest") != kernel_source_digest(kernel):
        return None
    return d.get("traffic_bytes_per_launch")


def make_problem(args):
    """(problem, workload name, data description) for --workload."""
    from paper_1003_3272_gb300 import synth
    if args.workload == "planted":
        pr = synth.planted(iters=args.iters)
        return pr, "planted_8192x8192_r50", "synthetic (seeded planted low-rank matrix; no dataset)"
    if args.workload == "faces":
        pr = synth.faces()
        return pr, pr.name, "synthetic (seeded iid uniform [0,1), faces-matrix shape; no dataset)"
    if args.workload == "tall":
        pr = synth.tall(args.rank)
        return pr, pr.name, "synthetic (seeded iid uniform [0,1); no dataset)"
    pr = synth.large()
    return pr, pr.name, "synthetic (seeded iid Exponential(1); no dataset)"


def time_planted(pr, prec, steps, warmup, ws, local, sample_clocks=False, profile=True,
                 V_dev=None):
    """Time `steps` benchmark steps of one precision on problem `pr` (the
    planted problem unless --workload says otherwise).  Returns the
    measurement dict (updates/s, per-launch stream time, ...).  `V_dev`: V
    already on the device (else it is copied from pr.V)."""
    import torch
    from paper_1003_3272_gb300 import nmf
    p, n, r, iters = pr.p, pr.n, pr.r, pr.iters
    seed = pr.seed
    V = V_dev if V_dev is not None else torch.from_numpy(pr.V).cuda()
    W = torch.empty(p, r, device="cuda")
    H = torch.empty(r, n, device="cuda")
    stream = torch.cuda.current_stream()
    ctx = nmf.NMF(V, W, H, eps=pr.eps, prec=prec, seed=seed, init_from_seed=True,
                  stream=stream)
    f_prev = [None]

    def step():
        ctx.restart(seed)
        ctx.step(iters)
        f = ctx.objective()
        # Section 3's stopping statistic on successive objective evaluations
        if f_prev[0] is not None:
            _ = abs(f - f_prev[0]) / (abs(f_prev[0]) + 1.0) < 1e-9
        f_prev[0] = f
        return f

    sampler = ClockSampler(local) if sample_clocks else None
    if sampler:
        sampler.start()
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    if profile:
        ctx.profile(True)
    barrier(ws)
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    l0 = nmf.kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fs = [step() for _ in range(steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    w1 = time.perf_counter()
    launches = nmf.kernel_launches() - l0
    barrier(ws)
    clocks = sampler.stop((w0, w1)) if sampler else None
    ms = max_over_ranks(e0.elapsed_time(e1), ws)
    res = {"prec": prec, "ms": ms, "steps": steps, "launches": int(launches),
           "clocks": clocks, "objective": fs[-1],
           "value": job_rate(iters * steps, ms / 1e3, ws)}
    if profile:
        res["kinds"] = {k: ctx.profile_read(i) for i, k in
                        enumerate(["stream_products", "gram_reductions", "objective", "restart"])}
        ctx.profile(False)
    ctx.close()
    del V, W, H
    torch.cuda.empty_cache()
    return res


def roofline(prec, p, n, r, res, clocks, workload="planted_8192x8192_r50"):
    pk = peaks()
    bytes_l, flops_l = algorithmic(prec, p, n, r)
    st_ms, st_n = res["kinds"]["stream_products"]
    avg_s = (st_ms / max(st_n, 1)) / 1e3
    if prec == "fp32":
        mhz = (clocks or {}).get("sm_mhz") or pk.get("sm_max_mhz", 2070.0)
        peak = SMS * FFMA_PER_SM_PER_CLK * 2 * mhz * 1e6 / 1e12
        achieved = flops_l / avg_s / 1e12
        roof = {"bound": "alu", "achieved": round(achieved, 2), "peak": round(peak, 2),
                "unit": "TFLOP/s", "frac": round(achieved / peak, 4),
                "peak_source": f"152 SMs x 128 FP32 FMA/clk x 2 x {mhz:.0f} MHz "
                               "(median sampled SM clock)",
                "kernel": "k_stream_f32"}
    else:
        peak = pk["hbm_gbs"]
        achieved = bytes_l / avg_s / 1e9
        roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4),
                "peak_source": f"{pk['_source']} hbm_gbs (copy bandwidth, MEASURED_PEAKS.json)",
                "kernel": "k_stream_tc"}
    roof["traffic"] = read_traffic(f"{roof['kernel']}/{prec}/{workload}")
    roof["algorithmic_bytes_per_launch"] = int(bytes_l)
    roof["algorithmic_flops_per_launch"] = float(flops_l)
    roof["avg_launch_us"] = round(avg_s * 1e6, 2)
    roof["launches_timed"] = int(st_n)
    return roof


def pass_bounds(prec, p, n, r, value):
    """The whole-step update rate against the two HBM bounds of an
    iteration: V streamed twice (the H and the W update each read it once;
    the bound of record) and V streamed once (an iteration that keeps column
    panels of V in L2 between the two products).  Each bound is the measured
    copy bandwidth over the algorithmic bytes of one or two streaming
    launches; `value` includes everything else a step does, so each fraction
    is a lower bound on the streams' own."""
    pk = peaks()
    bytes_l, _ = algorithmic(prec, p, n, r)
    two = pk["hbm_gbs"] * 1e9 / (2.0 * bytes_l)
    one = pk["hbm_gbs"] * 1e9 / bytes_l
    return {"unit": "updates/s", "bytes_per_pass": int(bytes_l), "peak_gbs": pk["hbm_gbs"],
            "two_pass": {"bound": round(two, 1), "frac": round(value / two, 4)},
            "one_pass": {"bound": round(one, 1), "frac": round(value / one, 4)}}


def batched_stored_objectives():
    """The float64 oracle's objectives after 100 iterations of sampled
    instances of the batched workload, from tests/golden/batched_objectives.json
    (written by tests/golden/make_batched_objectives.py from the oracle
    alone), or None."""
    path = os.path.join(ROOT, "tests", "golden", "batched_objectives.json")
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return None


def time_singles(probs, prec, iters, Vs):
    """The same instances one at a time, each through its own context and
    nmf_step (two launches per iteration each): the comparison for the
    grouped launch.  Returns instance-iterations/s."""
    import torch
    from paper_1003_3272_gb300 import nmf
    stream = torch.cuda.current_stream()
    ctxs, facs = [], []
    for pr, V in zip(probs, Vs):
        W = torch.from_numpy(pr.W0).cuda()
        H = torch.from_numpy(pr.H0).cuda()
        facs.append((W, H))
        ctxs.append(nmf.NMF(V, W, H, eps=pr.eps, prec=prec, stream=stream))
    for m in ctxs:
        m.step(1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for m in ctxs:
        m.step(iters)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    for m in ctxs:
        m.close()
    del facs
    torch.cuda.empty_cache()
    return len(probs) * iters / (ms / 1e3)


def time_batched(prec, steps, warmup, iters, ws, singles=True):
    """The batched workload: 512 independent problems (p, n in 64..2048, r in
    4..32), `iters` MM iterations per step through nmf_batched_step (one
    grouped persistent launch per half step, CUDA graph; the timing does not
    depend on the values).  Beside it the same instances one by one through nmf_step
    in plain FP32 and in the same precision, and the objective error after
    100 iterations against the stored oracle values of sampled instances."""
    import numpy as np
    import torch
    from paper_1003_3272_gb300 import nmf, synth
    probs = synth.batch(iters=iters)
    Vs = [torch.from_numpy(pr.V).cuda() for pr in probs]
    W0 = [torch.from_numpy(pr.W0).cuda() for pr in probs]
    H0 = [torch.from_numpy(pr.H0).cuda() for pr in probs]
    Ws = [w.clone() for w in W0]
    Hs = [h.clone() for h in H0]
    b = nmf.Batch(Vs, Ws, Hs, prec=prec)
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        b.step(iters)
    torch.cuda.synchronize()
    barrier(ws)
    l0 = nmf.kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        b.step(iters)
    e1.record(stream)
    torch.cuda.synchronize()
    launches = nmf.kernel_launches() - l0
    ms = max_over_ranks(e0.elapsed_time(e1), ws)
    schedule = b.schedule
    b.close()
    # accuracy: 100 iterations from the seeded start, sampled instances
    acc = None
    stored = batched_stored_objectives()
    if stored:
        for w, w0 in zip(Ws, W0):
            w.copy_(w0)
        for h, h0 in zip(Hs, H0):
            h.copy_(h0)
        b2 = nmf.Batch(Vs, Ws, Hs, prec=prec)
        b2.step(stored["iters"])
        f = b2.objective()
        b2.close()
        errs = {k: abs(f[int(k)] - v) / v for k, v in stored["objective"].items()}
        acc = {"iterations": stored["iters"], "instances": sorted(int(k) for k in errs),
               "max": float(f"{max(errs.values()):.3e}"),
               "median": float(f"{np.median(list(errs.values())):.3e}"),
               "source": "tests/golden/batched_objectives.json (float64 oracle, "
                         "tests/golden/make_batched_objectives.py)"}
    vb = {"fp32": 4, "tf32": 4, "bf16x3": 4, "bf16": 2}[prec]
    bytes_it = sum(2 * pr.p * pr.n * vb for pr in probs)
    per_it_s = ms / 1e3 / (steps * iters)
    value = len(probs) * iters * steps * ws / (ms / 1e3)
    out = {"metric": "instance MM iterations/s", "precision": prec, "instances": len(probs),
           "iters_per_step": iters, "steps": steps, "ms_per_step": round(ms / steps, 3),
           "value": round(value, 1), "unit": "instance-iterations/s",
           "aggregate_gbs": round(bytes_it / per_it_s / 1e9, 1),
           "hbm_frac": round(bytes_it / per_it_s / 1e9 / peaks()["hbm_gbs"], 4),
           "V_bytes_per_iteration": int(bytes_it), "gpu_launches": int(launches),
           "schedule": schedule, "rel_objective_error_vs_fp64_oracle": acc,
           "config": "synth.batch(): 512 instances, p,n ~ U{64..2048}, r ~ U{4..32}, "
                     "V ~ U[0,1), seeded"}
    if singles:
        sing = {}
        for sp in ("fp32", prec):
            rate = time_singles(probs, sp, max(2, iters // 10), Vs)
            sing[sp] = {"value": round(rate, 1), "unit": "instance-iterations/s",
                        "api": f"one context per instance, nmf_step, {sp}"}
        out["one_by_one"] = sing
        out["speedup_vs_fp32"] = round(value / sing["fp32"]["value"], 2)
        out["speedup_vs_one_by_one_same_precision"] = round(value / sing[prec]["value"], 2)
    del Vs, Ws, Hs, W0, H0
    torch.cuda.empty_cache()
    return out


def time_poisson_prec(ws, clocks, prec, steps=3, iters=10):
    """The Poisson model of Section 3.1 (simultaneous square-root MM update)
    on the counts workload (8192 x 8192 counts ~ Poisson(W* H*), mean 5,
    r = 50) in one precision: iterations/s through nmf_step with the inputs
    resident.  fp32: 8pnr flops per iteration on the float32 FMA pipes
    (b = WH formed once per pass, two passes) against the FFMA peak at the
    sampled clock.  bf16x3: the contractions run on the tensor cores and
    each iteration streams V twice, 2 x 4pn bytes, against the measured HBM
    copy bandwidth (the whole iteration's time: both passes and the fused
    update)."""
    import torch
    from paper_1003_3272_gb300 import nmf, synth
    pr = synth.counts()
    p, n, r = pr.p, pr.n, pr.r
    V = torch.from_numpy(pr.V).cuda()
    W = torch.from_numpy(pr.W0).cuda()
    H = torch.from_numpy(pr.H0).cuda()
    stream = torch.cuda.current_stream()
    with nmf.NMF(V, W, H, eps=pr.eps, model="poisson", prec=prec, seed=pr.seed,
                 stream=stream) as m:
        L0 = m.objective()
        m.step(2)
        torch.cuda.synchronize()
        m.profile(True)
        barrier(ws)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            m.step(iters)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = max_over_ranks(e0.elapsed_time(e1), ws)
        it_ms, it_n = m.profile_read(0)
        m.profile(False)
        L1 = m.objective()
    done = steps * iters
    per_it = it_ms / max(1, it_n)
    pk = peaks()
    if prec == "fp32":
        flops = 8.0 * p * n * r
        mhz = (clocks or {}).get("sm_mhz") or pk.get("sm_max_mhz", 2070.0)
        peak = SMS * FFMA_PER_SM_PER_CLK * 2 * mhz * 1e6 / 1e12
        achieved = flops / (per_it * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": round(achieved, 2), "peak": round(peak, 1),
                "unit": "TFLOP/s", "frac": round(achieved / peak, 4),
                "peak_source": "152 SMs x 128 FFMA x 2 x sampled SM clock",
                "flops_per_iteration": flops}
    else:
        nbytes = 2.0 * 4 * p * n
        achieved = nbytes / (per_it * 1e-3) / 1e9
        peak = pk["hbm_gbs"]
        roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": round(peak, 1),
                "unit": "GB/s", "frac": round(achieved / peak, 4),
                "peak_source": f"{pk['_source']} hbm_gbs (copy bandwidth, MEASURED_PEAKS.json)",
                "bytes_per_iteration": nbytes}
    del V, W, H
    torch.cuda.empty_cache()
    return {"precision": prec, "iterations": done,
            "value": round(job_rate(done, ms / 1e3, ws), 1), "unit": "iterations/s",
            "ms_per_iteration": round(per_it, 4), "roofline": roof,
            "loglik_start": L0, "loglik_end": L1}


def time_poisson(ws, clocks):
    """Both forms of the Poisson model on the counts workload, each from the
    same start for the same number of iterations; the BF16x3 form's
    loglikelihood is reported relative to the float32 form's."""
    from paper_1003_3272_gb300 import synth
    by = {prec: time_poisson_prec(ws, clocks, prec) for prec in ("fp32", "bf16x3")}
    ref = by["fp32"]["loglik_end"]
    by["bf16x3"]["loglik_rel_diff_vs_fp32"] = abs(by["bf16x3"]["loglik_end"] - ref) / abs(ref)
    by["bf16x3"]["speedup_vs_fp32"] = round(by["bf16x3"]["value"] / by["fp32"]["value"], 2)
    return {"workload": synth.COUNTS["name"] + " (counts ~ Poisson(W* H*), mean 5)",
            "model": "poisson", "by_precision": by}


def pet_stored_objectives(name):
    """The float64 oracle's objectives per penalty constant on a PET
    workload, from tests/golden/pet_objectives.json (written by
    tests/golden/make_pet_objectives.py from the oracle alone), or None."""
    path = os.path.join(ROOT, "tests", "golden", "pet_objectives.json")
    try:
        with open(path) as fh:
            return json.load(fh)[name]
    except (OSError, ValueError, KeyError):
        return None


def time_pet(ws, steps=3):
    """Penalised PET reconstruction (Section 3.2, Algorithm 2) through
    pet_step, inputs resident: the paper's example shape (64 x 64 pixels,
    2016 lines, E 33 MB: L2-resident, so launch- and latency-bound) and a
    larger scanner (128 x 128 pixels, 8128 lines, E 532 MB: HBM-bound), each
    with the four penalty constants reconstructed together (one pass over E
    serves all four) and with one image alone.  One step = the workload's
    iterations from lambda = 1.  Per iteration the two kernels each stream E
    once: 4 d p bytes each (plus vectors of d and p), the roofline's
    algorithmic bytes per launch."""
    import numpy as np
    import torch
    from paper_1003_3272_gb300 import nmf, synth
    pk = peaks()
    out = {}
    stream = torch.cuda.current_stream()
    for build in (synth.pet, synth.pet_large):
        pr = build()
        E = torch.from_numpy(pr.E).cuda()
        y = torch.from_numpy(pr.y).cuda()
        ent = {"d": pr.d, "p": pr.p, "iters_per_step": pr.iters,
               "E_bytes": int(pr.E.nbytes), "l2_resident": bool(pr.E.nbytes < 100e6)}
        stored = pet_stored_objectives(pr.name)
        for mu in (pr.mu, pr.mu[-1:]):
            k = len(mu)
            lam = torch.ones(k, pr.p, device="cuda")
            with nmf.PET(E, y, pr.nbr_ptr, pr.nbr_idx, mu, lam=lam, stream=stream) as m:
                m.step(2)                                   # warm-up
                torch.cuda.synchronize()
                m.profile(True)
                barrier(ws)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                fs = None
                e0.record(stream)
                for _ in range(steps):
                    m.restart()                             # Algorithm 2's start
                    m.step(pr.iters)
                e1.record(stream)
                torch.cuda.synchronize()
                ms = max_over_ranks(e0.elapsed_time(e1), ws)
                fw_ms, fw_n = m.profile_read(0)
                bk_ms, bk_n = m.profile_read(1)
                m.profile(False)
                fs = m.objective()
            its = steps * pr.iters
            bytes_l = 4.0 * pr.d * pr.p + 4.0 * k * (pr.d + pr.p)
            fw_us = fw_ms / max(fw_n, 1) * 1e3
            bk_us = bk_ms / max(bk_n, 1) * 1e3
            leg = {"images": k, "mu": list(mu),
                   "value": round(job_rate(its * k, ms / 1e3, ws), 1),
                   "unit": "image-iterations/s",
                   "iterations_per_s": round(job_rate(its, ms / 1e3, ws), 1),
                   "ms_per_iteration": round(ms / its, 5),
                   "forward_us": round(fw_us, 2), "back_us": round(bk_us, 2),
                   "roofline": {"bound": "hbm", "unit": "GB/s", "peak": pk["hbm_gbs"],
                                "algorithmic_bytes_per_launch": int(bytes_l),
                                "achieved_forward": round(bytes_l / (fw_us * 1e-6) / 1e9, 1),
                                "achieved_back": round(bytes_l / (bk_us * 1e-6) / 1e9, 1),
                                "frac_forward": round(bytes_l / (fw_us * 1e-6) / 1e9 / pk["hbm_gbs"], 4),
                                "frac_back": round(bytes_l / (bk_us * 1e-6) / 1e9 / pk["hbm_gbs"], 4),
                                "frac_iteration": round(2 * bytes_l / (ms / its * 1e-3) / 1e9
                                                        / pk["hbm_gbs"], 4),
                                "traffic": None},
                   "objective": [float(v) for v in fs]}
            if stored and stored.get("iters") == pr.iters:
                errs = []
                for kk, mk in enumerate(mu):
                    fo = stored["objective"][repr(float(mk))][str(pr.iters)]
                    errs.append(float(f"{abs(fs[kk] - fo) / abs(fo):.3e}"))
                leg["rel_objective_error_vs_fp64_oracle"] = errs
            ent["images_%d" % k] = leg
        out[pr.name] = ent
        del E, y
        torch.cuda.empty_cache()
    return out


def time_converge(ws, prec="fp32", tol=1e-9, max_iters=100000):
    """Section 3's protocol on the CBCL-shaped workload (faces 361 x 2429,
    r = 10): iterate until the relative objective change drops below tol
    (1e-9) or max_iters (1e5), testing after every iteration, once with the
    loop on the host (nmf_run: one synchronisation per test) and once on the
    device (nmf_converge: one CUDA graph, one synchronisation)."""
    import numpy as np
    import torch
    from paper_1003_3272_gb300 import nmf, synth
    pr = synth.faces()
    res = {}
    finals = {}
    for method in ("converge", "run"):
        V = torch.from_numpy(pr.V).cuda()
        W = torch.from_numpy(pr.W0).cuda()
        H = torch.from_numpy(pr.H0).cuda()
        with nmf.NMF(V, W, H, eps=pr.eps, prec=prec) as m:
            t0 = time.perf_counter()
            getattr(m, method)(1, tol=tol, check_every=1)    # builds the graph (converge)
            tb = time.perf_counter() - t0
            m.restart(synth.BASE_SEED)                       # a fresh seeded start
            torch.cuda.synchronize()
            barrier(ws)
            t0 = time.perf_counter()
            done, f = getattr(m, method)(max_iters, tol=tol, check_every=1)
            te = max_over_ranks(time.perf_counter() - t0, ws)
            finals[method] = (done, f, W.cpu().numpy(), H.cpu().numpy())
        res[method] = {"iterations": done, "seconds": round(te, 4),
                       "iters_per_s": round(done * ws / te, 1), "objective": f,
                       "first_call_ms": round(tb * 1e3, 2)}
    a, b = finals["converge"], finals["run"]
    resident = None
    if prec == "fp32":
        # every iteration in one persistent launch (nmf_converge_resident):
        # float32 rounding differs from the streaming kernels', so its count
        # and objective are reported beside the device loop's
        V = torch.from_numpy(pr.V).cuda()
        W = torch.from_numpy(pr.W0).cuda()
        H = torch.from_numpy(pr.H0).cuda()
        with nmf.NMF(V, W, H, eps=pr.eps, prec=prec) as m:
            m.converge_resident(1, tol=tol, check_every=1)
            m.restart(synth.BASE_SEED)
            torch.cuda.synchronize()
            barrier(ws)
            t0 = time.perf_counter()
            done, f = m.converge_resident(max_iters, tol=tol, check_every=1)
            te = max_over_ranks(time.perf_counter() - t0, ws)
        resident = {"iterations": done, "seconds": round(te, 4),
                    "iters_per_s": round(done * ws / te, 1), "objective": f,
                    "rel_objective_diff_vs_device_loop": float(f"{abs(f - a[1]) / a[1]:.3e}"),
                    "over_device_loop": round(res["converge"]["seconds"] / te, 2)}
    return {"workload": "faces_361x2429_r10 (seeded start from nmf_restart)",
            "precision": prec, "tol": tol, "max_iters": max_iters, "check_every": 1,
            "device_loop": res["converge"], "host_loop": res["run"],
            "resident": resident,
            "device_over_host": round(res["run"]["seconds"] / res["converge"]["seconds"], 3),
            "identical_results": bool(a[0] == b[0] and a[1] == b[1]
                                      and np.array_equal(a[2], b[2])
                                      and np.array_equal(a[3], b[3]))}


def time_workloads(ws, local, clocks, tall_ranks=(16, 32, 64, 128)):
    """The other measured workloads, one timed step each (restart + the
    workload's iterations + objective, after one warm-up step), V generated
    once per workload and kept on the device across the forms:
      faces 361 x 2429, r = 10, 50 iterations, all four forms (L2-resident,
            launch-bound: absolute time);
      tall 65536 x 4096, r in {16, 32, 64, 128}, 20 iterations, all four forms;
      large 131072 x 16384, r = 64, 20 iterations, FP32 and BF16x3.
    Each entry: updates/s, the roofline of its dominant kernel (CUDA-event
    average of the streaming launches) and the relative objective error
    against the stored float64 oracle trajectory."""
    import dataclasses
    import torch
    from paper_1003_3272_gb300 import synth
    out = {}

    def run(pr, precs, wname):
        V = torch.from_numpy(pr.V).cuda()
        ent, objs = {}, {}
        for prec in precs:
            res = time_planted(pr, prec, 1, 1, ws, local, V_dev=V)
            rf = roofline(prec, pr.p, pr.n, pr.r, res, clocks, wname)
            objs[prec] = res["objective"]
            ent[prec] = {"updates_per_s": round(res["value"], 1),
                         "ms_per_step": round(res["ms"], 3),
                         "roofline": {k: rf[k] for k in ("bound", "achieved", "peak", "unit",
                                                         "frac", "avg_launch_us", "kernel",
                                                         "traffic")}}
        acc = accuracy(wname, pr.iters, objs)
        for prec in precs:
            e = acc.get("rel_objective_error_vs_fp64_oracle")
            ent[prec]["rel_objective_error_vs_fp64_oracle"] = e.get(prec) if e else None
        ent["iterations"] = pr.iters
        del V
        torch.cuda.empty_cache()
        return ent

    all4 = ["fp32", "tf32", "bf16x3", "bf16"]
    pr = synth.faces()
    out[pr.name] = run(pr, all4, pr.name)
    out[pr.name]["resident_fp32"] = time_resident(pr, ws)
    base = synth.tall(tall_ranks[0])
    for r in tall_ranks:
        W0, H0 = synth.starting_factors(base.seed, base.p, base.n, r)
        pr = dataclasses.replace(base, W0=W0, H0=H0, r=r, name=f"{synth.TALL['name']}_r{r}")
        out[pr.name] = run(pr, all4, pr.name)
    del base, pr
    pr = synth.large()
    out[pr.name] = run(pr, ["fp32", "bf16x3"], pr.name)
    del pr
    return out


def time_resident(pr, ws, reps=5):
    """A small workload's iterations through nmf_converge_resident (one
    persistent launch; tol = 0, one objective at the end), FP32: the median
    wall time of `reps` calls from the seeded start, the call's whole cost
    (the starting objective, the launch, the final synchronisation)."""
    import torch
    from paper_1003_3272_gb300 import nmf
    V = torch.from_numpy(pr.V).cuda()
    W = torch.from_numpy(pr.W0).cuda()
    H = torch.from_numpy(pr.H0).cuda()
    W0, H0 = W.clone(), H.clone()
    times = []
    with nmf.NMF(V, W, H, eps=pr.eps) as m:
        m.converge_resident(pr.iters, tol=0.0, check_every=pr.iters)
        for _ in range(reps):
            W.copy_(W0)
            H.copy_(H0)
            torch.cuda.synchronize()
            barrier(ws)
            t0 = time.perf_counter()
            done, f = m.converge_resident(pr.iters, tol=0.0, check_every=pr.iters)
            times.append(max_over_ranks(time.perf_counter() - t0, ws))
    t = sorted(times)[len(times) // 2]
    acc = accuracy(pr.name, pr.iters, {"fp32": f})
    e = acc.get("rel_objective_error_vs_fp64_oracle")
    return {"updates_per_s": round(done * ws / t, 1), "ms_per_step": round(t * 1e3, 3),
            "api": "nmf_converge_resident (one persistent launch, wall time of the call)",
            "rel_objective_error_vs_fp64_oracle": e.get("fp32") if e else None}


def oracle_objective(workload, iters):
    """The float64 oracle's objective after `iters` iterations from the seeded
    start on `workload`, as stored in tests/golden/objectives.json (written by
    tests/golden/make_objectives.py from the oracle alone), or None."""
    path = os.path.join(ROOT, "tests", "golden", "objectives.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return d[workload]["objective"].get(str(iters))
    except (OSError, ValueError, KeyError):
        return None


def accuracy(workload, iters, objectives):
    """Relative objective error of each timed form against the stored float64
    oracle trajectory (same seeds, same iteration count)."""
    fo = oracle_objective(workload, iters)
    if fo is None:
        return {"rel_objective_error_vs_fp64_oracle": None,
                "note": f"no stored oracle objective for {workload} at {iters} iterations"}
    return {"rel_objective_error_vs_fp64_oracle":
                {k: float(f"{abs(f - fo) / fo:.3e}") for k, f in objectives.items()},
            "oracle_objective": fo, "iterations": iters,
            "source": "tests/golden/objectives.json (float64 oracle trajectory, "
                      "tests/golden/make_objectives.py)"}


def run_batched_line(args, ws, local):
    """--workload batched: the 512-instance batched workload as the line."""
    import torch
    torch.cuda.set_device(local)
    sampler = ClockSampler(local)
    sampler.start()
    w0 = time.perf_counter()
    b = time_batched(args.prec, args.steps, args.warmup, 100, ws, singles=not args.no_extras)
    clocks = sampler.stop((w0, time.perf_counter()))
    pk = peaks()
    return {
        "metric": METRIC, "value": b["value"], "unit": b["unit"], "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": b["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": args.prec, "data": "synthetic (seeded iid uniform [0,1); no dataset)",
        "config": {"workload": "batched_512", "instances": b["instances"],
                   "iters_per_step": b["iters_per_step"], "precision": args.prec,
                   "shapes": b["config"], "global_batch": ws,
                   "parallelism": f"replicas x{ws}",
                   "l2": "inputs larger than L2 (about 2.3 GB of V)"},
        "roofline": {"bound": "hbm", "achieved": b["aggregate_gbs"], "peak": pk["hbm_gbs"],
                     "unit": "GB/s", "frac": b["hbm_frac"], "traffic": None,
                     "kernel": "k_batched_tc (whole graph-captured iteration)"},
        "e2e": None, "gpu_launches": b["gpu_launches"], "clocks": clocks,
        "schedule": b["schedule"],
        "accuracy": b["rel_objective_error_vs_fp64_oracle"],
        "one_by_one": b.get("one_by_one"), "speedup_vs_fp32": b.get("speedup_vs_fp32"),
    }


def run_gpu(args, ws, rank, local):
    import torch
    from paper_1003_3272_gb300 import synth

    torch.cuda.set_device(local)
    if args.workload == "batched":
        return run_batched_line(args, ws, local), None
    pr, wname, data = make_problem(args)
    p, n, r, iters = pr.p, pr.n, pr.r, pr.iters
    stream = torch.cuda.current_stream()
    main = time_planted(pr, args.prec, args.steps, args.warmup, ws, local, sample_clocks=True)
    clocks = main["clocks"]
    roof = roofline(args.prec, p, n, r, main, clocks, wname)

    # End to end through the public one-call API with host buffers.
    e2e = None
    if not args.no_e2e:
        from paper_1003_3272_gb300 import nmf
        Vh = torch.from_numpy(pr.V).pin_memory().numpy()
        Wh0 = torch.from_numpy(pr.W0).pin_memory().numpy()
        Hh0 = torch.from_numpy(pr.H0).pin_memory().numpy()
        Wh = torch.empty(p, r).pin_memory().numpy()
        Hh = torch.empty(r, n).pin_memory().numpy()
        ne = max(1, min(args.steps, 5))
        nmf.solve(Vh, Wh, Hh, 2, eps=pr.eps, prec=args.prec, stream=stream)  # warm
        barrier(ws)
        t0 = time.perf_counter()
        for _ in range(ne):
            Wh[...] = Wh0
            Hh[...] = Hh0
            nmf.solve(Vh, Wh, Hh, iters, eps=pr.eps, prec=args.prec, stream=stream)
        te = time.perf_counter() - t0
        te = max_over_ranks(te, ws)
        e2e = {"value": round(iters * ne * ws / te, 2), "unit": "updates/s",
               "h2d_bytes_per_step": int(Vh.nbytes + Wh.nbytes + Hh.nbytes),
               "d2h_bytes_per_step": int(Wh.nbytes + Hh.nbytes + 8),
               "steps": ne, "api": f"nmf_solve (host V, W, H; allocation, operand copies, "
                                   f"{iters} iterations, objective, copies back)"}

    kinds = main["kinds"]
    out = {
        "metric": METRIC, "value": round(main["value"], 2), "unit": "updates/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(main["ms"] / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "tf32": "tf32", "bf16x3": "bf16x3", "bf16": "bf16"}[args.prec],
        "data": data,
        "config": {"workload": wname, "p": p, "n": n, "r": r,
                   "iters_per_step": iters, "precision": args.prec, "order": "h_first",
                   "eps": pr.eps, "global_batch": ws, "parallelism": f"replicas x{ws}",
                   "l2": (f"inputs larger than L2 (V is {p * n * 4 / 1e6:.0f} MB fp32; L2 129 MB)"
                          if p * n * 4 > 129e6 else
                          f"V ({p * n * 4 / 1e6:.1f} MB) fits in L2: the L2-resident case"),
                   "step": f"restart (operand copies + seeded W,H + Grams) + {iters} MM "
                           "iterations + objective + stopping test"},
        "roofline": roof, "e2e": e2e, "gpu_launches": main["launches"], "clocks": clocks,
        "pass_bounds": pass_bounds(args.prec, p, n, r, main["value"]),
        "objective": main["objective"],
        "breakdown_ms_per_step": {k: round(v[0] / args.steps, 3) for k, v in kinds.items()},
    }
    if not args.no_extras:
        # the plain FP32 form and the other precisions on the same workload
        by = {}
        objs = {}
        for prec in ["fp32", "tf32", "bf16x3", "bf16"]:
            if prec == args.prec:
                res, rf = main, roof
            else:
                res = time_planted(pr, prec, max(2, args.steps // 2), 2, ws, local)
                rf = roofline(prec, p, n, r, res, clocks, wname)
            objs[prec] = res["objective"]
            by[prec] = {"updates_per_s": round(res["value"], 1),
                        "ms_per_step": round(res["ms"] / res["steps"], 3),
                        "roofline_frac": rf["frac"], "roofline_bound": rf["bound"],
                        "achieved": rf["achieved"], "unit": rf["unit"],
                        "avg_launch_us": rf["avg_launch_us"]}
        base = by["fp32"]["updates_per_s"]
        for prec in by:
            by[prec]["speedup_vs_fp32"] = round(by[prec]["updates_per_s"] / base, 2)
        out["by_precision"] = by
        out["accuracy"] = accuracy(wname, iters, objs)
        if args.workload == "planted":
            out["batched"] = time_batched("bf16x3", 2, 2, 100, ws)
            out["converge"] = time_converge(ws)
            out["poisson"] = time_poisson(ws, clocks)
            out["pet"] = time_pet(ws)
            if not args.no_workloads:
                out["by_workload"] = time_workloads(ws, local, clocks)
    else:
        out["accuracy"] = accuracy(wname, iters, {args.prec: main["objective"]})
    return out, pr


def oracle_iterations(V, W0, H0, eps, budget_s):
    """MM iterations of the float64 oracle as it stands until `budget_s`
    seconds have passed (at least 2, after one warm-up): (count, seconds)."""
    import numpy as np
    from oracle import nmf_oracle as orc
    W = W0.astype(np.float64)
    H = H0.astype(np.float64)
    orc.step(V, W, H, eps)  # warm BLAS
    t0 = time.perf_counter()
    k = 0
    while True:
        W, H = orc.step(V, W, H, eps)
        k += 1
        if time.perf_counter() - t0 > budget_s and k >= 2:
            break
    return k, time.perf_counter() - t0


SINGLE_THREAD_ENV = {"OMP_NUM_THREADS": "1", "OPENBLAS_NUM_THREADS": "1",
                     "MKL_NUM_THREADS": "1", "BLIS_NUM_THREADS": "1",
                     "VECLIB_MAXIMUM_THREADS": "1", "NUMEXPR_NUM_THREADS": "1"}


def _single_thread_leg(pr, budget_s):
    """The same oracle iterations in a child interpreter whose BLAS runs one
    thread (the paper's one-core CPU protocol); V, W0, H0 pass through a
    temporary .npz file.  The child is a fresh process (fork + exec), so it
    shares no CUDA state with this one."""
    import tempfile
    import numpy as np
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "prob.npz")
        np.savez(path, V=pr.V, W0=pr.W0, H0=pr.H0)
        code = ("import json, sys, numpy as np; sys.path.insert(0, %r); import bench; "
                "z = np.load(%r); k, dt = bench.oracle_iterations(z['V'], z['W0'], z['H0'], "
                "%r, %r); print(json.dumps([k, dt]))" % (ROOT, path, pr.eps, budget_s))
        env = dict(os.environ, **SINGLE_THREAD_ENV)
        try:
            res = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                                 env=env, timeout=budget_s * 10 + 120)
            k, dt = json.loads(res.stdout.strip().splitlines()[-1])
        except (subprocess.SubprocessError, ValueError, IndexError, OSError) as e:
            return {"value": None, "unit": "updates/s", "cores": 1, "kind": "oracle",
                    "sample": f"not run: {type(e).__name__}"}
    return {"value": round(k / dt, 4), "unit": "updates/s", "cores": 1, "kind": "oracle",
            "sample": f"{k} MM iterations of the {pr.p}x{pr.n} r={pr.r} {pr.name} problem "
                      f"in float64 numpy/BLAS on one thread ({', '.join(sorted(SINGLE_THREAD_ENV))}"
                      f" = 1), {dt:.1f} s"}


def cpu_baseline(pr, budget_s, single_thread=True):
    """The FP64 oracle as it stands, timed on this host's cores on a bounded
    sample of the same workload: MM iterations of the full problem, once with
    BLAS on all cores (value, cores) and once on one thread (single_thread),
    as the paper timed its CPU baseline on one core."""
    if pr.V.size > (1 << 29):
        return {"value": None, "unit": "updates/s", "cores": os.cpu_count(), "kind": "oracle",
                "sample": "not run: the oracle widens V to float64 for every product "
                          f"({pr.V.size * 8 / 1e9:.0f} GB per copy); the sampled parity "
                          "tests cover this workload"}
    k, dt = oracle_iterations(pr.V, pr.W0, pr.H0, pr.eps, budget_s)
    out = {"value": round(k / dt, 4), "unit": "updates/s", "cores": os.cpu_count(),
           "kind": "oracle",
           "sample": f"{k} MM iterations (H then W update) of the {pr.p}x{pr.n} r={pr.r} "
                     f"{pr.name} problem in float64 numpy/BLAS on all cores, {dt:.1f} s"}
    if single_thread:
        out["single_thread"] = _single_thread_leg(pr, budget_s)
    return out


def run_reference_batched(args):
    """Reference arm on the batched workload: each step is one MM iteration of
    each of the first 32 instances (a bounded sample)."""
    import numpy as np
    from oracle import nmf_oracle as orc
    from paper_1003_3272_gb300 import synth
    probs = synth.batch(count=512)[:32]
    st = [(pr.W0.astype(np.float64), pr.H0.astype(np.float64)) for pr in probs]
    def one():
        for i, pr in enumerate(probs):
            st[i] = orc.step(pr.V, st[i][0], st[i][1], pr.eps)
    for _ in range(args.warmup):
        one()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one()
    dt = time.perf_counter() - t0
    value = len(probs) * args.steps / dt
    return {
        "impl": "reference", "metric": METRIC, "value": round(value, 2),
        "unit": "instance-iterations/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded iid uniform [0,1); no dataset)",
        "config": {"workload": "batched_512", "sample": "first 32 of the 512 instances",
                   "iters_per_step": 1, "precision": "f64 oracle"},
        "cpu_baseline": {"value": round(value, 2), "unit": "instance-iterations/s",
                         "cores": os.cpu_count(), "kind": "oracle",
                         "sample": "each step = 1 MM iteration of each of the first 32 "
                                   "instances (float64 numpy/BLAS)"},
        "e2e": {"value": round(value, 2), "unit": "instance-iterations/s",
                "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def run_reference(args):
    """Reference arm: the FP64 CPU oracle on the bench's workload; each step is
    one MM iteration (a bounded sample of the 200-iteration run)."""
    import numpy as np
    from oracle import nmf_oracle as orc
    if args.workload == "batched":
        return run_reference_batched(args)
    pr, wname, data = make_problem(args)
    W = pr.W0.astype(np.float64)
    H = pr.H0.astype(np.float64)
    for _ in range(args.warmup):
        W, H = orc.step(pr.V, W, H, pr.eps)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        W, H = orc.step(pr.V, W, H, pr.eps)
    dt = time.perf_counter() - t0
    value = args.steps / dt
    return {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "updates/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": data,
        "config": {"workload": wname, "p": pr.p, "n": pr.n, "r": pr.r,
                   "iters_per_step": 1, "precision": "f64 oracle"},
        "cpu_baseline": {"value": round(value, 4), "unit": "updates/s", "cores": os.cpu_count(),
                         "kind": "oracle",
                         "sample": f"each step = 1 MM iteration of the {pr.p}x{pr.n} r={pr.r} "
                                   f"{wname} problem (float64 numpy/BLAS)"},
        "e2e": {"value": round(value, 4), "unit": "updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--prec", default="bf16x3", choices=["fp32", "tf32", "bf16x3", "bf16"])
    ap.add_argument("--iters", type=int, default=200,
                    help="MM iterations per step on the planted workload")
    ap.add_argument("--workload", default="planted",
                    choices=["planted", "faces", "tall", "large", "batched"])
    ap.add_argument("--rank", type=int, default=64, choices=[16, 32, 64, 128],
                    help="rank of the tall workload")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the other precisions, the batched workload and the accuracy check")
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the by_workload block (faces, tall sweep, large)")
    args = ap.parse_args()

    if args.impl == "reference":
        rank = int(os.environ.get("RANK", "0"))
        if rank != 0:
            return 0
        print(json.dumps(run_reference(args)), flush=True)
        return 0

    ws, rank, local = dist_setup(args.gpus)
    out, pr = run_gpu(args, ws, rank, local)
    if rank == 0:
        if ws == 1 and not args.no_cpu_baseline and pr is not None:
            out["cpu_baseline"] = cpu_baseline(pr, args.cpu_budget)
        else:
            out["cpu_baseline"] = None
        print(json.dumps(out), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
