"""Benchmark: time to relative fit 1e-3 of ADMoM non-negative CP factorization on GB300.

One step = one whole factorization of the workload (default: the 1000x1000x1000 rank-32
tensor, U[0,1] factors, 30 dB Gaussian noise, drawn on the device; L = 5 inner iterations,
Khatri-Rao of the auxiliaries, rho = trace(G)/R, uniform start) from the start until the
relative error is within 1e-3 of the converged value RFE* (RFE_k <= RFE* (1 + 1e-3)), RFE*
the error of the plain FP32 method after the workload's outer-iteration budget, found
before the timed region.  The timed form (--form) defaults to BF16 tensor storage with the
learned warm start in the first sweep (network trained before the timed region on rows of
other tensors of the same generator; harvest and training times reported apart).  Every form
(plain FP32, plain BF16, BF16 + learned) is also timed to the fit target and to the same
KKT tolerance (eq. KKT_NTF: the scaled dual infeasibility and complementarity of every
factor's last update), and the learned form is compared with plain BF16 on held-out tensors.
The other workloads of the evaluation (600^3 rank 50 with sparse factors, the 4-way
200x200x200x50 rank-16 collinear stress case) are measured the same way under `variants`,
each with the live roofline of its dominant contraction.  The metric is the time of one
factorization (lower is better); the JSON line carries the live roofline of the dominant
tensor contraction (HBM GB/s from CUDA events inside the timed steps), an end-to-end time
through host buffers, and the FP64 oracle timed on the host cores (on a slab of the tensor,
scaled: extrapolated).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ntf|reference]
                  [--workload NAME] [--no-variants]

Multi-GPU: replicas only (each rank factorizes its own tensor of a different seed; no
collective on the data path); value = max over ranks of the time per factorization.

  python bench.py --study table1|table2 [--realizations R] [--study-cases 0,1,...]

runs the scenarios of the paper's Table 1 (or Table 2, stopping tolerances 1e-3) in paper
mode (restarts included) and prints, per scenario, the mean relative error beside the
printed one and the time per factorization.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time to rel. fit 1e-3 (s) & MTTKRP HBM GB/s; BF16+learned vs plain FP32 GPU"
FIT_TOL = 1e-3

# The evaluation workloads (the recipe of synth.WORKLOADS, drawn on the device).  max_outer:
# the outer-iteration budget whose plain FP32 error defines the fit target.  kkt: the common
# KKT tolerance (scaled dual infeasibility, scaled complementarity) every form is run to.
# fit_iters: outer iterations the plain FP32 method needs to reach the fit target (measured on
# GB300; the FP64 oracle runs the same iteration and tracks it within 1e-4 in the error), used
# to scale the oracle's per-iteration time into a time to fit.
WORKLOADS = {
    "1000x1000x1000_r32": dict(dims=(1000, 1000, 1000), R=32, snr_db=30.0,
                               structure="uniform", max_outer=300, kkt=(1e-5, 1e-6),
                               fit_iters=77),
    "600x600x600_r50_sparse": dict(dims=(600, 600, 600), R=50, snr_db=20.0,
                                   structure="sparse", max_outer=200, kkt=(1e-5, 1e-6),
                                   fit_iters=13),
    "200x200x200x50_r16_collinear": dict(dims=(200, 200, 200, 50), R=16, snr_db=10.0,
                                         structure="collinear", max_outer=300,
                                         kkt=(1e-5, 1e-6), fit_iters=52),
    "400x400x400_r20": dict(dims=(400, 400, 400), R=20, snr_db=20.0, structure="uniform",
                            max_outer=200, kkt=(1e-5, 1e-6), fit_iters=43),
}
DEFAULT_WORKLOAD = "1000x1000x1000_r32"
# measured beside the default workload, under `variants`
VARIANT_WORKLOADS = ("600x600x600_r50_sparse", "200x200x200x50_r16_collinear")
# oracle sample: a slab of the tensor over its last mode with at most this many entries
ORACLE_SAMPLE_NUMEL = 100_000_000


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# Source files that define each timed kernel: a stored ncu traffic figure is used only while
# these files are unchanged since the capture.
KERNEL_SOURCES = {
    "k_umma": ["umma_kernels.cuh", "umma_bf16.cu", "umma_f32.cu", "umma_host.cu"],
    "k_gemm": ["mttkrp_kernels.cuh", "gemm_n_f32.cu", "gemm_n_bf16.cu", "gemm_t_f32.cu",
               "gemm_t_bf16.cu"],
}


def kernel_source_hash(family: str) -> str:
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[family]:
        with open(os.path.join(ROOT, "paper_1409_2383_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def _traffic_record(kernel: str, workload: str):
    """Per-launch DRAM bytes of `kernel` on `workload` from a committed ncu summary
    (profiles/traffic.json, key "kernel@workload"), if it was taken on the current sources of
    that kernel; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            entry = json.load(f).get(f"{kernel}@{workload}")
    except Exception:
        return None
    if not entry:
        return None
    family = "k_umma" if kernel.startswith("k_umma") else "k_gemm"
    if entry.get("source_sha256") != kernel_source_hash(family):
        return None
    return entry.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi sampling (every 20 ms) while the timed region runs; entering waits until the
    sampler is live, so that the samples fall inside the region."""
    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.skip = 0

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t0 = time.time()
            while not self.lines and self.proc.poll() is None and time.time() - t0 < 3.0:
                time.sleep(0.005)
            self.skip = len(self.lines)  # samples taken before the timed region
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        # the samples taken inside the timed region (all of them if it was shorter than the
        # sampling period)
        for ln in (self.lines[self.skip:] if len(self.lines) > self.skip else self.lines):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) != 6:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[2:]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def host_cores() -> int:
    """Cores this process may run on (its CPU affinity; the whole host's count as fallback):
    the threads the oracle's BLAS calls spread over."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def device_workload(name: str, seed: int):
    """(X FP32 on the device, start factors) of a named workload, drawn on the device."""
    from paper_1409_2383_gb300 import warmstart
    w = WORKLOADS[name]
    return warmstart.synthetic_tensor(w["dims"], w["R"], seed=seed, snr_db=w["snr_db"],
                                      structure=w["structure"])


def oracle_sample(name: str, seed: int = 0):
    """The oracle's bounded sample of a workload: the first slab of the tensor over its last
    mode with at most ORACLE_SAMPLE_NUMEL entries, drawn by the host generator with the
    workload's recipe (the whole tensor if it is small).  Returns (X, start factors, scale):
    scale = the full tensor's entries over the slab's."""
    import synth
    w = WORKLOADS[name]
    dims = list(w["dims"])
    full = math.prod(dims)
    rest = full // dims[-1]
    dims[-1] = max(1, min(dims[-1], ORACLE_SAMPLE_NUMEL // rest))
    kw = {} if w["structure"] == "uniform" else {"structure": w["structure"]}
    X, _, init = synth.workload(tuple(dims), w["R"], seed=seed, snr_db=w["snr_db"], **kw)
    return X, [f.astype(np.float32) for f in init], full / math.prod(dims)


def cpu_oracle_seconds_per_iteration(X, init, sweeps: int):
    """Median wall time of `sweeps` oracle outer iterations (FP64, numpy on all host cores)."""
    from oracle import ntf as o
    X64 = X.astype(np.float64)
    params = o.Params(inner_iters=5, kr_source="aux", rho_policy="trace")
    st = o.init_state([f.astype(np.float64) for f in init], params)
    ts = []
    for _ in range(sweeps):
        t0 = time.perf_counter()
        o.outer_iteration(X64, st, params)
        ts.append(time.perf_counter() - t0)
    return statistics.median(ts)


def max_over_ranks(values, device):
    """Whole-job figures of a replicas run: the maximum over ranks of each value (the slowest
    rank sets the job's time).  One all-reduce of a small vector; nothing else is exchanged."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def _workload_config(name: str) -> dict:
    w = WORKLOADS[name]
    return {"workload": name, "dims": list(w["dims"]), "rank": w["R"], "snr_db": w["snr_db"],
            "structure": w["structure"], "inner_iters": 5, "rho": "trace(G)/R",
            "kr_source": "aux", "fit_tol": FIT_TOL, "max_outer": w["max_outer"],
            "kkt_tol": {"dual": w["kkt"][0], "comp": w["kkt"][1]}}


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return
    name = getattr(args, "workload", None) or DEFAULT_WORKLOAD
    X, init, scale = oracle_sample(name)
    n_iter = WORKLOADS[name]["fit_iters"]
    sec = cpu_oracle_seconds_per_iteration(X, init, args.warmup + args.steps) * scale
    value = sec * n_iter
    cores = host_cores()
    shape = "x".join(str(d) for d in X.shape)
    sample = (f"{args.warmup + args.steps} oracle outer iterations on a {shape} slab of "
              f"{name} (median, x {scale:g} for the full tensor: extrapolated) x the {n_iter} "
              "outer iterations the method needs to reach the fit")
    cfg = _workload_config(name)
    cfg["step"] = ("one FP64 oracle outer iteration (slab, scaled); value = that time x the "
                   f"{n_iter} iterations to the fit")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1000.0,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": cfg,
        "cpu_baseline": {"value": value, "unit": "s", "cores": cores, "kind": "oracle",
                         "sample": sample, "extrapolated": True},
        "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


FORMS = {
    # form: (storage, learned warm start)
    "bf16_learned": ("bf16", True),
    "bf16": ("bf16", False),
    "fp32": ("fp32", False),
}


def train_network(name: str, args):
    """Warm-start network for a workload: rows harvested from the first sweeps of tensors of
    the workload's generator with other seeds (drawn on the device), trained by the library's
    kernels.  Returns (network, report)."""
    import torch
    from paper_1409_2383_gb300 import ntf, warmstart
    w = WORKLOADS[name]
    dims, R = w["dims"], w["R"]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rows = warmstart.training_set(dims, R, args.train_rows, sweeps=args.ws_sweeps,
                                  seed0=1000, snr_db=w["snr_db"], storage="bf16",
                                  structure=w["structure"])
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    H = 256
    groups, per_group = 256, 25                  # rows from many coefficient matrices per step
    net = ntf.Mlp(R, H, warmstart.init_params(R, H, seed=0),
                  max_rows=max(groups * per_group, 16 * max(dims)), max_groups=groups)
    loss0 = warmstart.eval_loss(net, rows, 16)
    steps = max(1, int(args.train_epochs * rows.rows / (groups * per_group)))
    warmstart.train(net, rows, steps=steps, groups_per_batch=groups, lr=1e-3, decay_at=0.7,
                    rows_per_group=per_group)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    rep = {"rows": rows.rows, "groups": len(rows.Gn), "tensor_dims": list(dims),
           "sweeps_harvested": args.ws_sweeps, "ws_sweeps": args.ws_sweeps,
           "harvest_s": t1 - t0, "train_s": t2 - t1, "steps": steps, "hidden": H,
           "loss_before": loss0, "loss_after": warmstart.eval_loss(net, rows, 16)}
    del rows
    return net, rep


# ntf_params.tensor_copy of every context the bench makes (--tensor-copy)
TENSOR_COPY = 0


def _params(kkt=None):
    from paper_1409_2383_gb300 import ntf
    if kkt is None:
        return ntf.default_params(paper_mode=False, eps_abs=0.0, eps_rel=0.0,
                                  tensor_copy=TENSOR_COPY)
    return ntf.default_params(paper_mode=False, eps_abs=0.0, eps_rel=0.0,
                              kkt_dual_tol=kkt[0], kkt_comp_tol=kkt[1],
                              tensor_copy=TENSOR_COPY)


def fit_target(X, R: int, init, max_outer: int) -> float:
    """The error of the plain method on the tensor X as stored (FP32 or BF16) after
    `max_outer` outer iterations, relaxed by the fit tolerance: the fit target of the forms
    that store the tensor so.  (A form's error is measured against its own stored tensor; BF16
    rounding of the data adds about 0.15% RMS relative noise, which at 30 dB is the size of
    the tolerance, so each storage is timed to the converged error of its own data and every
    form's final error is also reported against the FP32 tensor.)"""
    import torch
    from paper_1409_2383_gb300 import ntf
    A = [f.clone() for f in init]
    T = [f.clone() for f in init]
    Y = [torch.zeros_like(f) for f in init]
    with ntf.Context(X, R, _params()) as c:
        rs = c.run(A, T, Y, max_outer, check_every=max_outer)
    return rs["rel_err"] * (1 + FIT_TOL)


def _roofline_of(prof, storage: str, workload: str) -> dict:
    """Live HBM roofline of the dominant contraction (more device time) from a profile."""
    k = 0 if prof["contraction_ms"][0] >= prof["contraction_ms"][1] else 1
    # (the second contraction runs as a row-major product on the context's transposed copy
    # of the tensor where the context made one)
    names = ["k_umma<0,...> (X * KR_right, tcgen05)",
             "k_umma<0,...> (X^T * KR_left on the transposed tensor copy, tcgen05)"
             if prof.get("tensor_copy_bytes") else "k_umma<1,...> (X^T * KR_left, tcgen05)"]
    kernel_ids = [f"k_umma_n_{storage}", f"k_umma_t_{storage}"]
    avg_ms = prof["contraction_ms"][k] / max(prof["contractions"][k], 1)
    bytes_ = prof["contraction_bytes"][k]
    achieved = bytes_ / (avg_ms * 1e-3) / 1e9
    peak, peak_kind = _peaks()
    other = None
    if prof["contractions"][1 - k]:
        other = prof["contraction_bytes"][1 - k] / (
            prof["contraction_ms"][1 - k] / prof["contractions"][1 - k] * 1e-3) / 1e9
    return {"bound": "hbm", "kernel": names[k], "achieved": achieved, "peak": peak,
            "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
            "traffic": _traffic_record(kernel_ids[k], workload),
            "algorithmic_bytes_per_launch": bytes_,
            "avg_launch_ms": avg_ms, "other_contraction_gbs": other}


def time_form(X32, R: int, init, storage: str, net, target: float, kkt, max_outer: int,
              ws_sweeps: int, workload: str, repeats: int = 3) -> dict:
    """One form on one tensor: time (CUDA events, median of `repeats`) and outer iterations to
    the fit target and to the KKT tolerance, the final error against the FP32 tensor, and the
    live roofline of its dominant contraction."""
    import torch
    from paper_1409_2383_gb300 import ntf, warmstart
    from paper_1409_2383_gb300 import ntf as _n
    Xf = _n.to_bf16(X32) if storage == "bf16" else X32
    fit = warmstart.time_to_fit(Xf, R, init, target, max_outer, net=net, repeats=repeats,
                                ws_sweeps=ws_sweeps)
    kk = warmstart.time_to_fit(Xf, R, init, 0.0, max_outer, net=net, repeats=repeats,
                               ws_sweeps=ws_sweeps, params=_params(kkt))
    # the state after the KKT run: its error against the FP32 tensor and its live roofline
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        A = [f.clone() for f in init]
        T = [f.clone() for f in init]
        Y = [torch.zeros_like(f) for f in init]
        with ntf.Context(Xf, R, _params(kkt), stream=stream) as c:
            if net is not None:
                c.attach_warmstart(net, ws_sweeps)
            c.profile_enable(True)
            c.run(A, T, Y, max_outer)
            prof = c.profile_get()
        with ntf.Context(X32, R, _params(), stream=stream) as c32:
            err32 = c32.fit_explicit(T)
    del Xf
    return {"fit": fit, "kkt": kk, "final_rfe_vs_fp32_tensor": err32,
            "roofline": _roofline_of(prof, storage, workload)}


def robustness(name: str, args, net) -> dict:
    """Outer iterations and time to the fit target and to the KKT tolerance, plain BF16 vs
    BF16 + learned warm start, on held-out tensors of the workload's generator: the iteration
    count depends on the path through the slow phase of the factorization, so one tensor says
    little about the warm start."""
    from paper_1409_2383_gb300 import ntf, warmstart
    w = WORKLOADS[name]
    rows = []
    for seed in range(100, 100 + args.robust_tensors):
        X, init = device_workload(name, seed)
        Xb = ntf.to_bf16(X)
        del X
        target = fit_target(Xb, w["R"], init, w["max_outer"])
        r = {"seed": seed}
        for tag, nt in (("plain", None), ("learned", net)):
            f = warmstart.time_to_fit(Xb, w["R"], init, target, w["max_outer"], net=nt,
                                      ws_sweeps=args.ws_sweeps)
            k = warmstart.time_to_fit(Xb, w["R"], init, 0.0, w["max_outer"], net=nt,
                                      ws_sweeps=args.ws_sweeps, params=_params(w["kkt"]))
            r[f"{tag}_fit_iters"], r[f"{tag}_fit_s"] = f["iters"], f["seconds"]
            r[f"{tag}_kkt_iters"], r[f"{tag}_kkt_s"] = k["iters"], k["seconds"]
            r[f"{tag}_kkt_met"] = k["kkt_met"]
        rows.append(r)
        del Xb
    out = {"tensors": rows}
    for key in ("fit_iters", "fit_s", "kkt_iters", "kkt_s"):
        for tag in ("plain", "learned"):
            vals = [r[f"{tag}_{key}"] for r in rows]
            out[f"{tag}_{key}_mean"] = statistics.mean(vals)
            out[f"{tag}_{key}_std"] = statistics.stdev(vals) if len(vals) > 1 else 0.0
    out["learned_fewer_kkt_iters"] = sum(r["learned_kkt_iters"] < r["plain_kkt_iters"]
                                         for r in rows)
    out["learned_more_kkt_iters"] = sum(r["learned_kkt_iters"] > r["plain_kkt_iters"]
                                        for r in rows)
    return out


def measure_workload(name: str, args, net=None, training=None) -> dict:
    """Every form of a workload (seed 0) to the fit target and to the KKT tolerance, the
    learned form's network (trained here unless given) and its held-out comparison."""
    w = WORKLOADS[name]
    from paper_1409_2383_gb300 import ntf
    X, init = device_workload(name, 0)
    Xb = ntf.to_bf16(X)
    targets = {"fp32": fit_target(X, w["R"], init, w["max_outer"]),
               "bf16": fit_target(Xb, w["R"], init, w["max_outer"])}
    del Xb
    if net is None and not args.no_learned:
        net, training = train_network(name, args)
    out = {"config": _workload_config(name), "target_rfe": targets, "forms": {},
           "training": training}
    for form, (storage, learned) in FORMS.items():
        if learned and net is None:
            continue
        out["forms"][form] = time_form(X, w["R"], init, storage, net if learned else None,
                                       targets[storage], w["kkt"], w["max_outer"],
                                       args.ws_sweeps, name)
    f = out["forms"]
    if "fp32" in f:
        for form in f:
            f[form]["fit_speedup_vs_fp32"] = f["fp32"]["fit"]["seconds"] / f[form]["fit"]["seconds"]
            f[form]["kkt_speedup_vs_fp32"] = f["fp32"]["kkt"]["seconds"] / f[form]["kkt"]["seconds"]
    del X
    if net is not None and args.robust_tensors > 0:
        out["learned_vs_plain_held_out"] = robustness(name, args, net)
    return out, net


def run_ntf(args):
    import torch
    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_1409_2383_gb300 import ntf

    name = args.workload
    w = WORKLOADS[name]
    dims, R, max_outer = w["dims"], w["R"], w["max_outer"]
    storage, learned = FORMS[args.form]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        Xd, init_d = device_workload(name, rank)    # replicas: one tensor per rank
        A = [f.clone() for f in init_d]
        At = [f.clone() for f in init_d]
        Y = [torch.zeros_like(f) for f in init_d]

        def reset():
            for a, t, y, f in zip(A, At, Y, init_d):
                a.copy_(f)
                t.copy_(f)
                y.zero_()

        # the fit target: the converged error of the plain method on the tensor as this form
        # stores it, within the workload's iteration budget, relaxed by the fit tolerance
        target32 = fit_target(Xd, R, init_d, max_outer)
        with ntf.Context(Xd, R, _params(), stream=stream) as c32:
            reset()
            fp32_fit = c32.run(A, At, Y, max_outer, target_rfe=target32)["iters"]

        net, training = train_network(name, args) if learned else (None, None)
        Xf = ntf.to_bf16(Xd) if storage == "bf16" else Xd
        target = fit_target(Xf, R, init_d, max_outer) if storage == "bf16" else target32
        ctx = ntf.Context(Xf, R, _params(), stream=stream)
        if net is not None:
            ctx.attach_warmstart(net, args.ws_sweeps)
        for _ in range(args.warmup):
            reset()
            ctx.run(A, At, Y, max_outer, target_rfe=target)
        stream.synchronize()

        # timed region: K factorizations to the target, inputs resident in HBM
        ctx.profile_enable(True)
        iters = []
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clk:
            ev0.record(stream)
            for _ in range(args.steps):
                reset()
                rs = ctx.run(A, At, Y, max_outer, target_rfe=target)
                iters.append(rs["iters"])
            ev1.record(stream)
            torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        ms = ev0.elapsed_time(ev1) / args.steps
        prof = ctx.profile_get()
        ctx.profile_enable(False)
        final_rfe = rs["rel_err"]
        ctx.close()
        # error of the form's factors against the FP32 tensor (BF16 storage rounds the data)
        with ntf.Context(Xd, R, _params(), stream=stream) as c32:
            rfe_vs_fp32 = c32.fit_explicit(At)

        # end to end through the public API with host buffers: H2D of the FP32 tensor and the
        # start (BF16 form: the conversion kernel reads the pinned host tensor, so the copy and
        # the conversion are one pass), context creation (||X||^2), the factorization, D2H of
        # the factors
        Xh = Xd.cpu().pin_memory()
        init_h = [f.cpu().pin_memory() for f in init_d]
        out_h = [torch.empty_like(f).pin_memory() for f in init_h]
        if storage == "bf16":
            del Xd                               # room for the end-to-end copies
        torch.cuda.synchronize()
        e2e_steps = max(1, min(args.steps, 5))
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            if storage == "bf16":
                Xe = ntf.to_bf16(Xh, stream)
            else:
                Xe = torch.empty(Xh.shape, dtype=torch.float32, device="cuda")
                Xe.copy_(Xh, non_blocking=True)
            Ae = [torch.empty(f.shape, device="cuda") for f in init_h]
            Te = [torch.empty(f.shape, device="cuda") for f in init_h]
            for a, t, f in zip(Ae, Te, init_h):
                a.copy_(f, non_blocking=True)
                t.copy_(f, non_blocking=True)
            Ye = [torch.zeros(f.shape, device="cuda") for f in init_h]
            with ntf.Context(Xe, R, _params(), stream=stream) as c2:
                if net is not None:
                    c2.attach_warmstart(net, args.ws_sweeps)
                c2.run(Ae, Te, Ye, max_outer, target_rfe=target)
            for o_, t in zip(out_h, Te):
                o_.copy_(t, non_blocking=True)
            stream.synchronize()
            del Xe
        e2e_s = (time.perf_counter() - t0) / e2e_steps
        h2d = Xh.numel() * 4 + 2 * sum(f.numel() * 4 for f in init_h)
        d2h = sum(f.numel() * 4 for f in out_h)
        oracle_slab = None
        if not args.no_cpu_baseline and rank == 0:
            oracle_slab = oracle_sample(name)
        del Xh, Xf

        variants = None
        if not args.no_variants and rank == 0:
            torch.cuda.empty_cache()
            main_meas, net = measure_workload(name, args, net=net, training=training)
            variants = {name: main_meas}
            torch.cuda.empty_cache()
            variants["sparse_mttkrp_1000x1000x1000_nnz1e8_r32"] = measure_sparse(
                (1000, 1000, 1000), 100_000_000, 32)
            for other in VARIANT_WORKLOADS:
                if other == name:
                    continue
                torch.cuda.empty_cache()
                meas, onet = measure_workload(other, args)
                if onet is not None:
                    onet.close()
                variants[other] = meas
        if net is not None:
            net.close()

    value_s = ms / 1000.0
    if world > 1:
        value_s, e2e_s = max_over_ranks([value_s, e2e_s], "cuda")
    if rank != 0:
        return

    roofline = _roofline_of(prof, storage, name)
    sweep_ms = ms / statistics.mean(iters)

    cpu = None
    if oracle_slab is not None:
        Xs, init_s, scale = oracle_slab
        n_cpu = 2
        sec = cpu_oracle_seconds_per_iteration(Xs, init_s, n_cpu) * scale
        shape = "x".join(str(d) for d in Xs.shape)
        cpu = {"value": sec * fp32_fit, "unit": "s", "cores": host_cores(), "kind": "oracle",
               "extrapolated": True,
               "sample": f"{n_cpu} FP64 oracle outer iterations on a {shape} slab of {name} "
                         f"(median, x {scale:g} for the full tensor: {sec:.2f} s per "
                         f"iteration) x the {fp32_fit} outer iterations the plain method "
                         "needs to reach the fit"}

    cfg = _workload_config(name)
    cfg.update({"form": args.form, "storage": storage,
                "accumulate": "f32 (Gram, coefficient system: f64)",
                "warm_start": f"learned, first {args.ws_sweeps} sweep(s)" if learned else "none",
                "target_rfe": target,
                "target_from": "the plain method's converged error on the tensor as this form "
                               "stores it x (1 + tol)",
                "fp32_target_rfe": target32,
                "final_rfe": final_rfe, "final_rfe_vs_fp32_tensor": rfe_vs_fp32,
                "outer_iters_to_fit": statistics.mean(iters),
                "fp32_outer_iters_to_fit": fp32_fit, "ms_per_outer_iter": sweep_ms,
                "l2": "inputs larger than L2 (tensor streamed twice per iteration)",
                "parallelism": "replicas" if world > 1 else "single GPU"})
    line = {
        "metric": METRIC, "value": value_s, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16" if storage == "bf16" else "f32",
        "data": "synthetic (drawn on the device with the workload's recipe)",
        "config": cfg,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(prof["kernel_launches"]),
        "clocks": clk.summary(),
        "training": training,
        "variants": variants,
    }
    print(json.dumps(line), flush=True)


def run_kernel_case(args):
    """Standalone MTTKRP calls on a small-but-larger-than-L2 tensor (for ncu captures):
    mode 0 runs the X * KR_right contraction, the last mode the X^T * KR_left one.  Prints
    the CUDA-event time of each (contraction plus its small second-level reduction)."""
    import torch
    from paper_1409_2383_gb300 import ntf
    dims = tuple(int(d) for d in args.dims.split("x"))
    g = torch.Generator(device="cuda").manual_seed(0)    # U[0, 1] entries, drawn on the device
    X = torch.rand(dims, generator=g, device="cuda")
    if args.storage == "bf16":
        X = ntf.to_bf16(X)
    F = [torch.rand(d, args.rank, generator=g, device="cuda") for d in dims]
    engine = {"auto": ntf.NTF_CONTRACT_AUTO, "tensor": ntf.NTF_CONTRACT_TENSOR,
              "simt": ntf.NTF_CONTRACT_SIMT}[args.engine]
    times = {0: [], len(dims) - 1: []}
    with ntf.Context(X, args.rank,
                     ntf.default_params(contraction=engine, tensor_copy=TENSOR_COPY)) as ctx:
        for it in range(args.warmup + args.steps):
            for n in (0, len(dims) - 1):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                ctx.mttkrp(n, F)
                e1.record()
                e1.synchronize()
                if it >= args.warmup:
                    times[n].append(e0.elapsed_time(e1) * 1e3)
    nbytes = X.numel() * X.element_size()
    us = {f"mode{n}_us": statistics.median(v) for n, v in times.items()}
    gbs = {f"mode{n}_gbs": nbytes / (statistics.median(v) * 1e-6) / 1e9 for n, v in times.items()}
    print(json.dumps({"kernel_case": args.dims, "rank": args.rank, "storage": args.storage,
                      "engine": args.engine, "calls": 2 * (args.warmup + args.steps), **us,
                      **gbs}))


def measure_sparse(dims, nnz: int, R: int, reps: int = 5) -> dict:
    """Sparse-tensor MTTKRP (coordinate form, Sec. IV-A's sparse case) on nnz uniformly drawn
    coordinates of a tensor of shape dims (indices and U[0,1] values drawn on the device): the
    layout build time and, per mode, the MTTKRP time (CUDA events, median of `reps` after one
    warm-up) with its throughput against the HBM peak; algorithmic bytes per nonzero = the
    (N + 1) 4-byte words of the mode's layout streamed once (the factor rows it gathers are
    L2-resident; the output is I_n R floats)."""
    import torch
    from paper_1409_2383_gb300 import ntf
    g = torch.Generator(device="cuda").manual_seed(7)
    idx = torch.stack([torch.randint(0, int(d), (nnz,), generator=g, device="cuda",
                                     dtype=torch.int32) for d in dims], dim=1).contiguous()
    vals = torch.rand(nnz, generator=g, device="cuda")
    F = [torch.rand(int(d), R, generator=g, device="cuda") for d in dims]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sp = ntf.SparseTensor(idx, vals, dims)
    build_s = time.perf_counter() - t0
    del idx, vals
    peak, peak_kind = _peaks()
    N = len(dims)
    modes = []
    for n in range(N):
        out = torch.empty(int(dims[n]), R, device="cuda")
        sp.mttkrp(n, F, out=out)
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            sp.mttkrp(n, F, out=out)
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1) * 1e-3)
        t = statistics.median(ts)
        bytes_ = nnz * (N + 1) * 4 + int(dims[n]) * R * 4
        modes.append({"mode": n, "ms": t * 1e3, "gbs": bytes_ / t / 1e9,
                      "frac": bytes_ / t / 1e9 / peak, "gnnz_per_s": nnz / t / 1e9,
                      "gflops": 3 * nnz * R / t / 1e9})
    sp.close()
    return {"dims": list(dims), "nnz": nnz, "rank": R, "layout_build_s": build_s,
            "bytes_per_nonzero": (N + 1) * 4, "peak": peak, "peak_kind": peak_kind,
            "modes": modes}


def run_sparse_case(args):
    dims = tuple(int(d) for d in args.dims.split("x"))
    print(json.dumps({"sparse_case": measure_sparse(dims, args.nnz, args.rank,
                                                    reps=max(args.steps, 1))}))


def run_sweep_case(args):
    """A few outer iterations of the benchmark workload in the chosen storage (for ncu launch
    lists of the whole sweep): one eager sweep, then graph replays."""
    import torch
    from paper_1409_2383_gb300 import ntf
    w = WORKLOADS[args.workload]
    RANK = w["R"]
    Xd, init = device_workload(args.workload, 0)
    if args.storage == "bf16":
        Xd = ntf.to_bf16(Xd)
    p = ntf.default_params(paper_mode=False, eps_abs=0.0, eps_rel=0.0, tensor_copy=TENSOR_COPY)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        A = [f.clone() for f in init]
        At = [a.clone() for a in A]
        Y = [torch.zeros_like(a) for a in A]
        with ntf.Context(Xd, RANK, p, stream=stream) as ctx:
            ctx.trace_enable(args.trace)
            rs = ctx.run(A, At, Y, args.steps)
            trace = ctx.trace_get() if args.trace else None
        stream.synchronize()
    print(json.dumps({"sweep_case": args.workload, "storage": args.storage, "sweeps": args.steps,
                      "rel_err": rs["rel_err"], "trace_last_sweep": trace}))


def table_cases(name: str = "table1_rfe.txt"):
    """Scenarios of the paper's Table 1 (Sec. VI-A) with their printed mean RFE, from the
    stored fixture: (dims, F, sigma2, printed mean RFE)."""
    rows = []
    with open(os.path.join(ROOT, "tests", "golden", name)) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                I, J, K, F, s2, v = line.split()
                rows.append(((int(I), int(J), int(K)), int(F), float(s2), float(v)))
    return rows


def study_case(dims, F, sigma2, realizations, n_max, max_restarts, open_ctx, device,
               sync=lambda: None):
    """One scenario of the paper's experiments (Sec. VI-A) in paper mode: for realization r,
    X = [A, B, C] + N (U[0,1] factors of data seed r, i.i.d. N(0, sigma2) noise) is
    factorized from B0, C0 i.i.d. U[0,1] (attempt k of realization r: init seed
    1000 (r + 1) + k), auxiliaries and duals zero, rho0 = 1, until the residual test holds
    within n_max outer iterations, restarting from a new random point otherwise.
    `open_ctx(X, F)` opens a context; returns the scenario's statistics."""
    import torch
    from paper_1409_2383_gb300 import restarts
    import synth
    rfe, secs, nrest, iters, total, conv = [], [], [], [], [], 0
    for r in range(realizations):
        X, _, _ = synth.workload(dims, F, seed=r, snr_db=None, sigma2=sigma2)
        Xd = torch.as_tensor(X).to(device)
        A = [torch.zeros(d, F, device=device) for d in dims]
        At = [torch.zeros_like(a) for a in A]
        Y = [torch.zeros_like(a) for a in A]

        def draw(k, A, At, Y, r=r):
            init = synth.init_factors(dims, F, seed=1000 * (r + 1) + k)
            for a, t, y, f in zip(A, At, Y, init):
                a.copy_(torch.as_tensor(f, dtype=torch.float32))
                t.zero_()
                y.zero_()

        with open_ctx(Xd, F) as ctx:
            sync()
            t0 = time.perf_counter()
            rs = restarts.factorize(ctx, A, At, Y, n_max, draw, max_restarts=max_restarts)
            sync()
            secs.append(time.perf_counter() - t0)
            rfe.append(ctx.fit_explicit(At))
        conv += rs["converged"]
        nrest.append(rs["restarts"])
        iters.append(rs["iters"])
        total.append(rs["restarts"] * n_max + rs["iters"])
    return {"dims": list(dims), "F": F, "sigma2": sigma2, "realizations": realizations,
            "converged": conv, "mean_rfe": statistics.mean(rfe),
            "mean_s": statistics.mean(secs),
            "std_s": statistics.stdev(secs) if len(secs) > 1 else 0.0,
            "mean_restarts": statistics.mean(nrest), "mean_iters_last_attempt":
            statistics.mean(iters), "mean_iters_total": statistics.mean(total)}


def run_study(args, open_ctx=None, device="cuda"):
    """The scenarios of the paper's Table 1 (or Table 2) on the GPU in paper mode (L = 1,
    primal Khatri-Rao, adaptive rho, eps_abs = eps_rel = 1e-4 (Table 2: 1e-3), n_max = 400,
    restarts): one JSON line per scenario with the mean RFE beside the printed one and the
    time per factorization.
    (open_ctx / device: a stand-in context on the host, for tests of the loop.)"""
    import contextlib
    import torch
    from paper_1409_2383_gb300 import ntf
    # Table 2 relaxes the stopping tolerances to 1e-3 (Sec. VI-A)
    study = getattr(args, "study", None) or "table1"
    tol = 1e-3 if study == "table2" else 1e-4
    p = ntf.default_params(paper_mode=True, eps_abs=tol, eps_rel=tol)
    cases = table_cases(f"{study}_rfe.txt")
    if args.study_cases:
        keep = {int(i) for i in args.study_cases.split(",")}
        cases = [c for i, c in enumerate(cases) if i in keep]
    if device == "cuda":
        stream = torch.cuda.Stream()       # a non-default stream: sweeps replay as CUDA graphs
        scope, sync = (lambda: torch.cuda.stream(stream)), torch.cuda.synchronize
        if open_ctx is None:
            open_ctx = lambda X, R: ntf.Context(X, R, p, stream=stream)  # noqa: E731
    else:
        scope, sync = contextlib.nullcontext, (lambda: None)
    for dims, F, s2, printed in cases:
        with scope():
            res = study_case(dims, F, s2, args.realizations, 400, args.max_restarts,
                             open_ctx, device, sync)
        res.update({"study": study, "printed_mean_rfe": printed,
                    "rfe_vs_printed": res["mean_rfe"] / printed, "data": "synthetic",
                    "settings": "L=1, kr_source=primal, adaptive rho (1, 8, 4, 2), "
                                f"eps {tol:g}, n_max 400"})
        print(json.dumps(res), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ntf", choices=["ntf", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip timing the other storage forms")
    ap.add_argument("--form", default="bf16_learned", choices=sorted(FORMS),
                    help="the timed form: BF16 or FP32 storage, with or without the learned "
                         "warm start")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS),
                    help="the evaluation workload of the headline line")
    ap.add_argument("--no-learned", action="store_true",
                    help="variants: skip the learned warm start (no network training)")
    ap.add_argument("--train-rows", type=int, default=1_000_000)
    ap.add_argument("--train-epochs", type=float, default=20.0)
    ap.add_argument("--robust-tensors", type=int, default=10,
                    help="other tensors on which the learned warm start is compared with plain")
    ap.add_argument("--ws-sweeps", type=int, default=1,
                    help="outer iterations of each run in which the network is consulted")
    ap.add_argument("--kernel-case", action="store_true",
                    help="standalone MTTKRP calls only (profiling case)")
    ap.add_argument("--dims", default="384x384x384")
    ap.add_argument("--rank", type=int, default=20)
    ap.add_argument("--storage", default="fp32", choices=["fp32", "bf16"])
    ap.add_argument("--engine", default="auto", choices=["auto", "tensor", "simt"])
    ap.add_argument("--sparse-case", action="store_true",
                    help="sparse-tensor MTTKRP on --nnz random coordinates of --dims")
    ap.add_argument("--nnz", type=int, default=100_000_000)
    ap.add_argument("--sweep-case", action="store_true",
                    help="run --steps outer iterations of the workload (for ncu launch lists)")
    ap.add_argument("--trace", action="store_true",
                    help="with --sweep-case: print the per-stream timeline of the last sweep")
    ap.add_argument("--study", choices=["table1", "table2"],
                    help="the scenarios of the paper's Table 1 or 2 in paper mode (one line "
                         "each)")
    ap.add_argument("--study-cases", default="",
                    help="with --study: comma-separated indices of the scenarios to run")
    ap.add_argument("--tensor-copy", type=int, default=0, choices=[-1, 0, 1],
                    help="ntf_params.tensor_copy: the second contraction on a transposed copy "
                         "of the tensor (0: FP32 storage where it fits, 1: also BF16, -1: never)")
    ap.add_argument("--realizations", type=int, default=10)
    ap.add_argument("--max-restarts", type=int, default=10)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    global TENSOR_COPY
    TENSOR_COPY = args.tensor_copy
    if args.study:
        run_study(args)
    elif args.kernel_case:
        run_kernel_case(args)
    elif args.sparse_case:
        run_sparse_case(args)
    elif args.sweep_case:
        run_sweep_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ntf(args)


if __name__ == "__main__":
    main()
