"""Record the FP64 oracle's relative-error trajectory on a named synthetic workload.

TEST INFRASTRUCTURE ONLY (writes stored expected values; calls nothing but ``oracle/`` and
the input generator).  Usage::

    python -m oracle.trajectory 400x400x400_r20 200 tests/golden/trajectory_400x400x400_r20.json

runs ``iters`` outer iterations of the fixed-penalty inner-loop form (L = 5, Khatri-Rao of
the auxiliaries, rho = trace(G)/R) from the uniform start of seed 1 on the workload of seed 0
and stores the relative error after every iteration plus the time per iteration.
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

import synth
from oracle import ntf as o


def run(name: str, iters: int, out_path: str) -> dict:
    spec = dict(synth.WORKLOADS[name])
    dims, R = spec.pop("dims"), spec.pop("R")
    X, _, init = synth.workload(dims, R, seed=0, **spec)
    X64 = X.astype(np.float64)
    init = [F.astype(np.float32).astype(np.float64) for F in init]
    params = o.Params(inner_iters=5, kr_source="aux", rho_policy="trace")
    st = o.init_state(init, params)
    hist, times = [], []
    for k in range(iters):
        t0 = time.perf_counter()
        o.outer_iteration(X64, st, params)
        times.append(time.perf_counter() - t0)
        hist.append(o.rfe(X64, st.aux))
        print(f"{k + 1} {hist[-1]:.10f} {times[-1]:.2f}s", flush=True)
    res = {"workload": name, "dims": list(dims), "R": R, "data_seed": 0, "init_seed": 1,
           "params": "L=5, kr_source=aux, rho=trace(G)/R", "rfe": hist,
           "seconds_per_iteration": float(np.median(times)), "threads": os.cpu_count()}
    with open(out_path, "w") as f:
        json.dump(res, f, indent=1)
    return res


if __name__ == "__main__":
    run(sys.argv[1], int(sys.argv[2]), sys.argv[3])
