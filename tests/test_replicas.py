"""Host logic of bench.py on CPU: the multi-process path (gloo, world size 2; replicas run
independently and the job's figures are the maximum over ranks), the reference arm (rank 0
only, the contract's keys), the clock summary, the slab partition of the paper's distributed
scheme on the oracle, and the loop of the Table 1 study on a stand-in context."""
import importlib.util
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    bench = _bench()
    w, r, local = bench._dist()
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # per-rank time and end-to-end time of a replica; the job's are the maxima
        got = bench.max_over_ranks([1.0 + rank, 10.0 - rank], "cpu")
        out.put((rank, (w, r, local), got))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, (w, r, local), got in res:
        assert (w, r, local) == (2, rank, rank)
        assert got == [2.0, 10.0]


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    bench = _bench()
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")

    class Args:
        gpus, steps, warmup, workload = 2, 1, 0, bench.DEFAULT_WORKLOAD

    called = []
    monkeypatch.setattr(bench, "oracle_sample", lambda name, seed=0: called.append(name))
    bench.run_reference(Args())
    assert called == [] and capsys.readouterr().out == ""


def test_reference_arm_line_on_rank_zero(monkeypatch, capsys):
    """Rank 0 of the reference arm prints one JSON line with the keys of the benchmark
    contract: the oracle's time per iteration on a slab, scaled to the full tensor, times the
    iterations the method needs to reach the fit."""
    import json
    bench = _bench()
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)

    class Args:
        gpus, steps, warmup, workload = 1, 2, 3, bench.DEFAULT_WORKLOAD

    monkeypatch.setattr(bench, "oracle_sample",
                        lambda name, seed=0: (np.zeros((4, 5, 6)), None, 10.0))
    monkeypatch.setattr(bench, "cpu_oracle_seconds_per_iteration", lambda X, init, n: 0.5)
    bench.run_reference(Args())
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    n_iter = bench.WORKLOADS[bench.DEFAULT_WORKLOAD]["fit_iters"]
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC
    assert d["value"] == pytest.approx(0.5 * 10.0 * n_iter) and d["higher_is_better"] is False
    assert d["cpu_baseline"]["value"] == d["value"] and d["cpu_baseline"]["kind"] == "oracle"
    assert d["cpu_baseline"]["extrapolated"] is True
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == bench.DEFAULT_WORKLOAD


def test_oracle_sample_is_a_slab_of_the_workload():
    """The oracle's sample of the 1000^3 workload is a slab over the last mode with at most
    1e8 entries; the scale brings its time per iteration to the full tensor."""
    bench = _bench()
    dims = bench.WORKLOADS[bench.DEFAULT_WORKLOAD]["dims"]
    rest = int(np.prod(dims[:-1]))
    last = max(1, min(dims[-1], bench.ORACLE_SAMPLE_NUMEL // rest))
    assert last * rest <= bench.ORACLE_SAMPLE_NUMEL
    assert (rest * dims[-1]) / (rest * last) == pytest.approx(10.0)
    X, init, scale = bench.oracle_sample("400x400x400_r20")   # small enough: the whole tensor
    assert X.shape == (400, 400, 400) and scale == 1.0 and len(init) == 3


def test_clock_summary_reads_the_samples_of_the_timed_region():
    bench = _bench()
    s = bench.ClockSampler(0)
    s.lines = ["1965, 2070, Not Active, Not Active, Not Active, Not Active",   # before the region
               "2070, 2070, Not Active, Not Active, Not Active, Active",
               "2055, 2070, Not Active, Not Active, Not Active, Not Active",
               "garbage line"]
    s.skip = 1
    got = s.summary()
    assert got["samples"] == 2 and got["sm_mhz"] == 2062.5 and got["sm_max_mhz"] == 2070.0
    assert got["reasons"] == ["sw_power_cap"]
    s.lines, s.skip = s.lines[:1], 1           # a region shorter than the sampling period
    assert s.summary()["samples"] == 1
    s.lines = []
    assert s.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def _slab_worker(rank, world, port, out):
    """Sec. V's block scheme on the oracle: each rank holds a slab of X along mode 1 and the
    factors; its MTTKRP of modes 2 and 3 over the slab are partial sums, added across ranks by
    one all-reduce; mode 1's rows are its own slab's."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import numpy as np
    import torch
    import torch.distributed as dist
    from oracle import ntf as o
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rng = np.random.default_rng(0)
        dims, R = (10, 7, 6), 3
        X = rng.random(dims)
        F = [rng.random((d, R)) for d in dims]
        lo, hi = rank * dims[0] // world, (rank + 1) * dims[0] // world
        Fs = [F[0][lo:hi], F[1], F[2]]
        got = []
        for n in (1, 2):
            part = torch.as_tensor(o.mttkrp(X[lo:hi], Fs, n))
            dist.all_reduce(part)
            got.append(part.numpy())
        rows0 = o.mttkrp(X[lo:hi], Fs, 0)
        want = [o.mttkrp(X, F, n) for n in (1, 2)]
        out.put((rank, all(np.allclose(g, w, rtol=1e-12, atol=0) for g, w in zip(got, want)),
                 np.allclose(rows0, o.mttkrp(X, F, 0)[lo:hi], rtol=1e-12, atol=0)))
    finally:
        dist.destroy_process_group()


def test_slab_partitioned_mttkrp_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_slab_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, True, True), (1, True, True)]


def _slab_iteration_worker(rank, world, port, out):
    """Sec. V-B on the oracle: whole outer iterations with the tensor and the first factor's
    rows split into slabs over the ranks.  The first factor's update is row-local (its
    coefficient matrix needs only the replicated factors); the others take their MTTKRP and
    the first factor's Gram as sums over the slabs (one all-reduce each) and are then updated
    identically on every rank.  The result equals the centralized iteration."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import numpy as np
    import torch
    import torch.distributed as dist
    import synth
    from oracle import ntf as o
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dims, R, L = (11, 7, 6), 3, 5
        X = synth.workload(dims, R, seed=3, snr_db=20.0)[0].astype(np.float64)
        init = synth.init_factors(dims, R, 4)
        ref = o.init_state(init, o.AO)
        lo, hi = rank * dims[0] // world, (rank + 1) * dims[0] // world
        At = [init[0][lo:hi].copy(), init[1].copy(), init[2].copy()]
        Y = [np.zeros_like(F) for F in At]

        def allsum(a):
            t = torch.as_tensor(np.ascontiguousarray(a))
            dist.all_reduce(t)
            return t.numpy()

        for _ in range(2):
            o.outer_iteration(X, ref, o.AO)
            Xs = X[lo:hi]
            # factor 1: rows of this slab, coefficient matrix from the replicated factors
            G = o.gram(At[1]) * o.gram(At[2])
            _, At[0], Y[0], _ = o.admm_factor_update(o.mttkrp(Xs, At, 0), G, At[0], Y[0],
                                                     o.rho_trace(G), L)
            GA = allsum(o.gram(At[0]))       # Gram of the split factor: a sum over slabs
            for n in (1, 2):
                M = allsum(o.mttkrp(Xs, At, n))
                G = GA * o.gram(At[3 - n])
                _, At[n], Y[n], _ = o.admm_factor_update(M, G, At[n], Y[n], o.rho_trace(G), L)
        ok = (np.allclose(At[0], ref.aux[0][lo:hi], rtol=1e-10, atol=1e-13)
              and np.allclose(Y[0], ref.dual[0][lo:hi], rtol=1e-10, atol=1e-13)
              and all(np.allclose(At[n], ref.aux[n], rtol=1e-10, atol=1e-13) and
                      np.allclose(Y[n], ref.dual[n], rtol=1e-10, atol=1e-13) for n in (1, 2)))
        out.put((rank, ok))
    finally:
        dist.destroy_process_group()


def test_slab_partitioned_outer_iterations_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_slab_iteration_worker, args=(r, 2, port, out))
             for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, True), (1, True)]


def test_table1_study_loop_on_a_stand_in_context():
    """The Table 1 study of bench.py (paper mode with restarts, Sec. VI-A): the scenarios come
    from the stored fixture; every attempt starts from its own random B0, C0 with zero
    auxiliaries and duals; the statistics count restarts and iterations over attempts."""
    import numpy as np
    import torch
    import synth
    bench = _bench()
    cases = bench.table_cases()
    assert len(cases) == 12 and cases[0] == ((3000, 50, 50), 3, 1e-2, 0.2156)
    assert cases[-1] == ((200, 200, 200), 30, 1e-4, 0.0026)

    seen = []

    class Ctx:
        def __init__(self, X, R):
            self.X, self.R, self.k = X, R, 0

        def __enter__(self):
            return self

        def __exit__(self, *exc):
            pass

        def run(self, A, At, Y, n_max, target_rfe=0.0, check_every=1):
            seen.append(([a.clone() for a in A], [float(t.abs().sum()) for t in At + Y]))
            self.k += 1
            ok = self.k >= 2                        # every realization restarts once
            return {"iters": 17 if ok else n_max, "converged": int(ok),
                    "reached_target": 0, "rel_err": 0.0}

        def fit_explicit(self, F):
            return float(self.X.abs().mean())

    dims, F = (6, 5, 4), 2
    res = bench.study_case(dims, F, 1e-2, 2, 30, 5, Ctx, "cpu")
    assert res["realizations"] == 2 and res["converged"] == 2
    assert res["mean_restarts"] == 1 and res["mean_iters_last_attempt"] == 17
    assert res["mean_iters_total"] == 30 + 17
    assert len(seen) == 4
    for i, (A, zeros) in enumerate(seen):
        r, k = divmod(i, 2)
        want = synth.init_factors(dims, F, seed=1000 * (r + 1) + k)
        for a, w in zip(A, want):
            assert np.array_equal(a.numpy(), w.astype(np.float32))
        assert zeros == [0.0] * 6
    X0 = synth.workload(dims, F, seed=0, snr_db=None, sigma2=1e-2)[0]
    X1 = synth.workload(dims, F, seed=1, snr_db=None, sigma2=1e-2)[0]
    assert res["mean_rfe"] == pytest.approx((np.abs(X0).mean() + np.abs(X1).mean()) / 2,
                                            rel=1e-6)


def test_table1_study_lines(capsys):
    """run_study prints one JSON line per chosen scenario, the mean error beside the printed
    one (stand-in context on the host whose error is the printed value)."""
    import json
    bench = _bench()

    class Args:
        study, study_cases, realizations, max_restarts = "table1", "8", 2, 0

    class Ctx:
        def __init__(self, X, R):
            pass

        def __enter__(self):
            return self

        def __exit__(self, *exc):
            pass

        def run(self, A, At, Y, n_max, target_rfe=0.0, check_every=1):
            return {"iters": 40, "converged": 1, "reached_target": 0, "rel_err": 0.0}

        def fit_explicit(self, F):
            return 0.14

    bench.run_study(Args(), open_ctx=Ctx, device="cpu")
    lines = [json.loads(ln) for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = lines[0]
    assert d["study"] == "table1" and d["dims"] == [200, 200, 200] and d["F"] == 5
    assert d["sigma2"] == 1e-2 and d["printed_mean_rfe"] == 0.14
    assert d["rfe_vs_printed"] == pytest.approx(1.0) and d["converged"] == 2
    assert d["mean_iters_total"] == 40 and d["mean_restarts"] == 0
