"""Learned warm start for the factor updates: harvest training rows from the plain method,
train the network with the library's kernels, attach it to a factorization.

Everything that computes runs in ``libntf.so``; this module only orchestrates calls and
holds the training rows in device memory.

Training rows: during outer iterations of the plain method on synthetic tensors, every
factor update contributes its coefficient matrix G (without rho) and its MTTKRP rows m_i;
the target of a row is the non-negative least-squares solution reached by running the same
row iteration to convergence (``conv_iters`` inner iterations, fixed rho = trace(G)/R) from
the carried-over state, paired with its dual: [x* ; y*/s], s = trace(G)/R.  The network is
consulted in the first sweeps of a factorization (the cold start), so the training rows come
from the first sweeps of many tensors of the workload's generator (``training_set``).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import ntf


def init_params(R: int, H: int, seed: int) -> torch.Tensor:
    """Glorot-uniform weights, zero biases, in the flat parameter layout of the ABI."""
    g = np.random.default_rng(seed)
    Din, Dout = R * R + 2 * R, 2 * R

    def glorot(fo, fi):
        a = math.sqrt(6.0 / (fi + fo))
        return g.uniform(-a, a, (fo, fi))

    parts = [glorot(H, Din), np.zeros(H), glorot(H, H), np.zeros(H), glorot(Dout, H),
             np.zeros(Dout)]
    return torch.as_tensor(np.concatenate([p.reshape(-1) for p in parts]), dtype=torch.float32)


@dataclass
class RowSet:
    """Training rows grouped by coefficient matrix (device tensors)."""
    R: int
    Gn: List[torch.Tensor] = field(default_factory=list)       # [R*R] each
    mrows: List[torch.Tensor] = field(default_factory=list)    # [rows, 2R] each: [m/s ; z]
    targets: List[torch.Tensor] = field(default_factory=list)  # [rows, 2R] each
    _packed: Optional[tuple] = None

    @property
    def rows(self) -> int:
        return sum(int(m.shape[0]) for m in self.mrows)

    def batch(self, idx: Sequence[int]):
        """Whole groups idx as one batch: (Gn [g, R^2], CSR offsets, row inputs, targets)."""
        Gn = torch.stack([self.Gn[i] for i in idx])
        mr = torch.cat([self.mrows[i] for i in idx])
        tg = torch.cat([self.targets[i] for i in idx])
        offs = [0]
        for i in idx:
            offs.append(offs[-1] + int(self.mrows[i].shape[0]))
        return Gn, torch.tensor(offs, dtype=torch.int32, device=mr.device), mr, tg

    def sample(self, groups: int, rows_per_group: int, gen: torch.Generator):
        """A training batch of `rows_per_group` random rows from each of `groups` random
        groups: many coefficient matrices per step (whole-group batches see only a few and
        train markedly worse)."""
        if self._packed is None or self._packed[0] != len(self.Gn):
            sizes = torch.tensor([int(m.shape[0]) for m in self.mrows], device=self.Gn[0].device)
            start = torch.cumsum(sizes, 0) - sizes
            self._packed = (len(self.Gn), torch.stack(self.Gn), torch.cat(self.mrows),
                            torch.cat(self.targets), start, sizes)
        n, G_all, M_all, T_all, start, sizes = self._packed
        dev = G_all.device
        gi = torch.randint(n, (groups,), generator=gen, device=dev)
        u = torch.rand(groups, rows_per_group, generator=gen, device=dev)
        ridx = (start[gi][:, None] + (u * sizes[gi][:, None]).long()).reshape(-1)
        offs = torch.arange(0, groups * rows_per_group + 1, rows_per_group, dtype=torch.int32,
                            device=dev)
        return (G_all[gi].contiguous(), offs, M_all[ridx].contiguous(),
                T_all[ridx].contiguous())


def _collinear_weight(congruence: float) -> float:
    """Mixing weight a of columns a u0 + (1 - a) u_r (u0, u_r i.i.d. U[0,1]) whose expected
    congruence is `congruence` (moments of U[0,1]: E[u^2] = 1/3, E[u u'] = 1/4), by
    bisection."""
    def c(a):
        cross = a * a / 3 + a * (1 - a) / 2 + (1 - a) ** 2 / 4
        return cross / (a * a / 3 + a * (1 - a) / 2 + (1 - a) ** 2 / 3)
    lo, hi = 0.0, 1.0
    for _ in range(100):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if c(mid) < congruence else (lo, mid)
    return 0.5 * (lo + hi)


def synthetic_tensor(dims: Sequence[int], R: int, seed: int, snr_db: float = 20.0,
                     device: str = "cuda", structure: str = "uniform",
                     zero_frac: float = 0.5, congruence: float = 0.9):
    """Tensor and start of a synthetic workload, drawn on the device with the device's random
    streams: factors i.i.d. uniform[0, 1] (``structure="sparse"``: each entry zeroed with
    probability `zero_frac`; ``"collinear"``: column r = a u0 + (1 - a) u_r with the weight a
    of expected congruence `congruence`), X = [F_1, ..., F_N] + i.i.d. Gaussian noise at
    `snr_db` (SNR = ||X_0||^2 / (numel sigma^2), ||X_0||^2 from the Hadamard product of the
    factors' Grams), start factors i.i.d. uniform[0, 1].  The recipe of the host generator of
    the tests."""
    g = torch.Generator(device=device).manual_seed(int(seed))
    F = []
    for d in dims:
        f = torch.rand(int(d), R, generator=g, device=device)
        if structure == "sparse":
            f[torch.rand(int(d), R, generator=g, device=device) < zero_frac] = 0.0
            for r in (f.max(dim=0).values <= 0).nonzero().flatten().tolist():
                while not bool((f[:, r] > 0).any()):  # an all-zero column: draw it again
                    col = torch.rand(int(d), generator=g, device=device)
                    col[torch.rand(int(d), generator=g, device=device) < zero_frac] = 0.0
                    f[:, r] = col
        elif structure == "collinear":
            a = _collinear_weight(congruence)
            u0 = torch.rand(int(d), 1, generator=g, device=device)
            f = a * u0 + (1 - a) * f
        elif structure != "uniform":
            raise ValueError(f"unknown structure {structure!r}")
        F.append(f)
    # X = KR(leading factors) KR(trailing factors)^T as one product, then the tensor's shape
    def kr(fs):
        t = fs[0]
        for f in fs[1:]:
            t = (t[:, None, :] * f[None, :, :]).reshape(-1, R)
        return t
    s = 2 if len(dims) == 4 else 1
    X = (kr(F[:s]) @ kr(F[s:]).T).reshape([int(d) for d in dims])
    G = torch.ones(R, R, dtype=torch.float64, device=device)
    for f in F:
        G *= f.double().T @ f.double()
    numel = X.numel()
    sigma = math.sqrt(float(G.sum()) / numel / 10.0 ** (snr_db / 10.0))
    X.add_(torch.randn(X.shape, generator=g, device=device), alpha=sigma)
    init = [torch.rand(int(d), R, generator=g, device=device) for d in dims]
    return X, init


def training_set(dims: Sequence[int], R: int, rows: int, sweeps: int = 2, seed0: int = 1,
                 snr_db: float = 20.0, conv_iters: int = 300, storage: str = "fp32",
                 **structure) -> RowSet:
    """Rows of the first `sweeps` outer iterations of synthetic tensors with seeds seed0,
    seed0 + 1, ... until at least `rows` rows are collected (`structure`: the keyword
    arguments of the generator's factor structure)."""
    from . import ntf as _ntf
    out = RowSet(R)
    seed = seed0
    while out.rows < rows:
        X, init = synthetic_tensor(dims, R, seed, snr_db, **structure)
        if storage == "bf16":
            X = _ntf.to_bf16(X)
        harvest(X, R, init, outer=sweeps, rows=out, conv_iters=conv_iters)
        del X
        seed += 1
    return out


def harvest(X: torch.Tensor, R: int, init: Sequence[torch.Tensor], outer: int,
            rows: RowSet, conv_iters: int = 300, params: Optional[ntf.Params] = None,
            every: int = 1) -> RowSet:
    """Run ``outer`` outer iterations of the plain method (Gauss-Seidel over the factors,
    exactly the updates of ``Context.run``) and add the rows of every ``every``-th sweep's
    factor updates to ``rows``."""
    p = params or ntf.default_params(paper_mode=False, eps_abs=0.0, eps_rel=0.0)
    pc = ntf.default_params(paper_mode=False, inner_iters=conv_iters,
                            rho_policy=ntf.NTF_RHO_TRACE, eps_abs=0.0, eps_rel=0.0)
    dims = tuple(int(d) for d in X.shape)
    A = [f.clone() for f in init]
    At = [f.clone() for f in init]
    Y = [torch.zeros_like(f) for f in init]
    with ntf.Context(X, R, p) as ctx, ntf.Context(X, R, pc) as conv:
        for m in range(len(dims)):
            ctx.gram(m, At[m])
            conv.gram(m, At[m])
        for k in range(outer):
            for n in range(len(dims)):
                M = ctx.mttkrp(n, At)
                if k % every == 0:
                    Ac, Tc, Yc = A[n].clone(), At[n].clone(), Y[n].clone()
                    conv.admm_update(n, M, Ac, Tc, Yc, stats=False)
                    # inputs [G/s], [m/s ; z] and targets [x* ; y*/s], formed by the library
                    # with this update's own coefficient system (z = (G + s I)^{-1} m)
                    Gn, mr, tg, _ = conv.warmstart_rows(n, M, Tc, Yc)
                    rows.Gn.append(Gn.reshape(-1))
                    rows.mrows.append(mr)
                    rows.targets.append(tg)
                    conv.gram(n, At[n])  # restore: the converged update refreshed its Gram
                ctx.admm_update(n, M, A[n], At[n], Y[n], stats=False)
                conv.gram(n, At[n])
    torch.cuda.synchronize()
    return rows


def train(net: ntf.Mlp, rows: RowSet, steps: int, groups_per_batch: int, lr: float,
          seed: int = 0, log_every: int = 0, decay_at: float = 1.0,
          rows_per_group: int = 25) -> List[float]:
    """Adam on random batches of `rows_per_group` rows from each of `groups_per_batch` random
    groups (learning rate divided by 10 after a fraction `decay_at` of the steps); returns
    the loss of every logged step."""
    gen = torch.Generator(device=rows.Gn[0].device).manual_seed(seed)
    losses = []
    for t in range(steps):
        Gn, offs, mr, tg = rows.sample(groups_per_batch, rows_per_group, gen)
        want = bool(log_every) and (t % log_every == 0 or t == steps - 1)
        lr_t = lr if t < decay_at * steps else 0.1 * lr
        loss = net.train_step(Gn, offs, mr, tg, lr_t, apply=True, want_loss=want)
        if want:
            losses.append(loss)
    return losses


def eval_loss(net: ntf.Mlp, rows: RowSet, groups_per_batch: int) -> float:
    """Mean loss over all rows (no update)."""
    tot, cnt = 0.0, 0
    for i in range(0, len(rows.Gn), groups_per_batch):
        idx = list(range(i, min(i + groups_per_batch, len(rows.Gn))))
        Gn, offs, mr, tg = rows.batch(idx)
        loss = net.train_step(Gn, offs, mr, tg, 0.0, apply=False, want_loss=True)
        tot += loss * tg.numel()
        cnt += tg.numel()
    return tot / max(cnt, 1)


def time_to_fit(X: torch.Tensor, R: int, init: Sequence[torch.Tensor], target: float,
                max_outer: int, net: Optional[ntf.Mlp] = None, repeats: int = 1,
                params: Optional[ntf.Params] = None, ws_sweeps: int = 1):
    """Time (CUDA events) of factorizations from `init` until rel_err <= target (or another
    stopping rule of `params`: the KKT tolerances), on a fresh non-default stream (so the
    sweep is replayed as a CUDA graph).  Returns a dict with the median seconds, iterations,
    final error, the rules met, the KKT measures and the warm-start row counts."""
    p = params or ntf.default_params(paper_mode=False, eps_abs=0.0, eps_rel=0.0)
    stream = torch.cuda.Stream()
    times, res = [], None
    with torch.cuda.stream(stream):
        A = [f.clone() for f in init]
        At = [f.clone() for f in init]
        Y = [torch.zeros_like(f) for f in init]
        with ntf.Context(X, R, p, stream=stream) as ctx:
            if net is not None:
                ctx.attach_warmstart(net, ws_sweeps)
            ctx.profile_enable(True)             # recorded in the graph from the first run
            prof0 = prof = ctx.profile_get()
            for rep in range(repeats + 1):      # the first run records the graph
                for a, t, y, f in zip(A, At, Y, init):
                    a.copy_(f)
                    t.copy_(f)
                    y.zero_()
                prof0 = ctx.profile_get()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                res = ctx.run(A, At, Y, max_outer, target_rfe=target)
                e1.record(stream)
                e1.synchronize()
                prof = ctx.profile_get()
                if rep > 0 or repeats == 0:
                    times.append(e0.elapsed_time(e1) / 1000.0)
    return {"seconds": float(np.median(times)), "iters": res["iters"],
            "rel_err": res["rel_err"], "reached": bool(res["reached_target"]),
            "kkt_met": bool(res["kkt_met"]), "kkt_dual": res["kkt_dual"],
            "kkt_comp": res["kkt_comp"],
            "ws_considered": prof["ws_rows_considered"] - prof0["ws_rows_considered"],
            "ws_accepted": prof["ws_rows_accepted"] - prof0["ws_rows_accepted"]}
