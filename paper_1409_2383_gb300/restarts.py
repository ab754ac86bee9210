"""Restarts of the outer driver (Sec. VI-A).

The paper runs ADMoM for up to n_max outer iterations (400 in its experiments); if the
stopping test of Sec. IV-C has not held by then, it starts again from another random initial
point, and repeats until the method converges.  This module is that loop on the host around
``Context.run`` (``ntf_run``): every attempt runs on the GPU; the attempts are bounded by
``max_restarts`` (the paper's loop has no bound), and the caller supplies the initial points,
so that the random numbers are the caller's.  Every attempt is a fresh start of the method:
under the adaptive penalty policy the penalties go back to their initial value rho0 (1 in the
paper's experiments) before it, as they do at the start of the paper's method."""
from __future__ import annotations

from typing import Callable, Sequence

import torch

from . import ntf as _ntf


def factorize(ctx, A: Sequence[torch.Tensor], At: Sequence[torch.Tensor],
              Y: Sequence[torch.Tensor], n_max: int,
              draw_init: Callable[[int, Sequence[torch.Tensor], Sequence[torch.Tensor],
                                   Sequence[torch.Tensor]], None],
              max_restarts: int = 10, target_rfe: float = 0.0, check_every: int = 1) -> dict:
    """Runs attempt 0, 1, ... until one converges (the residual test, or rel_err <=
    target_rfe when a target is given) within n_max outer iterations.  Before attempt k,
    ``draw_init(k, A, At, Y)`` writes that attempt's initial state into the tensors in place;
    under the adaptive penalty policy (``ctx.params``) every factor's rho is then reset to
    rho0.
    Returns the last attempt's run statistics with ``restarts`` (attempts before it) and
    ``converged`` (whether it met a rule)."""
    if n_max < 1 or max_restarts < 0:
        raise ValueError("n_max must be >= 1 and max_restarts >= 0")
    params = getattr(ctx, "params", None)
    reset_rho = params is not None and params.rho_policy == _ntf.NTF_RHO_ADAPTIVE
    for attempt in range(max_restarts + 1):
        draw_init(attempt, A, At, Y)
        if reset_rho:
            for m in range(len(A)):
                ctx.set_rho(m, params.rho0)
        rs = ctx.run(A, At, Y, n_max, target_rfe=target_rfe, check_every=check_every)
        met = bool(rs["converged"] or rs["reached_target"])
        if met:
            break
    out = dict(rs)
    out["restarts"] = attempt
    out["converged"] = int(met)
    return out
