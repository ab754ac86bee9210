"""The restart strategy of Sec. VI-A: the oracle's loop on its pins, and the host driver of the
GPU path on a stand-in context (its runs are the library's ntf_run, covered elsewhere)."""
import numpy as np
import pytest

import synth
from oracle import ntf as o


def _draws(dims, R, n):
    return [synth.workload(dims, R, seed=0, snr_db=20.0)[2] if k == 0 else
            [np.random.default_rng(100 + k).random((d, R)) for d in dims] for k in range(n)]


def test_oracle_first_attempt_converges():
    dims, R = (12, 10, 8), 2
    X = synth.workload(dims, R, seed=0, snr_db=20.0)[0].astype(np.float64)
    draws = _draws(dims, R, 3)
    st, hist, conv, restarts = o.factorize_with_restarts(X, draws, o.PAPER, 400)
    assert conv and restarts == 0
    st0, _, conv0 = o.factorize(X, draws[0], o.PAPER, 400)
    for a, b in zip(st.aux, st0.aux):
        assert np.array_equal(a, b)              # the same run as without the loop


def test_oracle_restarts_until_the_draws_run_out_when_nothing_converges():
    dims, R = (12, 10, 8), 2
    X = synth.workload(dims, R, seed=0, snr_db=20.0)[0].astype(np.float64)
    draws = _draws(dims, R, 3)
    st, hist, conv, restarts = o.factorize_with_restarts(X, draws, o.PAPER, 1)
    assert not conv and restarts == 2 and len(hist) == 1
    st2, _, _ = o.factorize(X, draws[2], o.PAPER, 1)
    for a, b in zip(st.aux, st2.aux):
        assert np.array_equal(a, b)              # the state is the last attempt's
    with pytest.raises(ValueError):
        o.factorize_with_restarts(X, [], o.PAPER, 1)


class _Ctx:
    """Stand-in for Context: run k converges from attempt `good` on."""

    def __init__(self, good):
        self.good, self.calls = good, []

    def run(self, A, At, Y, max_outer, target_rfe=0.0, check_every=1):
        k = len(self.calls)
        self.calls.append((max_outer, target_rfe, check_every, A[0]))
        ok = self.good is not None and k >= self.good
        return {"iters": 7 if ok else max_outer, "converged": int(ok and target_rfe == 0.0),
                "reached_target": int(ok and target_rfe > 0.0), "rel_err": 0.1 + k}


def test_driver_restarts_until_an_attempt_converges():
    import torch
    from paper_1409_2383_gb300 import restarts
    drawn = []

    def draw(k, A, At, Y):
        drawn.append(k)
        A[0].fill_(k)

    A, At, Y = [torch.zeros(2)], [torch.zeros(2)], [torch.zeros(2)]
    ctx = _Ctx(good=2)
    rs = restarts.factorize(ctx, A, At, Y, 400, draw, max_restarts=5)
    assert drawn == [0, 1, 2] and rs["restarts"] == 2 and rs["converged"] == 1
    assert rs["rel_err"] == 2.1 and [c[0] for c in ctx.calls] == [400] * 3
    ctx = _Ctx(good=1)
    rs = restarts.factorize(ctx, A, At, Y, 50, draw, max_restarts=5, target_rfe=0.2,
                            check_every=3)
    assert rs["restarts"] == 1 and rs["converged"] == 1 and ctx.calls[0][1:3] == (0.2, 3)


def test_driver_gives_up_after_max_restarts():
    import torch
    from paper_1409_2383_gb300 import restarts
    drawn = []
    A, At, Y = [torch.zeros(2)], [torch.zeros(2)], [torch.zeros(2)]
    rs = restarts.factorize(_Ctx(good=None), A, At, Y, 1, lambda k, *_: drawn.append(k),
                            max_restarts=3)
    assert drawn == [0, 1, 2, 3] and rs["restarts"] == 3 and rs["converged"] == 0
    with pytest.raises(ValueError):
        restarts.factorize(_Ctx(good=0), A, At, Y, 0, lambda *_: None)


class _CtxRho(_Ctx):
    """Stand-in that also records the penalties it is given."""

    def __init__(self, good, policy):
        super().__init__(good)
        from paper_1409_2383_gb300 import ntf
        self.params = ntf.Params(rho_policy=policy, rho0=1.0)
        self.rho_calls = []

    def set_rho(self, m, rho):
        self.rho_calls.append((len(self.calls), m, rho))


def test_driver_resets_adaptive_penalties_before_every_attempt():
    """A restart is a fresh start (Sec. VI-A): rho back to rho0 for every factor before each
    attempt under the adaptive policy, as the oracle's init_state does; the trace and fixed
    policies keep the caller's penalties."""
    import torch
    from paper_1409_2383_gb300 import ntf, restarts
    A = [torch.zeros(2) for _ in range(3)]
    At, Y = [a.clone() for a in A], [a.clone() for a in A]
    ctx = _CtxRho(good=1, policy=ntf.NTF_RHO_ADAPTIVE)
    rs = restarts.factorize(ctx, A, At, Y, 10, lambda *_: None, max_restarts=4)
    assert rs["restarts"] == 1
    assert ctx.rho_calls == [(k, m, 1.0) for k in range(2) for m in range(3)]
    for policy in (ntf.NTF_RHO_TRACE, ntf.NTF_RHO_FIXED):
        ctx = _CtxRho(good=1, policy=policy)
        restarts.factorize(ctx, A, At, Y, 10, lambda *_: None, max_restarts=4)
        assert ctx.rho_calls == []
