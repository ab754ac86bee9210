"""What the trained warm-start network gains over the plain method.

The network is trained (by the library's kernels) on rows harvested from the first
sweep of tensors of the workload generator with other seeds, then consulted in the first
sweep of factorizations of held-out tensors.  The test requires that the network wins a
substantial share of the first sweep's rows under the judge (smaller row objective and smaller
KKT residual than the carried-over start), that the error after the first sweep is lower with
it, and that the final fit is the plain method's (the plain iterations refine every row either
way).  On four held-out tensors it also runs both forms to the same KKT tolerance (eq.
KKT_NTF: scaled dual infeasibility <= 1e-5, complementarity <= 1e-6) and asserts the measured
effect on the number of outer iterations: both forms reach the tolerance and the mean counts
differ by less than a quarter -- the first sweep's gain does not carry through the slow phase
of the factorization (the benchmark's ten held-out tensors per workload say the same at full
size)."""
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ntf():
    from paper_1409_2383_gb300 import build, ntf as binding
    build.build()
    binding.lib()
    return binding


def _history(ntf, X, R, init, sweeps, net=None):
    p = ntf.default_params(paper_mode=False, eps_abs=0.0, eps_rel=0.0)
    A = [f.clone() for f in init]
    At = [f.clone() for f in init]
    Y = [torch.zeros_like(f) for f in init]
    with ntf.Context(X, R, p) as ctx:
        if net is not None:
            ctx.attach_warmstart(net, 1)
        ctx.profile_enable(True)
        h = ctx.run(A, At, Y, sweeps, history=True)["history"]
        prof = ctx.profile_get()
    return h, prof


def test_trained_network_on_held_out_tensor(ntf):
    from paper_1409_2383_gb300 import warmstart
    dims, R, H = (64, 64, 64), 8, 128
    rows = warmstart.training_set(dims, R, rows=60000, sweeps=1, seed0=1)
    net = ntf.Mlp(R, H, warmstart.init_params(R, H, seed=0), max_rows=16 * max(dims),
                  max_groups=64)
    before = warmstart.eval_loss(net, rows, 16)
    warmstart.train(net, rows, steps=2000, groups_per_batch=64, lr=1e-3, decay_at=0.7,
                    rows_per_group=16)
    after = warmstart.eval_loss(net, rows, 16)
    assert after < 0.2 * before

    X, init = warmstart.synthetic_tensor(dims, R, seed=999999)
    plain, _ = _history(ntf, X, R, init, 150)
    learned, prof = _history(ntf, X, R, init, 150, net)
    considered, accepted = prof["ws_rows_considered"], prof["ws_rows_accepted"]
    target = plain[-1] * (1 + 1e-3)
    it_plain = next(i + 1 for i, v in enumerate(plain) if v <= target)
    it_learned = next((i + 1 for i, v in enumerate(learned) if v <= target), None)
    print(f"\nloss {before:.4g} -> {after:.4g}; first sweep: network kept for "
          f"{accepted}/{considered} rows; rel. error after sweeps 1-3: plain "
          f"{plain[:3]}, learned {learned[:3]}; iterations to the fit: plain {it_plain}, "
          f"learned {it_learned}")
    assert considered == sum(dims)               # consulted in the first sweep only
    assert accepted >= 0.2 * considered
    assert learned[0] < plain[0]
    assert it_learned is not None
    assert abs(learned[-1] - plain[-1]) <= 1e-3 * plain[-1]
    net.close()


def test_iterations_to_the_kkt_tolerance_on_held_out_tensors(ntf):
    from paper_1409_2383_gb300 import warmstart
    dims, R, H = (64, 64, 64), 8, 128
    rows = warmstart.training_set(dims, R, rows=60000, sweeps=1, seed0=1)
    net = ntf.Mlp(R, H, warmstart.init_params(R, H, seed=0), max_rows=16 * max(dims),
                  max_groups=64)
    warmstart.train(net, rows, steps=2000, groups_per_batch=64, lr=1e-3, decay_at=0.7,
                    rows_per_group=16)
    p = ntf.default_params(paper_mode=False, eps_abs=0.0, eps_rel=0.0, kkt_dual_tol=1e-5,
                           kkt_comp_tol=1e-6)
    plain, learned = [], []
    for seed in range(500000, 500004):
        X, init = warmstart.synthetic_tensor(dims, R, seed=seed)
        a = warmstart.time_to_fit(X, R, init, 0.0, 400, params=p)
        b = warmstart.time_to_fit(X, R, init, 0.0, 400, net=net, params=p)
        assert a["kkt_met"] and b["kkt_met"]
        assert abs(a["rel_err"] - b["rel_err"]) <= 1e-3 * a["rel_err"]
        plain.append(a["iters"])
        learned.append(b["iters"])
    mp, ml = sum(plain) / 4, sum(learned) / 4
    print(f"\niterations to the KKT tolerance: plain {plain} (mean {mp}), learned {learned} "
          f"(mean {ml})")
    assert abs(ml - mp) < 0.25 * mp
    net.close()
