"""GPU parity of the warm-start network against the FP64 oracle (oracle/mlp.py), through the
C ABI: forward outputs, every gradient, the Adam step; training reduces the loss on NNLS rows
solved by the oracle; the warm start inside a factor update keeps, row by row, the candidate
with the smaller KKT residual.  The oracle uses the same BF16-rounded weights as the GPU."""
import math

import numpy as np
import pytest
import torch

from oracle import mlp as om
from oracle import ntf as o

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ntf():
    from paper_1409_2383_gb300 import build, ntf as binding
    build.build()
    binding.lib()
    return binding


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _split(flat, R, H):
    """Flat parameter array -> oracle dict, weights rounded to BF16 as the GPU products use."""
    Din, D = R * R + 2 * R, 2 * R
    sizes = [("W1", (H, Din)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (D, H)),
             ("b3", (D,))]
    out, i = {}, 0
    for k, shp in sizes:
        n = int(np.prod(shp))
        v = torch.as_tensor(flat[i:i + n].copy())
        if k.startswith("W"):
            v = v.to(torch.bfloat16).float()
        out[k] = v.double().numpy().reshape(shp)
        i += n
    return out


def _batch(R, groups, rows_per, seed):
    rng = np.random.default_rng(seed)
    Gn, M, T = [], [], []
    for g in range(groups):
        K = rng.random((3 * R, R))
        G = K.T @ K
        s = np.trace(G) / R
        m = rng.standard_normal((rows_per[g], R)) * s
        X = np.zeros_like(m)
        Yd = np.zeros_like(m)
        for i in range(rows_per[g]):
            X[i], Yd[i] = om.nnls_row(G, m[i])
        U, _ = om.features(G, m)
        Gn.append(G / s)
        M.append(U[:, R * R:])                   # per-row inputs [m/s ; z]
        T.append(om.targets(G, X, Yd, s))
    offs = np.concatenate([[0], np.cumsum(rows_per)]).astype(np.int32)
    return Gn, M, T, offs


def _dev(Gn, M, T, offs):
    return (torch.as_tensor(np.stack([g.reshape(-1) for g in Gn]), dtype=torch.float32).cuda(),
            torch.as_tensor(offs).cuda(),
            torch.as_tensor(np.concatenate(M), dtype=torch.float32).cuda(),
            torch.as_tensor(np.concatenate(T), dtype=torch.float32).cuda())


def _dense_U(Gn, M, offs):
    rows = []
    for g, G in enumerate(Gn):
        for r in range(offs[g], offs[g + 1]):
            rows.append(np.concatenate([G.reshape(-1), M[g][r - offs[g]]]))
    return np.array(rows)


@pytest.mark.parametrize("R,H", [(4, 32), (8, 64), (20, 256), (32, 256), (50, 256)])
def test_forward_and_gradients_match_oracle(ntf, R, H):
    from paper_1409_2383_gb300 import warmstart
    flat = warmstart.init_params(R, H, seed=R).numpy()
    flat[H * (R * R + 2 * R):H * (R * R + 2 * R) + H] = 0.05      # non-zero biases
    net = ntf.Mlp(R, H, torch.as_tensor(flat), max_rows=256, max_groups=8)
    Gn, M, T, offs = _batch(R, 3, [7, 30, 11], seed=R + 1)
    dG, doffs, dM, dT = _dev(Gn, M, T, offs)
    p = _split(flat, R, H)
    U = _dense_U([g.astype(np.float32).astype(np.float64) for g in Gn],
                 [m.astype(np.float32).astype(np.float64) for m in M], offs)
    Tn = np.concatenate(T).astype(np.float32).astype(np.float64)
    out_o, cache = om.forward(p, U)
    out_g = net.forward(dG, doffs, dM).cpu().numpy()
    assert rel(out_g, out_o) <= 1e-4
    grad = torch.empty(net.count, device="cuda")
    loss = net.train_step(dG, doffs, dM, dT, 0.0, apply=False, grad_out=grad)
    assert math.isclose(loss, om.loss(out_o, Tn), rel_tol=1e-4)
    g_o = om.backward(p, cache, out_o, Tn)
    flat_g = grad.cpu().numpy()
    i = 0
    for k, shp in [("W1", (H, R * R + 2 * R)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)),
                   ("W3", (2 * R, H)), ("b3", (2 * R,))]:
        n = int(np.prod(shp))
        assert rel(flat_g[i:i + n].reshape(shp), g_o[k]) <= 2e-4, k
        i += n
    net.close()


def test_adam_first_step(ntf):
    from paper_1409_2383_gb300 import warmstart
    R, H, lr = 4, 16, 1e-3
    flat = warmstart.init_params(R, H, seed=3)
    net = ntf.Mlp(R, H, flat, max_rows=64, max_groups=4)
    Gn, M, T, offs = _batch(R, 2, [5, 9], seed=4)
    dG, doffs, dM, dT = _dev(Gn, M, T, offs)
    grad = torch.empty(net.count, device="cuda")
    net.train_step(dG, doffs, dM, dT, lr, apply=True, grad_out=grad)
    after = net.params().numpy().astype(np.float64)
    g = grad.cpu().numpy().astype(np.float64)
    p = {"w": flat.numpy().astype(np.float64)}
    om.adam_step(p, {"w": g}, {"w": np.zeros_like(g)}, {"w": np.zeros_like(g)}, 1, lr)
    assert np.allclose(after, p["w"], atol=1e-7, rtol=1e-6)
    net.close()


def test_training_reduces_loss(ntf):
    from paper_1409_2383_gb300 import warmstart
    R, H = 5, 64
    rows = warmstart.RowSet(R)
    Gn, M, T, offs = _batch(R, 24, [40] * 24, seed=11)
    for g in range(24):
        rows.Gn.append(torch.as_tensor(Gn[g].reshape(-1), dtype=torch.float32).cuda())
        rows.mrows.append(torch.as_tensor(M[g], dtype=torch.float32).cuda())
        rows.targets.append(torch.as_tensor(T[g], dtype=torch.float32).cuda())
    net = ntf.Mlp(R, H, warmstart.init_params(R, H, seed=5), max_rows=24 * 40, max_groups=24)
    before = warmstart.eval_loss(net, rows, 8)
    warmstart.train(net, rows, steps=400, groups_per_batch=8, lr=2e-3)
    after = warmstart.eval_loss(net, rows, 8)
    assert after < 0.25 * before
    net.close()


@pytest.mark.parametrize("H", [32, 320])  # the fused inference kernels; the GEMM path (H > 256)
def test_warm_start_judge_in_factor_update(ntf, H):
    """Warm start of one factor update: every row starts from the network's candidate if it
    has both the smaller row objective and the smaller KKT residual, else from the
    carried-over state (replayed in FP64 with the oracle network and oracle judge); the final
    state is the oracle update from that start."""
    from paper_1409_2383_gb300 import warmstart
    rng = np.random.default_rng(9)
    dims, R = (40, 30, 20), 4
    X = rng.random(dims).astype(np.float32)
    fs = [rng.random((d, R)).astype(np.float32) for d in dims]
    flat = warmstart.init_params(R, H, seed=2)
    net = ntf.Mlp(R, H, flat, max_rows=64, max_groups=2)
    p = ntf.default_params(inner_iters=2)
    F64 = [f.astype(np.float64) for f in fs]
    n = 0
    M = o.mttkrp(X.astype(np.float64), F64, n).astype(np.float32)
    G = o.coeff_matrix(F64, n)
    At0 = np.maximum(rng.standard_normal((dims[n], R)), 0).astype(np.float32)
    Y0 = (-np.abs(rng.standard_normal((dims[n], R))) * (At0 == 0)).astype(np.float32)
    with ntf.Context(torch.as_tensor(X).cuda(), R, p) as ctx:
        for m in range(3):
            ctx.gram(m, torch.as_tensor(fs[m]).cuda())
        ctx.attach_warmstart(net)
        ctx.profile_enable(True)
        A_d = torch.empty(dims[n], R, device="cuda")
        At_d, Y_d = torch.as_tensor(At0).cuda(), torch.as_tensor(Y0).cuda()
        ctx.admm_update(n, torch.as_tensor(M).cuda(), A_d, At_d, Y_d)
        prof = ctx.profile_get()
    assert prof["ws_rows_considered"] == dims[n]
    # replay in FP64: network candidate vs carried state, judged as the oracle judge does
    Gf = G.astype(np.float32).astype(np.float64)
    U, sf = om.features(Gf, M.astype(np.float64))
    out, _ = om.forward(_split(flat.numpy(), R, H), U)
    xc, yc = om.decode(out, sf, R)

    M64, X0 = M.astype(np.float64), At0.astype(np.float64)
    rc, ro = om.kkt_residual(G, M64, xc), om.kkt_residual(G, M64, X0)
    qc, qo = om.row_objective(G, M64, xc), om.row_objective(G, M64, X0)

    def sure(a, b):  # a < b (+1) or a > b (-1) by a margin FP32 rounding cannot flip; else 0
        gap = 1e-3 * np.maximum(np.abs(a), np.abs(b))
        return np.where(a < b - gap, 1, np.where(a > b + gap, -1, 0))

    kr, kq = sure(rc, ro), sure(qc, qo)
    take_sure = (kr == 1) & (kq == 1)
    keep_sure = (kr == -1) | (kq == -1)
    clear = take_sure | keep_sure
    take = om.judge(G, M64, xc, X0)
    assert np.array_equal(take[clear], take_sure[clear])
    start_t = np.where(take[:, None], xc, At0)
    start_y = np.where(take[:, None], yc, Y0)
    _, At_w, Y_w, _ = o.admm_factor_update(M.astype(np.float64), G, start_t, start_y,
                                           o.rho_trace(G), 2)
    got_t = At_d.cpu().numpy()
    assert rel(got_t[clear], At_w[clear]) <= 1e-3
    assert prof["ws_rows_accepted"] >= int(np.sum(take_sure))
    assert prof["ws_rows_accepted"] <= int(np.sum(~keep_sure))
    assert np.all(got_t >= 0)
    net.close()


def test_harvest_rows_are_converged_nnls_solutions(ntf):
    """Harvested targets solve the row NNLS of their coefficient matrix (KKT of eq. KKT_NTF);
    the z inputs are the first ADMM primal iterates from zero."""
    from paper_1409_2383_gb300 import warmstart
    import synth
    dims, R = (30, 28, 26), 4
    X, _, init = synth.workload(dims, R, seed=3, snr_db=20.0)
    rows = warmstart.harvest(torch.as_tensor(X).cuda(), R,
                             [torch.as_tensor(f, dtype=torch.float32).cuda() for f in init],
                             outer=2, rows=warmstart.RowSet(R), conv_iters=400)
    assert len(rows.Gn) == 6 and rows.rows == 2 * sum(dims)
    for g in range(len(rows.Gn)):
        G = rows.Gn[g].double().cpu().numpy().reshape(R, R)
        u = rows.mrows[g].double().cpu().numpy()
        m, z = u[:, :R], u[:, R:]
        t = rows.targets[g].double().cpu().numpy()
        k = o.kkt_nnls(G, m, t[:, :R], t[:, R:])
        assert k["neg_x"] == 0 and k["dual"] < 1e-4 and k["comp"] < 1e-5
        # z = (G + s I)^{-1} m in the normalised variables: (G/s + I)^{-1} (m/s)
        assert rel(z, np.linalg.solve(G + np.eye(R), m.T).T) <= 1e-5
