"""Structural constraints of Sec. IV-E on the GPU against the FP64 oracle.

The factor update with the auxiliary projected onto a box, or onto the non-negative matrices
with at most c nonzero entries (eq. g_new_def), must match ``oracle.admm_factor_update`` with
the same projection (``project_box``, ``project_nonneg_sparse``, each pinned against brute
force in ``tests/test_oracle_constraints.py``) to relative Frobenius error 1e-5, and the
sparse auxiliary must have the oracle's support.  A whole run with one sparse-constrained
factor (recorded and replayed as a CUDA graph) must track the oracle's outer iterations."""
import numpy as np
import pytest
import torch

import synth
from oracle import ntf as o

pytestmark = pytest.mark.gpu

TOL = 1e-5


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


def _updates(ntf, dims, R, L, policy, cons, seed=11):
    """One factor update per mode from the same random state on the GPU and in the oracle;
    cons(I) -> (kind, lo, hi, c, projection).  Yields (GPU At, oracle At) after checking
    A, At, Y and the residual norms."""
    rng = np.random.default_rng(seed)
    X = (rng.random(dims) - 0.3).astype(np.float32)
    fs = [rng.random((d, R)).astype(np.float32) for d in dims]
    F64 = [F.astype(np.float64) for F in fs]
    pol = ntf.NTF_RHO_TRACE if policy == "trace" else ntf.NTF_RHO_FIXED
    p = ntf.default_params(inner_iters=L, rho_policy=pol, kr_source=ntf.NTF_KR_AUX)
    with ntf.Context(torch.as_tensor(X).cuda(), R, p) as ctx:
        for m in range(len(dims)):
            ctx.gram(m, torch.as_tensor(fs[m]).cuda())
            kind, lo, hi, c, _ = cons(dims[m])
            ctx.set_constraint(m, kind, lo, hi, c)
        for n in range(len(dims)):
            I = dims[n]
            project = cons(I)[4]
            M = o.mttkrp(X.astype(np.float64), F64, n).astype(np.float32)
            At0 = np.maximum(rng.standard_normal((I, R)), 0).astype(np.float32)
            Y0 = (-np.abs(rng.standard_normal((I, R))) * (At0 == 0)).astype(np.float32)
            G = o.coeff_matrix(F64, n)
            rho = o.rho_trace(G) if policy == "trace" else 0.37 * o.rho_trace(G)
            if policy == "fixed":
                ctx.set_rho(n, rho)
            A_d = torch.empty(I, R, device="cuda")
            At_d = torch.as_tensor(At0).cuda()
            Y_d = torch.as_tensor(Y0).cuda()
            st = ctx.admm_update(n, torch.as_tensor(M).cuda(), A_d, At_d, Y_d)
            A, At, Y, s = o.admm_factor_update(M.astype(np.float64), G, At0.astype(np.float64),
                                               Y0.astype(np.float64), rho, L, project=project)
            got_t = At_d.cpu().numpy()
            assert rel(A_d.cpu().numpy(), A) <= TOL, n
            assert rel(got_t, At) <= TOL, n
            # the dual in units of rho At: inside a box it is zero up to FP32 rounding of x - At
            dy = np.linalg.norm(Y_d.cpu().numpy().astype(np.float64) - Y)
            assert dy <= TOL * max(np.linalg.norm(Y), rho * np.linalg.norm(At)), n
            for k in ("primal_res", "dual_res", "norm_A", "norm_At", "norm_Y"):
                want = getattr(s, k)
                assert abs(st[k] - want) <= TOL * max(want, s.norm_At), k
            # the update refreshed the stored Gram of this factor from its new auxiliary
            # (Khatri-Rao source aux): the next modes see that factor -- unless it is zero
            # (c = 0), which would leave them no coefficient matrix: keep the old one then
            if np.any(got_t):
                F64[n] = got_t.astype(np.float64)
                ctx.gram(n, At_d)
            else:
                ctx.gram(n, torch.as_tensor(fs[n]).cuda())
            yield got_t, At


@pytest.mark.parametrize("dims,R,L,policy,lo,hi", [
    ((40, 30, 20), 5, 3, "trace", 0.05, 0.6),
    ((64, 48, 40), 20, 5, "trace", -0.2, 0.4),       # a box that allows negative entries
    ((60, 30, 20), 40, 2, "fixed", 0.0, 0.3),        # R > 32: two lanes per row, FP64 rows
    ((33, 20, 10), 12, 4, "fixed", 0.1, float("inf")),
])
def test_box_constrained_update_matches_oracle(ntf, dims, R, L, policy, lo, hi):
    cons = lambda I: (ntf.NTF_CONSTRAINT_BOX, lo, hi, 0,  # noqa: E731
                      lambda V: o.project_box(V, lo, hi))
    for got, want in _updates(ntf, dims, R, L, policy, cons):
        assert got.min() >= np.float32(lo) and got.max() <= np.float32(hi)


@pytest.mark.parametrize("dims,R,L,policy,frac", [
    ((40, 30, 20), 5, 1, "trace", 0.25),
    ((64, 48, 40), 20, 5, "trace", 0.3),
    ((50, 30, 20), 40, 3, "trace", 0.2),              # R > 32 and the LDL^T system
    ((33, 20, 10), 12, 4, "fixed", 0.1),              # FP64 rows
    ((20, 16, 12), 6, 2, "trace", 1.0),               # c = I R: the non-negative projection
    ((20, 16, 12), 6, 2, "fixed", 0.0),               # c = 0: everything zero
])
def test_sparse_constrained_update_matches_oracle(ntf, dims, R, L, policy, frac):
    def cons(I):
        c = int(frac * I * R)
        return (ntf.NTF_CONSTRAINT_SPARSE, 0.0, float("inf"), c,
                lambda V: o.project_nonneg_sparse(V, c))
    for got, want in _updates(ntf, dims, R, L, policy, cons):
        c = int(frac * got.shape[0] * R)
        assert np.count_nonzero(got) <= c and got.min() >= 0
        assert np.array_equal(got != 0, want != 0)      # the oracle's support


def test_run_with_a_sparse_factor_tracks_the_oracle(ntf):
    """Six outer iterations (L = 5, trace penalty, Khatri-Rao of the auxiliaries) with factor
    0 limited to 30% nonzeros, replayed as a CUDA graph, against the oracle's iterations with
    the same projection on factor 0 (composed from the oracle's steps)."""
    dims, R, iters = (40, 36, 32), 6, 6
    X, _, init = synth.workload(dims, R, seed=5, snr_db=20.0)
    init = [F.astype(np.float32).astype(np.float64) for F in init]
    c0 = int(0.3 * dims[0] * R)
    X64 = X.astype(np.float64)
    aux = [F.copy() for F in init]
    dual = [np.zeros_like(F) for F in init]
    for _ in range(iters):
        for n in range(3):
            M = o.mttkrp(X64, aux, n)
            G = o.coeff_matrix(aux, n)
            proj = (lambda V: o.project_nonneg_sparse(V, c0)) if n == 0 else o.project_nonneg
            _, aux[n], dual[n], _ = o.admm_factor_update(M, G, aux[n], dual[n], o.rho_trace(G),
                                                        5, project=proj)
    want_rfe = o.rfe(X64, aux)
    p = ntf.default_params(paper_mode=False, eps_abs=0.0, eps_rel=0.0)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        A = [torch.as_tensor(F, dtype=torch.float32).cuda() for F in init]
        At = [a.clone() for a in A]
        Y = [torch.zeros_like(a) for a in A]
        with ntf.Context(torch.as_tensor(X).cuda(), R, p, stream=stream) as ctx:
            ctx.set_constraint(0, ntf.NTF_CONSTRAINT_SPARSE, max_nonzeros=c0)
            rs = ctx.run(A, At, Y, iters, check_every=1, history=True)
        stream.synchronize()
    assert torch.count_nonzero(At[0]) <= c0
    for n in range(3):
        assert rel(At[n].cpu().numpy(), aux[n]) <= 1e-4, n
    assert abs(rs["rel_err"] - want_rfe) <= 1e-4
