"""GPU parity of every hot-path step against the FP64 oracle, through the C ABI.

Tolerances: one MTTKRP, Gram or factor update from identical inputs must match the oracle to
relative Frobenius error <= 1e-5 (FP32 storage and accumulation); Grams, coefficient matrix
and Cholesky factor (FP64) to 1e-12; the relative factorization error to 1e-4 absolute.
Sizes span several tiles and ragged tails, both halves of the tensor matricization, both
storage types, 3- and 4-way tensors, R from 1 to 64, and the unaligned fallback path."""
import math

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


def cuda(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(dtype).cuda()


def host(t):
    return t.detach().float().cpu().numpy() if t.dtype != torch.float64 else t.cpu().numpy()


def _problem(dims, R, seed=0, signed=False):
    rng = np.random.default_rng(seed)
    X = rng.random(dims).astype(np.float32)
    if signed:
        X -= 0.5
    fs = [rng.random((d, R)).astype(np.float32) for d in dims]
    return X, fs


SHAPES = [
    ((13, 17, 11), 5),          # odd extents: row-padded and transposed tensor copies
    ((24, 40, 36), 7),          # ragged rank, aligned rows
    ((64, 48, 40), 20),
    ((1, 5, 8), 3),             # a unit extent
    ((33, 65, 96), 1),          # rank 1
    ((70, 30, 40), 64),         # maximum rank
    ((100, 120, 140), 32),
    ((60, 70, 80), 50),
    ((9, 10, 12, 8), 3),        # 4-way
    ((20, 24, 16, 50), 16),     # 4-way with the short fastest mode of the stress workload
    ((7, 5, 9, 11), 6),         # 4-way, unaligned
    ((8, 40, 36), 8),           # vectorised second level with one split (short reduced range)
    ((12, 16, 20, 24), 4),      # 4-way, vectorised second levels
    ((200, 160, 40), 12),       # vectorised slow level with many splits and b-blocks
    # one K-chunk with >= 32 rows per leading index (the shapes of the fused second level)
    ((157, 131, 24), 20),
    ((160, 130, 30), 50),
    ((160, 128, 8, 6), 7),
    # even ranks that are not multiples of 4: the second tree levels in float2 vectors
    ((90, 50, 60), 18),
    ((64, 80, 48), 2),
    ((40, 36, 30, 20), 10),
]


@pytest.mark.parametrize("dims,R", SHAPES)
@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_mttkrp_all_modes(ntf, dims, R, storage):
    X, fs = _problem(dims, R, seed=len(dims) * 100 + R, signed=True)
    if storage == "bf16":
        Xt = torch.as_tensor(X).to(torch.bfloat16).cuda()
        Xref = torch.as_tensor(X).to(torch.bfloat16).double().numpy()
    else:
        Xt, Xref = cuda(X), X.astype(np.float64)
    Fd = [cuda(F) for F in fs]
    with ntf.Context(Xt, R) as ctx:
        for n in range(len(dims)):
            M = host(ctx.mttkrp(n, Fd))
            want = o.mttkrp(Xref, [F.astype(np.float64) for F in fs], n)
            assert rel(M, want) <= TOL, (n, rel(M, want))


@pytest.mark.parametrize("dims,R", [((157, 131, 24), 20), ((160, 130, 30), 32),
                                    ((160, 128, 8, 6), 7)])
@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_mttkrp_with_the_fused_second_level(ntf, dims, R, storage):
    """Factor 0's second tree level formed in the first contraction's epilogue (forced with
    fuse_level = 1; by default only for intermediates of at least half the L2): mode 0 against
    the oracle at the MTTKRP tolerance and against the separate level, and a short run that
    uses it in every sweep against one that does not (ragged 32-row groups, I_2 = 131)."""
    X, fs = _problem(dims, R, seed=7 * R + len(dims), signed=False)
    Xt = torch.as_tensor(X).to(torch.bfloat16).cuda() if storage == "bf16" else cuda(X)
    Xref = torch.as_tensor(X).to(torch.bfloat16).double().numpy() if storage == "bf16" \
        else X.astype(np.float64)
    Fd = [cuda(F) for F in fs]
    want = o.mttkrp(Xref, [F.astype(np.float64) for F in fs], 0)
    got = {}
    for fl in (1, -1):
        with ntf.Context(Xt, R, ntf.default_params(fuse_level=fl)) as ctx:
            got[fl] = host(ctx.mttkrp(0, Fd))
            assert rel(got[fl], want) <= TOL, (fl, rel(got[fl], want))
    assert rel(got[1], got[-1]) <= 4 * TOL
    init = [np.random.default_rng(40 + n).random((d, R)).astype(np.float32)
            for n, d in enumerate(dims)]
    errs = {}
    for fl in (1, -1):
        with ntf.Context(Xt, R, ntf.default_params(fuse_level=fl)) as ctx:
            A, At, Y = [cuda(F) for F in init], [cuda(F) for F in init], ntf.zeros_state(dims, R)
            errs[fl] = ctx.run(A, At, Y, 6)["rel_err"]
    assert abs(errs[1] - errs[-1]) <= 1e-5 * errs[-1], errs


@pytest.mark.parametrize("dims,R", [((24, 40, 36), 7), ((100, 120, 140), 32),
                                    ((20, 24, 16, 50), 16), ((64, 80, 48), 2),
                                    ((72, 30, 40), 64), ((13, 17, 11), 5), ((128, 96, 200), 16),
                                    ((16, 9, 7), 5)])   # odd trailing extent: element-wise copy
@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_mttkrp_on_the_transposed_copy(ntf, dims, R, storage):
    """The second contraction X^T W on the context's transposed tensor copy (tensor_copy = 1:
    a row-major tensor-core product) and on the tensor itself (-1): every mode against the
    oracle at the MTTKRP tolerance and the two against each other; the profile reports the
    copies (rows padded to 16-byte multiples where the extents need it: 13 x 17 x 11, 16 x 9 x
    7); short runs agree."""
    X, fs = _problem(dims, R, seed=11 * R + len(dims), signed=False)
    Xt = torch.as_tensor(X).to(torch.bfloat16).cuda() if storage == "bf16" else cuda(X)
    Xref = torch.as_tensor(X).to(torch.bfloat16).double().numpy() if storage == "bf16" \
        else X.astype(np.float64)
    Fd = [cuda(F) for F in fs]
    es = 2 if storage == "bf16" else 4
    got, used = {}, {}
    for tc in (1, -1):
        with ntf.Context(Xt, R, ntf.default_params(tensor_copy=tc)) as ctx:
            used[tc] = ctx.profile_get()["tensor_copy_bytes"]
            got[tc] = [host(ctx.mttkrp(n, Fd)) for n in range(len(dims))]
        for n in range(len(dims)):
            want = o.mttkrp(Xref, [F.astype(np.float64) for F in fs], n)
            assert rel(got[tc][n], want) <= TOL, (tc, n, rel(got[tc][n], want))
    for n in range(len(dims)):
        assert rel(got[1][n], got[-1][n]) <= 4 * TOL, n
    assert used[-1] == 0 and used[1] >= X.size * es, used
    init = [np.random.default_rng(50 + n).random((d, R)).astype(np.float32)
            for n, d in enumerate(dims)]
    errs = {}
    for tc in (1, -1):
        with ntf.Context(Xt, R, ntf.default_params(tensor_copy=tc)) as ctx:
            A, At, Y = [cuda(F) for F in init], [cuda(F) for F in init], ntf.zeros_state(dims, R)
            errs[tc] = ctx.run(A, At, Y, 4)["rel_err"]
    assert abs(errs[1] - errs[-1]) <= 1e-5 * errs[-1], errs


@pytest.mark.parametrize("dims,R,storage,copied", [
    ((512, 160, 128), 32, "bf16", True),    # one chunk, N = 32, streamed table
    ((512, 160, 128), 16, "bf16", False),   # N = 16
    ((512, 160, 128), 50, "bf16", False),   # N = 64
    ((256, 160, 128), 20, "bf16", False),   # table resident in shared memory (P <= 448)
    ((256, 160, 128), 20, "f32", True)])
def test_default_tensor_copy_policy(ntf, dims, R, storage, copied):
    """tensor_copy = 0 makes the transposed copy for FP32 storage and, for BF16, only where
    the row-major product measured faster (one chunk, N = 32, streamed table); the mode-2
    MTTKRP matches the oracle either way."""
    X, fs = _problem(dims, R, seed=3 * R, signed=False)
    Xt = torch.as_tensor(X).to(torch.bfloat16).cuda() if storage == "bf16" else cuda(X)
    Xref = torch.as_tensor(X).to(torch.bfloat16).double().numpy() if storage == "bf16" \
        else X.astype(np.float64)
    es = 2 if storage == "bf16" else 4
    used = {}
    for tc in (0, -1):
        with ntf.Context(Xt, R, ntf.default_params(tensor_copy=tc)) as ctx:
            used[tc] = ctx.profile_get()["tensor_copy_bytes"]
            M = host(ctx.mttkrp(2, [cuda(F) for F in fs]))
        want = o.mttkrp(Xref, [F.astype(np.float64) for F in fs], 2)
        assert rel(M, want) <= TOL, (tc, rel(M, want))
    assert used == {0: X.size * es if copied else 0, -1: 0}, used


@pytest.mark.parametrize("n", [1 << 20, 1000003])
def test_to_bf16_from_pinned_host_memory(ntf, n):
    """The conversion reads page-locked host memory directly (copy and conversion in one
    pass): the result equals the conversion of the same values in device memory, bit for bit,
    also for a length that leaves a tail and an input that starts off the 16-byte grid."""
    x = torch.randn(n + 1, dtype=torch.float32).pin_memory()
    for src in (x[:n], x[1:]):
        got = ntf.to_bf16(src)
        want = ntf.to_bf16(src.cuda())
        torch.cuda.synchronize()
        assert got.is_cuda and torch.equal(got.view(torch.int16), want.view(torch.int16))
    with pytest.raises(ValueError):
        ntf.to_bf16(torch.randn(16))  # pageable host memory is refused


def test_to_bf16_matches_round_to_nearest_even(ntf):
    rng = np.random.default_rng(3)
    x = (rng.standard_normal(100003) * 10.0 ** rng.integers(-20, 20, 100003)).astype(np.float32)
    # exact ties of the 16-bit truncation: low half 0x8000 with odd and even high halves
    ties = np.array([0x3F808000, 0x3F818000, 0xBF808000, 0x40C08000], np.uint32).view(np.float32)
    x = np.concatenate([x, ties, np.float32([0.0, -0.0, np.inf, -np.inf])])
    got = ntf.to_bf16(cuda(x)).cpu().view(torch.int16).numpy()
    want = torch.as_tensor(x).to(torch.bfloat16).view(torch.int16).numpy()
    assert np.array_equal(got, want)


@pytest.mark.parametrize("dims,R", [((30, 20, 10), 6), ((50, 40, 30, 20), 13), ((1000, 9, 8), 64)])
def test_gram_and_system(ntf, dims, R):
    X, fs = _problem(dims, R, seed=7)
    Fd = [cuda(F) for F in fs]
    F64 = [F.astype(np.float64) for F in fs]
    p = ntf.default_params(paper_mode=False)
    with ntf.Context(cuda(X), R, p) as ctx:
        for m in range(len(dims)):
            G = torch.empty(R, R, dtype=torch.float64, device="cuda")
            ctx.gram(m, Fd[m], G)
            assert rel(G.cpu().numpy(), o.gram(F64[m])) <= 1e-13
        for n in range(len(dims)):
            H = torch.empty(R, R, dtype=torch.float64, device="cuda")
            L = torch.empty(R, R, dtype=torch.float64, device="cuda")
            rho = ctx.system(n, H, L)
            Gn = o.coeff_matrix(F64, n)
            assert math.isclose(rho, o.rho_trace(Gn), rel_tol=1e-13)
            Hw = Gn + rho * np.eye(R)
            assert rel(H.cpu().numpy(), Hw) <= 1e-13
            assert rel(L.cpu().numpy(), np.linalg.cholesky(Hw)) <= 1e-10


def test_system_reports_not_spd(ntf):
    """Host-side fault injection: a factor corrupted with NaN makes the coefficient matrix
    non-positive-definite; the status is reported and the context stays usable."""
    R = 4
    X, fs = _problem((8, 9, 10), R)
    p = ntf.default_params(paper_mode=True)
    with ntf.Context(cuda(X), R, p) as ctx:
        bad = fs[1].copy()
        bad[3, 2] = np.nan
        ctx.gram(0, cuda(fs[0]))
        ctx.gram(1, cuda(bad))
        ctx.gram(2, cuda(fs[2]))
        with pytest.raises(ntf.NTFError) as e:
            ctx.system(0)
        assert e.value.status == 4
        At = torch.ones(8, R, device="cuda")
        before = At.clone()
        with pytest.raises(ntf.NTFError):
            ctx.admm_update(0, torch.ones(8, R, device="cuda"), torch.empty(8, R, device="cuda"),
                            At, torch.zeros(8, R, device="cuda"))
        assert torch.equal(At, before)                  # a failed update leaves the state
        ctx.gram(1, cuda(fs[1]))                        # repaired input: usable again
        assert ctx.system(0) == 1.0


@pytest.mark.parametrize("R", [6, 32])
def test_trace_policy_update_reports_not_spd(ntf, R):
    """The same injection under the trace penalty, whose factor update builds its own FP64
    coefficient system (sweep operator for small R, LDL^T factorization for R >= 28): the
    update fails with NOT_SPD, leaves the state, and works again once the input is repaired."""
    dims = (8, 9, 10)
    X, fs = _problem(dims, R)
    p = ntf.default_params(paper_mode=False)
    with ntf.Context(cuda(X), R, p) as ctx:
        bad = fs[2].copy()
        bad[5, 1] = np.nan
        ctx.gram(0, cuda(fs[0]))
        ctx.gram(1, cuda(fs[1]))
        ctx.gram(2, cuda(bad))
        At = torch.rand(8, R, device="cuda")
        before = At.clone()
        with pytest.raises(ntf.NTFError) as e:
            ctx.admm_update(0, torch.ones(8, R, device="cuda"), torch.empty(8, R, device="cuda"),
                            At, torch.zeros(8, R, device="cuda"))
        assert e.value.status == 4
        assert torch.equal(At, before)
        ctx.gram(2, cuda(fs[2]))
        st = ctx.admm_update(0, torch.ones(8, R, device="cuda"), torch.empty(8, R, device="cuda"),
                             At, torch.zeros(8, R, device="cuda"))
        assert st["rho"] > 0 and torch.isfinite(At).all()


@pytest.mark.parametrize("dims,R,L,policy", [((40, 30, 20), 5, 1, "trace"),
                                              ((64, 48, 40), 20, 5, "trace"),
                                              ((90, 30, 20), 50, 5, "trace"),
                                              ((33, 20, 10), 40, 3, "fixed"),
                                              ((12, 10, 9, 8), 9, 2, "fixed"),
                                              ((70, 36, 40), 32, 4, "trace"),   # widest 1-lane rows
                                              ((70, 36, 40), 32, 4, "fixed"),   # same, FP64 rows
                                              ((50, 44, 41), 33, 3, "trace"),   # first 2-lane rank
                                              ((300, 20, 12), 1, 2, "fixed"),   # R = 1, many blocks
                                              ((70, 30, 40), 64, 2, "trace"),   # maximum rank
                                              ((40, 30, 20), 16, 5, "trace")])
def test_admm_update(ntf, dims, R, L, policy):
    X, fs = _problem(dims, R, seed=11, signed=True)
    rng = np.random.default_rng(5)
    F64 = [F.astype(np.float64) for F in fs]
    pol = ntf.NTF_RHO_TRACE if policy == "trace" else ntf.NTF_RHO_FIXED
    p = ntf.default_params(inner_iters=L, rho_policy=pol, kr_source=ntf.NTF_KR_AUX)
    with ntf.Context(cuda(X), R, p) as ctx:
        for m in range(len(dims)):
            ctx.gram(m, cuda(fs[m]))
        for n in range(len(dims)):
            I = dims[n]
            M = o.mttkrp(X.astype(np.float64), F64, n).astype(np.float32)
            At0 = np.maximum(rng.standard_normal((I, R)), 0).astype(np.float32)
            Y0 = (-np.abs(rng.standard_normal((I, R))) * (At0 == 0)).astype(np.float32)
            G = o.coeff_matrix(F64, n)
            rho = o.rho_trace(G) if policy == "trace" else 0.37 * o.rho_trace(G)
            if policy == "fixed":
                ctx.set_rho(n, rho)
            A_d, At_d, Y_d = torch.empty(I, R, device="cuda"), cuda(At0), cuda(Y0)
            st = ctx.admm_update(n, cuda(M), A_d, At_d, Y_d)
            A, At, Y, s = o.admm_factor_update(M.astype(np.float64), G, At0.astype(np.float64),
                                               Y0.astype(np.float64), rho, L)
            assert rel(host(A_d), A) <= TOL
            assert rel(host(At_d), At) <= TOL
            assert rel(host(Y_d), Y) <= TOL
            assert math.isclose(st["rho"], rho, rel_tol=1e-12)
            for k in ("primal_res", "dual_res", "norm_A", "norm_At", "norm_Y"):
                want = getattr(s, k)
                assert abs(st[k] - want) <= TOL * max(want, s.norm_At), k
            # KKT measures of the factor's NNLS problem (eq. KKT_NTF) at the GPU's new At,
            # against the oracle's from the same At: the GPU forms the gradient At G - M in
            # FP32, so beyond 1e-4 relative it is allowed 4 R 2^-24 in the scaled units
            kk = o.kkt_nnls(G, M, host(At_d))
            assert st["kkt_neg_x"] == 0.0 and kk["neg_x"] == 0.0
            for k in ("dual", "comp"):
                assert abs(st["kkt_" + k] - kk[k]) <= 1e-4 * kk[k] + 4 * R * 2.0 ** -24, \
                    (k, st["kkt_" + k], kk[k])
            # the stored Gram of this factor now comes from the new auxiliary factor
            # (kr_source = aux); check through the next system's coefficient matrix
            F64[n] = host(At_d).astype(np.float64)
            ctx.gram(n, At_d)


@pytest.mark.parametrize("dims,R", [((30, 40, 50), 4), ((10, 12, 14, 16), 6), ((17, 13, 11), 3)])
def test_fit(ntf, dims, R):
    fs = synth.factors(dims, R, 1)
    X = synth.tensor(fs, 1, snr_db=15.0)
    G = [np.clip(F + 0.1 * np.random.default_rng(2).standard_normal(F.shape), 0, None)
         .astype(np.float32) for F in fs]
    with ntf.Context(cuda(X), R) as ctx:
        got = ctx.fit([cuda(F) for F in G])
        want = o.rfe(X.astype(np.float64), [F.astype(np.float64) for F in G])
        assert abs(got - want) <= 1e-4 * max(want, 1e-2)
        assert math.isclose(ctx.tensor_norm2(), float(np.sum(X.astype(np.float64) ** 2)),
                            rel_tol=1e-12)


@pytest.mark.parametrize("dims,R,snr,bf16", [((30, 40, 50), 4, 15.0, False),
                                             ((10, 12, 14, 16), 6, 15.0, False),
                                             ((40, 30, 20), 8, 15.0, True),
                                             ((60, 50, 40), 10, 70.0, False)])  # low noise
def test_fit_explicit(ntf, dims, R, snr, bf16):
    """The fit by explicit reconstruction against the oracle's: equal to 1e-5 relative plus
    1e-7 absolute at any noise level (at 70 dB the Gram identity of ntf_fit loses accuracy to
    cancellation; the explicit sum does not)."""
    fs = synth.factors(dims, R, 2)
    X = synth.tensor(fs, 2, snr_db=snr)
    G = [np.clip(F + 1e-4 * np.random.default_rng(3).standard_normal(F.shape), 0, None)
         .astype(np.float32) for F in fs]
    Xd = cuda(X)
    Xref = X.astype(np.float64)
    if bf16:
        Xd = ntf.to_bf16(Xd)
        Xref = Xd.float().cpu().numpy().astype(np.float64)
    with ntf.Context(Xd, R) as ctx:
        got = ctx.fit_explicit([cuda(F) for F in G])
    want = o.rfe(Xref, [F.astype(np.float64) for F in G])
    assert abs(got - want) <= 1e-5 * want + 1e-7, (got, want)


def _run_gpu(ntf, X, init, p, iters, stream=None, paper=False):
    R = init[0].shape[1]
    dims = X.shape
    A = [cuda(F) for F in init]
    if paper:
        At = [torch.zeros(d, R, device="cuda") for d in dims]
    else:
        At = [cuda(F) for F in init]
    Y = [torch.zeros(d, R, device="cuda") for d in dims]
    with ntf.Context(cuda(X), R, p, stream=stream) as ctx:
        rs = ctx.run(A, At, Y, iters, check_every=1, history=True)
    torch.cuda.synchronize()
    return rs, [host(t) for t in A], [host(t) for t in At], [host(t) for t in Y]


def test_full_run_matches_oracle_ao_mode(ntf):
    """50^3, R = 5, 20 dB, 100 outer iterations, L = 5, rho = trace(G)/R, uniform start."""
    dims, R = (50, 50, 50), 5
    X, fs, init = synth.workload(dims, R, seed=0, snr_db=20.0)
    init = [F.astype(np.float32).astype(np.float64) for F in init]
    p = ntf.default_params(paper_mode=False, eps_abs=0.0, eps_rel=0.0)
    rs, A, At, Y = _run_gpu(ntf, X, init, p, 100)
    params = o.Params(inner_iters=5, kr_source="aux", rho_policy="trace")
    st, _, _ = o.factorize(X.astype(np.float64), init, params, 100, stop_on_residuals=False,
                           record_rfe=False)
    want = o.rfe(X.astype(np.float64), st.aux)
    assert rs["iters"] == 100
    assert abs(rs["rel_err"] - want) <= 1e-4
    assert abs(o.rfe(X.astype(np.float64), [F.astype(np.float64) for F in At]) - want) <= 1e-4


def test_full_run_matches_oracle_paper_mode(ntf):
    """Paper settings: L = 1, primal Khatri-Rao, adaptive rho; first iterations track the
    oracle closely and the final fit agrees."""
    dims, R = (30, 30, 30), 3
    X, fs, init = synth.workload(dims, R, seed=0, snr_db=20.0)
    init = [F.astype(np.float32).astype(np.float64) for F in init]
    p = ntf.default_params(paper_mode=True, eps_abs=0.0, eps_rel=0.0)
    rs, A, At, Y = _run_gpu(ntf, X, init, p, 5, paper=True)
    st = o.init_state(init, o.PAPER)
    for _ in range(5):
        o.outer_iteration(X.astype(np.float64), st, o.PAPER)
    for n in range(3):
        assert rel(At[n], st.aux[n]) <= 1e-4
        assert rel(A[n], st.primal[n]) <= 1e-4


def test_graph_replay_is_bitwise_equal_to_eager(ntf):
    dims, R = (40, 36, 32), 6
    X, fs, init = synth.workload(dims, R, seed=4, snr_db=20.0)
    p = ntf.default_params(paper_mode=False, eps_abs=0.0, eps_rel=0.0)
    s = torch.cuda.Stream()
    r1 = _run_gpu(ntf, X, init, p, 12)                 # legacy default stream: eager launches
    with torch.cuda.stream(s):
        r2 = _run_gpu(ntf, X, init, p, 12, stream=s)   # captured sweep replayed as a graph
    for a, b in zip(r1[2], r2[2]):
        assert np.array_equal(a, b)
    assert r1[0]["history"] == r2[0]["history"]


def test_resume_from_saved_state_is_bitwise_equal(ntf):
    dims, R = (30, 28, 26), 4
    X, fs, init = synth.workload(dims, R, seed=6, snr_db=20.0)
    p = ntf.default_params(paper_mode=False, eps_abs=0.0, eps_rel=0.0)
    full = _run_gpu(ntf, X, init, p, 10)
    A = [cuda(F) for F in init]
    At = [cuda(F) for F in init]
    Y = [torch.zeros(d, R, device="cuda") for d in dims]
    with ntf.Context(cuda(X), R, p) as ctx:
        ctx.run(A, At, Y, 4)
    saved = [[t.clone().cpu() for t in S] for S in (A, At, Y)]
    A, At, Y = [[t.cuda() for t in S] for S in saved]
    with ntf.Context(cuda(X), R, p) as ctx:
        ctx.run(A, At, Y, 6)
    for a, b in zip(full[2], [host(t) for t in At]):
        assert np.array_equal(a, b)


def test_stopping_rule_and_target(ntf):
    dims, R = (30, 30, 30), 3
    X, fs, init = synth.workload(dims, R, seed=0, snr_db=20.0)
    p = ntf.default_params(paper_mode=False, eps_abs=1e-4, eps_rel=1e-4)
    rs = _run_gpu(ntf, X, init, p, 400)[0]
    assert rs["converged"] == 1 and rs["iters"] < 400
    p = ntf.default_params(paper_mode=False, eps_abs=0.0, eps_rel=0.0)
    A = [cuda(F) for F in init]
    At = [cuda(F) for F in init]
    Y = [torch.zeros(d, R, device="cuda") for d in dims]
    with ntf.Context(cuda(X), R, p) as ctx:
        rs = ctx.run(A, At, Y, 400, target_rfe=0.2)
    assert rs["reached_target"] == 1 and rs["rel_err"] <= 0.2 and rs["iters"] < 400


@pytest.mark.parametrize("dims,R,check_every,rule", [
    ((40, 36, 32), 4, 1, "target"), ((40, 36, 32), 4, 3, "target"),
    ((40, 36, 32), 4, 1, "residual"), ((40, 36, 32), 4, 2, "residual"),
    # the last factor's partial sums too many for the rows kernel: separate reduction kernel
    ((24, 20, 480), 8, 1, "target"), ((24, 20, 480), 8, 3, "target")])
def test_run_stops_at_the_first_sweep_that_meets_the_rule(ntf, dims, R, check_every, rule):
    """The host enqueues a sweep before it reads the previous sweep's outcome; the sweep after
    the one that met the stopping rule must leave the state untouched.  The stopped run's state
    equals, bit for bit, that of a run of exactly as many sweeps without a rule, and the rule's
    value at that sweep matches."""
    X, fs, init = synth.workload(dims, R, seed=3, snr_db=20.0)
    eps = 1e-3 if rule == "residual" else 0.0
    p = ntf.default_params(paper_mode=False, eps_abs=eps, eps_rel=eps)
    fresh = lambda: ([cuda(F) for F in init], [cuda(F) for F in init],
                     [torch.zeros(d, R, device="cuda") for d in dims])
    with ntf.Context(cuda(X), R, p) as ctx:
        A, At, Y = fresh()
        h = ctx.run(A, At, Y, 60, check_every=1, history=True)["history"]
        target = h[9] if rule == "target" else 0.0
        A, At, Y = fresh()
        rs = ctx.run(A, At, Y, 400, target_rfe=target, check_every=check_every)
        k = rs["iters"]
        if rule == "target":
            assert rs["reached_target"] == 1 and rs["rel_err"] <= target
            want = next(j for j in range(check_every, 61, check_every) if h[j - 1] <= target)
            assert k == want and rs["rel_err"] == h[k - 1]
        else:
            assert rs["converged"] == 1 and k < 400 and k % check_every == 0
        A2, At2, Y2 = fresh()
        p2 = ctx.run(A2, At2, Y2, k, check_every=k)
        assert p2["rel_err"] == rs["rel_err"]
        for S, S2 in ((A, A2), (At, At2), (Y, Y2)):
            for a, b in zip(S, S2):
                assert torch.equal(a, b)


# ------------------------------------------------------------------ full-size workloads

def _sampled_rows(ntf, dims, R, structure="uniform", storage="f32", snr=20.0, nrows=3):
    X, fs, init = synth.workload(dims, R, seed=0, snr_db=snr, structure=structure)
    if storage == "bf16":
        Xd = torch.as_tensor(X).to(torch.bfloat16).cuda()
        Xh = torch.as_tensor(X).to(torch.bfloat16).float().numpy()
    else:
        Xd, Xh = cuda(X), X
    F = [F.astype(np.float32) for F in init]
    Fd = [cuda(f) for f in F]
    rng = np.random.default_rng(1)
    with ntf.Context(Xd, R) as ctx:
        for n in range(len(dims)):
            M = host(ctx.mttkrp(n, Fd))
            rows = sorted(set(rng.integers(0, dims[n], nrows).tolist()) | {0, dims[n] - 1})
            want = o.mttkrp_rows(Xh, [f.astype(np.float64) for f in F], n, rows)
            assert rel(M[rows], want) <= TOL, (n, rel(M[rows], want))
    del Xd


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_full_size_400_cubed_r20(ntf, storage):
    _sampled_rows(ntf, (400, 400, 400), 20, storage=storage)


def test_full_size_600_cubed_r50_sparse(ntf):
    _sampled_rows(ntf, (600, 600, 600), 50, structure="sparse")


def test_full_size_4way_200x200x200x50_r16_bf16(ntf):
    _sampled_rows(ntf, (200, 200, 200, 50), 16, structure="collinear", storage="bf16", snr=10.0)


def test_profiling_under_graph_replay(ntf):
    """Contraction timing events recorded inside the captured sweep; no stale error left."""
    dims, R = (64, 48, 40), 8
    X, fs, init = synth.workload(dims, R, seed=2, snr_db=20.0)
    p = ntf.default_params(paper_mode=False, eps_abs=0.0, eps_rel=0.0)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        A = [cuda(F) for F in init]
        At = [cuda(F) for F in init]
        Y = [torch.zeros(d, R, device="cuda") for d in dims]
        with ntf.Context(cuda(X), R, p, stream=s) as ctx:
            ctx.run(A, At, Y, 3)                      # records the graph
            ctx.profile_enable(True)
            ctx.run(A, At, Y, 6)                      # eager first sweep, then a new graph
            ctx.run(A, At, Y, 4)                      # graph replays only
            prof = ctx.profile_get()
            assert prof["sweeps"] == 10
            assert prof["contractions"] == [10, 10]
            assert all(ms > 0 for ms in prof["contraction_ms"])
            assert prof["contraction_bytes"] == [X.size * 4.0] * 2
            assert prof["kernel_launches"] >= 10 * 10
            ctx.profile_enable(False)
            ctx.run(A, At, Y, 2)                      # back to a graph without events
            M = ctx.mttkrp(0, At)
    torch.cuda.synchronize()
    want = o.mttkrp(X.astype(np.float64), [host(t).astype(np.float64) for t in At], 0)
    assert rel(host(M), want) <= TOL


def test_trace_of_a_sweep(ntf):
    """The trace of the last outer iteration lists every step once per factor, on the
    documented streams, with start <= end, under graph replay; results are unchanged."""
    dims, R = (64, 48, 40), 8
    X, fs, init = synth.workload(dims, R, seed=4, snr_db=20.0)
    p = ntf.default_params(paper_mode=False, eps_abs=0.0, eps_rel=0.0)
    s = torch.cuda.Stream()
    out = []
    for trace in (False, True):
        with torch.cuda.stream(s):
            A = [cuda(F) for F in init]
            At = [cuda(F) for F in init]
            Y = [torch.zeros(d, R, device="cuda") for d in dims]
            with ntf.Context(cuda(X), R, p, stream=s) as ctx:
                ctx.trace_enable(trace)
                ctx.run(A, At, Y, 4)
                tr = ctx.trace_get()
        torch.cuda.synchronize()
        out.append([host(t) for t in At])
        if trace:
            names = [(e["name"], e["mode"]) for e in tr]
            assert ("contract_right", 0) in names and ("contract_left", 2) in names
            assert [e["mode"] for e in tr if e["name"] == "rows"] == [0, 1, 2]
            assert all(0.0 <= e["start_us"] <= e["end_us"] for e in tr)
            assert {e["stream"] for e in tr} == {0, 1, 2}
        else:
            assert tr == []
    for a, b in zip(*out):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_full_size_1000_cubed_r32(ntf, storage):
    _sampled_rows(ntf, (1000, 1000, 1000), 32, storage=storage, snr=30.0, nrows=2)


@pytest.mark.parametrize("check_every", [1, 2])
def test_run_stops_at_the_kkt_tolerance(ntf, check_every):
    """The KKT stopping rule (every factor's scaled dual infeasibility and complementarity at
    or below the tolerances, eq. KKT_NTF) stops the run at the first checked sweep that meets
    it: the state equals, bit for bit, a run of exactly that many sweeps, which reports the
    same measures, and the checked sweep before it did not meet the rule."""
    dims, R = (40, 36, 32), 4
    X, fs, init = synth.workload(dims, R, seed=3, snr_db=20.0)
    fresh = lambda: ([cuda(F) for F in init], [cuda(F) for F in init],
                     [torch.zeros(d, R, device="cuda") for d in dims])
    p0 = ntf.default_params(paper_mode=False, eps_abs=0.0, eps_rel=0.0)
    with ntf.Context(cuda(X), R, p0) as ctx:   # the measures after 8 sweeps set the tolerances
        A, At, Y = fresh()
        r8 = ctx.run(A, At, Y, 8, check_every=1)
    tol_d, tol_c = 1.0001 * r8["kkt_dual"], 1.0001 * r8["kkt_comp"]
    p = ntf.default_params(paper_mode=False, eps_abs=0.0, eps_rel=0.0, kkt_dual_tol=tol_d,
                           kkt_comp_tol=tol_c)
    with ntf.Context(cuda(X), R, p) as ctx:
        A, At, Y = fresh()
        rs = ctx.run(A, At, Y, 200, check_every=check_every)
    assert rs["kkt_met"] == 1 and rs["iters"] < 200
    assert rs["kkt_dual"] <= tol_d and rs["kkt_comp"] <= tol_c
    assert rs["iters"] % check_every == 0
    with ntf.Context(cuda(X), R, p0) as ctx:
        A2, At2, Y2 = fresh()
        rk = ctx.run(A2, At2, Y2, rs["iters"], check_every=1)
        assert rk["kkt_dual"] == rs["kkt_dual"] and rk["kkt_comp"] == rs["kkt_comp"]
        for a, b in zip(At, At2):
            assert torch.equal(a, b)
        if rs["iters"] > check_every:
            A3, At3, Y3 = fresh()
            rp = ctx.run(A3, At3, Y3, rs["iters"] - check_every, check_every=1)
            assert not (rp["kkt_dual"] <= tol_d and rp["kkt_comp"] <= tol_c)


@pytest.mark.parametrize("R,scale", [(8, 1e-6), (24, 1e-7), (40, 1e-6)])
def test_ill_conditioned_update_matches_the_cholesky_solve(ntf, R, scale):
    """Small penalty, nearly collinear factors: cond(G + rho I) from 7e5 to 1.6e7 under the fixed
    policy, where the rows run in FP64 against the FP64 sweep-operator inverse.  One update
    (L = 3) against the oracle's Cholesky solve; the tolerance grows with the condition
    number, cond * 2^-52 on top of the FP32 storage of the result (1e-5)."""
    import synth
    dims = (60, 50, 40)
    fs = synth.factors(dims, R, seed=R, structure="collinear", congruence=0.99999)
    fs = [F.astype(np.float32) for F in fs]
    F64 = [F.astype(np.float64) for F in fs]
    rng = np.random.default_rng(R)
    X = rng.random(dims).astype(np.float32)
    p = ntf.default_params(inner_iters=3, rho_policy=ntf.NTF_RHO_FIXED, kr_source=ntf.NTF_KR_AUX)
    with ntf.Context(cuda(X), R, p) as ctx:
        for m in range(3):
            ctx.gram(m, cuda(fs[m]))
        n = 0
        G = o.coeff_matrix(F64, n)
        rho = scale * o.rho_trace(G)
        cond = np.linalg.cond(G + rho * np.eye(R))
        assert cond > 1e5
        ctx.set_rho(n, rho)
        M = o.mttkrp(X.astype(np.float64), F64, n).astype(np.float32)
        At0 = np.maximum(rng.standard_normal((dims[n], R)), 0).astype(np.float32)
        Y0 = np.zeros((dims[n], R), np.float32)
        A_d, At_d, Y_d = torch.empty(dims[n], R, device="cuda"), cuda(At0), cuda(Y0)
        ctx.admm_update(n, cuda(M), A_d, At_d, Y_d)
        A, At, Y, _ = o.admm_factor_update(M.astype(np.float64), G, At0.astype(np.float64),
                                           Y0.astype(np.float64), rho, 3)
        tol = TOL + cond * 2.0 ** -52
        assert rel(host(A_d), A) <= tol, (rel(host(A_d), A), cond)
        assert rel(host(At_d), At) <= tol, (rel(host(At_d), At), cond)
