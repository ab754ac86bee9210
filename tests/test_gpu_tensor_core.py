"""Parity of the tensor-core (tcgen05 + TMA) MTTKRP contractions against the FP64 oracle.

The context is created with the TENSOR engine, so both contractions of every mode run on the
tensor cores (BF16 storage: BF16 x 3-part BF16 split; FP32 storage: TF32 hi/lo split).
Shapes cover a single partial K stage, ragged 128-row tiles, R from 1 to 64 (N = 16..64),
4-way tensors, and split contraction ranges (chunk partial sums).  Tolerance: relative
Frobenius error <= 1e-5, as for the FP32 FMA path."""
import numpy as np
import pytest
import torch

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


def _problem(dims, R, seed):
    rng = np.random.default_rng(seed)
    X = (rng.random(dims) - 0.5).astype(np.float32)
    fs = [rng.random((d, R)).astype(np.float32) for d in dims]
    return X, fs


def _tensor(X, storage):
    if storage == "bf16":
        t = torch.as_tensor(X).to(torch.bfloat16)
        return t.cuda(), t.double().numpy()
    return torch.as_tensor(X).cuda(), X.astype(np.float64)


SHAPES = [
    ((64, 48, 40), 20),      # contraction shorter than one stage
    ((24, 40, 32), 7),       # N = 16, ragged tiles
    ((33, 65, 96), 1),       # rank 1
    ((100, 120, 136), 32),   # N = 32
    ((60, 70, 80), 50),      # N = 64 with ragged rank
    ((70, 30, 40), 64),      # maximum rank
    ((50, 40, 72), 40),      # N = 48
    ((512, 40, 48), 20),     # few output tiles: split contraction range
    ((20, 24, 16, 50), 16),  # 4-way
    ((64, 8, 8, 40), 24),    # 4-way, split contraction range
]

# Skewed shapes (FP32 storage): 200-byte rows of X[I1 I2, I3]; both passes on X[I1, I2 I3]
SKEWED = [((300, 50, 50), 10), ((1000, 50, 50), 3)]


@pytest.mark.parametrize("dims,R", SHAPES)
@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_tensor_core_mttkrp_all_modes(ntf, dims, R, storage):
    X, fs = _problem(dims, R, seed=sum(dims) + R)
    Xt, Xref = _tensor(X, storage)
    Fd = [torch.as_tensor(F).cuda() for F in fs]
    p = ntf.default_params(contraction=ntf.NTF_CONTRACT_TENSOR)
    with ntf.Context(Xt, R, p) as ctx:
        for n in range(len(dims)):
            M = ctx.mttkrp(n, Fd).cpu().numpy()
            want = o.mttkrp(Xref, [F.astype(np.float64) for F in fs], n)
            assert rel(M, want) <= TOL, (n, rel(M, want))
            again = ctx.mttkrp(n, Fd).cpu().numpy()
            assert np.array_equal(M, again)          # deterministic


@pytest.mark.parametrize("dims,R", SKEWED)
def test_tensor_core_mttkrp_skewed_fp32(ntf, dims, R):
    test_tensor_core_mttkrp_all_modes(ntf, dims, R, "f32")


@pytest.mark.parametrize("dims,R", [((64, 50, 50), 4), ((300, 50, 50), 10), ((13, 17, 11), 5),
                                    ((10, 6, 9, 7), 3)])
@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_unaligned_rows_run_on_padded_copies(ntf, dims, R, storage):
    """Rows that are not 16-byte multiples in any matrix view (BF16 I x 50 x 50: 100 and 5000
    bytes; odd extents): the tensor engine runs on the context's row-padded and transposed
    copies of the tensor (every mode against the oracle); with the copies switched off
    (tensor_copy = -1) it is refused where no matrix view has aligned rows (FP32 I x 50 x 50
    has one, X[I, 2500]) and the default engine takes the FMA kernels."""
    X, fs = _problem(dims, R, seed=sum(dims) + 7 * R)
    Xt, Xref = _tensor(X, storage)
    Fd = [torch.as_tensor(F).cuda() for F in fs]
    with ntf.Context(Xt, R, ntf.default_params(contraction=ntf.NTF_CONTRACT_TENSOR)) as ctx:
        assert ctx.profile_get()["tensor_copy_bytes"] >= X.size * (2 if storage == "bf16" else 4)
        for n in range(len(dims)):
            M = ctx.mttkrp(n, Fd).cpu().numpy()
            want = o.mttkrp(Xref, [F.astype(np.float64) for F in fs], n)
            assert rel(M, want) <= TOL, (n, rel(M, want))
    es = 2 if storage == "bf16" else 4
    trailing = [int(np.prod(dims[2:]))] if len(dims) == 4 else [dims[2], dims[1] * dims[2]]
    if any(t * es % 16 == 0 for t in trailing):
        ntf.Context(Xt, R, ntf.default_params(contraction=ntf.NTF_CONTRACT_TENSOR,
                                              tensor_copy=-1)).close()
    else:
        with pytest.raises(ntf.NTFError) as ei:
            ntf.Context(Xt, R, ntf.default_params(contraction=ntf.NTF_CONTRACT_TENSOR,
                                                  tensor_copy=-1))
        assert "UNSUPPORTED" in str(ei.value)


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_tensor_core_agrees_with_fma_path(ntf, storage):
    dims, R = (96, 80, 64), 20
    X, fs = _problem(dims, R, seed=5)
    Xt, _ = _tensor(X, storage)
    Fd = [torch.as_tensor(F).cuda() for F in fs]
    out = {}
    for eng in (ntf.NTF_CONTRACT_TENSOR, ntf.NTF_CONTRACT_SIMT):
        with ntf.Context(Xt, R, ntf.default_params(contraction=eng)) as ctx:
            out[eng] = [ctx.mttkrp(n, Fd).cpu().numpy() for n in range(3)]
    for n in range(3):
        assert rel(out[ntf.NTF_CONTRACT_TENSOR][n], out[ntf.NTF_CONTRACT_SIMT][n]) <= 2 * TOL


def test_skewed_run_matches_oracle(ntf):
    """Ten outer iterations on a 400 x 50 x 50 rank-6 tensor (FP32: both passes on the
    [400, 2500] view, tensor cores) against the oracle's, L = 5, trace penalty."""
    import synth
    dims, R = (400, 50, 50), 6
    X, _, init = synth.workload(dims, R, seed=2, snr_db=20.0)
    init = [F.astype(np.float32).astype(np.float64) for F in init]
    params = o.Params(inner_iters=5, kr_source="aux", rho_policy="trace")
    st, _, _ = o.factorize(X.astype(np.float64), init, params, 10, stop_on_residuals=False,
                           record_rfe=False)
    p = ntf.default_params(paper_mode=False, eps_abs=0.0, eps_rel=0.0,
                           contraction=ntf.NTF_CONTRACT_TENSOR)
    A = [torch.as_tensor(F, dtype=torch.float32).cuda() for F in init]
    At = [a.clone() for a in A]
    Y = [torch.zeros_like(a) for a in A]
    with ntf.Context(torch.as_tensor(X).cuda(), R, p) as ctx:
        rs = ctx.run(A, At, Y, 10)
    for n in range(3):
        assert rel(At[n].cpu().numpy(), st.aux[n]) <= 1e-4, n
    assert abs(rs["rel_err"] - o.rfe(X.astype(np.float64), st.aux)) <= 1e-4


def test_tensor_engine_without_copies_rejects_unaligned_rows(ntf):
    X = torch.rand(13, 17, 11, device="cuda")
    with pytest.raises(ntf.NTFError) as ei:
        ntf.Context(X, 4, ntf.default_params(contraction=ntf.NTF_CONTRACT_TENSOR,
                                             tensor_copy=-1))
    assert "UNSUPPORTED" in str(ei.value)
