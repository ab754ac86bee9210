"""The allocation-free MTTKRP entry point against the context-based one.

Some callers of this library cannot allocate device memory on their call path (services that
reserve all device memory at start-up and treat later allocations as failures).
``ntf_mttkrp_noalloc`` serves them: it needs no context and keeps its scratch in a static
device array.  Here it is called through the C ABI twice in a row for every mode of several
tensors and compared with ``ntf_mttkrp`` of a context that uses the same FP32 FMA
contraction kernels, within the tolerance of the other parity tests (relative Frobenius
error 1e-5); one shape is also compared with the FP64 oracle directly.  Arguments it must
refuse (host memory, an intermediate beyond the static array) are refused before any launch,
with a message."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def ntf():
    from paper_1409_2383_gb300 import build, ntf as binding
    build.build()
    binding.lib()
    return binding


def _rel(a, b):
    return float(torch.linalg.norm((a - b).double()) / torch.linalg.norm(b.double()))


CASES = [
    ((64, 48, 40), 20, torch.float32),        # split-K partials and the intermediate in scratch
    ((400, 400, 400), 20, torch.float32),     # the benchmark shape
    ((20, 24, 16, 50), 16, torch.bfloat16),   # 4-way: both halves need the intermediate
    ((13, 17, 11), 5, torch.float32),         # unaligned rows: plain fallback kernels
    ((200, 1000, 1000), 8, torch.float32),    # mode-3 intermediate of 8e6 floats: near the limit
]


@pytest.mark.parametrize("dims,R,dtype", CASES)
def test_noalloc_matches_context_mttkrp_on_two_calls(ntf, dims, R, dtype):
    g = torch.Generator().manual_seed(sum(dims) + R)
    X = (torch.rand(dims, generator=g) - 0.3).to(dtype).cuda()
    F = [torch.rand(d, R, generator=g).cuda() for d in dims]
    with ntf.Context(X, R, ntf.default_params(contraction=ntf.NTF_CONTRACT_SIMT)) as ctx:
        want = [ctx.mttkrp(n, F).clone() for n in range(len(dims))]
    outs = [torch.empty(d, R, device="cuda") for d in dims]
    for call in range(2):
        for n in range(len(dims)):
            outs[n].fill_(float("nan"))
            ntf.mttkrp_noalloc(X, n, F, out=outs[n])
        torch.cuda.synchronize()
        for n in range(len(dims)):
            assert _rel(outs[n], want[n]) <= TOL, (call, n, _rel(outs[n], want[n]))


def test_noalloc_unsplit_contraction_when_partials_do_not_fit(ntf):
    """Mode 3 of a 65536 x 32 x 32 tensor at R = 64: the 4.2e6-float Khatri-Rao table leaves
    no room for the split-K partial sums the contraction plan asks for, so the contraction
    range is not split; the result still matches the context's.  (Modes 1 and 2 of this shape
    need a 1.3e8-float intermediate and are refused.)"""
    dims, R = (65536, 32, 32), 64
    g = torch.Generator().manual_seed(7)
    X = (torch.rand(dims, generator=g) - 0.3).cuda()
    F = [torch.rand(d, R, generator=g).cuda() for d in dims]
    with ntf.Context(X, R, ntf.default_params(contraction=ntf.NTF_CONTRACT_SIMT)) as ctx:
        want = ctx.mttkrp(2, F).clone()
    out = torch.empty(dims[2], R, device="cuda")
    for call in range(2):
        out.fill_(float("nan"))
        ntf.mttkrp_noalloc(X, 2, F, out=out)
        torch.cuda.synchronize()
        assert _rel(out, want) <= TOL, (call, _rel(out, want))
    with pytest.raises(ntf.NTFError) as e:
        ntf.mttkrp_noalloc(X, 0, F)
    assert e.value.status == 1


def test_noalloc_rejects_an_intermediate_beyond_the_maximum(ntf):
    dims, R = (4, 2048, 2048), 4               # mode 3 needs a 2048*2048*4-float intermediate
    X = torch.zeros(dims, device="cuda")
    F = [torch.zeros(d, R, device="cuda") for d in dims]
    with pytest.raises(ntf.NTFError) as e:
        ntf.mttkrp_noalloc(X, 2, F)
    assert e.value.status == 1
    assert "scratch" in str(e.value) and "mode 2" in str(e.value)
    cdims = (ctypes.c_int64 * 3)(*dims)
    ptrs = (ctypes.c_void_p * 3)(*[f.data_ptr() for f in F])
    out = torch.empty(dims[2], R, device="cuda")
    assert ntf.lib().ntf_mttkrp_noalloc(3, cdims, R, 0, X.data_ptr(), 2, ptrs, out.data_ptr(),
                                        None) == 1
    # the leading modes need only a 4*2048*4-float intermediate and still work
    for n in (0, 1):
        M = ntf.mttkrp_noalloc(X, n, F)
        torch.cuda.synchronize()
        assert torch.count_nonzero(M) == 0


def test_noalloc_matches_the_oracle(ntf):
    import synth
    from oracle import ntf as o
    dims, R = (64, 48, 40), 20
    X, _, init = synth.workload(dims, R, seed=3, snr_db=20.0)
    F64 = [f.astype(np.float32).astype(np.float64) for f in init]
    Xd = torch.as_tensor(X).cuda()
    F = [torch.as_tensor(f, dtype=torch.float32).cuda() for f in F64]
    for call in range(2):
        for n in range(3):
            got = ntf.mttkrp_noalloc(Xd, n, F)
            torch.cuda.synchronize()
            want = o.mttkrp(X.astype(np.float64), F64, n)
            err = np.linalg.norm(got.cpu().double().numpy() - want) / np.linalg.norm(want)
            assert err <= TOL, (call, n, err)


def test_noalloc_refuses_host_memory_before_any_launch(ntf):
    dims, R = (16, 16, 16), 4
    Xh = np.ones(dims, dtype=np.float32)           # pageable host memory
    F = [torch.ones(d, R, device="cuda") for d in dims]
    out = torch.full((dims[0], R), float("nan"), device="cuda")
    cdims = (ctypes.c_int64 * 3)(*dims)
    ptrs = (ctypes.c_void_p * 3)(*[f.data_ptr() for f in F])
    st = ntf.lib().ntf_mttkrp_noalloc(3, cdims, R, 0, Xh.ctypes.data, 0, ptrs, out.data_ptr(),
                                      None)
    assert st == 1
    assert b"device memory" in ntf.lib().ntf_last_error()
    # a host factor is refused the same way
    Fh = np.ones((dims[1], R), dtype=np.float32)
    ptrs[1] = Fh.ctypes.data
    Xd = torch.ones(dims, device="cuda")
    assert ntf.lib().ntf_mttkrp_noalloc(3, cdims, R, 0, Xd.data_ptr(), 0, ptrs, out.data_ptr(),
                                        None) == 1
    torch.cuda.synchronize()
    assert torch.isnan(out).all()                 # nothing was launched
