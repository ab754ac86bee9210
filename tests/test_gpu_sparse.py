"""Sparse-tensor MTTKRP (the sparse case of Sec. IV-A) on the GPU against the FP64 oracle's
coordinate-form MTTKRP (``oracle.mttkrp_coo``, pinned against index loops and the dense
definition in ``tests/test_oracle_ntf.py``): relative Frobenius error <= 1e-5 for every mode,
3- and 4-way, ranks 1..64, duplicated coordinates, empty rows, a row spanning many chunks,
indices that need every radix pass, and bit-identical repeated calls."""
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
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def _check(ntf, dims, idx, vals, R, seed=0):
    rng = np.random.default_rng(seed)
    fs = [rng.random((d, R)).astype(np.float32) for d in dims]
    F = [torch.as_tensor(f).cuda() for f in fs]
    F64 = [f.astype(np.float64) for f in fs]
    with ntf.SparseTensor(torch.as_tensor(idx).cuda(), torch.as_tensor(vals).cuda(), dims) as sp:
        assert sp.nnz == len(vals)
        for n in range(len(dims)):
            got = sp.mttkrp(n, F)
            again = sp.mttkrp(n, F)
            torch.cuda.synchronize()
            want = o.mttkrp_coo(idx, vals.astype(np.float64), F64, n)
            assert rel(got.cpu().numpy(), want) <= TOL, (n, rel(got.cpu().numpy(), want))
            assert torch.equal(got, again)                  # a fixed summation order


@pytest.mark.parametrize("dims,nnz,R", [((30, 40, 50), 5000, 1), ((30, 40, 50), 5000, 5),
                                        ((30, 40, 50), 20000, 32), ((64, 20, 33), 9000, 33),
                                        ((50, 60, 70), 30000, 64), ((12, 10, 14, 16), 3000, 7),
                                        ((1000, 1000, 1000), 2_000_000, 32)])
def test_sparse_mttkrp_matches_oracle(ntf, dims, nnz, R):
    idx, vals = synth.sparse_tensor(dims, nnz, seed=nnz + R)
    _check(ntf, dims, idx, vals, R)


def test_duplicates_and_empty_rows(ntf):
    dims = (300, 200, 100)               # 5000 coordinates: most rows of every mode empty
    idx, vals = synth.sparse_tensor(dims, 5000, seed=3, duplicates=True)
    idx = np.concatenate([idx, idx[:500]])                  # exact duplicates as well
    vals = np.concatenate([vals, vals[:500]])
    _check(ntf, dims, idx, vals, 16)


def test_a_row_spanning_many_chunks(ntf):
    """Half of the nonzeros share the index 0 in mode 1 (a row of tens of thousands of entries
    in that mode's layout), the rest are spread; 4-way."""
    dims, nnz = (40, 30, 20, 25), 60000
    idx, vals = synth.sparse_tensor(dims, nnz, seed=5, duplicates=True)
    idx[: nnz // 2, 1] = 0
    _check(ntf, dims, idx, vals, 24)


def test_indices_needing_every_radix_pass(ntf):
    dims, nnz = (100_000, 300, 70_000), 100_000     # keys above 2^16: three passes
    idx, vals = synth.sparse_tensor(dims, nnz, seed=9)
    _check(ntf, dims, idx, vals, 8)
