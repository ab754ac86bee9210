"""Seeded synthetic inputs for non-negative CP factorization experiments.

This module only creates workloads; it holds none of the factorization method's
arithmetic.  Both the FP64 oracle and the CUDA library are fed from here, so the two see
byte-identical inputs.

Recipe (the experiments of Sec. VI-A of Liavas & Sidiropoulos, plus the structured variants
used for the stress workloads):

* factor entries i.i.d. U[0,1] (``structure="uniform"``);
* ``structure="sparse"``: each entry zeroed independently with probability ``zero_frac``,
  any all-zero column redrawn;
* ``structure="collinear"``: column r of factor n is ``a*u0 + (1-a)*u_r`` with u0, u_r
  i.i.d. U[0,1] vectors and ``a`` chosen so the expected congruence (cosine) between two
  columns equals ``congruence``;
* X = [F_1, ..., F_N] + noise with i.i.d. Gaussian noise, its variance given directly
  (``sigma2``, as in the paper) or through an SNR in dB,
  SNR = 10 log10(||X0||^2 / (numel * sigma2));
* the algorithm's random start is i.i.d. U[0,1].

Every random stream is a numpy PCG64 generator keyed by (seed, stream id, index), so the
result does not depend on chunking.
"""
from __future__ import annotations

import math
from typing import List, Optional, Sequence

import numpy as np

_FACTOR, _NOISE, _INIT = 0, 1, 2


def _rng(*key: int) -> np.random.Generator:
    return np.random.default_rng([int(k) for k in key])


def collinear_weight(congruence: float) -> float:
    """Mixing weight a for which E-moments of U[0,1] entries give the requested congruence.

    For f_r = a u0 + (1-a) u_r:  E[f_r f_s] = a^2/3 + a(1-a)/2 + (1-a)^2/4 (r != s) and
    E[f_r^2] = a^2/3 + a(1-a)/2 + (1-a)^2/3; solved for a by bisection.
    """
    if not 0.75 <= congruence < 1.0:
        raise ValueError("independent U[0,1] columns already have congruence 0.75")

    def c(a):
        cross = a * a / 3 + a * (1 - a) / 2 + (1 - a) ** 2 / 4
        self_ = a * a / 3 + a * (1 - a) / 2 + (1 - a) ** 2 / 3
        return cross / self_

    lo, hi = 0.0, 1.0
    for _ in range(100):
        mid = 0.5 * (lo + hi)
        if c(mid) < congruence:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def factors(dims: Sequence[int], R: int, seed: int, structure: str = "uniform",
            zero_frac: float = 0.5, congruence: float = 0.9) -> List[np.ndarray]:
    """Ground-truth non-negative factors, FP64, one [I_n, R] array per mode."""
    out = []
    for n, I in enumerate(dims):
        g = _rng(seed, _FACTOR, n)
        if structure == "uniform":
            F = g.random((I, R))
        elif structure == "sparse":
            F = g.random((I, R))
            F[g.random((I, R)) < zero_frac] = 0.0
            for r in range(R):
                while not np.any(F[:, r] > 0):
                    col = g.random(I)
                    col[g.random(I) < zero_frac] = 0.0
                    F[:, r] = col
        elif structure == "collinear":
            a = collinear_weight(congruence)
            u0 = g.random(I)
            F = a * u0[:, None] + (1 - a) * g.random((I, R))
        else:
            raise ValueError(f"unknown structure {structure!r}")
        out.append(F)
    return out


def init_factors(dims: Sequence[int], R: int, seed: int) -> List[np.ndarray]:
    """The algorithm's random start: i.i.d. U[0,1] entries, FP64."""
    return [_rng(seed, _INIT, n).random((I, R)) for n, I in enumerate(dims)]


def _tail(fs: Sequence[np.ndarray]) -> np.ndarray:
    """[prod(I_2..I_N), R] table whose row (i_2, ..., i_N) (last index fastest) holds the
    products F_2[i_2, r] * ... * F_N[i_N, r]."""
    t = fs[1]
    for F in fs[2:]:
        t = (t[:, None, :] * F[None, :, :]).reshape(-1, F.shape[1])
    return t


def _slab(fs: Sequence[np.ndarray], tail: np.ndarray, i0: int) -> np.ndarray:
    """Noise-free slab X0[i0, ...] = sum_r F_1[i0, r] * (outer product of the other columns)."""
    return (tail @ fs[0][i0]).reshape([F.shape[0] for F in fs[1:]])


def tensor(fs: Sequence[np.ndarray], seed: int, snr_db: Optional[float] = None,
           sigma2: Optional[float] = None, dtype=np.float32) -> np.ndarray:
    """Observed tensor X = [F_1..F_N] + N with i.i.d. N(0, sigma^2) noise (Sec. VI-A).

    Exactly one of ``snr_db`` / ``sigma2`` may be given (neither: noise-free).  Built slab by
    slab over the first mode; the noise of slab i0 comes from its own stream.
    """
    dims = [F.shape[0] for F in fs]
    numel = int(np.prod(dims))
    X = np.empty(dims, dtype=dtype)
    sq = 0.0
    tail = _tail(fs)
    for i0 in range(dims[0]):
        s = _slab(fs, tail, i0)
        sq += float(np.sum(s * s))
        X[i0] = s
    if snr_db is not None and sigma2 is not None:
        raise ValueError("give snr_db or sigma2, not both")
    if snr_db is not None:
        sigma2 = sq / (numel * 10.0 ** (snr_db / 10.0))
    if sigma2:
        sd = math.sqrt(sigma2)
        slab_shape = dims[1:]
        for i0 in range(dims[0]):
            noise = _rng(seed, _NOISE, i0).standard_normal(slab_shape)
            X[i0] = (X[i0].astype(np.float64) + sd * noise).astype(dtype)
    return X


def workload(dims: Sequence[int], R: int, seed: int = 0, snr_db: Optional[float] = 20.0,
             sigma2: Optional[float] = None, structure: str = "uniform", dtype=np.float32,
             **kw):
    """(X, true factors, init factors) for one synthetic problem."""
    fs = factors(dims, R, seed, structure, **kw)
    X = tensor(fs, seed, snr_db=snr_db, sigma2=sigma2, dtype=dtype)
    return X, fs, init_factors(dims, R, seed + 1)


# Named workloads with the shapes, ranks and structure of the evaluation configurations.
WORKLOADS = {
    "50x50x50_r5": dict(dims=(50, 50, 50), R=5, snr_db=20.0),
    "400x400x400_r20": dict(dims=(400, 400, 400), R=20, snr_db=20.0),
    "1000x1000x1000_r32": dict(dims=(1000, 1000, 1000), R=32, snr_db=30.0),
    "600x600x600_r50_sparse": dict(dims=(600, 600, 600), R=50, snr_db=20.0,
                                   structure="sparse"),
    "200x200x200x50_r16_collinear": dict(dims=(200, 200, 200, 50), R=16, snr_db=10.0,
                                         structure="collinear"),
}


def sparse_tensor(dims: Sequence[int], nnz: int, seed: int, R: Optional[int] = None,
                  duplicates: bool = False):
    """A sparse tensor in coordinate form: nnz coordinates drawn uniformly (distinct unless
    ``duplicates``), values U[0,1] or, with R, the values of a rank-R model of U[0,1] factors
    (seed's factor streams) at those coordinates.  Returns (indices int32 [nnz, N], values
    float32 [nnz])."""
    g = _rng(seed, _NOISE, 1 << 20)
    numel = int(np.prod(dims))
    if duplicates:
        flat = g.integers(0, numel, nnz)
    else:
        flat = g.choice(numel, size=nnz, replace=False) if nnz < numel // 4 else \
            g.permutation(numel)[:nnz]
    idx = np.stack(np.unravel_index(flat, dims), axis=1).astype(np.int32)
    if R is None:
        vals = g.random(nnz)
    else:
        fs = factors(dims, R, seed)
        prod = np.ones((nnz, R))
        for m, F in enumerate(fs):
            prod *= F[idx[:, m]]
        vals = prod.sum(axis=1)
    return idx, vals.astype(np.float32)
