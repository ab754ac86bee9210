"""Structural constraints of Sec. IV-E in the oracle: the projections against brute force,
and the factor update with them against its special cases."""
import itertools

import numpy as np
import pytest

from oracle import ntf as o


def _brute_sparse(V, c):
    """Nearest non-negative matrix with at most c nonzeros, over every support."""
    flat = V.ravel()
    best, best_d = None, np.inf
    for k in range(c + 1):
        for S in itertools.combinations(range(flat.size), k):
            P = np.zeros_like(flat)
            P[list(S)] = np.maximum(flat[list(S)], 0.0)  # nearest on a support: (v)_+
            d = np.sum((P - flat) ** 2)
            if d < best_d - 1e-15:
                best, best_d = P, d
    return best.reshape(V.shape), best_d


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("c", [0, 1, 2, 4])
def test_sparse_projection_is_the_nearest_point(seed, c):
    V = np.random.default_rng(seed).standard_normal((2, 3))
    P = o.project_nonneg_sparse(V, c)
    _, d = _brute_sparse(V, c)
    assert np.all(P >= 0) and np.count_nonzero(P) <= c
    assert np.isclose(np.sum((P - V) ** 2), d, rtol=0, atol=1e-12)


def test_sparse_projection_special_cases():
    V = np.random.default_rng(1).standard_normal((5, 4))
    assert np.array_equal(o.project_nonneg_sparse(V, V.size), np.maximum(V, 0))
    assert not np.any(o.project_nonneg_sparse(V, 0))
    P = o.project_nonneg_sparse(V, 3)
    assert np.array_equal(o.project_nonneg_sparse(P, 3), P)       # idempotent
    with pytest.raises(ValueError):
        o.project_nonneg_sparse(V, -1)


def test_box_projection():
    rng = np.random.default_rng(2)
    V = rng.standard_normal((6, 3)) * 3
    P = o.project_box(V, -0.5, 1.0)
    assert np.all((P >= -0.5) & (P <= 1.0))
    # nearest: no point of the box is closer, entry by entry, than the clamp
    for cand in rng.uniform(-0.5, 1.0, (200,) + V.shape):
        assert np.all(np.abs(P - V) <= np.abs(cand - V) + 1e-15)
    assert np.array_equal(o.project_box(V, 0.0, np.inf), np.maximum(V, 0))
    with pytest.raises(ValueError):
        o.project_box(V, 1.0, 0.0)


def _update_inputs(seed=3, I=9, R=4):
    rng = np.random.default_rng(seed)
    F = rng.random((I + 3, R))
    G = F.T @ F
    M = rng.standard_normal((I, R)) + rng.random((I, R))
    At = np.maximum(rng.standard_normal((I, R)), 0)
    Y = -np.abs(rng.standard_normal((I, R))) * (At == 0)
    return M, G, At, Y, o.rho_trace(G)


def test_update_reduces_to_the_plain_one():
    M, G, At, Y, rho = _update_inputs()
    plain = o.admm_factor_update(M, G, At, Y, rho, 5)
    for proj in (lambda V: o.project_nonneg_sparse(V, V.size),
                 lambda V: o.project_box(V, 0.0, np.inf)):
        got = o.admm_factor_update(M, G, At, Y, rho, 5, project=proj)
        for a, b in zip(got[:3], plain[:3]):
            assert np.array_equal(a, b)


def test_update_keeps_the_constraint():
    M, G, At, Y, rho = _update_inputs()
    _, At_s, _, _ = o.admm_factor_update(M, G, At, Y, rho, 7,
                                         project=lambda V: o.project_nonneg_sparse(V, 10))
    assert np.all(At_s >= 0) and np.count_nonzero(At_s) <= 10
    _, At_b, _, _ = o.admm_factor_update(M, G, At, Y, rho, 7,
                                         project=lambda V: o.project_box(V, 0.1, 0.6))
    assert np.all((At_b >= 0.1) & (At_b <= 0.6))
