"""Pins of the FP64 warm-start network oracle (oracle/mlp.py): central finite differences
for every gradient, the GELU derivative, Adam's first-step and convergence properties, the
NNLS targets against exhaustive enumeration, and the scale invariance of the features."""
import math

import numpy as np
import pytest

from oracle import mlp
from oracle import ntf as o


def _params(Din, H, Dout, seed=0):
    rng = np.random.default_rng(seed)
    return {
        "W1": rng.standard_normal((H, Din)) / math.sqrt(Din),
        "b1": rng.standard_normal(H) * 0.1,
        "W2": rng.standard_normal((H, H)) / math.sqrt(H),
        "b2": rng.standard_normal(H) * 0.1,
        "W3": rng.standard_normal((Dout, H)) / math.sqrt(H),
        "b3": rng.standard_normal(Dout) * 0.1,
    }


def test_gelu_grad_finite_difference():
    z = np.linspace(-6, 6, 241)
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    assert np.allclose(mlp.gelu_grad(z), fd, atol=1e-8)
    # GELU(z) = z * Phi(z): limits
    assert abs(mlp.gelu(np.array([8.0]))[0] - 8.0) < 1e-12
    assert abs(mlp.gelu(np.array([-8.0]))[0]) < 1e-12
    # the exact form (not the tanh approximation) at table values of the normal CDF:
    # Phi(1) = 0.8413447460685429, Phi(2) = 0.9772498680518208, Phi(0.5) = 0.6914624612740131
    z = np.array([0.0, 1.0, -1.0, 2.0, 0.5])
    want = z * np.array([0.5, 0.8413447460685429, 1 - 0.8413447460685429,
                         0.9772498680518208, 0.6914624612740131])
    assert np.allclose(mlp.gelu(z), want, rtol=1e-14, atol=1e-16)
    tanh_form = 0.5 * z * (1 + np.tanh(math.sqrt(2 / math.pi) * (z + 0.044715 * z ** 3)))
    assert not np.allclose(mlp.gelu(z), tanh_form, rtol=1e-6, atol=0)


def test_backward_matches_central_differences():
    R, H = 3, 7
    Din, Dout = R * R + 2 * R, 2 * R
    p = _params(Din, H, Dout)
    rng = np.random.default_rng(1)
    U = rng.standard_normal((5, Din))
    T = rng.standard_normal((5, Dout))
    out, cache = mlp.forward(p, U)
    g = mlp.backward(p, cache, out, T)
    h = 1e-6
    for k, P in p.items():
        flat = P.reshape(-1)
        for idx in range(0, flat.size, max(1, flat.size // 17)):
            old = flat[idx]
            flat[idx] = old + h
            lp = mlp.loss(mlp.forward(p, U)[0], T)
            flat[idx] = old - h
            lm = mlp.loss(mlp.forward(p, U)[0], T)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(g[k].reshape(-1)[idx] - fd) <= 1e-7 * (1 + abs(fd)), (k, idx)


def test_adam_first_step_is_lr_times_sign():
    """With zero moments, bias correction makes the first Adam step lr * g / |g|."""
    p = {"w": np.array([1.0, -2.0, 3.0])}
    g = {"w": np.array([0.5, -1e-3, 20.0])}
    m = {"w": np.zeros(3)}
    v = {"w": np.zeros(3)}
    mlp.adam_step(p, g, m, v, 1, lr=0.1, eps=0.0)
    assert np.allclose(p["w"], [0.9, -1.9, 2.9], rtol=1e-12)


def test_adam_constant_gradient_steps_are_all_lr():
    """With a constant gradient the bias-corrected moments are g and g^2 at every step, so
    every step is lr * sign(g) (eps = 0): a missing or misplaced bias correction makes the
    early steps differ."""
    p = {"w": np.array([0.0, 0.0])}
    g = {"w": np.array([0.3, -7.0])}
    m = {"w": np.zeros(2)}
    v = {"w": np.zeros(2)}
    for t in range(1, 6):
        mlp.adam_step(p, g, m, v, t, lr=0.01, eps=0.0)
        assert np.allclose(p["w"], [-0.01 * t, 0.01 * t], rtol=1e-12, atol=0)


def test_forward_and_loss_by_hand():
    """A one-unit network whose pre-activations land on table values of the normal CDF:
    z1 = 1, h1 = Phi(1); z2 = h1 / Phi(1) = 1, h2 = Phi(1); out = 2 h2 + 1.  The loss is the
    mean of the squared entries of the error."""
    phi1 = 0.8413447460685429
    p = {"W1": np.array([[1.0]]), "b1": np.array([0.0]), "W2": np.array([[1.0 / phi1]]),
         "b2": np.array([0.0]), "W3": np.array([[2.0]]), "b3": np.array([1.0])}
    out, _ = mlp.forward(p, np.array([[1.0]]))
    assert out[0, 0] == pytest.approx(2 * phi1 + 1, rel=1e-14)
    assert mlp.loss(np.array([[1.0, 2.0]]), np.array([[0.0, 0.0]])) == 2.5
    assert mlp.loss(np.array([[1.0], [3.0]]), np.array([[1.0], [1.0]])) == 2.0


def test_decode_clamps_to_the_kkt_signs():
    """Network output [x ; y/s] -> (max(0, x), min(0, s y)): a non-negative auxiliary and a
    non-positive dual, the signs eq. (KKT_NTF) fixes."""
    out = np.array([[1.5, -0.5, 0.25, -2.0]])
    aux, dual = mlp.decode(out, 4.0, 2)
    assert np.array_equal(aux, [[1.5, 0.0]]) and np.array_equal(dual, [[0.0, -8.0]])


def test_adam_minimises_quadratic():
    rng = np.random.default_rng(2)
    target = rng.standard_normal(10)
    p = {"w": np.zeros(10)}
    m = {"w": np.zeros(10)}
    v = {"w": np.zeros(10)}
    for t in range(1, 3001):
        mlp.adam_step(p, {"w": 2 * (p["w"] - target)}, m, v, t, lr=0.01)
    assert np.allclose(p["w"], target, atol=1e-3)


@pytest.mark.parametrize("R", [3, 6])
def test_nnls_row_against_exhaustive(R):
    rng = np.random.default_rng(R)
    K = rng.random((4 * R, R))
    G = K.T @ K
    for _ in range(8):
        m = rng.standard_normal(R) * np.trace(G) / R
        x, y = mlp.nnls_row(G, m)
        assert np.allclose(x, o.nnls_exhaustive(G, m), atol=1e-9)
        # KKT of eq. (KKT_NTF): y = m - G x <= 0 and y * x = 0
        assert np.all(y <= 1e-9) and np.all(np.abs(x * y) <= 1e-9)


def test_features_are_scale_invariant():
    rng = np.random.default_rng(4)
    K = rng.random((12, 4))
    G = K.T @ K
    M = rng.standard_normal((3, 4))
    U1, s1 = mlp.features(G, M)
    U2, s2 = mlp.features(7.5 * G, 7.5 * M)
    assert np.allclose(U1, U2) and math.isclose(s2, 7.5 * s1)
    # the NNLS solution is unchanged and the dual scales with the data
    x1, y1 = mlp.nnls_row(G, M[0])
    x2, y2 = mlp.nnls_row(7.5 * G, 7.5 * M[0])
    assert np.allclose(x1, x2, atol=1e-10) and np.allclose(7.5 * y1, y2, atol=1e-9)
    T1 = mlp.targets(G, x1[None], y1[None], s1)
    T2 = mlp.targets(7.5 * G, x2[None], y2[None], s2)
    assert np.allclose(T1, T2, atol=1e-9)
    ax, dy = mlp.decode(T1, s1, 4)
    assert np.allclose(ax[0], x1, atol=1e-12) and np.allclose(dy[0], np.minimum(y1, 0))


def test_row_objective_and_kkt_residual_pins():
    """q(x) against the Cholesky least-squares form 1/2||L^T x - L^{-1} m||^2 - 1/2||L^{-1} m||^2
    (G = L L^T); the KKT residual vanishes at the exhaustive NNLS solution and nowhere near it."""
    rng = np.random.default_rng(21)
    R = 5
    K = rng.random((3 * R, R))
    G = K.T @ K
    M = rng.standard_normal((6, R)) * np.trace(G) / R
    X = np.abs(rng.standard_normal((6, R)))
    L = np.linalg.cholesky(G)
    b = np.linalg.solve(L, M.T).T
    ls = 0.5 * np.sum((X @ L - b) ** 2, axis=1) - 0.5 * np.sum(b ** 2, axis=1)
    assert np.allclose(mlp.row_objective(G, M, X), ls, rtol=1e-12, atol=1e-9)
    Xs = np.array([o.nnls_exhaustive(G, m) for m in M])
    assert np.all(mlp.kkt_residual(G, M, Xs) < 1e-18 * np.sum(M ** 2))
    assert np.all(mlp.kkt_residual(G, M, Xs + 0.1) > 0)


def test_judge_needs_both_criteria():
    rng = np.random.default_rng(22)
    R = 4
    K = rng.random((3 * R, R))
    G = K.T @ K
    M = rng.standard_normal((8, R)) * np.trace(G) / R
    Xs = np.array([o.nnls_exhaustive(G, m) for m in M])
    Xp = np.maximum(Xs + 0.3 * rng.standard_normal(Xs.shape), 0.0)
    Xp[np.all(Xp == Xs, axis=1)] += 0.5      # no perturbed row may equal the solution
    # the solution minimises q over x >= 0 and has zero KKT residual: it always wins ...
    assert np.all(mlp.judge(G, M, Xs, Xp))
    # ... and is never replaced (no candidate has a smaller KKT residual than zero)
    assert not np.any(mlp.judge(G, M, Xp, Xs))
    # a candidate equal to the carried state is not taken (strict comparisons)
    assert not np.any(mlp.judge(G, M, Xp, Xp))


def test_z_feature_is_the_first_admm_iterate_from_zero():
    """The z part of the features equals the primal of one step of eq. (ADMM_NTF_ALS_C) from a
    zero auxiliary and dual with rho = trace(G)/R (the oracle's Cholesky-based update)."""
    rng = np.random.default_rng(23)
    R = 6
    K = rng.random((4 * R, R))
    G = K.T @ K
    M = rng.random((9, R)) * 3.0
    U, s = mlp.features(G, M)
    A, _, _, _ = o.admm_factor_update(M, G, np.zeros_like(M), np.zeros_like(M), s, 1)
    assert np.allclose(U[:, R * R + R:], A, rtol=1e-12, atol=1e-12)
    assert np.allclose(U[:, R * R:R * R + R], M / s)
