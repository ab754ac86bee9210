"""FP64 CPU oracle of the warm-start network for the per-row non-negative least squares.

TEST INFRASTRUCTURE ONLY (same import rule as ``oracle/ntf.py``).

With the other factors fixed, every row a_i of a factor solves
    min_{x >= 0} 1/2 x^T G x - m_i^T x          (G = coefficient matrix, m_i = MTTKRP row)
and the ADMoM iteration of eq. (ADMoM_NTF) converges to x* with dual y* = m_i - G x*
(eq. KKT_NTF: Y = M - A G, Y <= 0, Y (*) A = 0).  The network maps the normalised pair
(G / s, m_i / s, z_i), s = trace(G) / R, to (x*, y* / s), where z_i = (G + s I)^{-1} m_i is
the first primal iterate of the row's ADMM from zero (eq. ADMM_NTF_ALS_C with rho = s): a
fixed function of (G, m_i) that spares the network learning a matrix inverse.  The
normalisation uses the invariance of the problem under (G, m) -> (c G, c m): x* and z are
unchanged and y* scales by c.

Architecture: input [vec(G/s) ; m_i/s ; z_i] of size R^2 + 2R, two hidden layers of width H with
the exact GELU, x -> x Phi(x), and a linear output of size 2R; loss = mean squared error.
Adam as in Kingma & Ba (2015).  Everything in FP64, one dense layer after the other, with
the first layer applied to the full concatenated input (no per-G reuse), so it is the plain
definition that the GPU kernels are checked against.
"""
from __future__ import annotations

import math
from typing import Dict, Tuple

import numpy as np
import scipy.optimize
import scipy.special

Params = Dict[str, np.ndarray]


def gelu(z: np.ndarray) -> np.ndarray:
    return 0.5 * z * (1.0 + scipy.special.erf(z / math.sqrt(2.0)))


def gelu_grad(z: np.ndarray) -> np.ndarray:
    cdf = 0.5 * (1.0 + scipy.special.erf(z / math.sqrt(2.0)))
    pdf = np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)
    return cdf + z * pdf


def features(G: np.ndarray, M: np.ndarray) -> Tuple[np.ndarray, float]:
    """Rows [vec(G/s) ; m_i/s ; z_i] for every row m_i of M, z_i = (G + s I)^{-1} m_i, and the
    scale s = trace(G)/R."""
    G = np.asarray(G, np.float64)
    M = np.asarray(M, np.float64)
    R = G.shape[0]
    s = float(np.trace(G)) / R
    U = np.empty((M.shape[0], R * R + 2 * R))
    U[:, :R * R] = (G / s).reshape(1, -1)
    U[:, R * R:R * R + R] = M / s
    U[:, R * R + R:] = np.linalg.solve(G + s * np.eye(R), M.T).T
    return U, s


def forward(p: Params, U: np.ndarray):
    """Returns the output [B, 2R] and the cache needed by :func:`backward`."""
    z1 = U @ p["W1"].T + p["b1"]
    h1 = gelu(z1)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = gelu(z2)
    out = h2 @ p["W3"].T + p["b3"]
    return out, (U, z1, h1, z2, h2)


def loss(out: np.ndarray, T: np.ndarray) -> float:
    """Mean over all entries of the squared error."""
    d = out - T
    return float(np.mean(d * d))


def backward(p: Params, cache, out: np.ndarray, T: np.ndarray) -> Params:
    """Gradients of :func:`loss` with respect to every parameter (chain rule, layer by layer)."""
    U, z1, h1, z2, h2 = cache
    d_out = 2.0 * (out - T) / out.size
    g = {"W3": d_out.T @ h2, "b3": d_out.sum(0)}
    d_h2 = d_out @ p["W3"]
    d_z2 = d_h2 * gelu_grad(z2)
    g["W2"] = d_z2.T @ h1
    g["b2"] = d_z2.sum(0)
    d_h1 = d_z2 @ p["W2"]
    d_z1 = d_h1 * gelu_grad(z1)
    g["W1"] = d_z1.T @ U
    g["b1"] = d_z1.sum(0)
    return g


def adam_step(p: Params, g: Params, m: Params, v: Params, t: int, lr: float,
              beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8) -> None:
    """One Adam update (bias-corrected first and second moments), in place; t counts from 1."""
    for k in p:
        m[k] = beta1 * m[k] + (1 - beta1) * g[k]
        v[k] = beta2 * v[k] + (1 - beta2) * g[k] * g[k]
        mh = m[k] / (1 - beta1 ** t)
        vh = v[k] / (1 - beta2 ** t)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)


def nnls_row(G: np.ndarray, m: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """(x*, y*) of min_{x>=0} 1/2 x^T G x - m^T x via an active-set NNLS on the Cholesky
    form 1/2 ||L^T x - L^{-1} m||^2 (constant dropped); y* = m - G x*."""
    L = np.linalg.cholesky(np.asarray(G, np.float64))
    b = np.linalg.solve(L, np.asarray(m, np.float64))
    x, _ = scipy.optimize.nnls(L.T, b, maxiter=50 * G.shape[0])
    return x, m - G @ x


def targets(G: np.ndarray, X: np.ndarray, Y: np.ndarray, s: float) -> np.ndarray:
    """Training targets [x* ; y*/s] for rows (x*, y*)."""
    return np.concatenate([X, Y / s], axis=1)


def decode(out: np.ndarray, s: float, R: int) -> Tuple[np.ndarray, np.ndarray]:
    """Network output -> warm-start (aux, dual) rows: aux = max(0, x), dual = min(0, s y)."""
    return np.maximum(out[:, :R], 0.0), np.minimum(out[:, R:] * s, 0.0)


def row_objective(G: np.ndarray, M: np.ndarray, X: np.ndarray) -> np.ndarray:
    """q(x_i) = 1/2 x_i^T G x_i - m_i^T x_i per row: the part of the squared fit error that
    depends on row i of the factor being updated (eq. ADMM_NTF_ALS_C without the constant)."""
    return 0.5 * np.sum((X @ G) * X, axis=1) - np.sum(M * X, axis=1)


def kkt_residual(G: np.ndarray, M: np.ndarray, X: np.ndarray) -> np.ndarray:
    """||min(x_i, G x_i - m_i)||^2 per row: zero exactly at the NNLS solution (eq. KKT_NTF)."""
    return np.sum(np.minimum(X, X @ G - M) ** 2, axis=1)


def judge(G: np.ndarray, M: np.ndarray, Xc: np.ndarray, Xo: np.ndarray) -> np.ndarray:
    """Rows where the candidate Xc replaces the carried-over Xo: both the row objective and
    the KKT residual are smaller (strictly)."""
    return ((row_objective(G, M, Xc) < row_objective(G, M, Xo))
            & (kkt_residual(G, M, Xc) < kkt_residual(G, M, Xo)))
