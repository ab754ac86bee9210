"""Plain FP64 CPU oracle for ADMoM non-negative CP factorization (NTF).

Liavas & Sidiropoulos, "Parallel Algorithms for Constrained Tensor Factorization via
Alternating Direction Method of Multipliers" (arXiv 1409.2383).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
CPU-baseline leg may import this module.  The product path (the CUDA library and its Python
binding) never imports it, and this module imports nothing from the product package.

Every function follows the paper's definitions literally, in FP64, with no blocking, fusion
or reordering beyond what the definition states:

* matricization with the column order implied by Sec. II eq. (f_X_matr): the lowest-numbered
  remaining mode varies fastest (W^(1) = A (C (.) B)^T);
* the Khatri-Rao factor of mode n is F_N (.) ... (.) F_{n+1} (.) F_{n-1} (.) ... (.) F_1
  (Sec. II, App. A);
* MTTKRP = explicit unfolding times explicit Khatri-Rao matrix (Sec. IV-A, item 1);
* the coefficient matrix via the Gram identity (Sec. IV-A, item 2) and explicitly;
* the per-factor update of eq. (ADMM_NTF_ALS_C), solved with LAPACK Cholesky, followed by
  the projection and dual ascent of eq. (ADMoM_NTF);
* residuals and stopping test of Sec. IV-C, penalty rule of Sec. IV-D;
* the relative factorization error of Sec. VI-A by explicit reconstruction.

Where the paper is silent the readings are (each also listed in the design notes):
* ``inner_iters`` L repeats the closed-form update / projection / dual step L times per
  factor with the coefficient matrix fixed (the paper uses L = 1, Sec. IV footnote);
* ``kr_source`` chooses which factors feed the Khatri-Rao products: the unconstrained primal
  factors (the paper, eq. ADMM_NTF_ALS_C) or the non-negative auxiliaries;
* ``rho_policy`` "adaptive" is the rule of eq. (varying_penalty_rule) applied once per outer
  iteration; "trace" sets rho = trace(G)/R for every factor update;
* the dual is kept unscaled (Y, as in eq. ADMoM_NTF); the dual residual of an update with L
  inner iterations is rho * (aux after - aux before the update);
* reported factors are the non-negative auxiliaries.

Parity status: every function here is pinned by ``tests/test_oracle_*.py`` (the restart loop
by ``tests/test_restarts.py``) against brute force, closed forms, exhaustive NNLS, optimality
conditions or the paper's printed values.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np
import scipy.linalg


# ----------------------------------------------------------------------------------------
# Sec. II: matricization and Khatri-Rao products
# ----------------------------------------------------------------------------------------

def unfold(X: np.ndarray, n: int) -> np.ndarray:
    """Mode-n matricization X^(n) (Sec. II, eq. f_X_matr).

    Row index i_n; the column index enumerates the other modes with the lowest-numbered one
    varying fastest, e.g. X^(1)[i, j + J*k] = X[i, j, k] for a 3-way tensor, which is the
    ordering that makes W^(1) = A (C (.) B)^T hold.
    """
    others = [m for m in range(X.ndim) if m != n]
    # C-order reshape makes the LAST listed axis fastest, so list the others highest-first.
    Xt = np.transpose(X, [n] + others[::-1])
    return np.ascontiguousarray(Xt).reshape(X.shape[n], -1)


def fold(W: np.ndarray, n: int, shape: Sequence[int]) -> np.ndarray:
    """Inverse of :func:`unfold` for a tensor of the given shape."""
    others = [m for m in range(len(shape)) if m != n]
    perm = [n] + others[::-1]
    Wt = W.reshape([shape[p] for p in perm])
    return np.transpose(Wt, np.argsort(perm))


def khatri_rao(U: np.ndarray, V: np.ndarray) -> np.ndarray:
    """Column-wise Kronecker product U (.) V (Sec. I-A notation).

    Column r is kron(U[:, r], V[:, r]): row u * rows(V) + v holds U[u, r] * V[v, r].
    """
    if U.shape[1] != V.shape[1]:
        raise ValueError("Khatri-Rao operands need the same number of columns")
    R = U.shape[1]
    out = np.empty((U.shape[0] * V.shape[0], R), dtype=np.float64)
    for r in range(R):
        out[:, r] = np.kron(U[:, r], V[:, r])
    return out


def kr_others(factors: Sequence[np.ndarray], n: int) -> np.ndarray:
    """Khatri-Rao factor of mode n: F_N (.) ... (.) F_{n+1} (.) F_{n-1} (.) ... (.) F_1.

    Sec. II (3-way: C (.) B, C (.) A, B (.) A) and App. A (4-way: D (.) (C (.) B), ...).
    """
    others = [m for m in range(len(factors)) if m != n]
    K = np.asarray(factors[others[-1]], dtype=np.float64)
    for m in reversed(others[:-1]):
        K = khatri_rao(K, np.asarray(factors[m], dtype=np.float64))
    return K


def reconstruct(factors: Sequence[np.ndarray]) -> np.ndarray:
    """[F_1, ..., F_N] = sum_f f_1 o ... o f_N, built as fold(F_1 KR^T) (Sec. II)."""
    shape = [F.shape[0] for F in factors]
    W1 = np.asarray(factors[0], dtype=np.float64) @ kr_others(factors, 0).T
    return fold(W1, 0, shape)


# ----------------------------------------------------------------------------------------
# Sec. IV-A: MTTKRP and the coefficient matrix
# ----------------------------------------------------------------------------------------

def mttkrp(X: np.ndarray, factors: Sequence[np.ndarray], n: int) -> np.ndarray:
    """M_n = X^(n) (Khatri-Rao of the other factors): explicit unfolding times explicit KR.

    Sec. IV-A item 1 (the term X^(1)(C (.) B) of eq. ADMM_NTF_ALS_C).
    """
    return unfold(np.asarray(X, dtype=np.float64), n) @ kr_others(factors, n)


def mttkrp_rows(X: np.ndarray, factors: Sequence[np.ndarray], n: int,
                rows: Sequence[int]) -> np.ndarray:
    """Selected rows of M_n: the mode-n slices X[..., i, ...] for i in ``rows`` unfolded and
    multiplied by the explicit Khatri-Rao matrix (same definition as :func:`mttkrp`)."""
    Xs = np.take(np.asarray(X), list(rows), axis=n).astype(np.float64)
    return unfold(Xs, n) @ kr_others(factors, n)


def mttkrp_coo(indices: np.ndarray, values: np.ndarray, factors: Sequence[np.ndarray],
               n: int) -> np.ndarray:
    """MTTKRP of a sparse tensor in coordinate form (the sparse case of Sec. IV-A: with n
    nonzeros it costs 3nF flops for a 3-way tensor).  Entry (i_1, ..., i_N) with value v adds
    v * prod_{m != n} F_m[i_m, :] to row i_n of M (duplicate coordinates add up, as in the dense
    tensor they describe).  indices: [nnz, N] integers, values: [nnz]."""
    indices = np.asarray(indices)
    values = np.asarray(values, np.float64)
    R = np.asarray(factors[0]).shape[1]
    M = np.zeros((np.asarray(factors[n]).shape[0], R))
    prod = values[:, None] * np.ones((values.size, R))
    for m, F in enumerate(factors):
        if m != n:
            prod = prod * np.asarray(F, np.float64)[indices[:, m]]
    np.add.at(M, indices[:, n], prod)
    return M


def coo_to_dense(indices: np.ndarray, values: np.ndarray, dims: Sequence[int]) -> np.ndarray:
    """The dense tensor a coordinate list describes (duplicates add up)."""
    X = np.zeros(dims)
    np.add.at(X, tuple(np.asarray(indices).T), np.asarray(values, np.float64))
    return X


def gram(F: np.ndarray) -> np.ndarray:
    """F^T F in FP64."""
    F = np.asarray(F, dtype=np.float64)
    return F.T @ F


def coeff_matrix_explicit(factors: Sequence[np.ndarray], n: int) -> np.ndarray:
    """(KR)^T (KR) with the Khatri-Rao matrix formed explicitly (eq. ADMM_NTF_ALS_C)."""
    K = kr_others(factors, n)
    return K.T @ K


def coeff_matrix(factors: Sequence[np.ndarray], n: int) -> np.ndarray:
    """(KR)^T (KR) via the Hadamard-of-Grams identity of Sec. IV-A item 2."""
    G = None
    for m, F in enumerate(factors):
        if m == n:
            continue
        G = gram(F) if G is None else G * gram(F)
    return G


# ----------------------------------------------------------------------------------------
# eq. (ADMM_NTF_ALS_C) + eq. (ADMoM_NTF): one factor update
# ----------------------------------------------------------------------------------------

@dataclasses.dataclass
class UpdateStats:
    primal_res: float  # ||A - At||_F                       (eq. R_Mk_def)
    dual_res: float    # rho ||At_after - At_before||_F     (eq. D_Mk_def)
    norm_A: float
    norm_At: float
    norm_Y: float
    rho: float


def project_nonneg(V: np.ndarray) -> np.ndarray:
    """Projection onto the non-negative matrices (eq. ADMoM_NTF): (V)_+."""
    return np.maximum(V, 0.0)


def project_nonneg_sparse(V: np.ndarray, c: int) -> np.ndarray:
    """Projection onto the non-negative matrices with at most c nonzero entries (Sec. IV-E,
    eq. g_new_def), by sorting.  Keeping entry v costs (max(v, 0) - v)^2 and zeroing it v^2,
    so keeping it gains max(v, 0)^2: the projection keeps the c largest positive entries
    (ties broken by the lower flat index) and zeroes the rest."""
    if c < 0:
        raise ValueError("c must be >= 0")
    P = np.maximum(np.asarray(V, np.float64), 0.0)
    flat = P.ravel()
    if np.count_nonzero(flat) <= c:
        return P
    keep = np.argsort(-flat, kind="stable")[:c]
    out = np.zeros_like(flat)
    out[keep] = flat[keep]
    return out.reshape(P.shape)


def project_box(V: np.ndarray, lo: float, hi: float) -> np.ndarray:
    """Projection onto the box lo <= entry <= hi (Sec. IV-E, "box or other set
    constraints"): entrywise clamp."""
    if not lo <= hi:
        raise ValueError("lo must be <= hi")
    return np.clip(np.asarray(V, np.float64), lo, hi)


def admm_factor_update(M: np.ndarray, G: np.ndarray, At: np.ndarray, Y: np.ndarray,
                       rho: float, inner_iters: int = 1, project=project_nonneg):
    """Update one factor: L repetitions of

        A   = (M + rho At - Y) (G + rho I)^{-1}        (eq. ADMM_NTF_ALS_C)
        At  = (A + Y / rho)_+                          (eq. ADMoM_NTF, auxiliary)
        Y   = Y + rho (A - At)                         (eq. ADMoM_NTF, dual)

    with G + rho I factored once by Cholesky (Sec. IV-A item 2) and the common coefficient
    matrix shared by all rows (App. B).  ``project`` replaces (.)_+ for the structural
    constraints of Sec. IV-E (the only step that changes there).  Returns (A, At, Y,
    UpdateStats).
    """
    if not rho > 0:
        raise ValueError("rho must be positive")
    M = np.asarray(M, np.float64)
    G = np.asarray(G, np.float64)
    R = G.shape[0]
    Lc = np.linalg.cholesky(G + rho * np.eye(R))
    At_before = np.array(At, np.float64)
    At_k = At_before.copy()
    Y_k = np.array(Y, np.float64)
    A = None
    for _ in range(max(1, inner_iters)):
        rhs = M + rho * At_k - Y_k                               # I x R
        Z = scipy.linalg.solve_triangular(Lc, rhs.T, lower=True)
        A = scipy.linalg.solve_triangular(Lc.T, Z, lower=False).T
        At_k = project(A + Y_k / rho)
        Y_k = Y_k + rho * (A - At_k)
    st = UpdateStats(
        primal_res=float(np.linalg.norm(A - At_k)),
        dual_res=float(rho * np.linalg.norm(At_k - At_before)),
        norm_A=float(np.linalg.norm(A)),
        norm_At=float(np.linalg.norm(At_k)),
        norm_Y=float(np.linalg.norm(Y_k)),
        rho=float(rho),
    )
    return A, At_k, Y_k, st


def rho_trace(G: np.ndarray) -> float:
    """rho = trace(G) / R (the fixed-per-update penalty policy)."""
    return float(np.trace(G)) / G.shape[0]


def rho_adapt(rho: float, P: float, D: float, mu: float = 8.0, tau_incr: float = 4.0,
              tau_decr: float = 2.0) -> float:
    """Penalty rule of eq. (varying_penalty_rule), Sec. IV-D."""
    if P > mu * D:
        return tau_incr * rho
    if D > mu * P:
        return rho / tau_decr
    return rho


def small_residuals(st: UpdateStats, rows: int, R: int, eps_abs: float, eps_rel: float) -> bool:
    """Stopping test of eqs. (stopping_cond_prim_A_def) and (stopping_cond_dual_A_def)."""
    base = math.sqrt(rows * R) * eps_abs
    return (st.primal_res <= base + eps_rel * max(st.norm_A, st.norm_At)
            and st.dual_res <= base + eps_rel * st.norm_Y)


# ----------------------------------------------------------------------------------------
# Sec. VI-A: relative factorization error; Sec. IV-B: KKT conditions
# ----------------------------------------------------------------------------------------

def rfe(X: np.ndarray, factors: Sequence[np.ndarray]) -> float:
    """||X - [F_1..F_N]||_F / ||X||_F by explicit reconstruction (Sec. VI-A)."""
    X = np.asarray(X, np.float64)
    return float(np.linalg.norm(X - reconstruct(factors)) / np.linalg.norm(X))


def kkt_nnls(G: np.ndarray, M: np.ndarray, At: np.ndarray, Y: Optional[np.ndarray] = None):
    """KKT quantities of the non-negative least-squares problem of one factor.

    With the other factors fixed, the factor problem is min_{A >= 0} 1/2 ||X^(n) - A K^T||^2
    whose gradient is g = A G - M.  eq. (KKT_NTF) asks Y = M - A G (i.e. Y = -g), A = At,
    Y <= 0 and Y (*) At = 0.  Scaled with s_x = max|At| and s_g = max|G| s_x + max|M|:

      neg_x   = -min(At) / s_x            (primal feasibility; 0 by construction)
      dual    = max(-g) / s_g             (dual feasibility, -g <= 0)
      comp    = sum|At * g| / (n s_x s_g) (complementarity)
      y_gap   = ||Y - (M - At G)|| / (sqrt(n) s_g)   (only if Y is given)
    """
    G = np.asarray(G, np.float64)
    M = np.asarray(M, np.float64)
    At = np.asarray(At, np.float64)
    g = At @ G - M
    s_x = max(float(np.max(np.abs(At))), 1e-30)
    s_g = float(np.max(np.abs(G))) * s_x + float(np.max(np.abs(M)))
    out = {
        "neg_x": float(max(0.0, -np.min(At)) / s_x),
        "dual": float(max(0.0, np.max(-g)) / s_g),
        "comp": float(np.sum(np.abs(At * g)) / (At.size * s_x * s_g)),
    }
    if Y is not None:
        out["y_gap"] = float(np.linalg.norm(np.asarray(Y, np.float64) - (M - At @ G))
                             / (math.sqrt(At.size) * s_g))
    return out


def nnls_exhaustive(G: np.ndarray, m: np.ndarray) -> np.ndarray:
    """Exact solution of min_{x >= 0} 1/2 x^T G x - m^T x for SPD G by enumerating supports.

    For every support S the stationary point on S is G_SS x_S = m_S; the solution is the one
    with x_S >= 0 and gradient (G x - m) >= 0 off S.  Exponential in R: for R <= 10 only.
    """
    G = np.asarray(G, np.float64)
    m = np.asarray(m, np.float64)
    R = G.shape[0]
    if R > 10:
        raise ValueError("exhaustive NNLS is for R <= 10")
    best, best_val = None, math.inf
    for mask in range(1 << R):
        S = [j for j in range(R) if mask >> j & 1]
        x = np.zeros(R)
        if S:
            x[S] = np.linalg.solve(G[np.ix_(S, S)], m[S])
            if np.min(x[S]) < -1e-12:
                continue
        g = G @ x - m
        off = [j for j in range(R) if j not in S]
        if off and np.min(g[off]) < -1e-10 * (1 + np.max(np.abs(m))):
            continue
        val = 0.5 * x @ G @ x - m @ x
        if val < best_val:
            best, best_val = np.maximum(x, 0.0), val
    return best


# ----------------------------------------------------------------------------------------
# Outer iteration (eq. ADMoM_NTF with the alternating scheme of eq. ADMM_NTF_ALS_C)
# ----------------------------------------------------------------------------------------

@dataclasses.dataclass
class Params:
    inner_iters: int = 1          # L (paper: 1)
    kr_source: str = "primal"     # "primal" (paper) or "aux"
    rho_policy: str = "adaptive"  # "adaptive" (eq. varying_penalty_rule) or "trace"
    rho0: float = 1.0
    mu: float = 8.0
    tau_incr: float = 4.0
    tau_decr: float = 2.0
    eps_abs: float = 1e-4
    eps_rel: float = 1e-4


PAPER = Params()
AO = Params(inner_iters=5, kr_source="aux", rho_policy="trace")


@dataclasses.dataclass
class State:
    primal: List[np.ndarray]
    aux: List[np.ndarray]
    dual: List[np.ndarray]
    rho: List[float]


def init_state(init: Sequence[np.ndarray], params: Params) -> State:
    """Initial point of Sec. VI-A (paper mode) or the all-uniform start (aux mode).

    Paper mode: primal factors take the given non-negative random values (only those of
    modes 2..N are used), auxiliaries and duals are zero.  Aux mode: primal = aux = the
    given values, duals zero.
    """
    prim = [np.array(F, np.float64) for F in init]
    if params.kr_source == "primal":
        aux = [np.zeros_like(F) for F in prim]
    else:
        aux = [F.copy() for F in prim]
    dual = [np.zeros_like(F) for F in prim]
    return State(prim, aux, dual, [params.rho0] * len(prim))


def outer_iteration(X: np.ndarray, st: State, params: Params):
    """One ADMoM iteration: update factors 1..N in Gauss-Seidel order (eq. ADMM_NTF_ALS_C),
    each followed by its projection and dual step (eq. ADMoM_NTF); then the penalty rule.

    Returns the list of per-factor UpdateStats and the last factor's MTTKRP.
    """
    N = X.ndim
    stats = []
    M = None
    for n in range(N):
        src = st.primal if params.kr_source == "primal" else st.aux
        M = mttkrp(X, src, n)
        G = coeff_matrix(src, n)
        rho = rho_trace(G) if params.rho_policy == "trace" else st.rho[n]
        A, At, Y, s = admm_factor_update(M, G, st.aux[n], st.dual[n], rho, params.inner_iters)
        st.primal[n], st.aux[n], st.dual[n] = A, At, Y
        st.rho[n] = rho
        stats.append(s)
    if params.rho_policy == "adaptive":
        for n in range(N):
            st.rho[n] = rho_adapt(st.rho[n], stats[n].primal_res, stats[n].dual_res,
                                  params.mu, params.tau_incr, params.tau_decr)
    return stats, M


def factorize(X: np.ndarray, init: Sequence[np.ndarray], params: Params, max_iters: int,
              stop_on_residuals: bool = True, record_rfe: bool = True):
    """Run outer iterations until the stopping test (Sec. IV-C) holds for every factor or
    ``max_iters`` is reached.  Returns (State, history) with history a list of
    (iteration, rfe) pairs and the convergence flag."""
    st = init_state(init, params)
    hist = []
    converged = False
    for k in range(max_iters):
        stats, _ = outer_iteration(X, st, params)
        if record_rfe:
            hist.append((k + 1, rfe(X, st.aux)))
        if stop_on_residuals and all(
                small_residuals(s, st.aux[n].shape[0], st.aux[n].shape[1], params.eps_abs,
                                params.eps_rel) for n, s in enumerate(stats)):
            converged = True
            break
    return st, hist, converged


def factorize_with_restarts(X: np.ndarray, draws: Sequence[Sequence[np.ndarray]],
                            params: Params, n_max: int):
    """The restart strategy of Sec. VI-A: run ADMoM for up to n_max outer iterations; if the
    stopping test of Sec. IV-C has not held by then, start again from the next random initial
    point, until it converges.  The random initial points are inputs (draws[attempt], the
    factors that init_state takes); the paper repeats without bound, here the attempts end
    with the last draw.  Returns (State, history, converged, restarts) of the last attempt,
    restarts = the number of attempts before it."""
    if not draws:
        raise ValueError("at least one initial point is needed")
    for attempt, init in enumerate(draws):
        st, hist, converged = factorize(X, init, params, n_max)
        if converged:
            break
    return st, hist, converged, attempt
