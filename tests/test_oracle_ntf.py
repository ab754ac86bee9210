"""Pins of the FP64 oracle (oracle/ntf.py) against things other than itself:
brute-force loops, closed forms, exhaustive NNLS, optimality of the argmin, invariants of
the projection/dual step, the centralized = partitioned equivalence (App. B) and the
paper's printed Table 1 / Table 2 values.  CPU only."""
import itertools
import math
import os

import numpy as np
import pytest

import synth
from oracle import ntf as o

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand(shape, seed=0):
    return np.random.default_rng(seed).random(shape)


# ---------------------------------------------------------------- matricization (Sec. II)

@pytest.mark.parametrize("shape", [(3, 4, 5), (2, 3, 4, 5)])
def test_unfold_matches_index_definition(shape):
    X = _rand(shape)
    for n in range(len(shape)):
        U = o.unfold(X, n)
        others = [m for m in range(len(shape)) if m != n]
        for idx in itertools.product(*[range(s) for s in shape]):
            col, stride = 0, 1
            for m in others:                       # lowest remaining mode fastest
                col += idx[m] * stride
                stride *= shape[m]
            assert U[idx[n], col] == X[idx]
        assert np.array_equal(o.fold(U, n, shape), X)


def test_khatri_rao_definition():
    U, V = _rand((3, 2), 1), _rand((4, 2), 2)
    K = o.khatri_rao(U, V)
    for u in range(3):
        for v in range(4):
            for r in range(2):
                assert K[u * 4 + v, r] == U[u, r] * V[v, r]


@pytest.mark.parametrize("shape", [(3, 4, 5), (2, 3, 4, 5)])
def test_reconstruct_is_sum_of_outer_products(shape):
    R = 3
    fs = [_rand((s, R), 10 + i) for i, s in enumerate(shape)]
    W = np.zeros(shape)
    for r in range(R):
        t = fs[0][:, r]
        for F in fs[1:]:
            t = np.multiply.outer(t, F[:, r])
        W += t
    assert np.allclose(o.reconstruct(fs), W, rtol=1e-14, atol=1e-14)
    # eq. (f_X_matr): W^(n) = F_n (KR of the others)^T for every n
    for n in range(len(shape)):
        assert np.allclose(o.unfold(W, n), fs[n] @ o.kr_others(fs, n).T, rtol=1e-13)


# ---------------------------------------------------------------- MTTKRP (Sec. IV-A)

def test_mttkrp_brute_force_3way():
    I, J, K, R = 3, 4, 5, 2
    X = _rand((I, J, K), 3) - 0.3
    A, B, C = _rand((I, R), 4), _rand((J, R), 5), _rand((K, R), 6)
    want = [np.zeros((I, R)), np.zeros((J, R)), np.zeros((K, R))]
    for i in range(I):
        for j in range(J):
            for k in range(K):
                for r in range(R):
                    want[0][i, r] += X[i, j, k] * B[j, r] * C[k, r]
                    want[1][j, r] += X[i, j, k] * A[i, r] * C[k, r]
                    want[2][k, r] += X[i, j, k] * A[i, r] * B[j, r]
    for n in range(3):
        assert np.allclose(o.mttkrp(X, [A, B, C], n), want[n], rtol=1e-13, atol=1e-14)


def test_mttkrp_brute_force_4way():
    shape, R = (2, 3, 4, 5), 3
    X = _rand(shape, 7) - 0.5
    fs = [_rand((s, R), 20 + i) for i, s in enumerate(shape)]
    for n in range(4):
        want = np.zeros((shape[n], R))
        for idx in itertools.product(*[range(s) for s in shape]):
            w = np.ones(R)
            for m in range(4):
                if m != n:
                    w = w * fs[m][idx[m]]
            want[idx[n]] += X[idx] * w
        assert np.allclose(o.mttkrp(X, fs, n), want, rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("shape", [(3, 4, 5), (2, 3, 4, 5)])
def test_mttkrp_rows_brute_force(shape):
    """Selected rows of M_n (unordered, repeated) against the index loops of the MTTKRP
    definition (the sampled-row check of the full-size GPU parity tests relies on them)."""
    R = 3
    X = _rand(shape, 11) - 0.4
    fs = [_rand((s, R), 40 + i) for i, s in enumerate(shape)]
    for n in range(len(shape)):
        full = np.zeros((shape[n], R))
        for idx in itertools.product(*[range(s) for s in shape]):
            w = np.ones(R)
            for m in range(len(shape)):
                if m != n:
                    w = w * fs[m][idx[m]]
            full[idx[n]] += X[idx] * w
        rows = [shape[n] - 1, 0, shape[n] - 1, shape[n] // 2]
        assert np.allclose(o.mttkrp_rows(X, fs, n, rows), full[rows], rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("shape", [(6, 5, 4), (3, 4, 5, 2)])
def test_mttkrp_exact_low_rank_closed_form(shape):
    """X = [F] exactly  =>  M_n = F_n * (Hadamard of the other Grams)."""
    R = 3
    fs = [_rand((s, R), 30 + i) for i, s in enumerate(shape)]
    X = o.reconstruct(fs)
    for n in range(len(shape)):
        H = np.ones((R, R))
        for m, F in enumerate(fs):
            if m != n:
                H = H * (F.T @ F)
        assert np.allclose(o.mttkrp(X, fs, n), fs[n] @ H, rtol=1e-12)


def test_mttkrp_all_ones():
    I, J, K, R = 4, 5, 6, 3
    A, B, C = _rand((I, R), 1), _rand((J, R), 2), _rand((K, R), 3)
    M = o.mttkrp(np.ones((I, J, K)), [A, B, C], 0)
    assert np.allclose(M, np.tile(B.sum(0) * C.sum(0), (I, 1)), rtol=1e-13)


@pytest.mark.parametrize("shape", [(6, 5, 4), (3, 4, 5, 2)])
def test_coeff_matrix_hadamard_identity(shape):
    """(KR)^T (KR) = Hadamard of Grams (Sec. IV-A item 2)."""
    fs = [_rand((s, 4), 40 + i) for i, s in enumerate(shape)]
    for n in range(len(shape)):
        assert np.allclose(o.coeff_matrix(fs, n), o.coeff_matrix_explicit(fs, n), rtol=1e-13)


# ---------------------------------------------------------------- factor update

def _setup_update(seed=0, I=7, shape=(7, 6, 5), R=4):
    rng = np.random.default_rng(seed)
    X = rng.random(shape)
    fs = [rng.random((s, R)) for s in shape]
    At = np.maximum(rng.standard_normal((I, R)), 0)
    Y = -np.abs(rng.standard_normal((I, R))) * (At == 0)
    return X, fs, At, Y


def test_update_is_argmin_of_augmented_objective():
    """First line of eq. (ADMM_NTF_ALS_C): A^{k+1} minimises
    1/2||X^(1) - A K^T||^2 + Y*A + rho/2 ||A - At||^2  -- checked by evaluating the objective
    (explicit unfolding and Khatri-Rao) in random directions around the returned A."""
    X, fs, At, Y = _setup_update()
    rho = 0.7
    K = o.kr_others(fs, 0)
    X1 = o.unfold(X, 0)

    def f(A):
        return (0.5 * np.sum((X1 - A @ K.T) ** 2) + np.sum(Y * A)
                + 0.5 * rho * np.sum((A - At) ** 2))

    A, _, _, _ = o.admm_factor_update(o.mttkrp(X, fs, 0), o.coeff_matrix(fs, 0), At, Y, rho, 1)
    f0 = f(A)
    rng = np.random.default_rng(1)
    for _ in range(20):
        D = rng.standard_normal(A.shape)
        for t in (1e-2, 1e-4):
            assert f(A + t * D) >= f0
            # zero gradient: the objective is symmetric to first order around A
            assert abs(f(A + t * D) - f(A - t * D)) <= 1e-9 * abs(f0) + 1e-12


def test_projection_and_dual_invariants():
    """After every step of eq. (ADMoM_NTF): At >= 0, Y <= 0 and Y (*) At = 0 up to rounding,
    when the dual starts non-positive (it does: zero init).  A sign error in either step
    breaks this."""
    X, fs, At, Y = _setup_update(seed=2)
    X = X - 0.5                      # mixed signs so that some projections are active
    M, G = o.mttkrp(X, fs, 0), o.coeff_matrix(fs, 0)
    for L in (1, 2, 7):
        for rho in (1e-3, 0.5, 30.0):
            _, At2, Y2, _ = o.admm_factor_update(M, G, At, Y, rho, L)
            scale = rho * (np.max(np.abs(At2)) + 1) + np.max(np.abs(Y))
            assert np.all(At2 >= 0)
            assert np.all(Y2 <= 1e-14 * scale)
            assert np.all(np.abs(Y2 * At2) <= 1e-14 * scale * (np.max(At2) + 1))
            assert np.min(Y2) < -1e-3 * scale   # the dual is not trivially zero


def _nnls_case(R, seed):
    rng = np.random.default_rng(seed)
    K = rng.random((3 * R, R))
    G = K.T @ K
    M = rng.standard_normal((6, R)) * np.trace(G) / R
    return G, M


@pytest.mark.parametrize("R,seed", [(3, 0), (5, 1), (8, 2)])
def test_inner_loop_converges_to_exhaustive_nnls(R, seed):
    """With G and M fixed, L -> infinity takes the auxiliary factor to the exact NNLS
    solution, pinned by enumeration of supports, and satisfies eq. (KKT_NTF)."""
    G, M = _nnls_case(R, seed)
    At = np.zeros_like(M)
    Y = np.zeros_like(M)
    _, At, Y, st = o.admm_factor_update(M, G, At, Y, o.rho_trace(G), 3000)
    for i in range(M.shape[0]):
        x = o.nnls_exhaustive(G, M[i])
        assert np.allclose(At[i], x, atol=1e-8 * (1 + np.max(np.abs(x))))
    k = o.kkt_nnls(G, M, At, Y)
    assert k["neg_x"] == 0 and k["dual"] < 1e-9 and k["comp"] < 1e-10 and k["y_gap"] < 1e-9


def test_kkt_measures_on_a_hand_worked_problem():
    """eq. (KKT_NTF) on min_{x >= 0} 1/2 ||x||^2 - m^T x with m = (1, -1): x* = (1, 0),
    gradient g = x - m.  Each measure is zero at x* and positive exactly where its own
    condition fails (the scale is s_g = max|G| max|x| + max|m|)."""
    G, M = np.eye(2), np.array([[1.0, -1.0]])
    k = o.kkt_nnls(G, M, np.array([[1.0, 0.0]]), np.array([[0.0, -1.0]]))
    assert k == {"neg_x": 0.0, "dual": 0.0, "comp": 0.0, "y_gap": 0.0}
    k = o.kkt_nnls(G, M, np.array([[0.5, 0.0]]))           # g = (-0.5, 1): not dual feasible
    assert k["neg_x"] == 0.0 and k["dual"] == pytest.approx(0.5 / 1.5) and k["comp"] > 0
    k = o.kkt_nnls(G, M, np.array([[1.0, 0.5]]))           # g = (0, 1.5): x_2 g_2 != 0
    assert k["dual"] == 0.0 and k["comp"] == pytest.approx(0.75 / (2 * 1.0 * 2.0))
    k = o.kkt_nnls(G, M, np.array([[1.0, -0.25]]))         # infeasible x
    assert k["neg_x"] == pytest.approx(0.25)
    k = o.kkt_nnls(G, M, np.array([[1.0, 0.0]]), np.array([[0.0, -0.5]]))   # Y != M - x G
    assert k["y_gap"] == pytest.approx(0.5 / (math.sqrt(2) * 2.0))


def test_nnls_exhaustive_against_scipy():
    import scipy.optimize
    for seed in range(5):
        G, M = _nnls_case(6, seed)
        L = np.linalg.cholesky(G)
        for m in M:
            x, _ = scipy.optimize.nnls(L.T, np.linalg.solve(L, m))
            assert np.allclose(o.nnls_exhaustive(G, m), x, atol=1e-9)


def test_rho_rule_cases():
    """eq. (varying_penalty_rule): the three cases are exclusive for mu > 1."""
    assert o.rho_adapt(1.0, 9.0, 1.0) == 4.0
    assert o.rho_adapt(1.0, 1.0, 9.0) == 0.5
    assert o.rho_adapt(2.0, 1.0, 1.0) == 2.0
    assert o.rho_adapt(2.0, 8.0, 1.0) == 2.0          # boundary: strict inequality


def test_trace_penalty_bounds_the_condition_number():
    """rho = trace(G)/R: G = c I gives rho = c, and for any PSD G (rank-deficient included)
    the eigenvalues of G lie in [0, trace G], so cond(G + rho I) <= (trace G + rho) / rho
    = R + 1."""
    assert o.rho_trace(3.5 * np.eye(4)) == 3.5
    rng = np.random.default_rng(9)
    for R, rank in ((5, 5), (8, 2), (20, 1)):
        F = rng.standard_normal((30, rank)) @ rng.standard_normal((rank, R))
        G = F.T @ F
        rho = o.rho_trace(G)
        assert np.linalg.cond(G + rho * np.eye(R)) <= (R + 1) * (1 + 1e-12)
    G = np.diag([1.0] + [0.0] * 5)                      # the bound is reached
    assert np.linalg.cond(G + o.rho_trace(G) * np.eye(6)) == pytest.approx(7.0)


def test_stopping_test_scaling():
    st = o.UpdateStats(primal_res=1e-3, dual_res=1e-3, norm_A=1.0, norm_At=1.0, norm_Y=1.0,
                       rho=1.0)
    # sqrt(I F) eps_abs = 10 * 1e-4 = 1e-3 -> both equalities hold
    assert o.small_residuals(st, 10, 10, 1e-4, 0.0)
    assert not o.small_residuals(st, 10, 10, 0.9e-4, 0.0)


def test_stopping_test_relative_terms():
    """eqs. (stopping_cond_prim_A_def), (stopping_cond_dual_A_def) worked by hand: the primal
    bound takes the larger of ||A||, ||At||, the dual bound takes ||Y||, and both add the
    absolute term sqrt(I F) eps_abs."""
    def st(p, d, a, t, y):
        return o.UpdateStats(primal_res=p, dual_res=d, norm_A=a, norm_At=t, norm_Y=y, rho=1.0)
    # I F = 4: absolute term 0; relative: primal 0.1 * max(2, 5) = 0.5, dual 0.1 * 1 = 0.1
    assert o.small_residuals(st(0.5, 0.1, 2.0, 5.0, 1.0), 4, 1, 0.0, 0.1)
    assert o.small_residuals(st(0.3, 0.05, 2.0, 5.0, 1.0), 4, 1, 0.0, 0.1)      # > 0.1 min(.)
    assert o.small_residuals(st(0.3, 0.05, 5.0, 2.0, 1.0), 4, 1, 0.0, 0.1)      # either order
    assert not o.small_residuals(st(0.51, 0.1, 2.0, 5.0, 1.0), 4, 1, 0.0, 0.1)
    assert not o.small_residuals(st(0.1, 0.3, 2.0, 5.0, 1.0), 4, 1, 0.0, 0.1)   # dual: ||Y||
    # I F = 36: absolute 6 * 0.01 = 0.06; primal 0.06 + 0.1 * 1 = 0.16, dual 0.06 + 0.1 * 2
    assert o.small_residuals(st(0.16, 0.26, 1.0, 0.5, 2.0), 9, 4, 0.01, 0.1)
    assert not o.small_residuals(st(0.161, 0.26, 1.0, 0.5, 2.0), 9, 4, 0.01, 0.1)
    assert not o.small_residuals(st(0.16, 0.261, 1.0, 0.5, 2.0), 9, 4, 0.01, 0.1)


def test_partitioned_update_equals_centralized():
    """App. B / eq. (partitioned_update_Ak): row blocks of A computed from column-blocked
    unfoldings, sum_nC X_{nA,nC} (C_nC (.) B) and sum_nC (C_nC (.) B)^T (C_nC (.) B), equal
    the centralized update."""
    rng = np.random.default_rng(5)
    I, J, K, R = 9, 4, 7, 3
    X = rng.random((I, J, K))
    A, B, C = rng.random((I, R)), rng.random((J, R)), rng.random((K, R))
    At = rng.random((I, R))
    Y = -rng.random((I, R)) * 0.1
    rho = 0.9
    A_c, At_c, Y_c, _ = o.admm_factor_update(o.mttkrp(X, [A, B, C], 0),
                                             o.coeff_matrix([A, B, C], 0), At, Y, rho, 1)
    row_blocks = [range(0, 4), range(4, 9)]
    col_blocks = [range(0, 2), range(2, 5), range(5, 7)]
    for rb in row_blocks:
        rb = list(rb)
        Msum = np.zeros((len(rb), R))
        Gsum = np.zeros((R, R))
        for cb in col_blocks:
            cb = list(cb)
            KRb = o.khatri_rao(C[cb], B)
            Xb = o.unfold(X[rb][:, :, cb], 0)
            Msum += Xb @ KRb
            Gsum += KRb.T @ KRb
        A_b = (Msum + rho * At[rb] - Y[rb]) @ np.linalg.inv(Gsum + rho * np.eye(R))
        assert np.allclose(A_b, A_c[rb], rtol=1e-11)


# ---------------------------------------------------------------- whole runs

def test_rfe_special_cases():
    """Sec. VI-A's error: 0 for the exact factors of a noise-free tensor, 1 for zero
    factors, |1 - c| when the factors reproduce c X, and invariant to scaling X and one
    factor together."""
    fs = [_rand((s, 3), 60 + i) for i, s in enumerate((5, 4, 6))]
    X = o.reconstruct(fs)
    assert o.rfe(X, fs) < 1e-15
    assert o.rfe(X, [np.zeros_like(F) for F in fs]) == pytest.approx(1.0)
    assert o.rfe(X, [0.25 * fs[0], fs[1], fs[2]]) == pytest.approx(0.75)
    Xn = X + 0.01 * _rand(X.shape, 70)
    assert o.rfe(3.0 * Xn, [3.0 * fs[0], fs[1], fs[2]]) == pytest.approx(o.rfe(Xn, fs))


def test_exact_low_rank_fit_goes_to_zero():
    """Noise-free non-negative data: the relative error keeps falling (no floor, Sec. VI-C)."""
    dims = (12, 10, 8)
    fs = synth.factors(dims, 3, 0)
    X = synth.tensor(fs, 0, dtype=np.float64)
    st, hist, _ = o.factorize(X, synth.init_factors(dims, 3, 1), o.AO, 500,
                              stop_on_residuals=False, record_rfe=False)
    assert o.rfe(X, st.aux) < 2e-4


def test_noisy_fit_reaches_noise_floor_ao_mode():
    """Noisy data: the fitted error equals the noise level sqrt(||N||^2 / ||X||^2) reduced by
    the fraction of the data absorbed by the model's degrees of freedom."""
    dims = (24, 22, 20)
    fs = synth.factors(dims, 3, 3)
    X0 = synth.tensor(fs, 3, dtype=np.float64)
    X = synth.tensor(fs, 3, snr_db=20.0, dtype=np.float64)
    floor = np.linalg.norm(X - X0) / np.linalg.norm(X) * math.sqrt(1 - sum(dims) * 3 / X.size)
    st, _, _ = o.factorize(X, synth.init_factors(dims, 3, 4), o.AO, 150,
                           stop_on_residuals=False, record_rfe=False)
    assert abs(o.rfe(X, st.aux) / floor - 1) < 0.01


def test_paper_mode_converges_with_stopping_rule():
    """Paper settings (Sec. VI-A): L = 1, primal Khatri-Rao, rho0 = 1, mu = 8, tau = 4 / 2,
    eps = 1e-4, B0, C0 random, other state zero; converges within n_max = 400 and the final
    auxiliaries satisfy the KKT conditions of eq. (KKT_NTF) approximately."""
    dims = (30, 30, 30)
    fs = synth.factors(dims, 3, 0)
    X = synth.tensor(fs, 0, snr_db=20.0, dtype=np.float64)
    X0 = synth.tensor(fs, 0, dtype=np.float64)
    st, _, conv = o.factorize(X, synth.init_factors(dims, 3, 1), o.PAPER, 400,
                              record_rfe=False)
    assert conv
    floor = np.linalg.norm(X - X0) / np.linalg.norm(X) * math.sqrt(1 - sum(dims) * 3 / X.size)
    assert abs(o.rfe(X, st.aux) / floor - 1) < 0.01
    for n in range(3):
        k = o.kkt_nnls(o.coeff_matrix(st.aux, n), o.mttkrp(X, st.aux, n), st.aux[n])
        assert k["dual"] < 1e-2 and k["comp"] < 1e-4


# ---------------------------------------------------------------- printed values

def _golden(name):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        if line.strip() and not line.startswith("#"):
            I, J, K, F, s2, v = line.split()
            rows.append((int(I), int(J), int(K), int(F), float(s2), float(v)))
    return rows


@pytest.mark.parametrize("name", ["table1_rfe.txt", "table2_rfe.txt"])
def test_printed_rfe_matches_noise_model(name):
    """The printed mean RFE equals sqrt(s2 / (E[x0^2] + s2)) * sqrt(1 - dof/numel) with
    E[x0^2] = F/27 + F(F-1)/64 for i.i.d. U[0,1] factors: this pins the reading of the
    experiment's generator (U[0,1] factors, noise variance s2) and of the RFE definition."""
    for I, J, K, F, s2, printed in _golden(name):
        ex2 = F / 27 + F * (F - 1) / 64
        cf = math.sqrt(s2 / (ex2 + s2)) * math.sqrt(1 - (I + J + K) * F / (I * J * K))
        assert abs(cf / printed - 1) < 0.01, (I, J, K, F, s2)


def test_generator_moments():
    """E[x0^2] of the generator and the noise variance agree with the model used above."""
    for F in (3, 30):
        ratios = []
        for seed in range(40):
            fs = synth.factors((30, 30, 30), F, seed)
            X0 = synth.tensor(fs, seed, dtype=np.float64)
            ratios.append(np.mean(X0 ** 2) / (F / 27 + F * (F - 1) / 64))
        assert abs(np.mean(ratios) - 1) < 0.03
    fs = synth.factors((40, 40, 40), 5, 1)
    N = synth.tensor(fs, 1, sigma2=1e-2, dtype=np.float64) - synth.tensor(fs, 1, dtype=np.float64)
    assert abs(np.var(N) / 1e-2 - 1) < 0.01


def test_snr_definition():
    fs = synth.factors((20, 30, 40), 4, 2)
    X0 = synth.tensor(fs, 2, dtype=np.float64)
    X = synth.tensor(fs, 2, snr_db=10.0, dtype=np.float64)
    snr = 10 * math.log10(np.sum(X0 ** 2) / np.sum((X - X0) ** 2))
    assert abs(snr - 10.0) < 0.05


def test_structured_generators():
    fs = synth.factors((300, 200, 100), 8, 0, structure="sparse")
    for F in fs:
        assert abs(np.mean(F == 0) - 0.5) < 0.05
        assert np.all(np.any(F > 0, axis=0))
    fs = synth.factors((4000, 3000), 6, 0, structure="collinear", congruence=0.9)
    for F in fs:
        Fn = F / np.linalg.norm(F, axis=0)
        C = Fn.T @ Fn
        off = C[~np.eye(6, dtype=bool)]
        assert abs(np.mean(off) - 0.9) < 0.01


def test_stored_trajectory_is_the_oracles():
    """The stored relative-error trajectory of the 400^3 rank-20 workload (written by
    oracle/trajectory.py; the benchmark takes the oracle's iteration count from it) starts
    with what the oracle computes now: its first two outer iterations, recomputed."""
    import json
    with open(os.path.join(GOLDEN, "trajectory_400x400x400_r20.json")) as f:
        h = json.load(f)
    spec = dict(synth.WORKLOADS[h["workload"]])
    dims, R = spec.pop("dims"), spec.pop("R")
    X, _, init = synth.workload(dims, R, seed=h["data_seed"], **spec)
    X64 = X.astype(np.float64)
    params = o.Params(inner_iters=5, kr_source="aux", rho_policy="trace")
    st = o.init_state([F.astype(np.float32).astype(np.float64) for F in init], params)
    for k in range(2):
        o.outer_iteration(X64, st, params)
        assert o.rfe(X64, st.aux) == pytest.approx(h["rfe"][k], rel=1e-10)
    # it ends at its lowest value (the converged error the fit target is measured against)
    r = np.asarray(h["rfe"])
    assert len(r) == 200 and r[-1] <= r.min() * (1 + 1e-9)


def test_paper_mode_start_has_zero_auxiliaries_and_duals():
    """Sec. VI-A starts ADMoM from random non-negative B0, C0 with At0 = Y0 = 0 (A0 unused).
    Pinned against the first update written out from that start: with zero auxiliary and dual
    the first primal update of eq. (ADMM_NTF_ALS_C) is A1 = M (G + rho0 I)^{-1}, M and G from
    B0, C0 only; then At1 = (A1)_+ and Y1 = rho0 (A1 - At1).  A start whose auxiliaries were
    seeded with the random values (or whose A0 entered the update) gives another A1."""
    rng = np.random.default_rng(21)
    dims, R = (6, 5, 4), 3
    X = rng.random(dims)
    init = [rng.random((d, R)) for d in dims]
    st = o.init_state(init, o.PAPER)
    for n in range(3):
        assert np.array_equal(st.aux[n], np.zeros((dims[n], R)))
        assert np.array_equal(st.dual[n], np.zeros((dims[n], R)))
    assert st.rho == [1.0, 1.0, 1.0]
    # the first factor's update by hand, from B0 and C0 (explicit unfolding X^(1)[i, j + J k])
    B, C = init[1], init[2]
    X1 = np.zeros((dims[0], dims[1] * dims[2]))
    KR = np.zeros((dims[1] * dims[2], R))
    for i in range(dims[0]):
        for j in range(dims[1]):
            for k in range(dims[2]):
                X1[i, j + dims[1] * k] = X[i, j, k]
    for j in range(dims[1]):
        for k in range(dims[2]):
            KR[j + dims[1] * k] = C[k] * B[j]
    M = X1 @ KR
    A1 = np.linalg.solve((KR.T @ KR + np.eye(R)).T, M.T).T
    o.outer_iteration(X, st, o.PAPER)
    assert np.allclose(st.primal[0], A1, rtol=1e-12, atol=1e-12)
    assert np.allclose(st.aux[0], np.maximum(A1, 0.0), rtol=1e-12, atol=1e-12)
    assert np.allclose(st.dual[0], A1 - np.maximum(A1, 0.0), rtol=1e-12, atol=1e-12)
    # a start with seeded auxiliaries is not that start
    seeded = o.State([F.copy() for F in init], [F.copy() for F in init],
                     [np.zeros_like(F) for F in init], [1.0] * 3)
    o.outer_iteration(X, seeded, o.PAPER)
    assert not np.allclose(seeded.primal[0], A1, rtol=1e-6, atol=1e-9)


def test_mttkrp_coo_brute_force_and_dense_equivalent():
    """The sparse-tensor MTTKRP (Sec. IV-A, n nonzeros): against index loops on a tiny tensor
    with a duplicated coordinate, and against the dense definition on the tensor the
    coordinates describe (3- and 4-way, every mode)."""
    rng = np.random.default_rng(4)
    idx = np.array([[0, 1, 2], [2, 0, 1], [1, 1, 0], [0, 1, 2], [2, 2, 2]])
    vals = np.array([1.5, -2.0, 0.5, 0.25, 3.0])
    fs = [rng.random((3, 2)) for _ in range(3)]
    for n in range(3):
        want = np.zeros((3, 2))
        for e in range(len(vals)):
            for r in range(2):
                p = vals[e]
                for m in range(3):
                    if m != n:
                        p *= fs[m][idx[e, m], r]
                want[idx[e, n], r] += p
        assert np.allclose(o.mttkrp_coo(idx, vals, fs, n), want, rtol=1e-14, atol=1e-14)
    for dims, R, nnz in (((7, 6, 5), 3, 40), ((4, 5, 3, 6), 2, 60)):
        idx, vals = synth.sparse_tensor(dims, nnz, seed=1, duplicates=True)
        fs = [rng.random((d, R)) for d in dims]
        X = o.coo_to_dense(idx, vals, dims)
        for n in range(len(dims)):
            assert np.allclose(o.mttkrp_coo(idx, vals, fs, n), o.mttkrp(X, fs, n), rtol=1e-12,
                               atol=1e-12)
