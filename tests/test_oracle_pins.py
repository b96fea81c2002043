"""Pins of the CPU oracle against facts that do not come from the oracle:
the paper's printed values, closed forms, the mathematics of each step, and
dense LAPACK on tiny inputs (called, never retyped)."""
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

import oracle
import workloads as W
from closed_forms import gradient_singular_values, laplacian5_eigs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- generators

def test_splitmix64_reference_output():
    # SplitMix64 (Steele, Lea, Flood 2014): first output from state 0 is
    # 0xE220A8397B1DCDAF; entry (row 0, vector 0) of a block with seed 0 is
    # 2 * (z >> 11) * 2^-53 - 1 of that output.
    z = 0xE220A8397B1DCDAF
    expect = 2.0 * (z >> 11) * 2.0 ** -53 - 1.0
    assert oracle.random_block(0, 1, 1)[0, 0] == expect
    blk = oracle.random_block(123, 1000, 3)
    assert blk.min() >= -1.0 and blk.max() < 1.0
    assert abs(blk.mean()) < 0.05


def test_generators_match_their_definitions():
    L = W.laplacian5(5).to_scipy().toarray()
    assert np.allclose(L, L.T)
    assert np.allclose(np.sort(np.linalg.eigvalsh(L)), laplacian5_eigs(5), rtol=1e-12)
    G = W.gradient(5).to_scipy()
    assert G.shape == (2 * 5 * 6, 25)
    assert np.allclose((G.T @ G).toarray(), L)
    Le = W.laplacian5(6, 0.3).to_scipy().toarray()
    assert np.allclose(np.sort(np.linalg.eigvalsh(Le)), laplacian5_eigs(6, 0.3), rtol=1e-12)


# ---------------------------------------------------------------- Kaczmarz

def test_kaczmarz_single_row_is_exact_projection():
    # after projecting row i, a_i . x = b_i exactly (up to rounding)
    A = sp.csr_matrix(np.array([[2.0, -1.0, 0.5]]))
    x = np.array([[1.0], [2.0], [3.0]])
    oracle.kaczmarz_sweep(A, x, np.array([[7.0]]))
    assert abs((A @ x)[0, 0] - 7.0) < 1e-14
    # the change is along a_i: x - x0 parallel to (2, -1, 0.5)
    d = x.ravel() - np.array([1.0, 2.0, 3.0])
    assert np.allclose(np.cross(d, [2.0, -1.0, 0.5]), 0.0)


def test_kaczmarz_is_sequential_not_simultaneous():
    # hand computation on rows r1 = (1, 1), r2 = (1, -1), b = (2, 0), x0 = 0:
    # row 1: d = 2/2 -> x = (1, 1); row 2: d = (0 - 0)/2 -> x = (1, 1).
    # A simultaneous (Cimmino-like) update would give (0.5, 0.5) + (0, 0).
    A = sp.csr_matrix(np.array([[1.0, 1.0], [1.0, -1.0]]))
    x = np.zeros((2, 1))
    oracle.kaczmarz_sweep(A, x, np.array([[2.0], [0.0]]))
    assert np.allclose(x.ravel(), [1.0, 1.0])
    # order matters: rows (1, 0), (1, 1) with b = (1, 3), x0 = 0
    # row 1 -> x = (1, 0); row 2: d = (3 - 1)/2 = 1 -> x = (2, 1)
    A = sp.csr_matrix(np.array([[1.0, 0.0], [1.0, 1.0]]))
    x = np.zeros((2, 1))
    oracle.kaczmarz_sweep(A, x, np.array([[1.0], [3.0]]))
    assert np.allclose(x.ravel(), [2.0, 1.0])


def test_kaczmarz_converges_to_solution_of_consistent_system():
    rng = np.random.default_rng(1)
    A = sp.csr_matrix(rng.standard_normal((12, 8)))
    xs = rng.standard_normal((8, 3))
    b = A @ xs
    x = np.zeros((8, 3))
    for _ in range(3000):
        oracle.kaczmarz_sweep(A, x, b)
    assert np.allclose(x, xs, atol=1e-9)


def test_kaczmarz_shifted_rows_match_explicit_matrix():
    # rows of A - s_j B built explicitly give the same sweep as the merged form
    rng = np.random.default_rng(2)
    A = sp.random(9, 9, density=0.4, random_state=3, format="csr") + sp.eye(9)
    B = sp.random(9, 9, density=0.3, random_state=4, format="csr") + sp.eye(9)
    s = np.array([0.3, -1.2])
    x1 = rng.standard_normal((9, 2))
    x2 = x1.copy()
    rhs = rng.standard_normal((9, 2))
    oracle.kaczmarz_sweep(oracle.samg._csr(A), x1, rhs, B=oracle.samg._csr(B), shift=s)
    for j in range(2):
        R = oracle.samg._csr(A - s[j] * B)
        xj = np.ascontiguousarray(x2[:, j:j + 1])
        oracle.kaczmarz_sweep(R, xj, rhs[:, j:j + 1])
        x2[:, j] = xj[:, 0]
    assert np.allclose(x1, x2, atol=1e-13)


# ---------------------------------------------------------------- coarsening

def test_rs_coarsening_1d_laplacian_hand_computed():
    # tridiag(-1, 2, -1), n = 7: lambda = (1,2,2,2,2,2,1); pick 1 (C), F = {0, 2},
    # lambda_3 -> 3; pick 3 (C), F = {4}, lambda_5 -> 3; pick 5 (C), F = {6}.
    n = 7
    T = sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1], format="csr")
    S = oracle.strength(T, 0.25)
    cf = oracle.rs_coarsen(S)
    assert list(np.flatnonzero(cf)) == [1, 3, 5]


def test_rs_coarsening_invariants_2d():
    A = W.laplacian5(20, 0.4).to_scipy()
    S = oracle.strength(A, 0.06)
    cf = oracle.rs_coarsen(S)
    S = S.tocsr()
    for i in range(A.shape[0]):
        js = S.indices[S.indptr[i]:S.indptr[i + 1]]
        if not cf[i]:
            assert cf[js].any(), "F point without strong C influence"
    # C points are an independent set w.r.t. strong influence of earlier picks
    assert 0.2 < cf.mean() < 0.8


def test_strength_definition():
    N = sp.csr_matrix(np.array([[4.0, -1.0, -0.1], [-1.0, 4.0, -2.0], [-0.1, -2.0, 4.0]]))
    S = oracle.strength(N, 0.2).toarray()
    # row 0: sum 5.1, threshold 1.02: only j=1 weak?  |n01| = 1 < 1.02 -> none
    assert (S[0] == 0).all()
    # row 1: sum 7, threshold 1.4: j = 2 strong (2), j = 0 weak (1)
    assert S[1, 2] == 2.0 and S[1, 0] == 0.0
    # row 2: sum 6.1, threshold 1.22: j = 1 strong
    assert S[2, 1] == 2.0 and S[2, 0] == 0.0


# ---------------------------------------------------------------- LS interpolation

def test_ls_fit_recovers_exact_interpolation():
    # vectors exactly in range(P*) with P* sparse on the C^i pattern are fitted exactly
    A = W.laplacian5(10).to_scipy()
    S = oracle.strength(A, 0.06)
    cf = oracle.rs_coarsen(S)
    nc = int(cf.sum())
    rng = np.random.default_rng(5)
    ptr, cols = oracle.interp_sets(S, cf, 6)
    alpha = np.cumsum(cf) - 1
    Pstar = sp.lil_matrix((A.shape[0], nc))
    for i in range(A.shape[0]):
        if cf[i]:
            Pstar[i, alpha[i]] = 1.0
        else:
            for j in cols[ptr[i]:ptr[i + 1]]:
                Pstar[i, alpha[j]] = rng.uniform(0.1, 1.0)
    Pstar = Pstar.tocsr()
    Y = np.ascontiguousarray(Pstar @ rng.standard_normal((nc, 12)))
    P = oracle.fit_interp(S, cf, Y, Y, rng.uniform(0.5, 2.0, 12))
    assert np.allclose(P.toarray(), Pstar.toarray(), atol=1e-10)


def test_ls_fit_weights_multiply_squared_residuals():
    # R13: for data no interpolation fits exactly, each F row's weights are
    # the minimiser of sum_k w_k (y_k(i) - sum_j p_j y_k(c_j))^2, i.e. the
    # ordinary least-squares solution of the rows scaled by sqrt(w_k)
    # (numpy's lstsq, called); weighting by w_k unsquared or by w_k^2 fails
    A = W.laplacian5(9).to_scipy()
    S = oracle.strength(A, 0.06)
    cf = oracle.rs_coarsen(S)
    rng = np.random.default_rng(13)
    nf = 10
    Y = rng.standard_normal((A.shape[0], nf))
    w = rng.uniform(0.1, 5.0, nf)
    P = oracle.fit_interp(S, cf, Y, Y, w).tocsr()
    ptr, cols = oracle.interp_sets(S, cf, nf - 1)
    alpha = np.cumsum(cf) - 1
    checked = 0
    for i in np.flatnonzero(cf == 0):
        C = cols[ptr[i]:ptr[i + 1]]
        if len(C) == 0:
            continue
        G = Y[C].T * np.sqrt(w)[:, None]           # nf x |C^i|
        p_ref = np.linalg.lstsq(G, Y[i] * np.sqrt(w), rcond=None)[0]
        row = dict(zip(P.indices[P.indptr[i]:P.indptr[i + 1]], P.data[P.indptr[i]:P.indptr[i + 1]]))
        got = np.array([row[alpha[j]] for j in C])
        assert np.allclose(got, p_ref, rtol=1e-9, atol=1e-12)
        checked += 1
    assert checked > 10


def test_interpolatory_sets_keep_the_strongest_up_to_the_cap():
    # R15: C^i holds the cap strongest strong C-point influences (ties to the
    # lowest index), hand-built strength row
    S = sp.csr_matrix(np.array([
        [0, 3, 1, 3, 2, 5, 0],
        [0, 0, 0, 0, 0, 0, 0],
        [0, 0, 0, 0, 0, 0, 0],
        [0, 0, 0, 0, 0, 0, 0],
        [0, 0, 0, 0, 0, 0, 0],
        [0, 0, 0, 0, 0, 0, 0],
        [0, 0, 0, 0, 0, 0, 0]], dtype=float))
    cf = np.array([0, 1, 1, 1, 1, 1, 0])
    ptr, cols = oracle.interp_sets(S, cf, 3)
    assert list(cols[ptr[0]:ptr[1]]) == [5, 1, 3]      # 5 (5), then the tie 3/3 -> 1, 3
    ptr, cols = oracle.interp_sets(S, cf, 10)
    assert sorted(cols[ptr[0]:ptr[1]]) == [1, 2, 3, 4, 5]


def test_minimal_test_vectors_have_unit_norm_after_relaxation():
    # R16: minimal kind, test vectors scaled to unit B (C) norm after each
    # block of mu_t relaxations, whatever their scale before
    A = W.gradient(10).to_scipy()
    m, n = A.shape
    L0 = oracle.Level(A, sp.identity(m, format="csr"), sp.identity(n, format="csr"))
    Ut = oracle.random_block(3, m, 4) * 7.0
    Vt = oracle.random_block(4, n, 4) * 0.2
    oracle.relax_test(L0, False, "minimal", Ut, Vt, 3, 0.7)
    assert np.allclose(np.linalg.norm(Ut, axis=0), 1.0, atol=1e-12)
    assert np.allclose(np.linalg.norm(Vt, axis=0), 1.0, atol=1e-12)


def test_block_order_v_then_u():
    # R1/R2: one minimal block Gauss-Seidel relaxation updates v from the rows
    # of A, then u from the rows of A^t.  A Kaczmarz sweep leaves its last
    # row satisfied exactly (P8), so afterwards the last row of
    # A^t u - s C v = tau holds with the final v; the reverse order would
    # leave the last row of A v - s B u = kappa exact instead.
    A = W.gradient(9).to_scipy()
    m, n = A.shape
    L0 = oracle.Level(A, sp.identity(m, format="csr"), sp.identity(n, format="csr"))
    rng = np.random.default_rng(21)
    sig = np.array([2.0, 3.5, 5.0])
    U, V = rng.standard_normal((m, 3)), rng.standard_normal((n, 3))
    K, T = rng.standard_normal((m, 3)), rng.standard_normal((n, 3))
    oracle.relax_boot(L0, False, "minimal", sig, U, V, K, T, 0.7)
    last_t = (A.T @ U - sig * V)[-1] - T[-1]
    last_k = (A @ V - sig * U)[-1] - K[-1]
    assert np.allclose(last_t, 0.0, atol=1e-12)
    assert np.abs(last_k).min() > 1e-6


def test_coarsest_rule():
    # R6: levels are added while max(m_l, n_l) > coarsest_max (and coarsening
    # still reduces); the coarsest has max(m_L, n_L) <= coarsest_max here
    A = W.gradient(24).to_scipy()
    H, s, U, V = oracle.setup(A, 4, "minimal", "svd", dict(W.GRAD_PARAMS, seed=2, n_mult=2,
                                                           coarsest_max=60))
    sizes = [max(L.A.shape) for L in H.levels]
    assert sizes[-1] <= 60 and all(x > 60 for x in sizes[:-1]), sizes


# ---------------------------------------------------------------- Galerkin

def test_galerkin_matches_dense_triple_product():
    rng = np.random.default_rng(6)
    A = sp.random(30, 20, density=0.2, random_state=7, format="csr")
    P = sp.random(30, 9, density=0.3, random_state=8, format="csr")
    Q = sp.random(20, 7, density=0.3, random_state=9, format="csr")
    L = oracle.Level(A, sp.identity(30, format="csr"), sp.identity(20, format="csr"))
    L.P, L.Q = P, Q
    Lc = oracle.galerkin(L, False)
    Ad, Pd, Qd = A.toarray(), P.toarray(), Q.toarray()
    assert np.allclose(Lc.A.toarray(), Pd.T @ Ad @ Qd)
    assert np.allclose(Lc.B.toarray(), Pd.T @ Pd)
    assert np.allclose(Lc.C.toarray(), Qd.T @ Qd)
    x = rng.standard_normal(7)
    assert np.allclose(Lc.A @ x, P.T @ (A @ (Q @ x)))


# ---------------------------------------------------------------- generalized SVD

def _spd(n, seed):
    r = np.random.default_rng(seed).standard_normal((n, n))
    return r @ r.T + n * np.eye(n)


@pytest.mark.parametrize("m,n", [(9, 6), (6, 9), (7, 7)])
def test_generalized_svd_theorem(m, n):
    rng = np.random.default_rng(m * 10 + n)
    A = rng.standard_normal((m, n))
    B, C = _spd(m, 1), _spd(n, 2)
    L = oracle.Level(sp.csr_matrix(A), sp.csr_matrix(B), sp.csr_matrix(C))
    X, Y = oracle.dense_XY(L, False)
    w = np.sort(sla.eigh(X, Y, eigvals_only=True))
    # change of variables D = B^-1/2 A C^-1/2 (proof of the existence theorem)
    Bh = sla.sqrtm(B).real
    Ch = sla.sqrtm(C).real
    D = np.linalg.solve(Bh, A) @ np.linalg.inv(Ch)
    s = np.linalg.svd(D, compute_uv=False)
    l = min(m, n)
    expect = np.sort(np.concatenate([s, -s, np.zeros(m + n - 2 * l)]))
    assert np.allclose(w, expect, atol=1e-10)
    for target in ("dominant", "minimal"):
        sig, U, V = oracle.coarsest_triplets(L, False, target, 3)
        ref = s[:3] if target == "dominant" else np.sort(s)[:3]
        assert np.allclose(sig, ref, rtol=1e-10)
        assert np.allclose(U.T @ B @ U, np.eye(3), atol=1e-10)
        assert np.allclose(V.T @ C @ V, np.eye(3), atol=1e-10)
        assert np.allclose(A @ V, B @ U * sig, atol=1e-9)
        assert np.allclose(A.T @ U, C @ V * sig, atol=1e-9)


def test_coarsest_pinv_drops_only_smallest_singular_value():
    # symmetric diagonal S = X - s Y with Y = I: pinv leaves out the entry of
    # smallest |d| and inverts the rest
    d = np.array([3.0, -0.01, 2.0, -5.0])
    X = np.diag(d + 0.5)
    Y = np.eye(4)
    K = np.arange(1.0, 5.0)[:, None]
    out, _ = oracle.coarsest_pinv_apply((X, Y), np.array([0.5]), K, None, True)
    expect = K[:, 0] / d
    expect[1] = 0.0
    assert np.allclose(out[:, 0], expect)
    # the two-value variant also leaves out the next smallest |d| (2.0)
    out, _ = oracle.coarsest_pinv_apply((X, Y), np.array([0.5]), K, None, True, drop=2)
    expect[2] = 0.0
    assert np.allclose(out[:, 0], expect)


# ---------------------------------------------------------------- Ritz

def test_ritz_exact_on_exact_subspaces():
    A = W.gradient(8).to_scipy()
    U, s, Vt = np.linalg.svd(A.toarray(), full_matrices=False)
    rng = np.random.default_rng(11)
    idx = np.argsort(s)[:5]
    R1 = rng.standard_normal((5, 5))
    R2 = rng.standard_normal((5, 5))
    sig, Uo, Vo = oracle.ritz(A, False, "minimal", U[:, idx] @ R1, Vt[idx].T @ R2)
    assert np.allclose(sig, np.sort(s)[:5], rtol=1e-12)
    assert np.allclose(A @ Vo, Uo * sig, atol=1e-10)
    idx = np.argsort(-s)[:4]
    sig, Uo, Vo = oracle.ritz(A, False, "dominant", U[:, idx] @ R1[:4, :4], Vt[idx].T)
    assert np.allclose(sig, np.sort(s)[::-1][:4], rtol=1e-12)


# ---------------------------------------------------------------- relaxation fixed points

def _exact_pairs(A, idx):
    # dense LAPACK SVD (called): exact singular triplets of a tiny operator
    U, s, Vt = np.linalg.svd(A.toarray(), full_matrices=False)
    return s[idx], U[:, idx].copy(), Vt[idx].T.copy()


def test_rayleigh_quotient_of_exact_triplets():
    # Eq. Rayleigh on exact pairs returns sigma_j; flipping v flips its sign
    A = W.gradient(7).to_scipy()
    m, n = A.shape
    L0 = oracle.Level(A, sp.identity(m, format="csr"), sp.identity(n, format="csr"))
    s, U, V = _exact_pairs(A, np.arange(4))
    assert np.allclose(oracle.rayleigh(L0, False, 3.0 * U, 0.5 * V), s, rtol=1e-12)
    assert np.allclose(oracle.rayleigh(L0, False, U, -V), -s, rtol=1e-12)


def test_minimal_block_gauss_seidel_fixes_exact_triplets():
    # A v = s u and A^t u = s v make every Kaczmarz row residual of
    # A v - s u = 0 and A^t u - s v = 0 vanish: the relaxation (Sec. 5.3,
    # kappa = tau = 0) leaves exact triplets unchanged, and moves a perturbed one
    A = W.gradient(7).to_scipy()
    m, n = A.shape
    L0 = oracle.Level(A, sp.identity(m, format="csr"), sp.identity(n, format="csr"))
    s, U, V = _exact_pairs(A, np.argsort(np.linalg.svd(A.toarray(), compute_uv=False))[:3])
    U0, V0 = U.copy(), V.copy()
    oracle.relax_boot(L0, False, "minimal", s, U, V, np.zeros_like(U), np.zeros_like(V), 0.7)
    assert np.abs(U - U0).max() < 1e-12 and np.abs(V - V0).max() < 1e-12
    oracle.relax_boot(L0, False, "minimal", -s, U, V, np.zeros_like(U), np.zeros_like(V), 0.7)
    assert np.abs(V - V0).max() > 1e-3  # the sign of the shift matters


def test_dominant_jacobi_fixes_exact_triplets():
    # u <- u - w D^-1 (u - (A v - kappa) / s) vanishes for A v = s u (Sec. 3.5)
    A = W.gradient(7).to_scipy()
    m, n = A.shape
    L0 = oracle.Level(A, sp.identity(m, format="csr"), sp.identity(n, format="csr"))
    s, U, V = _exact_pairs(A, np.arange(3))
    U0, V0 = U.copy(), V.copy()
    oracle.relax_boot(L0, False, "dominant", s, U, V, np.zeros_like(U), np.zeros_like(V), 0.7)
    assert np.abs(U - U0).max() < 1e-12 and np.abs(V - V0).max() < 1e-12
    oracle.relax_boot(L0, False, "dominant", 1.1 * s, U, V, np.zeros_like(U), np.zeros_like(V), 0.7)
    assert np.abs(U - U0).max() > 1e-3


def test_spd_shifted_kaczmarz_fixes_exact_eigenpairs():
    # rows of A - lam B with B = I: (A - lam I) x = 0 for an exact eigenpair
    A = W.laplacian5(6).to_scipy()
    n = A.shape[0]
    L0 = oracle.Level(A, sp.identity(n, format="csr"), None)
    lam, X = np.linalg.eigh(A.toarray())
    lam, X = lam[:3], X[:, :3].copy()
    X0 = X.copy()
    oracle.relax_boot(L0, True, "minimal", lam, X, None, np.zeros_like(X), None, 0.7)
    assert np.abs(X - X0).max() < 1e-12
    assert np.allclose(lam, laplacian5_eigs(6)[:3], rtol=1e-12)


# ---------------------------------------------------------------- setup readings

def test_coarsest_triplets_are_normalized_generalized_triplets():
    # Thm genSVD: A v = s B u, A^t u = s C v with u^t B u = v^t C v = 1, for
    # random SPD B, C; the SVD of B^-1/2 A C^-1/2 (LAPACK, called) gives s
    rng = np.random.default_rng(17)
    m, n = 9, 6
    A = rng.standard_normal((m, n))
    Rb = rng.standard_normal((m, m))
    Rc = rng.standard_normal((n, n))
    B = Rb @ Rb.T + m * np.eye(m)
    C = Rc @ Rc.T + n * np.eye(n)
    L = oracle.Level(sp.csr_matrix(A), sp.csr_matrix(B), sp.csr_matrix(C))
    for target in ("dominant", "minimal"):
        s, U, V = oracle.coarsest_triplets(L, False, target, 3)
        assert np.allclose(A @ V, B @ U * s, atol=1e-10)
        assert np.allclose(A.T @ U, C @ V * s, atol=1e-10)
        assert np.allclose(np.einsum("ij,ij->j", U, B @ U), 1.0, atol=1e-10)
        assert np.allclose(np.einsum("ij,ij->j", V, C @ V), 1.0, atol=1e-10)
        Bh = sla.sqrtm(np.linalg.inv(B)).real
        Ch = sla.sqrtm(np.linalg.inv(C)).real
        ref = np.sort(np.linalg.svd(Bh @ A @ Ch, compute_uv=False))
        want = ref[::-1][:3] if target == "dominant" else ref[:3]
        assert np.allclose(s, want, rtol=1e-10)


def test_r14_jacobi_weight_never_amplifies():
    # R14: the weight 2 omega / g (g the Gershgorin bound of D^-1 N) keeps
    # every eigenvalue of I - w D^-1 N in [-1, 1] for omega <= 1, so repeated
    # steps never grow the D-norm; the plain weight omega = 0.7 on A A^t of the
    # gradient (g = 4) amplifies its high modes
    A = W.gradient(6).to_scipy()
    m, n = A.shape
    L = oracle.Level(A, sp.identity(m, format="csr"), sp.identity(n, format="csr"))
    N = (A @ A.T).toarray()
    d = np.diag(N)
    rng = np.random.default_rng(3)
    Y0 = rng.standard_normal((m, 4))
    Y = Y0.copy()
    dnorm = lambda Z: np.sqrt(np.einsum("ij,i,ij->", Z, d, Z))
    for _ in range(30):
        Y = oracle.samg._jacobi_on_N(L, False, "u", Y, 0.7)
    assert dnorm(Y) <= dnorm(Y0) * (1 + 1e-12)
    Z = Y0.copy()
    for _ in range(30):
        Z = Z - 0.7 * (N @ Z) / d[:, None]
    assert dnorm(Z) > 10 * dnorm(Y0)


def test_r21_induced_interpolation_structure():
    # minimal SVD kind with m >= n: P_0 = A Q_0 and P_l = Q_l below, so that
    # A_1 = P_0^t A Q_0 = Q_0^t A^t A Q_0 equals B_1 = P_0^t P_0 (symmetric)
    A = W.gradient(12).to_scipy()
    H, s, U, V = oracle.setup(A, 4, "minimal", "svd",
                              dict(W.GRAD_PARAMS, n_mult=1, seed=7, coarsest_max=40))
    assert len(H.levels) >= 3
    L0 = H.levels[0]
    assert abs(L0.P - A @ L0.Q).max() < 1e-12
    L1 = H.levels[1]
    assert abs(L1.A - L1.B).max() < 1e-9 * abs(L1.A).max()
    assert abs(L1.A - L1.A.T).max() < 1e-9 * abs(L1.A).max()
    for L in H.levels[1:-1]:
        assert abs(L.P - L.Q).max() == 0


# ---------------------------------------------------------------- additive cycle

def test_additive_equals_multiplicative_when_x_in_range_of_P():
    # Eq. e: with x in range(P) and an exact coarse solve, one additive
    # two-level step (no relaxation) returns the exact eigenvector direction.
    A = W.laplacian5(8).to_scipy()
    w, X = np.linalg.eigh(A.toarray())
    x = X[:, 0]
    rng = np.random.default_rng(3)
    Pd = np.column_stack([x, rng.standard_normal((64, 5))])
    L0 = oracle.Level(A, sp.identity(64, format="csr"))
    L0.P = sp.csr_matrix(Pd)
    H = oracle.Hierarchy("spd", "minimal", [L0, oracle.galerkin(L0, True)],
                         dict(oracle.DEFAULTS, mu_b=0))
    u0 = np.ascontiguousarray((Pd @ rng.standard_normal(6))[:, None])
    U = u0.copy()
    oracle.vcycle(H, 0, np.array([w[0]]), U, None, np.zeros_like(U), None)
    u = U[:, 0] / np.linalg.norm(U[:, 0])
    assert abs(abs(u @ x) - 1.0) < 1e-10


def test_defect_correction_form_equals_paper_form():
    # R12: relaxation is affine in (iterate, rhs); a V-cycle on the error
    # equation with zero initial guess, added to the iterate, equals the
    # V-cycle on the iterate itself (FP64, to rounding).
    A = W.gradient(12).to_scipy()
    H, s, U, V = oracle.setup(A, 4, "minimal", "svd",
                              dict(W.GRAD_PARAMS, n_mult=2, seed=5))
    U1, V1 = U.copy(), V.copy()
    oracle.vcycle(H, 0, s, U1, V1, np.zeros_like(U), np.zeros_like(V))
    r, t = oracle.level_residual(H.levels[0], False, s, U, V, np.zeros_like(U), np.zeros_like(V))
    Eu, Ev = np.zeros_like(U), np.zeros_like(V)
    oracle.vcycle(H, 0, s, Eu, Ev, r, t)
    assert np.allclose(U + Eu, U1, atol=1e-11 * np.abs(U1).max())
    assert np.allclose(V + Ev, V1, atol=1e-11 * np.abs(V1).max())


# ---------------------------------------------------------------- whole method

def _table_fd():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "table_values_fd.txt"))
            if l.strip() and not l.startswith("#")]
    return np.array([float(r[1]) for r in rows]), np.array([float(r[2]) for r in rows])


def test_fd_minimal_matches_paper_table_values():
    # Sec. 6.2 setting: FD 32x32, 8 minimal eigenpairs, theta = 0.06, n_t = 6,
    # mu_t = 8, mu_b = 4, 15 multiplicative cycles, then additive cycles.
    lge, sm = _table_fd()
    A = W.laplacian5(32).to_scipy() / 33.0 ** 2       # unscaled 4, -1 stencil
    H, s, U, V = oracle.setup(A, 8, "minimal", "spd", dict(W.FD_PARAMS, seed=W.problem_seed(1)))
    assert len(H.levels) == 5                           # "Five levels are used"
    # Sec. 6.2 reports a coarsest level of 64 points; the C/F splitting's
    # tie-breaking is a reading (R9), so the size is pinned to within 10%
    assert abs(H.levels[-1].A.shape[0] - 64) <= 6.4, H.levels[-1].A.shape
    s, U, V, hist = oracle.solve(H, s, U, V, tol=1e-12, max_outer=40)
    assert hist[-1].max() <= 1e-12
    assert len(hist) - 1 <= 30                          # machine accuracy in <= 30 cycles
    assert np.allclose(s, sm, rtol=5e-7)
    assert np.allclose(s, laplacian5_eigs(32)[:8] / 33.0 ** 2, rtol=1e-12)


def test_fd_dominant_matches_paper_table_values():
    # Sec. 6.2, dominant case: same setting, the 8 largest eigenpairs; the
    # paper reports four levels and the Table's "FD lge" column, printed to
    # 7 decimals (half a unit of the last place is 5e-8).
    lge, sm = _table_fd()
    A = W.laplacian5(32).to_scipy() / 33.0 ** 2
    H, s, U, V = oracle.setup(A, 8, "dominant", "spd", dict(W.FD_PARAMS, seed=W.problem_seed(1)))
    assert len(H.levels) == 4                           # "Four levels are used"
    # a coarsest level of 52 points in the paper (within 10%, as above)
    assert abs(H.levels[-1].A.shape[0] - 52) <= 5.2, H.levels[-1].A.shape
    s, U, V, hist = oracle.solve(H, s, U, V, tol=1e-12, max_outer=150)
    assert hist[-1].max() <= 1e-12
    # the paper notes that the additive phase converges more slowly here
    # than in the minimal case (at most 30 cycles there)
    assert len(hist) - 1 > 30
    assert np.all(np.abs(s - lge) <= 5.01e-8)
    assert np.allclose(s, laplacian5_eigs(32)[::-1][:8] / 33.0 ** 2, rtol=1e-12)
    assert np.allclose(A @ U, U * s, atol=1e-11 * s.max())


def test_laplacian_workload_minimal_closed_form():
    wl = W.workload(1)
    A = wl.build().to_scipy()
    H, s, U, V = oracle.setup(A, wl.nb, wl.target, wl.kind,
                              dict(wl.params, seed=W.problem_seed(1)))
    s, U, V, hist = oracle.solve(H, s, U, V, tol=1e-10, max_outer=40)
    assert np.allclose(s, laplacian5_eigs(32)[:4], rtol=1e-10)
    assert np.allclose(U.T @ U, np.eye(4), atol=1e-10)


def test_gradient_minimal_closed_form_and_lapack():
    N = 24
    A = W.gradient(N).to_scipy()
    H, s, U, V = oracle.setup(A, 8, "minimal", "svd", dict(W.GRAD_PARAMS, seed=W.problem_seed(2)))
    s, U, V, hist = oracle.solve(H, s, U, V, tol=1e-10, max_outer=60)
    assert hist[-1].max() <= 1e-10
    exact = gradient_singular_values(N)[:8]
    assert np.allclose(s, exact, rtol=1e-10)
    lap = np.sort(np.linalg.svd(A.toarray(), compute_uv=False))[:8]
    assert np.allclose(s, lap, rtol=1e-10)
    assert np.allclose(A @ V, U * s, atol=1e-8 * s.max())
    assert np.allclose(A.T @ U, V * s, atol=1e-8 * s.max())
    assert np.allclose(U.T @ U, np.eye(8), atol=1e-10)
    assert np.allclose(V.T @ V, np.eye(8), atol=1e-10)


def test_dominant_svd_lapack():
    A = W.laplacian5(16).to_scipy()
    H, s, U, V = oracle.setup(A, 4, "dominant", "svd",
                              dict(W.FD_PARAMS, seed=9, coarsest_max=40))
    assert len(H.levels) >= 3
    s, U, V, hist = oracle.solve(H, s, U, V, tol=1e-9, max_outer=150)
    assert hist[-1].max() <= 1e-9
    ref = np.sort(np.linalg.svd(A.toarray(), compute_uv=False))[::-1][:4]
    assert np.allclose(s, ref, rtol=1e-10)


def test_residual_norms_hand_built_triplets():
    """R11 pinned on triplets whose residuals are worked out by hand.

    A = [[3, 0], [0, 1], [0, 0]], sigma = 3, u = e1, v = (e1 + e2)/sqrt(2):
      A v - sigma u   = (3/r - 3, 1/r, 0)      with r = sqrt(2)
      A^t u - sigma v = (3 - 3/r, -3/r)
    so |A v - s u|^2 + |A^t u - s v|^2 = 2 (3 - 3/r)^2 + 1/2 + 9/2 and
    rho = sqrt(2 (3 - 3/r)^2 + 5) / 3.  Dropping either term, using the
    wrong sign of sigma, dividing by sigma^2 or skipping the unit scaling of
    u and v changes the value.  The SPD form: A = diag(2, 5), lam = 2,
    x = (1, 1)/sqrt(2): A x - lam x = (0, 3/r), rho = (3/r)/2."""
    r = np.sqrt(2.0)
    A = sp.csr_matrix(np.array([[3.0, 0.0], [0.0, 1.0], [0.0, 0.0]]))
    U = np.array([[1.0], [0.0], [0.0]])
    V = np.array([[1.0], [1.0]]) / r
    want = np.sqrt(2.0 * (3.0 - 3.0 / r) ** 2 + 5.0) / 3.0
    got = oracle.residual_norms(A, False, np.array([3.0]), U, V)
    assert abs(got[0] - want) < 1e-15 * want
    # the scale of u and v does not matter (R11 takes unit vectors)
    got2 = oracle.residual_norms(A, False, np.array([3.0]), 7.0 * U, 0.25 * V)
    assert abs(got2[0] - want) < 1e-15 * want
    # (3, e1, e1) is an exact triplet: both terms vanish
    got3 = oracle.residual_norms(A, False, np.array([3.0]), U, np.array([[1.0], [0.0]]))
    assert got3[0] < 1e-16
    # one side nonzero: u = e2, v = e2, sigma = 1 is exact; sigma = 2 gives
    # A v - s u = (0, -1, 0), A^t u - s v = (0, -1): rho = sqrt(2)/2
    e2u = np.array([[0.0], [1.0], [0.0]])
    e2v = np.array([[0.0], [1.0]])
    assert oracle.residual_norms(A, False, np.array([1.0]), e2u, e2v)[0] < 1e-16
    assert abs(oracle.residual_norms(A, False, np.array([2.0]), e2u, e2v)[0] - r / 2.0) < 1e-15
    # u with a component in null(A^t) = span(e3): A^t u is unchanged but
    # A v - s u gains -s e3/|u|.  u = (e2 + e3)/r, v = e2, s = 1:
    # A v - s u = (0, 1 - 1/r, -1/r), A^t u - s v = (0, 1/r - 1)
    u = np.array([[0.0], [1.0], [1.0]]) / r
    want4 = np.sqrt(2.0 * (1.0 - 1.0 / r) ** 2 + 0.5)
    assert abs(oracle.residual_norms(A, False, np.array([1.0]), u, e2v)[0] - want4) < 1e-15
    # SPD form
    D = sp.csr_matrix(np.diag([2.0, 5.0]))
    x = np.array([[1.0], [1.0]]) / r
    assert abs(oracle.residual_norms(D, True, np.array([2.0]), x, None)[0] - (3.0 / r) / 2.0) < 1e-15
    # several columns at once are independent
    got5 = oracle.residual_norms(A, False, np.array([3.0, 2.0]), np.hstack([U, e2u]),
                                 np.hstack([V, e2v]))
    assert abs(got5[0] - want) < 1e-15 * want and abs(got5[1] - r / 2.0) < 1e-15


def test_coarse_geneig_variant_pins():
    """The generalized-eigen form of the coarsest solve (a variant of R7).

    * With Y = I the generalized eigenpairs are the eigenpairs of the
      symmetric X, the singular values of X - s I are |lam_k - s|, and the
      mode nearest s is the smallest singular value: the variant equals the
      paper's SVD pseudo-inverse.
    * For any SPD Y: X - s Y = Y W (Lam - s) W^t Y and W W^t = Y^-1, so the
      variant's z satisfies (X - s Y) z = r - Y w* (w*^t r), w* the dropped
      generalized eigenvector; and w*^t Y z = 0."""
    rng = np.random.default_rng(31)
    n = 9
    X = rng.standard_normal((n, n))
    X = X + X.T
    I = np.eye(n)
    K = rng.standard_normal((n, 3))
    s = np.array([0.3, -1.1, 2.0])
    zs, _ = oracle.coarsest_pinv_apply((X, I), s, K, None, True)
    zg, _ = oracle.coarsest_pinv_apply((X, I), s, K, None, True, form="geneig")
    assert np.abs(zs - zg).max() < 1e-11 * np.abs(zs).max()
    G = rng.standard_normal((n, n))
    Y = G @ G.T + n * I
    lam, Wm = oracle.coarse_geneig((X, Y))
    zg, _ = oracle.coarsest_pinv_apply((X, Y), s, K, None, True, form="geneig")
    for j in range(3):
        k = int(np.argmin(np.abs(lam - s[j])))
        w = Wm[:, k]
        lhs = (X - s[j] * Y) @ zg[:, j]
        rhs = K[:, j] - Y @ w * (w @ K[:, j])
        assert np.abs(lhs - rhs).max() < 1e-10 * np.abs(K).max()
        assert abs(w @ Y @ zg[:, j]) < 1e-10 * np.abs(zg).max()
    # the SVD kind splits [kappa; tau] into the two blocks in order
    m1 = 4
    zu, zv = oracle.coarsest_pinv_apply((X, Y), s, K[:m1], K[m1:], False, form="geneig")
    full, _ = oracle.coarsest_pinv_apply((X, Y), s, K, None, True, form="geneig")
    assert np.array_equal(np.vstack([zu, zv]), full)


def test_paper_row_form_collapses_onto_null_At_on_the_gradient():
    """Why R21 replaces the paper's row coarsening for the minimal SVD kind.

    With the rows coarsened on A A^t and a two-sided Ritz step (Secs. 3.7,
    4.3), the setup's left boot vectors of the 16 x 16 gradient end up almost
    entirely in null(A^t) -- the |m - n| zero modes of Thm genSVD -- and the
    Ritz values fall far below the true smallest singular value.  R21 (rows
    from A, left basis A V_b) keeps u in range(A) and finds the closed-form
    values."""
    A = W.gradient(16).to_scipy()
    exact = gradient_singular_values(16)[:8]
    Q, _ = np.linalg.qr(A.toarray())          # orthonormal basis of range(A)
    prm = dict(W.GRAD_PARAMS, seed=14, coarsest_max=40, n_mult=5)
    H, s, U, V = oracle.setup(A, 8, "minimal", "svd", dict(prm, row_form="paper"))
    Un = U / np.linalg.norm(U, axis=0)
    outside = np.linalg.norm(Un - Q @ (Q.T @ Un), axis=0)
    assert outside.min() > 0.99, outside
    assert s.max() < 0.2 * exact[0], s
    H, s, U, V = oracle.setup(A, 8, "minimal", "svd", dict(prm, row_form="induced"))
    Un = U / np.linalg.norm(U, axis=0)
    assert np.linalg.norm(Un - Q @ (Q.T @ Un), axis=0).max() < 1e-10
    s, U, V, hist = oracle.solve(H, s, U, V, tol=1e-10, max_outer=60)
    assert hist[-1].max() <= 1e-10
    assert np.abs(s - exact).max() < 1e-10 * exact.max()


def test_coloured_order_pins():
    """The coloured-order variant of the sweep (not the paper's order).

    * The greedy colouring is proper (rows of one colour share no column)
      and greedy: a row of colour c > 0 has, for every c' < c, an earlier
      row of colour c' sharing a column with it.
    * On the N x N gradient it is worked out by hand: the x-edge rows
      alternate colours 0, 1 along a grid row; a y-edge row meets up to two
      x-edges at each end, which hold both 0 and 1, so y-edges take 2 and 3:
      4 colours for the rows of A.  The rows of A^t (nodes) conflict when
      adjacent, and the natural order gives the checkerboard: 2 colours.
    * A coloured sweep is the natural-order sweep of the rows permuted by
      colour, and reordering rows inside a colour does not change it (they
      commute); after it the rows of the last colour hold exactly."""
    A = W.gradient(12).to_scipy()
    for R, want in ((A, 4), (sp.csr_matrix(A.T), 2)):
        col = oracle.row_colours(R)
        assert col.max() + 1 == want
        S = (abs(R) @ abs(R).T).tocsr()       # rows sharing a column
        for i in range(R.shape[0]):
            nbr = S.indices[S.indptr[i]:S.indptr[i + 1]]
            nbr = nbr[nbr != i]
            assert not np.any(col[nbr] == col[i])
            earlier = set(col[nbr[nbr < i]].tolist())
            assert all(c in earlier for c in range(col[i]))
    rng = np.random.default_rng(3)
    R = sp.random(60, 40, density=0.08, random_state=4, format="csr") + sp.eye(60, 40, format="csr")
    R = oracle.samg._csr(R)
    X0 = rng.standard_normal((40, 3))
    rhs = rng.standard_normal((60, 3))
    col = oracle.row_colours(R)
    order = np.argsort(col, kind="stable")
    X1 = X0.copy()
    oracle.kaczmarz_sweep_coloured(R, X1, rhs)
    # plain projections in the permuted order
    X2 = X0.copy()
    D = R.toarray()
    for i in order:
        a = D[i]
        if a @ a > 0:                        # an empty row projects nothing
            X2 += np.outer(a, (rhs[i] - a @ X2) / (a @ a))
    assert np.abs(X1 - X2).max() < 1e-12
    # rows shuffled inside each colour
    shuf = np.concatenate([rng.permutation(np.flatnonzero(col == c)) for c in range(col.max() + 1)])
    X3 = X0.copy()
    oracle.kaczmarz_sweep_coloured(R, X3, rhs, order=shuf)
    assert np.abs(X1 - X3).max() < 1e-12
    last = np.flatnonzero((col == col.max()) & (np.abs(D).sum(axis=1) > 0))
    assert last.size and np.abs(D[last] @ X1 - rhs[last]).max() < 1e-12


def test_square_forms_keep_square_levels_and_reach_lapack():
    """R23 (Sec. 5.1): with the C/F splitting and sparsity patterns of P and
    Q taken from A, every level of a square nonsymmetric operator stays
    square; with P = Q shared, B_c = C_c on every level.  The converged
    triplets equal a dense LAPACK SVD (called) of the 20 x 20 upwind
    convection-diffusion operator: its 4 largest (from A and shared) and its
    4 smallest (shared) singular values."""
    A = W.convdiff5(20, 8.0).to_scipy()
    assert abs(A - A.T).max() > 0
    sv = np.sort(np.linalg.svd(A.toarray(), compute_uv=False))
    cases = [("dominant", "from_A", W.FD_PARAMS), ("dominant", "shared", W.FD_PARAMS),
             ("minimal", "shared", W.GRAD_PARAMS)]
    for target, form, base in cases:
        prm = dict(base, seed=W.problem_seed(2), coarsest_max=40, n_mult=10, square_form=form)
        H, s, U, V = oracle.setup(A, 4, target, "svd", prm)
        for L in H.levels:
            assert L.A.shape[0] == L.A.shape[1]
        if form == "shared":
            for l, L in enumerate(H.levels[:-1]):
                assert L.Q is L.P
                if l > 0:
                    assert abs(L.B - L.C).max() == 0
        s, U, V, hist = oracle.solve(H, s, U, V, tol=1e-10, max_outer=120)
        ref = sv[::-1][:4] if target == "dominant" else sv[:4]
        assert hist[-1].max() <= 1e-10, (target, form, hist[-1])
        assert np.allclose(s, ref, rtol=1e-12), (target, form, s, ref)
        assert np.allclose(A @ V, U * s, atol=1e-9 * sv[-1])
