"""GPU path vs the FP64 CPU oracle, through the C ABI (float64, float32 and
bfloat16-storage arithmetic).

Each step of the additive cycle (Sec. 4) -- Galerkin operators, block
Gauss-Seidel relaxation (Kaczmarz or Jacobi blocks), residual + restriction,
interpolation + correction, coarsest pseudo-inverse solve, one V-cycle, the
Ritz step -- runs on the GPU on the oracle's own hierarchy and the same
seeded inputs, and is compared element by element with the oracle.

Tolerances: float64 steps agree to 1e-10 relative to the largest entry
(only the rounding of fused multiply-adds and of summation order differs);
float32 steps to 2e-4 (a few float32 ulps amplified by a sweep); converged
singular values to 1e-10 relative, residuals below the requested tolerance.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

samg = pytest.importorskip("paper_1102_0919_gb300")

TOL64 = 1e-10
TOL32 = 2e-4
# bfloat16 vector storage: unit roundoff u = 2^-8 = 3.9e-3 per stored value; a
# relaxation, transfer or V-cycle step stores an entry up to about 8 times
# (every row update that touches it, then the output), so its error relative
# to the largest entry stays within 8u = 3.1e-2
TOLB16 = 3.2e-2


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _case(name):
    if name == "spd_min":
        A = W.laplacian5(20, 0.37).to_scipy()
        prm = dict(W.FD_PARAMS, seed=11, coarsest_max=40)
        return A, 4, "minimal", "spd", prm
    if name == "svd_min":
        A = W.gradient(20).to_scipy()
        prm = dict(W.GRAD_PARAMS, seed=12, coarsest_max=40)
        return A, 8, "minimal", "svd", prm
    if name == "svd_min_paper":
        # the paper's own form of the minimal SVD kind (rows coarsened on
        # A A^t, two-sided Ritz step), step by step against the oracle's
        A = W.gradient(20).to_scipy()
        prm = dict(W.GRAD_PARAMS, seed=14, coarsest_max=40, row_form="paper")
        return A, 8, "minimal", "svd", prm
    if name == "svd_dom":
        A = W.laplacian5(16).to_scipy()
        prm = dict(W.FD_PARAMS, seed=13, coarsest_max=40)
        return A, 4, "dominant", "svd", prm
    raise ValueError(name)


CASES = ["spd_min", "svd_min", "svd_min_paper", "svd_dom"]


@pytest.fixture(scope="module", params=CASES)
def case(request):
    A, nb, target, kind, prm = _case(request.param)
    H, s, U, V = oracle.setup(A, nb, target, kind, prm)
    Ps = [L.P for L in H.levels[:-1]]
    Qs = None if kind == "spd" else [L.Q for L in H.levels[:-1]]
    g = samg.Solver.from_hierarchy(A, Ps, Qs, nb, s, U, V, target, kind, prec="fp64", **prm)
    yield dict(name=request.param, A=A, nb=nb, H=H, s=s, U=U, V=V, g=g, kind=kind, prm=prm)
    g.close()


def _vecs(c, l, seed):
    rng = np.random.default_rng(seed)
    L = c["H"].levels[l]
    m, n = L.A.shape
    spd = c["kind"] == "spd"
    U = rng.standard_normal((n if spd else m, c["nb"]))
    V = None if spd else rng.standard_normal((n, c["nb"]))
    K = rng.standard_normal(U.shape)
    T = None if spd else rng.standard_normal(V.shape)
    sig = c["s"] * (1.0 + 0.01 * rng.standard_normal(c["nb"]))
    return sig, U, V, K, T


def test_galerkin_operators(case):
    H, g = case["H"], case["g"]
    assert len(g.levels()) == len(H.levels)
    for l, L in enumerate(H.levels):
        mats = [("A", L.A)] + ([("B", L.B)] if l > 0 else [])
        if case["kind"] != "spd" and l > 0:
            mats.append(("C", L.C))
        for which, ref in mats:
            rp, ci, v, shape = g.level_matrix(l, which)
            got = sp.csr_matrix((v, ci, rp), shape=shape)
            assert got.shape == ref.shape
            d = abs(got - ref).max()
            assert d <= TOL64 * abs(ref).max(), (l, which, d)


@pytest.mark.parametrize("prec,tol", [("fp64", TOL64), ("fp32", TOL32), ("bf16", TOLB16)])
def test_relaxation_each_level(case, prec, tol):
    H, g = case["H"], case["g"]
    g.set_precision(prec)
    spd = case["kind"] == "spd"
    for l in range(len(H.levels) - 1):
        sig, U, V, K, T = _vecs(case, l, 100 + l)
        Ug, Vg = g.relax(l, sig, U, V, K, T, count=2)
        Ur, Vr = U.copy(), None if spd else V.copy()
        for _ in range(2):
            oracle.relax_boot(H.levels[l], spd, H.target, sig, Ur, Vr, K, T, H.params["omega_J"])
        assert rel(Ug, Ur) < tol, (l, rel(Ug, Ur))
        if not spd:
            assert rel(Vg, Vr) < tol, (l, rel(Vg, Vr))
    g.set_precision("fp64")


@pytest.mark.parametrize("band_rows,float_windows", [(1, False), (2, True), (8, False), (64, True)])
def test_relaxation_under_other_sweep_bandings(case, band_rows, float_windows):
    """The sweep programs' banding (samg_set_sweep_banding: rows per level a
    band grows to, float32-only windows) and the claim order change the
    parallel schedule only: every level's smoothing phase still equals the
    oracle's sequential block Gauss-Seidel relaxations, in float64 and
    float32."""
    H, g = case["H"], case["g"]
    spd = case["kind"] == "spd"
    try:
        g.set_sweep_banding(band_rows, float_windows)
        for prec, tol in (("fp64", TOL64), ("fp32", TOL32)):
            g.set_precision(prec)
            for l in range(len(H.levels) - 1):
                sig, U, V, K, T = _vecs(case, l, 170 + l)
                Ug, Vg = g.relax(l, sig, U, V, K, T, count=3)
                Ur, Vr = U.copy(), None if spd else V.copy()
                for _ in range(3):
                    oracle.relax_boot(H.levels[l], spd, H.target, sig, Ur, Vr, K, T,
                                      H.params["omega_J"])
                assert rel(Ug, Ur) < tol, (prec, l, rel(Ug, Ur))
                if not spd:
                    assert rel(Vg, Vr) < tol, (prec, l, rel(Vg, Vr))
    finally:
        g.set_sweep_banding()
        g.set_precision("fp64")


@pytest.mark.parametrize("prec,tol", [("fp64", TOL64), ("fp32", TOL32), ("bf16", TOLB16)])
def test_relaxation_coloured_each_level(case, prec, tol):
    """relax_order = 1 (the coloured variant): every level's smoothing phase
    against the oracle's coloured sweeps (the same greedy colouring)."""
    H, g = case["H"], case["g"]
    if H.target != "minimal":
        pytest.skip("the coloured order applies to the Kaczmarz (minimal) relaxation")
    g.set_precision(prec)
    g.set_relax_order("coloured")
    spd = case["kind"] == "spd"
    try:
        for l in range(len(H.levels) - 1):
            sig, U, V, K, T = _vecs(case, l, 150 + l)
            Ug, Vg = g.relax(l, sig, U, V, K, T, count=3)
            Ur, Vr = U.copy(), None if spd else V.copy()
            for _ in range(3):
                oracle.relax_boot(H.levels[l], spd, H.target, sig, Ur, Vr, K, T,
                                  H.params["omega_J"], "coloured")
            assert rel(Ug, Ur) < tol, (l, rel(Ug, Ur))
            if not spd:
                assert rel(Vg, Vr) < tol, (l, rel(Vg, Vr))
    finally:
        g.set_relax_order("natural")
        g.set_precision("fp64")


@pytest.mark.parametrize("prec,tol", [("fp64", TOL64), ("fp32", TOL32), ("bf16", TOLB16)])
def test_residual_restrict_and_interpolate(case, prec, tol):
    H, g = case["H"], case["g"]
    g.set_precision(prec)
    spd = case["kind"] == "spd"
    for l in range(len(H.levels) - 1):
        L, Lc = H.levels[l], H.levels[l + 1]
        sig, U, V, K, T = _vecs(case, l, 200 + l)
        mc, nc = Lc.A.shape
        Kc, Tc = g.residual_restrict(l, sig, U, V, K, T, nc if spd else mc, nc)
        r, s = oracle.level_residual(L, spd, sig, U, V, K, T)
        assert rel(Kc, L.P.T @ r) < tol
        if not spd:
            assert rel(Tc, L.Q.T @ s) < tol
        rng = np.random.default_rng(300 + l)
        Uc = rng.standard_normal(Kc.shape)
        Vc = None if spd else rng.standard_normal(Tc.shape)
        Ug, Vg = g.interpolate(l, U, V, Uc, Vc)
        assert rel(Ug, U + L.P @ Uc) < tol
        if not spd:
            assert rel(Vg, V + L.Q @ Vc) < tol
    g.set_precision("fp64")


def test_coarsest_pseudo_inverse(case):
    H, g = case["H"], case["g"]
    spd = case["kind"] == "spd"
    l = len(H.levels) - 1
    sig, U, V, K, T = _vecs(case, l, 400)
    mL, nL = H.levels[l].A.shape
    ug, vg = g.coarsest_solve(sig, K, T, nL if spd else mL, nL)
    ur, vr = oracle.coarsest_pinv_apply(oracle.dense_XY(H.levels[l], spd), sig, K, T, spd)
    assert rel(ug, ur) < 1e-9
    if not spd:
        assert rel(vg, vr) < 1e-9


def test_coarsest_geneig_variant(case):
    """coarse_pinv = 1 (the generalized-eigen variant of the Sec. 4.2 coarsest
    solve) against the oracle's definition of the same variant."""
    H, g = case["H"], case["g"]
    spd = case["kind"] == "spd"
    l = len(H.levels) - 1
    sig, U, V, K, T = _vecs(case, l, 401)
    mL, nL = H.levels[l].A.shape
    g.set_coarse_pinv(1)
    try:
        ug, vg = g.coarsest_solve(sig, K, T, nL if spd else mL, nL)
    finally:
        g.set_coarse_pinv(0)
    XY = oracle.dense_XY(H.levels[l], spd)
    ur, vr = oracle.coarsest_pinv_apply(XY, sig, K, T, spd, form="geneig")
    assert rel(ug, ur) < 1e-9
    if not spd:
        assert rel(vg, vr) < 1e-9


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-9), ("fp32", 5e-4), ("bf16", 2 * TOLB16)])
def test_one_vcycle(case, prec, tol):
    H, g = case["H"], case["g"]
    g.set_precision(prec)
    spd = case["kind"] == "spd"
    rng = np.random.default_rng(500)
    U = case["U"] + 1e-3 * rng.standard_normal(case["U"].shape)
    V = None if spd else case["V"] + 1e-3 * rng.standard_normal(case["V"].shape)
    sig = case["s"] * (1 + 1e-3)
    Ug, Vg = g.vcycle(sig, U, V)
    Ur, Vr = U.copy(), None if spd else V.copy()
    oracle.vcycle(H, 0, sig, Ur, Vr, np.zeros_like(Ur), None if spd else np.zeros_like(Vr))
    # compare the corrections (the iterate itself is common to both)
    assert rel(Ug - U, Ur - U) < tol, rel(Ug - U, Ur - U)
    if not spd:
        assert rel(Vg - V, Vr - V) < tol
    g.set_precision("fp64")


def _match_up_to_sign(X, Y):
    s = np.sign(np.einsum("ij,ij->j", X, Y))
    s[s == 0] = 1
    return X * s


def test_ritz_step(case):
    H, g = case["H"], case["g"]
    spd = case["kind"] == "spd"
    rng = np.random.default_rng(600)
    U = case["U"] + 1e-2 * rng.standard_normal(case["U"].shape)
    V = None if spd else case["V"] + 1e-2 * rng.standard_normal(case["V"].shape)
    sg, Ug, Vg, rg = g.ritz(U, V)
    sr, Ur, Vr = oracle.ritz(H.levels[0].A, spd, H.target, U, V,
                             H.params.get("row_form", "induced"))
    rr = oracle.residual_norms(H.levels[0].A, spd, sr, Ur, Vr)
    assert rel(sg, sr) < 1e-12
    assert rel(rg, rr) < 1e-7
    # vectors are unique up to sign where sigma is simple
    gaps = np.abs(np.diff(np.sort(sr)))
    if gaps.min() > 1e-8 * np.abs(sr).max():
        assert rel(_match_up_to_sign(Ug, Ur), Ur) < 1e-9


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_solve_matches_oracle(case, prec):
    if case["name"] == "svd_min_paper":
        pytest.skip("the paper's row form collapses onto the null(A^t) zero modes of the "
                    "gradient in the oracle too (sigma -> 0); its steps are compared above")
    H, g = case["H"], case["g"]
    spd = case["kind"] == "spd"
    g.set_precision(prec)
    g.set_triplets(case["s"], case["U"], case["V"])
    tol = 1e-10
    ok, it = g.solve(tol, 200)
    sg, Ug, Vg, rg = g.triplets()
    so, Uo, Vo, hist = oracle.solve(H, case["s"], case["U"], case["V"], tol=tol, max_outer=200)
    assert ok and rg.max() <= tol, (ok, rg)
    assert hist[-1].max() <= tol
    assert rel(sg, so) < 1e-10, (sg, so)
    A = H.levels[0].A
    ref = np.linalg.svd(A.toarray(), compute_uv=False)
    ref = np.sort(ref)[: case["nb"]] if H.target == "minimal" else np.sort(ref)[::-1][: case["nb"]]
    assert rel(sg, ref) < 1e-10
    if prec == "fp64":
        # the defect form equals the paper form to rounding: same iteration counts
        assert abs(it - (len(hist) - 1)) <= 1
    g.set_precision("fp64")


def test_solve_coloured_matches_oracle(case):
    """The solve with the coloured variant reaches the oracle's triplets, and
    the FP64 path takes the oracle's coloured iteration count to within 1."""
    H, g = case["H"], case["g"]
    if H.target != "minimal" or case["name"] == "svd_min_paper":
        pytest.skip("coloured order: minimal target, converging form")
    g.set_precision("fp64")
    g.set_relax_order("coloured")
    try:
        g.set_triplets(case["s"], case["U"], case["V"])
        ok, it = g.solve(1e-10, 200)
        sg, Ug, Vg, rg = g.triplets()
        Hc = oracle.hierarchy_from_interp(H.levels[0].A, [L.P for L in H.levels[:-1]],
                                          None if case["kind"] == "spd" else
                                          [L.Q for L in H.levels[:-1]],
                                          case["kind"], H.target, dict(H.params, relax_order="coloured"))
        so, Uo, Vo, hist = oracle.solve(Hc, case["s"], case["U"], case["V"], tol=1e-10, max_outer=200)
        assert ok and rg.max() <= 1e-10
        assert rel(sg, so) < 1e-10
        assert abs(it - (len(hist) - 1)) <= 1
    finally:
        g.set_relax_order("natural")


# ----------------------------------------------------------- Kaczmarz stress
@pytest.mark.parametrize("nb", [3, 8, 10])
def test_kaczmarz_sweep_many_bands_random_rectangular(nb):
    # a random rectangular operator with ragged rows spans many bands and
    # levels; the GPU sweep must equal the sequential natural-order sweep.
    # A few long rows (33..80 entries) make lanes walk several entries; n_b
    # of 3, 8 and 10 give vector blocks of 4, 8 and 12 columns.
    rng = np.random.default_rng(21)
    m, n = 30011, 9007
    lens = rng.integers(1, 7, size=m)
    long_rows = rng.random(m) < 0.02
    lens[long_rows] = rng.integers(33, 81, size=int(long_rows.sum()))
    rows = np.repeat(np.arange(m), lens)
    cols = rng.integers(0, n, size=rows.size)
    A = sp.csr_matrix((rng.standard_normal(rows.size), (rows, cols)), shape=(m, n))
    A.sum_duplicates()
    A = oracle.samg._csr(A)
    agg_u = np.minimum(np.arange(m) // 211, 99)
    agg_v = np.minimum(np.arange(n) // 97, 89)
    P = sp.csr_matrix((np.ones(m), (np.arange(m), agg_u)), shape=(m, 100))
    Q = sp.csr_matrix((np.ones(n), (np.arange(n), agg_v)), shape=(n, 90))
    L0 = oracle.Level(A, sp.identity(m, format="csr"), sp.identity(n, format="csr"))
    sig = np.linspace(0.5, 2.0, nb)
    U = rng.standard_normal((m, nb))
    V = rng.standard_normal((n, nb))
    g = samg.Solver.from_hierarchy(A, [P], [Q], nb, sig, U, V, "minimal", "svd", prec="fp64",
                                   mu_b=1)
    K = rng.standard_normal((m, nb))
    T = rng.standard_normal((n, nb))
    for prec, tol in (("fp64", 1e-11), ("fp32", 1e-3)):
        g.set_precision(prec)
        Ug, Vg = g.relax(0, sig, U, V, K, T, count=1)
        Ur, Vr = U.copy(), V.copy()
        oracle.relax_boot(L0, False, "minimal", sig, Ur, Vr, K, T, 0.7)
        assert rel(Vg, Vr) < tol, (prec, rel(Vg, Vr))
        assert rel(Ug, Ur) < tol, (prec, rel(Ug, Ur))
    g.close()
