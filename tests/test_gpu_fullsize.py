"""Single steps of the solve phase at the full size of the 1024 x 1024
gradient workload (m = 2,099,200, n = 1,048,576), against the oracle, element
by element.  The hierarchy is a two-level aggregation (P, Q piecewise
constant) imported into the library, so the test needs no setup phase: what is
checked is the Kaczmarz block Gauss-Seidel relaxation over thousands of bands
and chunks, the fused residual + restriction, and the interpolation, each at
the workload's size and block width."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

samg = pytest.importorskip("paper_1102_0919_gb300")


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.fixture(scope="module")
def big():
    A = W.gradient(1024).to_scipy()
    m, n = A.shape
    nb = 8
    P = sp.csr_matrix((np.ones(m), (np.arange(m), np.minimum(np.arange(m) // 21000, 99))),
                      shape=(m, 100))
    Q = sp.csr_matrix((np.ones(n), (np.arange(n), np.minimum(np.arange(n) // 11700, 89))),
                      shape=(n, 90))
    rng = np.random.default_rng(1024)
    sig = np.linspace(4.0, 12.0, nb)
    U = rng.standard_normal((m, nb))
    V = rng.standard_normal((n, nb))
    g = samg.Solver.from_hierarchy(A, [P], [Q], nb, sig, U, V, "minimal", "svd", prec="fp64",
                                   mu_b=1)
    L0 = oracle.Level(A, sp.identity(m, format="csr"), sp.identity(n, format="csr"), P=P, Q=Q)
    yield dict(A=A, g=g, L0=L0, sig=sig, U=U, V=V, nb=nb, rng=rng)
    g.close()


def _fp32_bound(A, count):
    """Max-norm bound of a float32 relaxation program relative to its largest
    entry: every row update rounds its correction and each updated value
    (3 roundings of u = 2^-24), the projections do not amplify earlier
    errors, and a value's error collects at most one update per level along
    the longest chain of dependent rows -- the program's dependency depth D
    (from the schedule builder's plan).  Twice 3 u D."""
    _, depth, _ = samg.sweep_plan(A, count)
    return 2.0 * 3.0 * 2.0 ** -24 * depth


@pytest.mark.parametrize("count", [4])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_fused_relaxations_full_size(big, prec, count):
    """The fused program of four block Gauss-Seidel relaxations (12.6 M rows
    over about 190 bands at this size) against four sequential relaxations
    of the oracle, element by element."""
    g, L0, sig, U, V = big["g"], big["L0"], big["sig"], big["U"], big["V"]
    tol = 1e-10 if prec == "fp64" else _fp32_bound(big["A"], count)
    rng = np.random.default_rng(9)
    K = rng.standard_normal(U.shape)
    T = rng.standard_normal(V.shape)
    g.set_precision(prec)
    Ug, Vg = g.relax(0, sig, U, V, K, T, count=count)
    Ur, Vr = U.copy(), V.copy()
    for _ in range(count):
        oracle.relax_boot(L0, False, "minimal", sig, Ur, Vr, K, T, 0.7)
    assert rel(Vg, Vr) < tol, (rel(Vg, Vr), tol)
    assert rel(Ug, Ur) < tol, (rel(Ug, Ur), tol)
    g.set_precision("fp64")


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_relaxation_full_size(big, prec):
    g, L0, sig, U, V = big["g"], big["L0"], big["sig"], big["U"], big["V"]
    tol = 1e-10 if prec == "fp64" else _fp32_bound(big["A"], 1)
    rng = np.random.default_rng(7)
    K = rng.standard_normal(U.shape)
    T = rng.standard_normal(V.shape)
    g.set_precision(prec)
    Ug, Vg = g.relax(0, sig, U, V, K, T, count=1)
    Ur, Vr = U.copy(), V.copy()
    oracle.relax_boot(L0, False, "minimal", sig, Ur, Vr, K, T, 0.7)
    assert rel(Vg, Vr) < tol, rel(Vg, Vr)
    assert rel(Ug, Ur) < tol, rel(Ug, Ur)
    g.set_precision("fp64")


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-4)])
def test_residual_restrict_interpolate_full_size(big, prec, tol):
    g, L0, sig, U, V = big["g"], big["L0"], big["sig"], big["U"], big["V"]
    rng = np.random.default_rng(8)
    K = rng.standard_normal(U.shape)
    T = rng.standard_normal(V.shape)
    g.set_precision(prec)
    Kc, Tc = g.residual_restrict(0, sig, U, V, K, T, 100, 90)
    r, s = oracle.level_residual(L0, False, sig, U, V, K, T)
    assert rel(Kc, L0.P.T @ r) < tol
    assert rel(Tc, L0.Q.T @ s) < tol
    Uc = rng.standard_normal(Kc.shape)
    Vc = rng.standard_normal(Tc.shape)
    Ug, Vg = g.interpolate(0, U, V, Uc, Vc)
    assert rel(Ug, U + L0.P @ Uc) < tol
    assert rel(Vg, V + L0.Q @ Vc) < tol
    g.set_precision("fp64")
