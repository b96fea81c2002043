"""Parity of the relaxations and the Ritz step at the block widths the
workloads use besides n_b = 8: n_b = 3 (vector rows of 4) and n_b = 10 (rows
of 12, the term-document workload), on random operators with ragged rows.
Covers the shifted Kaczmarz sweep of the SPD kind (rows of A - lambda_j B)
and the weighted-Jacobi relaxation of the dominant kind."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle

pytestmark = pytest.mark.gpu

samg = pytest.importorskip("paper_1102_0919_gb300")


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _ragged(rng, m, n):
    lens = rng.integers(1, 7, size=m)
    long_rows = rng.random(m) < 0.02
    lens[long_rows] = rng.integers(33, 81, size=int(long_rows.sum()))
    rows = np.repeat(np.arange(m), lens)
    cols = rng.integers(0, n, size=rows.size)
    A = sp.csr_matrix((rng.standard_normal(rows.size), (rows, cols)), shape=(m, n))
    A.sum_duplicates()
    return A


def _agg(k, kc):
    return sp.csr_matrix((np.ones(k), (np.arange(k), np.minimum(np.arange(k) * kc // k, kc - 1))),
                         shape=(k, kc))


@pytest.mark.parametrize("nb", [3, 10])
def test_shifted_kaczmarz_spd(nb):
    # symmetric, diagonally dominant (SPD) operator with ragged rows
    rng = np.random.default_rng(31 + nb)
    n = 20011
    R = _ragged(rng, n, n)
    A = (R + R.T).tocsr()
    A = (A + sp.diags(np.asarray(abs(A).sum(axis=1)).ravel() + 1.0)).tocsr()
    A = oracle.samg._csr(A)
    P = _agg(n, 100)
    sig = np.linspace(0.5, 3.0, nb)
    U = rng.standard_normal((n, nb))
    g = samg.Solver.from_hierarchy(A, [P], None, nb, sig, U, None, "minimal", "spd",
                                   prec="fp64", mu_b=1)
    K = rng.standard_normal((n, nb))
    L0 = oracle.Level(A, sp.identity(n, format="csr"), None)
    for prec, tol in (("fp64", 1e-10), ("fp32", 1e-3)):
        g.set_precision(prec)
        Ug, _ = g.relax(0, sig, U, None, K, None, count=1)
        Ur = U.copy()
        oracle.relax_boot(L0, True, "minimal", sig, Ur, None, K, None, 0.7)
        assert rel(Ug, Ur) < tol, (prec, rel(Ug, Ur))
    g.close()


@pytest.mark.parametrize("nb", [3, 10])
def test_dominant_jacobi_and_ritz(nb):
    rng = np.random.default_rng(41 + nb)
    m, n = 30011, 9007
    A = oracle.samg._csr(_ragged(rng, m, n))
    P, Q = _agg(m, 100), _agg(n, 90)
    sig = np.linspace(20.0, 10.0, nb)
    U = rng.standard_normal((m, nb))
    V = rng.standard_normal((n, nb))
    g = samg.Solver.from_hierarchy(A, [P], [Q], nb, sig, U, V, "dominant", "svd", prec="fp64",
                                   mu_b=1)
    K = rng.standard_normal((m, nb))
    T = rng.standard_normal((n, nb))
    L0 = oracle.Level(A, sp.identity(m, format="csr"), sp.identity(n, format="csr"))
    for prec, tol in (("fp64", 1e-10), ("fp32", 1e-4)):
        g.set_precision(prec)
        Ug, Vg = g.relax(0, sig, U, V, K, T, count=1)
        Ur, Vr = U.copy(), V.copy()
        oracle.relax_boot(L0, False, "dominant", sig, Ur, Vr, K, T, 0.7)
        assert rel(Ug, Ur) < tol, (prec, rel(Ug, Ur))
        assert rel(Vg, Vr) < tol, (prec, rel(Vg, Vr))
    g.set_precision("fp64")
    sg, Ug, Vg, rg = g.ritz(U, V)
    sr, Ur, Vr = oracle.ritz(A, False, "dominant", U, V)
    assert rel(sg, sr) < 1e-12
    assert rel(rg, oracle.residual_norms(A, False, sr, Ur, Vr)) < 1e-7
    g.close()
