"""The library's host steps of the setup phase against the oracle, on the
CPU (no GPU needed): strength + Ruge-Stueben coarsening bit for bit, and the
weighted LS interpolation operator (Sec. 3.7-3.8) entry by entry."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import workloads as W

samg = pytest.importorskip("paper_1102_0919_gb300")


def _operators():
    G = W.gradient(12).to_scipy()
    rng = np.random.default_rng(9)
    R = sp.random(500, 500, density=0.01, random_state=rng, format="csr")
    S = (R + R.T + sp.diags(np.asarray(abs(R + R.T).sum(axis=1)).ravel() + 1.0)).tocsr()
    return {
        "laplacian": W.laplacian5(16).to_scipy(),
        "aniso": W.laplacian5(14, 0.05).to_scipy(),
        "gradient_AAt": (G @ G.T).tocsr(),
        "gradient_AtA": (G.T @ G).tocsr(),
        "random_spd": S,
    }


@pytest.mark.parametrize("name", ["laplacian", "aniso", "gradient_AAt", "gradient_AtA", "random_spd"])
@pytest.mark.parametrize("theta", [0.06, 0.25])
def test_coarsening_bit_exact(name, theta):
    N = oracle.samg._csr(_operators()[name])
    cf_lib = samg.host_coarsen(N, theta)
    cf_ref = oracle.rs_coarsen(oracle.strength(N, theta))
    assert np.array_equal(cf_lib.astype(np.int32), cf_ref.astype(np.int32))


@pytest.mark.parametrize("name", ["laplacian", "gradient_AtA", "random_spd"])
def test_ls_interpolation_matches_oracle(name):
    N = oracle.samg._csr(_operators()[name])
    theta = 0.06
    S = oracle.strength(N, theta)
    cf = oracle.rs_coarsen(S)
    rng = np.random.default_rng(4)
    n = N.shape[0]
    nf = 6
    Yc = rng.standard_normal((n, nf))
    Yf = Yc + 0.1 * rng.standard_normal((n, nf))
    w = rng.uniform(0.5, 2.0, nf)
    P_lib = samg.host_ls_interp(N, theta, cf, Yf, Yc, w)
    P_ref = oracle.fit_interp(S, cf, Yf, Yc, w)
    assert P_lib.shape == P_ref.shape
    P_lib.sort_indices()
    assert np.array_equal(P_lib.indptr, P_ref.indptr)
    assert np.array_equal(P_lib.indices, P_ref.indices)
    assert np.abs(P_lib.data - P_ref.data).max() <= 1e-10 * max(np.abs(P_ref.data).max(), 1.0)


def _strength_cases():
    G = W.gradient(12).to_scipy()
    td = W.termdoc(6000, 1500, seed=77, kmax=300).to_scipy()      # > 4096 rows: threaded path
    ti = td.copy()
    ti.data = np.round(np.expm1(ti.data))                          # integer counts tf
    E = sp.lil_matrix((40, 30))                                    # empty rows and columns
    rng = np.random.default_rng(2)
    for i in range(0, 40, 3):
        E[i, rng.choice(25, 4, replace=False)] = rng.integers(1, 5, 4)
    return {"gradient": G, "laplacian": W.laplacian5(16).to_scipy(), "termdoc_counts": ti,
            "termdoc": td, "empty_rows": sp.csr_matrix(E)}


@pytest.mark.parametrize("name", ["gradient", "laplacian", "termdoc_counts", "termdoc",
                                  "empty_rows"])
@pytest.mark.parametrize("side", ["AAt", "AtA"])
def test_strength_of_product_matches_oracle(name, side):
    # the setup's strength graph of A A^t (or A^t A) formed from A alone
    # equals the oracle's strength of the explicit product: bit for bit for
    # integer entries (every sum exact), pattern exact and values to rounding
    # otherwise
    A = oracle.samg._csr(_strength_cases()[name])
    if side == "AtA":
        A = oracle.samg._csr(A.T)
    theta = 0.03 if name.startswith("termdoc") else 0.06
    S_lib = samg.host_strength_product(A, theta)
    S_ref = oracle.strength(A @ A.T, theta)
    S_lib.sort_indices()
    S_ref.sort_indices()
    assert np.array_equal(S_lib.indptr, S_ref.indptr)
    assert np.array_equal(S_lib.indices, S_ref.indices)
    if name == "termdoc":
        assert np.allclose(S_lib.data, S_ref.data, rtol=1e-13, atol=0)
    else:
        assert np.array_equal(S_lib.data, S_ref.data)
    # and the coarsening on it is the oracle's
    assert np.array_equal(oracle.rs_coarsen(S_lib), oracle.rs_coarsen(S_ref))


def test_strength_of_product_rejects_malformed_input():
    bad = sp.csr_matrix(np.eye(3))
    bad.indices = bad.indices.copy()
    bad.indices[1] = 7
    with pytest.raises(samg.SamgError):
        samg.host_strength_product(bad, 0.06)
