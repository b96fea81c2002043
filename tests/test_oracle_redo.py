"""Pins of the oracle's redo-P remedy (Sec. 6.3): the interpolation is
redetermined by one downward sweep of the multiplicative phase with the LS
weights of the test vectors and of the converged boot vectors divided by
1000."""
import numpy as np

import oracle
import oracle.samg as osamg
import workloads as W
from closed_forms import laplacian5_eigs


def _fd_dominant(N=20):
    A = W.laplacian5(N).to_scipy()
    H, s, U, V = oracle.setup(A, 4, "dominant", "spd", dict(W.FD_PARAMS, seed=3, coarsest_max=40))
    return A, H, s, U


def test_redo_keeps_the_iterate_and_replaces_the_hierarchy():
    A, H, s, U = _fd_dominant()
    s0, U0, Ut0 = s.copy(), U.copy(), H.Ut.copy()
    old = H.levels
    osamg.redo_interpolation(H, s, U, None, np.array([True, False, False, True]))
    assert np.array_equal(s, s0) and np.array_equal(U, U0)
    assert H.levels is not old
    assert np.array_equal(H.levels[0].A.toarray(), old[0].A.toarray())
    assert H.levels[0].P is not None and not np.array_equal(Ut0, H.Ut)  # test vectors relaxed on


def _fit_residual(L, theta, Y, cols, w):
    """sum over cols k of w_k |Y_k - P Y_k[C]|^2 on level L (SPD kind; the
    coarse copy of a vector is its values at the C-points, in order)."""
    cpts = np.flatnonzero(oracle.rs_coarsen(oracle.strength(L.A, theta)))
    assert L.P.shape[1] == len(cpts)
    tot = 0.0
    for k in cols:
        r = Y[:, k] - L.P @ Y[cpts, k]
        tot += w[k] * float(r @ r)
    return tot


def test_reweighting_favours_the_unconverged_vectors():
    # For a weighted LS fit, lowering the weights of the other equations by
    # eps < 1 cannot raise the weighted misfit of the kept ones; the level-0
    # fit of the dominant SPD kind is a plain weighted LS on [U_t, U_b].
    A, H, s, U = _fd_dominant()
    conv = np.array([True, True, False, False])
    nt = H.Ut.shape[1]
    res = {}
    for name, f in (("plain", 1.0), ("redo", 1e-3)):
        Ut = H.Ut.copy()
        ub = U.copy()
        wscale = np.concatenate([np.full(nt, f), np.where(conv, f, 1.0)])
        levels, _, _, _ = osamg._down_sweep(A.tocsr(), True, "dominant", 4, H.params, Ut, None,
                                            s.copy(), ub, None, wscale)
        L0 = levels[0]
        Y = np.hstack([Ut, ub])            # level-0 vectors as fitted (relaxed in place)
        w = np.abs(osamg.rayleigh(L0, True, Y, None))
        res[name] = _fit_residual(L0, H.params["theta"], Y, [nt + 2, nt + 3], w)
        # the other side: the down-weighted vectors may only fit worse
        res[name + "_rest"] = _fit_residual(L0, H.params["theta"], Y, list(range(nt + 2)), w)
    assert res["redo"] <= res["plain"] * (1 + 1e-12)
    assert res["redo"] < 0.9 * res["plain"]
    assert res["redo_rest"] >= res["plain_rest"] * (1 - 1e-12)


def test_solve_with_redo_reaches_the_closed_form():
    A = W.laplacian5(32).to_scipy()
    H, s, U, V = oracle.setup(A, 4, "minimal", "spd", dict(W.FD_PARAMS, seed=W.problem_seed(1)))
    s, U, V, hist = oracle.solve(H, s, U, V, tol=1e-10, max_outer=60, redo_tol=1e-6)
    assert hist[-1].max() <= 1e-10
    assert len(H.redos) >= 1
    assert np.allclose(s, laplacian5_eigs(32)[:4], rtol=1e-10)
    assert np.allclose(U.T @ U, np.eye(4), atol=1e-10)
