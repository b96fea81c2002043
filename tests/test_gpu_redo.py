"""The redo of the interpolation for lagging triplets (Sec. 6.3) on the GPU:
one downward sweep of the multiplicative phase from the setup's fine test
vectors and copies of the boot triplets, the LS weights of the test vectors
and of the converged triplets divided by 1000.

On a two-level hierarchy the whole setup depends on A and the seeded draws
only (the one splitting is A's), so the library's and the oracle's setups
agree to rounding; the redo is then compared operator by operator with the
oracle's.  On the gradient, a solve with redo_tol redoes the interpolation
on its own and still reaches the closed form."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import oracle.samg as osamg
import workloads as W
from closed_forms import gradient_singular_values

pytestmark = pytest.mark.gpu

samg = pytest.importorskip("paper_1102_0919_gb300")


def _mat(s, l, which):
    rp, ci, v, shape = s.level_matrix(l, which)
    return sp.csr_matrix((v, ci, rp), shape=shape)


def _rel(a, b):
    d = abs(a - b).max() if sp.issparse(a) else np.abs(a - b).max()
    ref = abs(b).max() if sp.issparse(b) else np.abs(b).max()
    return float(d / ref)


def test_redo_matches_the_oracle_on_two_levels():
    # anisotropic Laplacian: simple eigenvalues, so the coarsest boot
    # vectors are unique up to sign on both sides
    A = W.laplacian5(20, 0.37).to_scipy()
    prm = dict(W.FD_PARAMS, seed=W.problem_seed(1), coarsest_max=40, max_levels=2)
    # redo_tol > 0 keeps the setup's test vectors; 1e-300 never triggers
    s = samg.Solver.setup(A, 4, "dominant", "spd", prec="fp64", redo_tol=1e-300, **prm)
    try:
        H, so, Uo, _ = oracle.setup(A, 4, "dominant", "spd", dict(prm))
        assert len(s.levels()) == 2 and len(H.levels) == 2
        P0 = _mat(s, 0, "P")
        assert P0.shape == H.levels[0].P.shape
        assert _rel(P0, H.levels[0].P) <= 1e-8
        n_it = 3
        s.solve(1e-300, n_it)
        sg, U, _, _ = s.triplets()
        so, Uo, _, _ = oracle.solve(H, so, Uo, None, tol=1e-300, max_outer=n_it)
        assert np.allclose(sg, so, rtol=1e-10), (sg, so)
        conv = np.array([True, True, False, False])
        s.redo_interpolation(conv)
        osamg.redo_interpolation(H, so, Uo, None, conv)
        # the iterate is unchanged, the hierarchy replaced
        sg2, U2, _, _ = s.triplets()
        assert np.array_equal(sg, sg2) and np.array_equal(U, U2)
        P1 = _mat(s, 0, "P")
        assert _rel(P1, P0) > 1e-6
        assert P1.shape == H.levels[0].P.shape
        assert _rel(P1, H.levels[0].P) <= 1e-6
        assert _rel(_mat(s, 1, "A"), H.levels[1].A) <= 1e-6
        # the solve goes on with the new hierarchy on both sides
        s.solve(1e-300, 2)
        so, Uo, _, hist = oracle.solve(H, so, Uo, None, tol=1e-300, max_outer=2)
        sg3 = s.triplets()[0]
        assert np.allclose(sg3, so, rtol=1e-9), (sg3, so)
    finally:
        s.close()


def test_solve_with_redo_reaches_the_closed_form():
    N = 32
    A = W.gradient(N).to_scipy()
    s = samg.Solver.setup(A, 8, "minimal", "svd", prec="fp64", redo_tol=1e-6,
                          **dict(W.GRAD_PARAMS, seed=W.problem_seed(2)))
    try:
        Q0 = _mat(s, 0, "Q")
        ok, it = s.solve(1e-10, 150)
        sig, U, V, res = s.triplets()
        assert ok and res.max() <= 1e-10, res
        assert np.allclose(sig, gradient_singular_values(N)[:8], rtol=1e-10)
        # the triplets cross 1e-6 at different outer iterations: at least one
        # redo replaced the interpolation
        assert _rel(_mat(s, 0, "Q"), Q0) > 1e-8
    finally:
        s.close()


def test_redo_needs_the_setup_state():
    A = W.laplacian5(12).to_scipy()
    s = samg.Solver.setup(A, 2, "minimal", "spd", prec="fp64",
                          **dict(W.FD_PARAMS, seed=5, coarsest_max=40))
    try:
        with pytest.raises(samg.SamgError):
            s.redo_interpolation([1, 0])
    finally:
        s.close()
