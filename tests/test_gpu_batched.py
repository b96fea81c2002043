"""The batched workload's API on the GPU: independent anisotropic 5-point
diffusion problems of uneven sizes (the seeded draw of the batched
workload), set up and solved through samg_setup_batched /
samg_solve_batched, each problem's 4 smallest eigenvalues against the closed
form lam_kl = 4(N+1)^2 [eps sin^2(k pi h/2) + sin^2(l pi h/2)]."""
import numpy as np
import pytest

import workloads as W
from closed_forms import laplacian5_eigs

pytestmark = pytest.mark.gpu

samg = pytest.importorskip("paper_1102_0919_gb300")


def _problems(ids):
    draw = W.aniso_batch()
    return [draw[p] for p in ids]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batched_problems_closed_form(prec):
    # problems whose gap after the 4 sought eigenvalues is at least 1.1
    ids = [0, 2, 5, 6, 9, 10]
    probs = _problems(ids)
    As = [W.laplacian5(N, e).to_scipy() for N, e in probs]
    b = samg.Batch.setup(As, 4, "minimal", "spd", prec=prec,
                         **dict(W.FD_PARAMS, seed=W.problem_seed(5)))
    try:
        ok, done = b.solve(1e-10, 200)
        assert ok, done
        for k, (N, e) in enumerate(probs):
            lam, X, _, res = b.problem(k).triplets()
            exact = laplacian5_eigs(N, e)[:4]
            assert res.max() <= 1e-10, (ids[k], res)
            assert np.allclose(lam, exact, rtol=1e-9), (ids[k], lam, exact)
            assert np.allclose(X.T @ X, np.eye(4), atol=1e-9)
    finally:
        b.close()


def test_batched_small_gap_with_guard_pairs():
    # problem 7 (N = 81, eps = 0.61) has lam_5 / lam_4 = 1.0072; two guard
    # pairs (n_b = 6, the first 4 converged) keep the block complete
    probs = _problems([7, 4])
    As = [W.laplacian5(N, e).to_scipy() for N, e in probs]
    b = samg.Batch.setup(As, 6, "minimal", "spd", prec="fp32", n_conv=4,
                         **dict(W.FD_PARAMS, seed=W.problem_seed(5)))
    try:
        ok, done = b.solve(1e-10, 300)
        assert ok, done
        for k, (N, e) in enumerate(probs):
            lam, _, _, res = b.problem(k).triplets()
            assert res[:4].max() <= 1e-10
            assert np.allclose(lam[:4], laplacian5_eigs(N, e)[:4], rtol=1e-9)
    finally:
        b.close()


def test_concurrent_rounds_match_solving_each_problem_alone():
    # samg_solve_batched runs the problems in rounds on their own streams;
    # each problem's iterations and triplets equal those of its own context
    # solved alone (same setup, same arithmetic, float64)
    ids = [0, 5, 9, 10]
    probs = _problems(ids)
    As = [W.laplacian5(N, e).to_scipy() for N, e in probs]
    prm = dict(W.FD_PARAMS, seed=W.problem_seed(5))
    b = samg.Batch.setup(As, 4, "minimal", "spd", prec="fp64", **prm)
    try:
        ok, done = b.solve(1e-10, 200)
        assert ok, done
        for k, A in enumerate(As):
            s = samg.Solver.setup(A, 4, "minimal", "spd", prec="fp64", **prm)
            try:
                ok1, it1 = s.solve(1e-10, 200)
                assert ok1 and it1 == done[k], (ids[k], it1, done[k])
                lam1 = s.triplets()[0]
                lam = b.problem(k).triplets()[0]
                assert np.allclose(lam, lam1, rtol=1e-13), (ids[k], lam, lam1)
            finally:
                s.close()
    finally:
        b.close()
