"""The library's own setup (multiplicative phase on the GPU + host
coarsening) followed by the solve, checked against closed forms, dense
LAPACK and the invariants A v = sigma u, A^t u = sigma v.  The hierarchy
itself is not compared with the oracle's: from the second coarsening down
it depends on rounding (the oracle's own level sizes change with the number
of BLAS threads), so the two setups build different, equally valid
hierarchies."""
import time

import numpy as np
import pytest

import oracle
import workloads as W
from closed_forms import gradient_singular_values, laplacian5_eigs

pytestmark = pytest.mark.gpu
samg = pytest.importorskip("paper_1102_0919_gb300")


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_laplacian_workload_minimal_eigenpairs(prec):
    wl = W.workload(1)
    A = wl.build().to_scipy()
    t0 = time.perf_counter()
    s = samg.Solver.setup(A, wl.nb, wl.target, wl.kind, prec=prec,
                          **dict(wl.params, seed=W.problem_seed(1)))
    wall = time.perf_counter() - t0
    # the setup's stage clock: every stage accounted, none above the wall time
    st = s.setup_times()
    assert set(st) == set(samg.Solver.SETUP_STAGES)
    assert all(v >= 0.0 for v in st.values()) and 0.0 < sum(st.values()) <= wall
    assert st["test_relax"] > 0.0 and st["strength_rs"] > 0.0 and st["ls_fit"] > 0.0
    levels = s.levels()
    ok, it = s.solve(1e-10, 60)
    sig, U, _, res = s.triplets()
    s.close()
    assert ok and res.max() <= 1e-10
    assert np.allclose(sig, laplacian5_eigs(32)[:4], rtol=1e-10)
    assert np.allclose(U.T @ U, np.eye(4), atol=1e-9)
    assert 4 <= len(levels) <= 6 and levels[-1][0] <= 100


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_gradient_minimal_triplets(prec):
    N = 32
    A = W.gradient(N).to_scipy()
    s = samg.Solver.setup(A, 8, "minimal", "svd", prec=prec,
                          **dict(W.GRAD_PARAMS, seed=W.problem_seed(2)))
    ok, it = s.solve(1e-10, 80)
    sig, U, V, res = s.triplets()
    s.close()
    assert ok and res.max() <= 1e-10, res
    assert np.allclose(sig, gradient_singular_values(N)[:8], rtol=1e-10)
    assert np.allclose(A @ V, U * sig, atol=1e-8 * sig.max())
    assert np.allclose(A.T @ U, V * sig, atol=1e-8 * sig.max())
    assert np.allclose(V.T @ V, np.eye(8), atol=1e-9)


def test_dominant_svd_lapack():
    A = W.laplacian5(16).to_scipy()
    s = samg.Solver.setup(A, 4, "dominant", "svd", prec="fp64",
                          **dict(W.FD_PARAMS, seed=9, coarsest_max=40))
    assert len(s.levels()) >= 3
    ok, it = s.solve(1e-9, 200)
    sig, U, V, res = s.triplets()
    s.close()
    assert ok
    ref = np.sort(np.linalg.svd(A.toarray(), compute_uv=False))[::-1][:4]
    assert np.allclose(sig, ref, rtol=1e-10)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_gradient_256_full_size(prec):
    # workload: 8 minimal triplets of the 256 x 256 gradient (m = 131584, n = 65536)
    wl = W.workload(2)
    A = wl.build().to_scipy()
    s = samg.Solver.setup(A, wl.nb, wl.target, wl.kind, prec=prec,
                          **dict(wl.params, seed=W.problem_seed(2)))
    ok, it = s.solve(1e-8, 300)
    sig, U, V, res = s.triplets()
    s.close()
    assert ok and res.max() <= 1e-8, (it, res)
    exact = gradient_singular_values(256)[:8]
    # Weyl bound from the augmented operator: |s~ - s| <= rho s / sqrt(2)
    assert np.all(np.abs(sig - exact) <= res * sig / np.sqrt(2) + 1e-12 * exact)
    assert np.allclose(sig, exact, rtol=1e-9)
