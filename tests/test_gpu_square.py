"""Square SVD kind (Sec. 5.1) on the GPU: the C/F splitting and the sparsity
patterns of P and Q taken from A itself (square_form "from_A"), or one
operator P = Q for both sides ("shared"), on the 20 x 20 upwind
convection-diffusion operator (a square nonsymmetric 5-point matrix).

Checked through the C ABI: every level of the library's hierarchy is square;
the first coarse level has the oracle's size (the splitting depends on A
only); with P = Q the library's Q_l equals its P_l and B_l = C_l; the
library's solve reaches a dense LAPACK SVD (called); and, on the library's
own interpolation operators given to the oracle, the two solves' residual
histories agree outer iteration by outer iteration."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

samg = pytest.importorskip("paper_1102_0919_gb300")

CASES = [("dominant", "from_A"), ("dominant", "shared"), ("minimal", "shared")]


def _prm(target, form):
    base = W.FD_PARAMS if target == "dominant" else W.GRAD_PARAMS
    return dict(base, seed=W.problem_seed(2), coarsest_max=40, n_mult=10, square_form=form)


@pytest.mark.parametrize("target,form", CASES)
def test_square_forms_on_the_gpu(target, form):
    A = W.convdiff5(20, 8.0)
    As = A.to_scipy()
    sv = np.sort(np.linalg.svd(As.toarray(), compute_uv=False))
    prm = _prm(target, form)
    s = samg.Solver.setup(A, 4, target, "svd", prec="fp64", **prm)
    try:
        lv = s.levels()
        assert len(lv) >= 2
        for m, n, _ in lv:
            assert m == n, lv
        H, _, _, _ = oracle.setup(As, 4, target, "svd", prm)
        assert lv[1][0] == H.levels[1].A.shape[0], (lv, [L.A.shape for L in H.levels])

        def mat(l, which):
            rp, ci, v, shape = s.level_matrix(l, which)
            return sp.csr_matrix((v, ci, rp), shape=shape)

        nl = len(lv)
        Ps = [mat(l, "P") for l in range(nl - 1)]
        Qs = [mat(l, "Q") for l in range(nl - 1)]
        if form == "shared":
            for l in range(nl - 1):
                assert abs(Ps[l] - Qs[l]).max() == 0
            for l in range(1, nl):
                assert abs(mat(l, "B") - mat(l, "C")).max() <= 1e-14 * abs(mat(l, "B")).max()

        # iterate parity on the library's hierarchy (float64 both sides)
        Ho = oracle.hierarchy_from_interp(As, Ps, Qs, "svd", target, dict(prm))
        sig0, U0, V0, r0 = s.triplets()
        n_it = 5
        gpu = [float(r0.max())]
        for _ in range(n_it):
            s.solve(1e-300, 1)
            gpu.append(float(s.triplets()[3].max()))
        _, _, _, hist = oracle.solve(Ho, sig0, U0, V0, tol=1e-300, max_outer=n_it)
        ora = [float(h.max()) for h in hist]
        assert np.allclose(gpu, ora, rtol=1e-6), (gpu, ora)

        # the library's own solve reaches LAPACK
        s.solve(1e-10, 150)
        sg, U, V, res = s.triplets()
        ref = sv[::-1][:4] if target == "dominant" else sv[:4]
        assert res.max() <= 1e-10, res
        assert np.allclose(sg, ref, rtol=1e-10), (sg, ref)
        assert np.abs(As @ V - U * sg).max() <= 1e-9 * sv[-1]
    finally:
        s.close()
