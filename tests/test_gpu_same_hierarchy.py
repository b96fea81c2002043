"""Iterate parity at a real size on one hierarchy: the library's own setup of
the 256 x 256 gradient (8 minimal triplets), its interpolation operators read
back through the C ABI and given to the oracle (which forms its own Galerkin
operators), then both solves run from the same boot triplets and their
residual histories are compared outer iteration by outer iteration."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

samg = pytest.importorskip("paper_1102_0919_gb300")


def test_gpu_and_oracle_histories_on_the_library_hierarchy():
    wl = W.workload(2)
    A = wl.build()
    prm = dict(wl.params, seed=W.problem_seed(2))
    s = samg.Solver.setup(A, wl.nb, wl.target, wl.kind, prec="fp64", **prm)
    try:
        nl = len(s.levels())

        def mat(l, which):
            rp, ci, v, shape = s.level_matrix(l, which)
            return sp.csr_matrix((v, ci, rp), shape=shape)

        H = oracle.hierarchy_from_interp(A.to_scipy(), [mat(l, "P") for l in range(nl - 1)],
                                         [mat(l, "Q") for l in range(nl - 1)], wl.kind,
                                         wl.target, dict(prm))
        # the library's coarse operators equal the oracle's Galerkin products
        for l in range(1, nl):
            d = abs(mat(l, "A") - H.levels[l].A).max()
            assert d <= 1e-10 * abs(H.levels[l].A).max(), (l, d)
        sig0, U0, V0, r0 = s.triplets()
        n_it = 6
        gpu = [float(r0.max())]
        for _ in range(n_it):
            s.solve(1e-300, 1)
            gpu.append(float(s.triplets()[3].max()))
        so, Uo, Vo, hist = oracle.solve(H, sig0, U0, V0, tol=1e-300, max_outer=n_it)
        ora = [float(h.max()) for h in hist]
        assert len(ora) == len(gpu)
        # float64 on both sides: the histories agree to the rounding of the
        # row-sum order inside the sweeps, amplified over a few cycles
        assert np.allclose(gpu, ora, rtol=1e-6), (gpu, ora)
        sg = s.triplets()[0]
        assert np.allclose(sg, so, rtol=1e-9), (sg, so)
    finally:
        s.close()
