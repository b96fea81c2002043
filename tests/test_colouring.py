"""The library's greedy row colouring (coloured sweep variant) against the
oracle's, on the CPU: the colours are integers, so they must agree exactly."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import workloads as W

samg = pytest.importorskip("paper_1102_0919_gb300")


@pytest.mark.parametrize("name", ["grad", "gradT", "lap", "random", "galerkin"])
def test_library_colouring_matches_oracle(name):
    if name == "grad":
        R = W.gradient(40).to_scipy()
    elif name == "gradT":
        R = sp.csr_matrix(W.gradient(40).to_scipy().T)
    elif name == "lap":
        R = W.laplacian5(30, 0.3).to_scipy()
    elif name == "random":
        R = sp.random(3000, 1700, density=0.004, random_state=7, format="csr")
    else:
        A = W.gradient(24).to_scipy()
        H, s, U, V = oracle.setup(A, 4, "minimal", "svd", dict(W.GRAD_PARAMS, n_mult=1, seed=5,
                                                               coarsest_max=40))
        R = H.levels[2].A
    R = oracle.samg._csr(R)
    got, k = samg.row_colours(R)
    want = oracle.row_colours(R)
    assert k == want.max() + 1
    assert np.array_equal(got, want)
