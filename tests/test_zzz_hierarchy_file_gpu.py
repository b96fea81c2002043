"""samg_export -> samg_import_file on the GPU: the file holds the context's
operators and boot triplets exactly, and a solve from the imported context
repeats the original's (the Galerkin operators are rebuilt by the same
products in the same order)."""
import numpy as np
import pytest

import workloads as W
from test_hierarchy_file import _parse, _same

pytestmark = pytest.mark.gpu
samg = pytest.importorskip("paper_1102_0919_gb300")


@pytest.mark.parametrize("case", ["spd", "svd"])
def test_export_import_file_round_trip(case, tmp_path):
    import scipy.sparse as sp

    if case == "spd":
        wl = W.workload(1)
        A = wl.build().to_scipy()
        args = (A, wl.nb, wl.target, wl.kind)
        prm = dict(wl.params, seed=W.problem_seed(1))
    else:
        A = W.gradient(32).to_scipy()
        args = (A, 8, "minimal", "svd")
        prm = dict(W.GRAD_PARAMS, seed=W.problem_seed(2))
    s = samg.Solver.setup(*args, prec="fp64", **prm)
    path = str(tmp_path / "h.samg")
    s.export(path)
    d = _parse(path)
    lv = s.levels()
    assert d["nlev"] == len(lv) and _same(d["A"], A)
    for l in range(len(lv) - 1):
        rp, ci, v, shape = s.level_matrix(l, "P")
        assert _same(d["P"][l], sp.csr_matrix((v, ci, rp), shape=shape))
        if case == "svd":
            rp, ci, v, shape = s.level_matrix(l, "Q")
            assert _same(d["Q"][l], sp.csr_matrix((v, ci, rp), shape=shape))
    sig0, U0, V0, r0 = s.triplets()
    assert np.array_equal(d["sig"], sig0) and np.array_equal(d["U"], U0)
    t = samg.Solver.from_file(path, prec="fp64", **prm)
    assert t.levels() == lv
    sig1, U1, V1, r1 = t.triplets()
    assert np.array_equal(sig1, sig0) and np.array_equal(U1, U0)
    assert np.allclose(r1, r0, rtol=1e-12, atol=0)
    ok0, it0 = s.solve(1e-10, 80)
    ok1, it1 = t.solve(1e-10, 80)
    assert ok0 and ok1 and abs(it0 - it1) <= 1
    assert np.allclose(t.triplets()[0], s.triplets()[0], rtol=1e-12, atol=0)
    s.close()
    t.close()
