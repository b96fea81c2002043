"""The paper's own worked example on the GPU (Sec. 6.2, Table "values"): the
8 largest and the 8 smallest eigenvalues of the unscaled 5-point FD
Laplacian on a 32 x 32 grid, found by the library's setup and solve (SPD
kind, the FD parameter set), against the Table's FD-lge and FD-sm columns
printed to 7 and 8 digits (half a unit of the last printed place), and
against the closed form.  The C client of the ABI runs here too."""
import os
import subprocess
import sys

import numpy as np
import pytest

import workloads as W
from closed_forms import laplacian5_eigs

pytestmark = pytest.mark.gpu

samg = pytest.importorskip("paper_1102_0919_gb300")

HERE = os.path.dirname(os.path.abspath(__file__))


def _table():
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "table_values_fd.txt"))
            if l.strip() and not l.startswith("#")]
    return np.array([float(r[1]) for r in rows]), np.array([float(r[2]) for r in rows])


@pytest.mark.parametrize("target", ["dominant", "minimal"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_fd_laplacian_table_values_on_gpu(target, prec):
    lge, sm = _table()
    A = W.laplacian5(32).to_scipy() / 33.0 ** 2          # entries 4, -1
    s = samg.Solver.setup(A, 8, target, "spd", prec=prec,
                          **dict(W.FD_PARAMS, seed=W.problem_seed(1)))
    try:
        ok, it = s.solve(1e-10, 300)
        sig, U, _, res = s.triplets()
    finally:
        s.close()
    assert ok and res.max() <= 1e-10, (it, res)
    exact = laplacian5_eigs(32) / 33.0 ** 2
    if target == "dominant":
        # the Table prints 7 decimals: within half a unit of the last place
        assert np.all(np.abs(sig - lge) <= 5.01e-8), sig - lge
        assert np.allclose(sig, exact[::-1][:8], rtol=1e-12)
    else:
        assert np.all(np.abs(sig - sm) <= 5.01e-9), sig - sm
        assert np.allclose(sig, exact[:8], rtol=1e-10)
    assert np.allclose(U.T @ U, np.eye(8), atol=1e-9)
    assert np.allclose(A @ U, U * sig, atol=1e-9 * np.abs(sig).max())


def test_c_client_runs_on_gpu(tmp_path):
    """tests/c_abi_client.c, a plain C99 program, sets up and solves through
    the C ABI on the GPU and exits 0."""
    import shutil

    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    root = os.path.dirname(HERE)
    lib = samg.LIB_PATH
    exe = str(tmp_path / "client")
    cmd = [gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(root, "include"),
           os.path.join(HERE, "c_abi_client.c"), "-o", exe, "-L", os.path.dirname(lib),
           "-l:" + os.path.basename(lib), "-Wl,-rpath," + os.path.dirname(lib)]
    out = subprocess.run(cmd, capture_output=True, text=True)
    assert out.returncode == 0, out.stderr
    run = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    assert run.returncode == 0, (run.stdout, run.stderr)
