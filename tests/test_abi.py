"""The C-ABI library loads and exports every entry point that include/samg.h
declares (no GPU needed; no compute calls)."""
import ctypes
import os
import re

import pytest


@pytest.fixture(scope="module")
def lib(repo_root):
    import importlib.util

    spec = importlib.util.spec_from_file_location(
        "_samg_build", os.path.join(repo_root, "paper_1102_0919_gb300", "build.py"))
    libbuild = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(libbuild)
    path = libbuild.build()
    return ctypes.CDLL(path), path


def declared(repo_root):
    hdr = open(os.path.join(repo_root, "include", "samg.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(samg_[a-z_0-9]+)\s*\(", hdr)))


def test_header_declares_the_boundary(repo_root):
    names = declared(repo_root)
    for need in ("samg_setup", "samg_solve", "samg_get_triplets", "samg_import", "samg_destroy",
                 "samg_last_error", "samg_default_params"):
        assert need in names


def test_library_exports_every_declared_symbol(lib, repo_root):
    so, path = lib
    for name in declared(repo_root):
        assert hasattr(so, name), name


def test_binding_covers_every_declared_symbol(lib, repo_root):
    import paper_1102_0919_gb300 as samg

    assert sorted(samg.EXPORTED) == declared(repo_root)


def test_default_params_and_null_handling(lib):
    import paper_1102_0919_gb300 as samg

    p = samg.make_params()
    assert p.n_t == 8 and abs(p.theta - 0.06) < 1e-15 and p.mu_b == 4
    assert abs(p.omega_J - 0.7) < 1e-15 and p.prec == samg.FP32 and p.n_conv == 0
    # argument errors are reported without touching a GPU
    assert samg.samg_solve(None, 1e-8, 1, None) == samg.E_INVALID
    assert samg.samg_setup(None, 4, 1, 0, None, None, None) == samg.E_INVALID


def test_header_serves_a_plain_c_client(lib, repo_root, tmp_path):
    # the header compiles as C99 with warnings as errors, a client links
    # against the library, and without a GPU the library says so (status
    # SAMG_E_CUDA, exit 2) instead of computing anywhere else
    import shutil
    import subprocess

    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    so, path = lib
    exe = str(tmp_path / "client")
    cmd = [gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(repo_root, "include"),
           os.path.join(repo_root, "tests", "c_abi_client.c"), "-o", exe,
           "-L", os.path.dirname(path), "-l:" + os.path.basename(path),
           "-Wl,-rpath," + os.path.dirname(path)]
    out = subprocess.run(cmd, capture_output=True, text=True)
    assert out.returncode == 0, out.stderr
    run = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    # the binding's parameter struct has the header's layout
    import paper_1102_0919_gb300 as samg

    head = run.stdout.split()
    assert head[:1] == ["sizeof(samg_params)"], run.stdout
    assert int(head[1]) == ctypes.sizeof(samg.Params)
    assert int(head[3]) == samg.Params.n_conv.offset
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except ImportError:
        has_gpu = False
    if has_gpu:
        assert run.returncode == 0, run.stderr
    else:
        assert run.returncode == 2, (run.returncode, run.stderr)


def _lap(N=12):
    import scipy.sparse as sp

    T = sp.diags([-1.0, 2.0, -1.0], [-1, 0, 1], shape=(N, N))
    return sp.csr_matrix(sp.kron(sp.identity(N), T) + sp.kron(T, sp.identity(N)))


class _RawCsr:
    """A CSR given by its raw arrays (possibly malformed on purpose)."""

    def __init__(self, m, n, rp, ci, v):
        import numpy as np

        self.m, self.n = m, n
        self.row_ptr = np.asarray(rp, dtype=np.int64)
        self.col = np.asarray(ci, dtype=np.int32)
        self.val = np.asarray(v, dtype=np.float64)


def _setup_status(samg, A, nb=2, target=1, kind=1, **params):
    c = samg._csr(A)
    if isinstance(A, _RawCsr):      # keep nnz as given by row_ptr's last entry
        c.nnz = int(A.row_ptr[-1])
    p = samg.make_params(**params)
    ctx = samg._CTX()
    st = samg.samg_setup(ctypes.byref(c), nb, target, kind, ctypes.byref(p), None, ctypes.byref(ctx))
    assert not ctx.value                  # no context on failure
    return st


def test_argument_errors_are_reported_before_any_device_call(lib):
    # Every argument check of samg_setup / samg_import / the no-alloc Gram
    # runs on the host before the device is touched, so these statuses are
    # the same with or without a GPU (no compute call is made).
    import numpy as np

    import paper_1102_0919_gb300 as samg

    A = _lap()
    good = _RawCsr(A.shape[0], A.shape[1], A.indptr, A.indices, A.data)
    assert _setup_status(samg, good, nb=0) == samg.E_INVALID
    assert _setup_status(samg, good, nb=17) == samg.E_INVALID
    assert _setup_status(samg, good, kind=7) == samg.E_INVALID
    assert _setup_status(samg, good, target=9) == samg.E_INVALID
    assert _setup_status(samg, good, n_t=0, nb=1) == samg.E_NT_TOO_SMALL
    assert _setup_status(samg, good, n_t=17) == samg.E_INVALID
    assert _setup_status(samg, good, prec=5) == samg.E_INVALID
    rect = _RawCsr(3, 2, [0, 1, 2, 3], [0, 1, 1], [1.0, 1.0, 1.0])
    assert _setup_status(samg, rect, nb=1, kind=samg.SPD_EIG) == samg.E_INVALID
    assert _setup_status(samg, rect, nb=3, kind=samg.SVD) == samg.E_INVALID   # n_b > min(m, n)
    # malformed CSR
    rp, ci, v = A.indptr.copy(), A.indices.copy(), A.data.copy()
    bad_rp = rp.copy()
    bad_rp[1] = rp[-1] + 50                          # a row running past nnz
    cases = {
        "row past nnz": (bad_rp, ci, v),
        "decreasing row_ptr": (np.r_[rp[:3], rp[1], rp[4:]], ci, v),
        "unsorted columns": (rp, np.r_[ci[1], ci[0], ci[2:]], v),
        "column out of range": (rp, np.r_[ci[:-1], A.shape[1]], v),
        "NaN value": (rp, ci, np.r_[v[:-1], np.nan]),
    }
    for name, (r, c, x) in cases.items():
        st = _setup_status(samg, _RawCsr(A.shape[0], A.shape[1], r, c, x))
        assert st == samg.E_INVALID, name
        assert samg.samg_last_error(None).decode().startswith("csr:"), name
    # import: P with the wrong number of rows
    c = samg._csr(A)
    P = samg._csr(_RawCsr(A.shape[0] - 1, 4, np.zeros(A.shape[0], np.int64), [], []))
    p = samg.make_params()
    ctx = samg._CTX()
    st = samg.samg_import(ctypes.byref(c), 2, ctypes.byref(P), None, 2, samg.MINIMAL, samg.SPD_EIG,
                          ctypes.byref(p), None, None, None, None, ctypes.byref(ctx))
    assert st == samg.E_INVALID and not ctx.value
    # the no-alloc Gram rejects sizes beyond its fixed scratch (no pointer is used)
    fake = ctypes.c_void_p(256)
    assert samg.samg_block_gram_noalloc(fake, fake, 1 << 40, 8, 8, fake, None) == samg.E_INVALID


def test_well_formed_setup_without_a_gpu_reports_the_device(lib):
    import paper_1102_0919_gb300 as samg

    try:
        import torch

        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    st = _setup_status(samg, _lap())
    assert st == samg.E_CUDA
    assert "device" in samg.samg_last_error(None).decode()


def test_batched_setup_checks_every_problem_before_the_device(lib):
    import paper_1102_0919_gb300 as samg

    good = [_lap(6), _lap(8), _lap(5)]
    A = _lap(7)
    bad = _RawCsr(A.shape[0], A.shape[1], A.indptr, A.indices, A.data.copy())
    bad.val[3] = float("nan")
    with pytest.raises(samg.SamgError) as e:
        samg.Batch.setup(good + [bad], 2, "minimal", "spd")
    assert e.value.status == samg.E_INVALID and "problem 3" in str(e.value)
    rect = _RawCsr(3, 2, [0, 1, 2, 3], [0, 1, 1], [1.0, 1.0, 1.0])
    with pytest.raises(samg.SamgError) as e:
        samg.Batch.setup([good[0], rect], 2, "minimal", "spd")
    assert e.value.status == samg.E_INVALID and "problem 1" in str(e.value)
    with pytest.raises(samg.SamgError) as e:
        samg.Batch.setup([], 2, "minimal", "spd")
    assert e.value.status == samg.E_INVALID
    assert samg.samg_solve_batched(None, 1e-8, 1, None) == samg.E_INVALID
    assert samg.samg_batch_size(None) == 0


def test_batched_setup_without_a_gpu_reports_the_device(lib):
    import paper_1102_0919_gb300 as samg

    try:
        import torch

        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    with pytest.raises(samg.SamgError) as e:
        samg.Batch.setup([_lap(6), _lap(8)], 2, "minimal", "spd")
    assert e.value.status == samg.E_CUDA and "problem 0" in str(e.value)
