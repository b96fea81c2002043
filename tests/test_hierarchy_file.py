"""Hierarchy files (samg_write_hierarchy / samg_import_file / samg_export):
the host side on the CPU.  The file written from the oracle's hierarchy is
parsed here from its documented layout and compared array by array; damaged
files are rejected before any device call."""
import os

import numpy as np
import pytest

import oracle
import workloads as W

samg = pytest.importorskip("paper_1102_0919_gb300")


def _parse(path):
    """Independent reader of the documented layout."""
    b = open(path, "rb").read()
    assert b[:8] == b"SAMGHIER"
    h = 1469598103934665603
    for x in b[:-8]:
        h = ((h ^ x) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    assert int.from_bytes(b[-8:], "little") == h
    at = 8
    ver, kind, target, nb, nlev = np.frombuffer(b[at:at + 20], "<u4")
    at += 20

    def csr():
        nonlocal at
        m, n = np.frombuffer(b[at:at + 8], "<i4")
        nnz = int(np.frombuffer(b[at + 8:at + 16], "<i8")[0])
        at += 16
        rp = np.frombuffer(b[at:at + 8 * (m + 1)], "<i8"); at += 8 * (m + 1)
        ci = np.frombuffer(b[at:at + 4 * nnz], "<i4"); at += 4 * nnz
        v = np.frombuffer(b[at:at + 8 * nnz], "<f8"); at += 8 * nnz
        return int(m), int(n), rp, ci, v

    def f64(count):
        nonlocal at
        x = np.frombuffer(b[at:at + 8 * count], "<f8")
        at += 8 * count
        return x

    A = csr()
    P, Q = [], []
    for _ in range(nlev - 1):
        P.append(csr())
        if kind == 0:
            Q.append(csr())
    sig = f64(nb)
    U = f64((A[0] if kind == 0 else A[1]) * nb).reshape(-1, nb)
    V = f64(A[1] * nb).reshape(-1, nb) if kind == 0 else None
    assert at == len(b) - 8
    return dict(ver=ver, kind=kind, target=target, nb=nb, nlev=nlev, A=A, P=P, Q=Q, sig=sig, U=U, V=V)


def _same(csr_tuple, M):
    M = M.tocsr()
    M.sort_indices()
    m, n, rp, ci, v = csr_tuple
    return (m, n) == M.shape and np.array_equal(rp, M.indptr) and np.array_equal(ci, M.indices) \
        and np.array_equal(v, M.data)


@pytest.fixture(scope="module")
def hier():
    A = W.gradient(12).to_scipy()
    H, s, U, V = oracle.setup(A, 4, "minimal", "svd", dict(W.GRAD_PARAMS, seed=3, n_mult=3))
    return A, H, s, U, V


def test_written_file_holds_the_hierarchy_as_documented(hier, tmp_path):
    A, H, s, U, V = hier
    path = str(tmp_path / "h.samg")
    Ps = [L.P for L in H.levels[:-1]]
    Qs = [L.Q for L in H.levels[:-1]]
    samg.write_hierarchy(path, A, Ps, Qs, s, U, V, target="minimal", kind="svd")
    d = _parse(path)
    assert (d["ver"], d["kind"], d["target"], d["nb"], d["nlev"]) == (1, samg.SVD, samg.MINIMAL, 4,
                                                                      len(H.levels))
    assert _same(d["A"], A)
    for l in range(len(H.levels) - 1):
        assert _same(d["P"][l], Ps[l]) and _same(d["Q"][l], Qs[l])
    assert np.array_equal(d["sig"], s) and np.array_equal(d["U"], U) and np.array_equal(d["V"], V)


def test_spd_file_has_no_q_or_v(tmp_path):
    A = W.laplacian5(16).to_scipy()
    H, s, U, _ = oracle.setup(A, 4, "minimal", "spd", dict(W.FD_PARAMS, seed=1, n_mult=2))
    path = str(tmp_path / "s.samg")
    samg.write_hierarchy(path, A, [L.P for L in H.levels[:-1]], None, s, U, None, kind="spd")
    d = _parse(path)
    assert d["kind"] == samg.SPD_EIG and d["Q"] == [] and d["V"] is None
    assert np.array_equal(d["U"], U)


def _import_status(path):
    p = samg.make_params()
    ctx = samg._CTX()
    st = samg.samg_import_file(os.fsencode(path), samg.ctypes.byref(p), None, samg.ctypes.byref(ctx))
    assert not ctx.value
    return st, samg.samg_last_error(None).decode()


def test_damaged_files_are_rejected_before_the_device(hier, tmp_path):
    A, H, s, U, V = hier
    good = str(tmp_path / "g.samg")
    samg.write_hierarchy(good, A, [L.P for L in H.levels[:-1]], [L.Q for L in H.levels[:-1]], s, U, V)
    raw = open(good, "rb").read()
    cases = {
        "missing": None,
        "truncated": raw[:len(raw) // 2],
        "flipped byte": raw[:100] + bytes([raw[100] ^ 1]) + raw[101:],
        "not a hierarchy": b"hello" * 20,
        "other version": raw[:8] + (2).to_bytes(4, "little") + raw[12:],
    }
    for name, content in cases.items():
        path = str(tmp_path / ("bad_" + name.replace(" ", "_")))
        if content is not None:
            open(path, "wb").write(content)
        st, msg = _import_status(path)
        assert st == samg.E_INVALID, name
        assert msg.startswith("hierarchy file"), (name, msg)


def test_well_formed_file_reaches_the_device_check(hier, tmp_path):
    try:
        import torch

        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    A, H, s, U, V = hier
    path = str(tmp_path / "ok.samg")
    samg.write_hierarchy(path, A, [L.P for L in H.levels[:-1]], [L.Q for L in H.levels[:-1]], s, U, V)
    st, msg = _import_status(path)
    assert st == samg.E_CUDA and "device" in msg


def test_write_rejects_inconsistent_levels(hier, tmp_path):
    A, H, s, U, V = hier
    Ps = [L.P for L in H.levels[:-1]]
    Qs = [L.Q for L in H.levels[:-1]]
    with pytest.raises(samg.SamgError):            # P_0 with Q_0's rows (n instead of m)
        samg.write_hierarchy(str(tmp_path / "x"), A, [Qs[0]] + Ps[1:], Qs, s, U, V)
    c = samg._csr(A)
    P = (samg._Csr * len(Ps))(*[samg._csr(x) for x in Ps])
    Q = (samg._Csr * len(Qs))(*[samg._csr(x) for x in Qs])
    sg = np.ascontiguousarray(s)
    st = samg.samg_write_hierarchy(os.fsencode(str(tmp_path / "y")), samg.ctypes.byref(c),
                                   len(Ps) + 1, P, Q, 4, samg.MINIMAL, samg.SVD, samg._ptr(sg),
                                   None, None)             # triplets missing
    assert st == samg.E_INVALID
    assert not os.path.exists(str(tmp_path / "x")) and not os.path.exists(str(tmp_path / "y"))
