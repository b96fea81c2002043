"""Host logic of the exact-order Kaczmarz schedules, on the CPU: the library's
level assignment (samg_sweep_plan, no GPU) against a direct computation of
the dependency levels of the same row program, and the invariants that make
the parallel sweep equal to the sequential one (Sec. 5.3)."""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W

samg = pytest.importorskip("paper_1102_0919_gb300")


def _levels(rows, ncols):
    # level of a row = 1 + the level of the latest earlier row sharing a column
    last = np.full(ncols, -1, dtype=np.int64)
    out = np.empty(len(rows), dtype=np.int64)
    for r, cols in enumerate(rows):
        lv = int(last[cols].max()) + 1 if len(cols) else 0
        out[r] = lv
        last[cols] = lv
    return out


def _rows(M):
    M = M.tocsr()
    return [M.indices[M.indptr[i]:M.indptr[i + 1]] for i in range(M.shape[0])]


def _fused_rows(A, count):
    # per relaxation: rows of A over [v; u] (v columns, then u_i), then rows
    # of A^t (v_j, then u columns)
    m, n = A.shape
    At = A.T.tocsr()
    ra = [np.concatenate([c, [n + i]]) for i, c in enumerate(_rows(A))]
    rt = [np.concatenate([[j], n + c]) for j, c in enumerate(_rows(At))]
    return (ra + rt) * count


@pytest.mark.parametrize("N", [7, 24])
def test_single_sweep_levels(N):
    A = W.gradient(N).to_scipy()
    lv, depth, nb = samg.sweep_plan(A, 0)
    ref = _levels(_rows(A), A.shape[1])
    assert np.array_equal(lv, ref)
    assert depth == ref.max() + 1 and nb >= 1


@pytest.mark.parametrize("count", [1, 2, 4])
def test_fused_program_levels(count):
    A = W.gradient(16).to_scipy()
    m, n = A.shape
    lv, depth, nb = samg.sweep_plan(A, count)
    prog = _fused_rows(A, count)
    ref = _levels(prog, m + n)
    assert len(lv) == len(prog) == count * (m + n)
    assert np.array_equal(lv, ref)
    # rows of one level touch disjoint columns, so they commute
    for l in range(depth):
        cols = np.concatenate([prog[r] for r in np.flatnonzero(lv == l)])
        assert len(cols) == len(np.unique(cols)), l


def test_fused_program_is_far_shallower_than_its_sweeps_in_sequence():
    A = W.gradient(32).to_scipy()
    _, d_a, _ = samg.sweep_plan(A, 0)
    _, d_at, _ = samg.sweep_plan(sp.csr_matrix(A.T), 0)
    _, d4, _ = samg.sweep_plan(A, 4)
    assert d4 * 3 < 4 * (d_a + d_at), (d4, d_a, d_at)


def test_sweep_plan_rejects_malformed_input():
    A = W.gradient(5).to_scipy()
    bad = sp.csr_matrix((A.data, A.indices.copy(), A.indptr), shape=A.shape)
    bad.indices[0] = A.shape[1] + 3  # a column out of range
    with pytest.raises(samg.SamgError):
        samg.sweep_plan(bad, 0)
