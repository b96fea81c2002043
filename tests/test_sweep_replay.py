"""The exact-order sweep schedules the kernels receive, replayed on the CPU
(tests/sweep_replay.py) against the oracle's sequential Kaczmarz sweeps:
single sweeps and fused block Gauss-Seidel relaxation programs, on operators
whose schedules span many bands, chunks and cross-band requirements.  The
replay runs the bands in the most eager order the recorded requirements
allow, so a missing requirement reads a stale value."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import workloads as W
from sweep_replay import check_claim_order, claim_model, parse, replay

samg = pytest.importorskip("paper_1102_0919_gb300")


def _rand_rect(m, n, seed, dens=0.02):
    rng = np.random.default_rng(seed)
    R = sp.random(m, n, density=dens, random_state=rng, format="csr")
    # a few long rows (more than 32 entries) and no empty row
    for i in rng.choice(m, 3, replace=False):
        R[i, rng.choice(n, 40, replace=False)] = 1.0
    R = R + sp.csr_matrix((np.ones(m), (np.arange(m), np.arange(m) % n)), shape=(m, n))
    R = sp.csr_matrix(R)
    R.sort_indices()
    return R


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("name", ["gradient48", "laplacian40", "random"])
def test_single_sweep_schedule_replays_the_sequential_sweep(name):
    A = {"gradient48": lambda: W.gradient(48).to_scipy(),
         "laplacian40": lambda: W.laplacian5(40).to_scipy(),
         "random": lambda: _rand_rect(3000, 1200, 5)}[name]()
    A = oracle.samg._csr(A)
    S = parse(samg.sweep_schedule(A, 0))
    assert S["mode"] == 0 and S["rows"] == A.shape[0]
    rng = np.random.default_rng(1)
    X = rng.standard_normal((A.shape[1], 8))
    rhs = rng.standard_normal((A.shape[0], 8))
    got = replay(S, X.copy(), rhs)
    ref = X.copy()
    oracle.kaczmarz_sweep(A, ref, rhs)
    assert rel(got, ref) < 1e-11, rel(got, ref)


# (256, 4) is the bench workload's level-0 smoothing program (49 bands)
@pytest.mark.parametrize("N,count", [(32, 1), (32, 4), (96, 4), (256, 4)])
def test_fused_relaxation_schedule_replays_block_gauss_seidel(N, count):
    A = W.gradient(N).to_scipy()
    m, n = A.shape
    S = parse(samg.sweep_schedule(A, count))
    assert S["mode"] == 2 and S["rows"] == count * (m + n)
    if N == 96:
        assert S["nbands"] >= 8 and len(S["req"]) >= 8     # many bands and requirements
    rng = np.random.default_rng(N + count)
    sig = np.linspace(3.0, 9.0, 8)
    U = rng.standard_normal((m, 8))
    V = rng.standard_normal((n, 8))
    K = rng.standard_normal((m, 8))
    T = rng.standard_normal((n, 8))
    z = replay(S, np.vstack([V, U]), np.vstack([K, T]), sig)
    L0 = oracle.Level(A, sp.identity(m, format="csr"), sp.identity(n, format="csr"))
    Ur, Vr = U.copy(), V.copy()
    for _ in range(count):
        oracle.relax_boot(L0, False, "minimal", sig, Ur, Vr, K, T, 0.7)
    assert rel(z[:n], Vr) < 1e-10, rel(z[:n], Vr)
    assert rel(z[n:], Ur) < 1e-10, rel(z[n:], Ur)


def test_fused_schedule_of_a_random_operator():
    A = _rand_rect(1500, 700, 9, dens=0.01)
    m, n = A.shape
    S = parse(samg.sweep_schedule(A, 2))
    rng = np.random.default_rng(3)
    sig = np.linspace(0.5, 2.0, 4)
    U, V = rng.standard_normal((m, 4)), rng.standard_normal((n, 4))
    K, T = rng.standard_normal((m, 4)), rng.standard_normal((n, 4))
    z = replay(S, np.vstack([V, U]), np.vstack([K, T]), sig)
    L0 = oracle.Level(A, sp.identity(m, format="csr"), sp.identity(n, format="csr"))
    Ur, Vr = U.copy(), V.copy()
    for _ in range(2):
        oracle.relax_boot(L0, False, "minimal", sig, Ur, Vr, K, T, 0.7)
    assert rel(z[:n], Vr) < 1e-10 and rel(z[n:], Ur) < 1e-10


@pytest.mark.parametrize("count", [1, 4])
def test_stacked_spd_schedule_replays_shifted_sweeps(count):
    # SPD kind: stacked sweeps over the rows of A - lambda_j I (norms per
    # column), as the oracle's shifted Kaczmarz relaxation
    A = oracle.samg._csr(W.laplacian5(40, 0.3).to_scipy())
    n = A.shape[0]
    S = parse(samg.sweep_schedule(A, count, spd=True))
    assert S["mode"] == 1 and S["rows"] == count * n
    rng = np.random.default_rng(count)
    lam = np.linspace(5.0, 60.0, 8)
    U = rng.standard_normal((n, 8))
    K = rng.standard_normal((n, 8))
    got = replay(S, U.copy(), K, lam)
    L0 = oracle.Level(A, sp.identity(n, format="csr"))
    ref = U.copy()
    for _ in range(count):
        oracle.relax_boot(L0, True, "minimal", lam, ref, None, K, None, 0.7)
    assert rel(got, ref) < 1e-10, rel(got, ref)


def test_replay_detects_a_dropped_requirement():
    # the replay is only evidence if it can fail: remove every cross-band
    # requirement of a multi-band schedule and the eager band order must
    # produce a different (stale) result
    A = W.gradient(96).to_scipy()
    m, n = A.shape
    S = parse(samg.sweep_schedule(A, 4))
    lvl = S["lvl"].copy()
    lvl[:, 1] = 0
    S["lvl"] = lvl
    rng = np.random.default_rng(2)
    z0 = rng.standard_normal((n + m, 8))
    rhs = rng.standard_normal((m + n, 8))
    with pytest.raises(AssertionError):
        z = replay(S, z0.copy(), rhs, np.linspace(3.0, 9.0, 8))
        good = replay(parse(samg.sweep_schedule(A, 4)), z0.copy(), rhs, np.linspace(3.0, 9.0, 8))
        assert rel(z, good) < 1e-12


@pytest.mark.parametrize("kind", ["svd", "spd"])
def test_coarse_level_programs_with_galerkin_b_and_c(kind):
    # the smoothing programs of coarse levels, where B and C are Galerkin
    # products (not the identity): taken from an oracle hierarchy
    if kind == "svd":
        A = W.gradient(40).to_scipy()
        H, s, U, V = oracle.setup(A, 8, "minimal", "svd", dict(W.GRAD_PARAMS, seed=4, n_mult=2))
    else:
        A = W.laplacian5(48, 0.4).to_scipy()
        H, s, U, V = oracle.setup(A, 4, "minimal", "spd", dict(W.FD_PARAMS, seed=4, n_mult=2))
    assert len(H.levels) >= 3
    L = H.levels[1]
    nb = len(s)
    rng = np.random.default_rng(6)
    sig = np.abs(s) * (1 + 0.01 * rng.standard_normal(nb))
    for count in (1, 3):
        if kind == "svd":
            m, n = L.A.shape
            S = parse(samg.sweep_schedule(L.A, count, B=L.B, C=L.C))
            Uc, Vc = rng.standard_normal((m, nb)), rng.standard_normal((n, nb))
            K, T = rng.standard_normal((m, nb)), rng.standard_normal((n, nb))
            z = replay(S, np.vstack([Vc, Uc]), np.vstack([K, T]), sig)
            Ur, Vr = Uc.copy(), Vc.copy()
            for _ in range(count):
                oracle.relax_boot(L, False, "minimal", sig, Ur, Vr, K, T, 0.7)
            assert rel(z[:n], Vr) < 1e-10 and rel(z[n:], Ur) < 1e-10, (rel(z[:n], Vr), rel(z[n:], Ur))
        else:
            n = L.A.shape[0]
            S = parse(samg.sweep_schedule(L.A, count, spd=True, B=L.B))
            Uc, K = rng.standard_normal((n, nb)), rng.standard_normal((n, nb))
            got = replay(S, Uc.copy(), K, sig)
            ref = Uc.copy()
            for _ in range(count):
                oracle.relax_boot(L, True, "minimal", sig, ref, None, K, None, 0.7)
            assert rel(got, ref) < 1e-10, rel(got, ref)


@pytest.mark.parametrize("band_rows,slot_cap", [(8, 0), (128, 0), (128, 2700), (512, 64)])
def test_bands_of_other_widths_replay_block_gauss_seidel(band_rows, slot_cap):
    # the bands' rows per level (samg_set_sweep_banding) and window size
    # change the schedule only: narrower bands (8 rows per level), wider ones
    # (more rows per level, longer sub-level lists, more live columns) and a
    # small window (64 columns, which stops a band's growth early) replay the
    # same relaxations
    A = W.gradient(96).to_scipy()
    m, n = A.shape
    count = 4
    plain = parse(samg.sweep_schedule(A, count))
    S = parse(samg.sweep_schedule(A, count, band_rows=band_rows, slot_cap=slot_cap))
    if band_rows < 32:
        assert S["nbands"] > plain["nbands"], (S["nbands"], plain["nbands"])
    elif slot_cap != 64:
        assert S["nbands"] < plain["nbands"], (S["nbands"], plain["nbands"])
    else:
        assert S["nbands"] > plain["nbands"], (S["nbands"], plain["nbands"])
    rng = np.random.default_rng(band_rows + slot_cap)
    sig = np.linspace(3.0, 9.0, 8)
    U, V = rng.standard_normal((m, 8)), rng.standard_normal((n, 8))
    K, T = rng.standard_normal((m, 8)), rng.standard_normal((n, 8))
    z = replay(S, np.vstack([V, U]), np.vstack([K, T]), sig)
    L0 = oracle.Level(A, sp.identity(m, format="csr"), sp.identity(n, format="csr"))
    Ur, Vr = U.copy(), V.copy()
    for _ in range(count):
        oracle.relax_boot(L0, False, "minimal", sig, Ur, Vr, K, T, 0.7)
    assert rel(z[:n], Vr) < 1e-10 and rel(z[n:], Ur) < 1e-10


def test_widened_bands_on_a_galerkin_level():
    A = W.gradient(40).to_scipy()
    H, s, U, V = oracle.setup(A, 8, "minimal", "svd", dict(W.GRAD_PARAMS, seed=4, n_mult=2))
    L = H.levels[1]
    m, n = L.A.shape
    nb = len(s)
    rng = np.random.default_rng(8)
    sig = np.abs(s) * (1 + 0.01 * rng.standard_normal(nb))
    S = parse(samg.sweep_schedule(L.A, 3, B=L.B, C=L.C, band_rows=512, slot_cap=2700))
    Uc, Vc = rng.standard_normal((m, nb)), rng.standard_normal((n, nb))
    K, T = rng.standard_normal((m, nb)), rng.standard_normal((n, nb))
    z = replay(S, np.vstack([Vc, Uc]), np.vstack([K, T]), sig)
    Ur, Vr = Uc.copy(), Vc.copy()
    for _ in range(3):
        oracle.relax_boot(L, False, "minimal", sig, Ur, Vr, K, T, 0.7)
    assert rel(z[:n], Vr) < 1e-10 and rel(z[n:], Ur) < 1e-10


def _nine_point(N):
    I = sp.identity(N, format="csr")
    T = sp.diags([np.full(N - 1, -1.0), np.full(N, 4.0), np.full(N - 1, -1.0)], [-1, 0, 1])
    E = sp.diags([np.ones(N - 1), np.ones(N), np.ones(N - 1)], [-1, 0, 1])
    return sp.csr_matrix(sp.kron(I, T) - 0.5 * sp.kron(sp.diags([np.ones(N - 1), np.ones(N - 1)],
                                                                [-1, 1]), E))


@pytest.mark.parametrize("name", ["gradient96", "nine_point80", "random", "galerkin"])
def test_claim_order_is_safe_for_any_cta_count(name):
    # the CTAs claim bands in the schedule's ticket order; every band's
    # required bands must hold earlier tickets, so that a run on any number
    # of CTAs finishes (a later band never holds the last free CTA while an
    # earlier one it waits for is unclaimed)
    if name == "gradient96":
        S = parse(samg.sweep_schedule(W.gradient(96).to_scipy(), 4, band_rows=8))
    elif name == "nine_point80":
        S = parse(samg.sweep_schedule(_nine_point(80), 4, band_rows=8))
        # a 2-D stencil: the rows of later lines start late, so the order
        # moves the next relaxation's first bands ahead of them
        assert list(S["order"]) != list(range(S["nbands"]))
    elif name == "random":
        S = parse(samg.sweep_schedule(_rand_rect(1500, 700, 9, dens=0.01), 2))
    else:
        A = W.gradient(40).to_scipy()
        H, s, U, V = oracle.setup(A, 8, "minimal", "svd", dict(W.GRAD_PARAMS, seed=4, n_mult=2))
        L = H.levels[1]
        S = parse(samg.sweep_schedule(L.A, 3, B=L.B, C=L.C, band_rows=8))
    assert S["nbands"] >= 4
    for ctas in (1, 2, 5, S["nbands"]):
        check_claim_order(S, ctas)


def test_claim_order_keeps_the_relaxations_wavefronts_resident():
    # with more bands than CTAs (here 3 per CTA, as on the coarse levels of
    # the 1024^2 gradient: about 500 bands on 152 SMs), program order makes
    # CTAs hold the bands of a sweep's last lines, which the wavefront
    # reaches late, while the next relaxation's first bands wait; in a model
    # of the claims (unit levels, handoffs of two) the schedule's own order
    # finishes at least a quarter sooner, and with a CTA per band both equal
    # the unlimited time
    S = parse(samg.sweep_schedule(_nine_point(120), 4, band_rows=4))
    nb = S["nbands"]
    assert nb >= 60
    ctas = nb // 3
    prog = claim_model(S, ctas, order=range(nb))
    mine = claim_model(S, ctas)
    free = claim_model(S, nb)
    assert mine <= 0.75 * prog, (mine, prog, free)
    assert claim_model(S, nb, order=range(nb)) == free <= mine


@pytest.mark.parametrize("spd", [False, True])
def test_no_band_crosses_a_sweep_of_a_fused_program(spd):
    # the next relaxation's first bands must depend only on the first bands
    # of the one before (the claim order relies on it): every band's rows
    # lie inside one sweep of the program (rows of A or of A^t of one
    # relaxation; one stacked sweep of the SPD kind)
    if spd:
        A = W.laplacian5(60, 0.3).to_scipy()
        count = 3
        S = parse(samg.sweep_schedule(A, count, spd=True, band_rows=8))
        seg = [k * A.shape[0] for k in range(1, count)]
    else:
        A = W.gradient(64).to_scipy()
        m, n = A.shape
        count = 3
        S = parse(samg.sweep_schedule(A, count, band_rows=8))
        seg = sorted({k * (m + n) for k in range(1, count)} | {k * (m + n) + m for k in range(count)})
    assert S["nbands"] > count
    # program rows of each band, from the images' row records: right-hand
    # side rows repeat per relaxation, so rebuild program rows from the
    # band's position in program order (bands are contiguous row ranges)
    starts = []
    row = 0
    bc = S["band_chunk"]
    for b in range(S["nbands"]):
        starts.append(row)
        for c in range(bc[b], bc[b + 1]):
            row += S["chunks"][c]["nr"]
    starts.append(row)
    assert row == S["rows"]
    for b in range(S["nbands"]):
        lo, hi = starts[b], starts[b + 1]
        assert not any(lo < x < hi for x in seg), (b, lo, hi)


def test_schedules_do_not_depend_on_the_host_thread_count(monkeypatch):
    # the builder analyses and writes bands on several host threads; every
    # ordering step is sequential, so one thread and several give the same
    # bytes (fused program with Galerkin-like 2-D rows, single sweep, SPD)
    import hashlib
    cases = [(_nine_point(70), 4, {}), (W.gradient(80).to_scipy(), 0, {}),
             (oracle.samg._csr(W.laplacian5(30, 0.3).to_scipy()), 2, {"spd": True})]
    for A, count, kw in cases:
        digests = []
        for threads in ("1", "3", "8"):
            monkeypatch.setenv("SAMG_HOST_THREADS", threads)
            digests.append(hashlib.sha256(samg.sweep_schedule(A, count, band_rows=8, **kw)).hexdigest())
        assert len(set(digests)) == 1, digests


def test_empty_rows_and_a_single_row():
    # rows without entries leave x unchanged; a one-row program is one level
    A = sp.csr_matrix(np.array([[0.0, 0.0, 0.0], [1.0, -2.0, 0.0], [0.0, 0.0, 0.0],
                                [0.0, 3.0, 1.0]]))
    S = parse(samg.sweep_schedule(A, 0))
    rng = np.random.default_rng(0)
    X = rng.standard_normal((3, 4))
    rhs = rng.standard_normal((4, 4))
    got = replay(S, X.copy(), rhs)
    ref = X.copy()
    oracle.kaczmarz_sweep(oracle.samg._csr(A), ref, rhs)
    assert rel(got, ref) < 1e-14
    one = sp.csr_matrix(np.array([[2.0, 0.0, -1.0]]))
    S1 = parse(samg.sweep_schedule(one, 0))
    assert S1["nbands"] == 1 and len(S1["lvl"]) == 1


def test_row_longer_than_a_staging_chunk_is_rejected():
    # a chunk holds at most 1024 entries; a longer row is an input error,
    # reported before any device work
    n = 1100
    A = sp.csr_matrix((np.ones(n), (np.zeros(n, dtype=int), np.arange(n))), shape=(1, n))
    with pytest.raises(samg.SamgError) as e:
        samg.sweep_schedule(A, 0)
    assert e.value.status == samg.E_INVALID and "staging chunk" in str(e.value)


def test_resident_band_mode_on_coarse_levels():
    # optional mode: a coarse level whose program keeps at most 4095 columns
    # live is one band with every column resident; all first touches are
    # then staged ahead (no global reads at compute time, no requirements),
    # and the replay still matches the oracle's relaxations
    A = W.gradient(64).to_scipy()
    H, s, U, V = oracle.setup(A, 8, "minimal", "svd", dict(W.GRAD_PARAMS, seed=4, n_mult=2))
    L = H.levels[3]
    m, n = L.A.shape
    assert m + n <= 4095
    base = parse(samg.sweep_schedule(L.A, 4, B=L.B, C=L.C))
    S = parse(samg.sweep_schedule(L.A, 4, B=L.B, C=L.C, resident_slots=4095))
    assert base["nbands"] > 1 and S["nbands"] == 1
    assert S["lvl"][:, 1].sum() == 0                      # no cross-band requirement
    from sweep_replay import _image
    for c in range(len(S["chunks"])):
        fl = _image(S, c)["ent"][:, 1]
        assert not np.any(((fl & 1) != 0) & ((fl & 4) == 0))   # every first touch staged
    rng = np.random.default_rng(8)
    sig = np.abs(s) * 1.01
    Uc, Vc = rng.standard_normal((m, 8)), rng.standard_normal((n, 8))
    K, T = rng.standard_normal((m, 8)), rng.standard_normal((n, 8))
    z = replay(S, np.vstack([Vc, Uc]), np.vstack([K, T]), sig)
    Ur, Vr = Uc.copy(), Vc.copy()
    for _ in range(4):
        oracle.relax_boot(L, False, "minimal", sig, Ur, Vr, K, T, 0.7)
    assert rel(z[:n], Vr) < 1e-10 and rel(z[n:], Ur) < 1e-10
    # a program with more live columns than the cap keeps the usual bands
    big = parse(samg.sweep_schedule(A, 4, resident_slots=64))
    assert big["nbands"] == parse(samg.sweep_schedule(A, 4))["nbands"]
