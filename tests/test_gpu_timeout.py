"""The bounded device waits of the Kaczmarz sweep, exercised without a GPU
fault: one band of a multi-band sweep is told never to publish its progress
(a flag that nothing sets), so the later bands that need it give up after
their 2 s bound.  The call must return SAMG_E_TIMEOUT, the context must
refuse further work, and a fresh context on the same GPU must run normally."""
import time

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

samg = pytest.importorskip("paper_1102_0919_gb300")

TIMEOUT = 6


def _context(A, P, Q, nb, rng):
    m, n = A.shape
    sig = np.linspace(5.0, 11.0, nb)
    U = rng.standard_normal((m, nb))
    V = rng.standard_normal((n, nb))
    g = samg.Solver.from_hierarchy(A, [P], [Q], nb, sig, U, V, "minimal", "svd", prec="fp64",
                                   mu_b=1)
    return g, sig, U, V


def test_cross_band_wait_times_out_and_the_gpu_stays_usable():
    # the 256 x 256 gradient: its sweep over the rows of A spans several bands,
    # and every band after the first needs the progress of the one before it
    A = W.gradient(256).to_scipy()
    m, n = A.shape
    nb = 8
    P = sp.csr_matrix((np.ones(m), (np.arange(m), np.minimum(np.arange(m) // 1400, 93))),
                      shape=(m, 94))
    Q = sp.csr_matrix((np.ones(n), (np.arange(n), np.minimum(np.arange(n) // 730, 89))),
                      shape=(n, 90))
    rng = np.random.default_rng(5)
    g, sig, U, V = _context(A, P, Q, nb, rng)
    K = rng.standard_normal(U.shape)
    T = rng.standard_normal(V.shape)
    g.relax(0, sig, U, V, K, T, count=1)  # publishes normally
    g.debug_mute_band(0, 2, 0)  # the fused relaxation program the call above built
    t0 = time.time()
    with pytest.raises(samg.SamgError) as err:
        g.relax(0, sig, U, V, K, T, count=1)
    dt = time.time() - t0
    assert err.value.status == TIMEOUT, err.value
    assert 1.5 < dt < 60.0, dt
    with pytest.raises(samg.SamgError):  # poisoned
        g.relax(0, sig, U, V, K, T, count=1)
    g.close()
    # a fresh context on the same device: the sweep runs and matches the oracle
    g2, sig, U, V = _context(A, P, Q, nb, np.random.default_rng(6))
    Ug, Vg = g2.relax(0, sig, U, V, K, T, count=1)
    g2.close()
    L0 = oracle.Level(A, sp.identity(m, format="csr"), sp.identity(n, format="csr"))
    Ur, Vr = U.copy(), V.copy()
    oracle.relax_boot(L0, False, "minimal", sig, Ur, Vr, K, T, 0.7)
    assert np.abs(Vg - Vr).max() <= 1e-10 * np.abs(Vr).max()
    assert np.abs(Ug - Ur).max() <= 1e-10 * np.abs(Ur).max()
