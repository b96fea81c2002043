"""The seeded input generators follow their stated recipes (shapes, value
distributions, determinism); they hold no method arithmetic."""
import numpy as np
import scipy.sparse as sp

import oracle
import workloads as W


def test_termdoc_recipe_small():
    A = W.termdoc(2000, 500, seed=123).to_scipy()
    assert A.shape == (2000, 500)
    k = np.diff(A.tocsc().indptr)  # entries per column = distinct rows
    assert k.min() >= 5 and k.max() <= 2000
    # values are fp32(log(1 + tf)) with tf >= 1: log 2 is the smallest
    assert np.all(A.data >= np.float32(np.log(2.0)) - 1e-7)
    assert np.array_equal(A.data, A.data.astype(np.float32).astype(np.float64))
    # Zipf(1.1): small counts dominate
    assert np.median(k) < np.mean(k)
    B = W.termdoc(2000, 500, seed=123).to_scipy()
    assert (A != B).nnz == 0  # deterministic for a seed


def test_aniso_batch_recipe():
    b = W.aniso_batch()
    assert len(b) == 64
    Ns = [N for N, _ in b]
    assert Ns[0] == 64 and Ns[-1] == 512 and all(x <= y for x, y in zip(Ns, Ns[1:]))
    eps = np.array([e for _, e in b])
    assert eps.min() >= 1e-3 and eps.max() <= 1.0
    assert W.aniso_batch() == b


def test_problem_seeds_differ_per_workload():
    seeds = {W.problem_seed(c, p) for c in range(1, 6) for p in range(4)}
    assert len(seeds) == 20


def test_oracle_dominant_triplets_of_a_small_termdoc_match_lapack():
    # the term-document family with the MEDLINE-like setup parameters, small
    # enough for a dense LAPACK SVD (called)
    A = W.termdoc(400, 120, seed=7).to_scipy()
    prm = dict(W.TD_PARAMS, seed=W.problem_seed(4), coarsest_max=40)
    H, s, U, V = oracle.setup(A, 4, "dominant", "svd", prm)
    s, U, V, hist = oracle.solve(H, s, U, V, tol=1e-10, max_outer=80)
    ref = np.sort(np.linalg.svd(A.toarray(), compute_uv=False))[::-1][:4]
    assert hist[-1].max() <= 1e-10
    assert np.allclose(s, ref, rtol=1e-9)
    assert np.allclose(A @ V, U * s, atol=1e-8 * s.max())


def test_oracle_on_the_first_batched_anisotropic_problem():
    # problem 0 of the batched family (N = 64, its own epsilon): the oracle
    # with the FD parameter set reaches the closed-form eigenvalues
    from closed_forms import laplacian5_eigs

    N, e = W.aniso_batch()[0]
    A = W.laplacian5(N, e).to_scipy()
    H, s, U, V = oracle.setup(A, 4, "minimal", "spd", dict(W.FD_PARAMS, seed=W.problem_seed(5, 0)))
    s, U, V, hist = oracle.solve(H, s, U, V, tol=1e-10, max_outer=60)
    assert hist[-1].max() <= 1e-10
    assert np.allclose(s, laplacian5_eigs(N, e)[:4], rtol=1e-12)
    assert np.allclose(A @ U, U * s, atol=1e-9 * s.max())


def test_oracle_guard_pairs_on_the_smallest_gap_batched_problem():
    # problem 7 of the batched family has lambda_5 / lambda_4 = 1.0072; with
    # two guard pairs (n_b = 6, n_conv = 4) the 4 wanted reach the closed form
    from closed_forms import laplacian5_eigs

    N, e = W.aniso_batch()[7]
    A = W.laplacian5(N, e).to_scipy()
    lam = laplacian5_eigs(N, e)
    assert lam[4] / lam[3] < 1.01
    H, s, U, V = oracle.setup(A, 6, "minimal", "spd", dict(W.FD_PARAMS, seed=W.problem_seed(5, 7)))
    s, U, V, hist = oracle.solve(H, s, U, V, tol=1e-10, max_outer=90, n_conv=4)
    assert hist[-1][:4].max() <= 1e-10
    assert np.allclose(s[:4], lam[:4], rtol=1e-12)
