"""CPU oracle (FP64) of the self-learning AMG triplet method, arXiv:1102.0919.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the GPU library.  The
oracle and the GPU path share no code; the only common dependency is the
input generator module ``workloads``, which holds no method arithmetic.

Pins (tests/test_oracle_*.py, run with ``-m "not gpu"``):
  * closed-form Dirichlet Laplacian / gradient spectra and the FD columns of
    the paper's Table "values" (Sec. 6.2);
  * dense LAPACK SVD / eigh on tiny inputs;
  * Theorem genSVD (spectrum +-s_j plus |m-n| zeros) and the change of
    variables D = B^-1/2 A C^-1/2 (Sec. 3.2);
  * a hand-computed Ruge-Stueben coarsening, exact LS recovery of a known
    interpolation, Galerkin matvec identities, Kaczmarz projection
    identities, Ritz exactness on exact subspaces, and the additive =
    multiplicative identity of Eq. e;
  * the square SVD forms of Sec. 5.1 (R23) against LAPACK on an upwind
    convection-diffusion operator, and the Sec. 6.3 redo (R22): iterate
    kept, weighted misfit of the favoured vectors not raised.

Parity unpinned: the per-cycle convergence rates of the figures (the
figures are not in the available text) and the setup constants the paper
leaves open (R5-R10, R13-R16 in samg.py) beyond the invariants above.
"""
from .samg import (DEFAULTS, Hierarchy, Level, coarse_geneig, coarsest_pinv_apply,  # noqa: F401
                   coarsest_triplets,
                   dense_XY, fit_interp, galerkin, hierarchy_from_interp, interp_sets, kaczmarz_sweep,
                   kaczmarz_sweep_coloured, colour_order, row_colours,
                   level_residual, random_block, rayleigh, redo_interpolation, relax_boot,
                   relax_test, residual_norms,
                   ritz, rs_coarsen, setup, solve, strength, vcycle)
