// dense.cuh -- float64 dense kernels: Ritz step (Sec. 4.3) and coarsest level.
#pragma once

#include "common.cuh"

namespace samg {

// Small Ritz problem (n_b <= 16) on one thread: Cholesky of the Gram
// matrices, M = R_U^-t (U^t A V) R_V^-1, its SVD (SPD: eigendecomposition),
// ordering, TU = R_U^-1 Y, TV = R_V^-1 Z.  status[0] = 1 if a Gram matrix is
// not positive definite.
void launch_ritz_small(const double *GU, const double *GV, const double *H, int nb, int ld,
                       bool spd, bool dominant, double *sigma, double *TU, double *TV,
                       int *status, cudaStream_t s);

// Xn = X T (rows x ld), and per-chunk partial sums of |W T2 - sigma o Xn|^2.
void launch_ritz_update(const double *X, const double *W, const double *T, const double *T2,
                        const double *sigma, int64_t rows, int nb, int ld, double *Xn,
                        double *part, cudaStream_t s);
// resid_j = sqrt(sum of both sides' partials) / |sigma_j|
void launch_ritz_resid(const double *pu, int64_t rows_u, const double *pv, int64_t rows_v,
                       int nb, const double *sigma, double *resid, cudaStream_t s);

// Dense scatter of a CSR block into an M x M row-major matrix at (r_off, c_off).
void dense_fill(const DCsr &a, int r_off, int c_off, int Mdim, double *D, bool transpose,
                cudaStream_t s);

// Generalized eigendecomposition X W = Y W Lam, W^t Y W = I (one CTA).
void launch_coarse_geneig(int M, const double *X, const double *Y, double *work, double *lam,
                          double *W, double *Wt, int *status, cudaStream_t s);

// Pseudo-inverse solve of (X - sigma_j Y) without its smallest singular value,
// one CTA per column (Sec. 4.2).  qwarm (coarse_warm_size doubles) keeps each
// column's subspace-iteration basis between calls; warm = 0 starts afresh.
template <typename T>
void launch_coarse_apply(int M, int m1, int ld, int nb, const double *lam, const double *W,
                         const double *Wt, const double *sigma, const T *k1, const T *k2, T *o1,
                         T *o2, double *qwarm, int warm, cudaStream_t s);
size_t coarse_warm_size(int M, int nb);

// The generalized-eigen variant of the coarsest solve (coarse_pinv = 1):
// z_j = sum over k != k*_j of w_k (w_k^t r_j) / (lam_k - s_j), k*_j the lam_k
// nearest s_j (ties: lowest k).  Two passes, each one warp per output row
// over all columns: c = D_j W^t r (into cbuf, M x ld float64), z = W c.
template <typename T>
void launch_coarse_apply_geneig(int M, int m1, int ld, int nb, const double *lam,
                                const double *W, const double *Wt, const double *sigma,
                                const T *k1, const T *k2, T *o1, T *o2, double *cbuf,
                                cudaStream_t s);

}  // namespace samg
