// kernels.cuh -- launch wrappers of the library's CUDA kernels.
#pragma once

#include "common.cuh"

namespace samg {

// ---------------------------------------------------------------- vec.cu --
// One row-combination pass over a vector block of ld columns:
//   out_i = a0 * in0_i + c1 * s1 o (M1 x1)_i + c2 * s2 o (M2 x2)_i
// where s_t[j] = sigma[j] when sig_t is set (else 1), M_t == identity when
// its row pointer is null, and o is the column-wise product.  TI is the
// arithmetic and input type, TO the output type.
// TI is the storage type of the vectors; the matrix coefficients and the
// arithmetic are Acc<TI>::T (float32 for bfloat16 storage).
template <typename TI>
struct Term {
    CsrView<typename Acc<TI>::T> M{0, 0, nullptr, nullptr, nullptr};
    const TI *x = nullptr;
    double c = 0.0;
    bool sig = false;
};

template <typename TI, typename TO>
void launch_combine(int rows, int ld, const TI *in0, double a0, const Term<TI> &t1,
                    const Term<TI> &t2, const double *sigma, TO *out, cudaStream_t s);

// Weighted-Jacobi block step (Sec. 3.5):
//   out_i = x_i - (omega / d_i) ((B x)_i - ((A y)_i - kappa_i) / sigma)
// B == identity (d = 1) when its row pointer is null; kappa may be null.
template <typename T>
void launch_jacobi(int rows, int ld, CsrView<typename Acc<T>::T> A, const T *y,
                   CsrView<typename Acc<T>::T> B, const typename Acc<T>::T *dB, const T *x,
                   const T *kappa, const double *sigma, double omega, T *out, cudaStream_t s);

template <typename TA, typename TB>
void launch_convert(size_t count, const TA *a, TB *b, cudaStream_t s);

// x += y (elementwise, y converted to float64)
template <typename TY>
void launch_add_to(size_t count, double *x, const TY *y, cudaStream_t s);

// Column-wise x_j^t (M y)_j, accumulated into out[j] (float64, out zeroed by
// the caller); M == identity when its row pointer is null.
template <typename T>
void launch_coldot(int rows, int nb, int ld, const T *x, CsrView<T> M, const T *y, double *out,
                   cudaStream_t s);

// x[:, j] *= scale[j] (scale on the device, ld entries)
template <typename T>
void launch_scale_cols(int rows, int ld, T *x, const double *scale, cudaStream_t s);

// gather rows: out[k, :] = x[idx[k], :] * (colscale ? 1 / colscale[j] : 1)
template <typename T>
void launch_gather_rows(int k, int ld, const int *idx, const T *x, const double *inv_colscale,
                        T *out, cudaStream_t s);

// 1 / sum_k a_ik^2 per row (0 for an all-zero row)
void launch_inv_rownorm2(const DCsr &a, DBuf<double> &outd, DBuf<float> &outf, cudaStream_t s);

// diagonal of a square CSR
void launch_diagonal(const DCsr &a, DBuf<double> &outd, DBuf<float> &outf, cudaStream_t s);

// -------------------------------------------------------- sparse_build.cu --
// C = A B on the device (float64 values; the float32 copy is refreshed).
void spgemm(const DCsr &A, const DCsr &B, DCsr &C, cudaStream_t s);
// C = A^t on the device, rows sorted.
void transpose(const DCsr &A, DCsr &C, cudaStream_t s);
// refresh the float32 copy of the values
void refresh_float(DCsr &A, cudaStream_t s);
// host checks of a caller's CSR (SAMG_E_INVALID): sizes, row_ptr monotone
// from 0 to nnz, columns in range and strictly increasing in a row, finite
// values; no device call
void validate_csr(const samg_csr &h);
// upload / download a host CSR (upload validates first)
void upload_csr(const HCsr &h, DCsr &d, cudaStream_t s);
void upload_csr(const samg_csr &h, DCsr &d, cudaStream_t s);
void download_csr(const DCsr &d, HCsr &h, cudaStream_t s);
// device exclusive scan of n int64 counts into out (n+1 entries)
void exclusive_scan(const int64_t *in, int64_t *out, int n, cudaStream_t s);

// -------------------------------------------------------------- dense.cu --
// G (nb x nb, row-major, device) = X^t Y over rows, deterministic two-stage
// reduction using the caller's workspace of gram_workspace(rows, nb) doubles.
size_t gram_workspace(int64_t rows, int nb);
void launch_gram(const double *X, const double *Y, int64_t rows, int nb, int ld, double *G,
                 double *work, cudaStream_t s);

}  // namespace samg
