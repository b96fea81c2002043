// vec.cu -- block sparse-matrix x vector-block kernels of the V-cycle:
// residual (Eq. add), restriction (Eq. addCoarse), interpolation + correction
// (Eq. corrAdd), right-hand sides of the Kaczmarz blocks (Eqs.
// genSVDresid1-2) and the weighted-Jacobi block step (Sec. 3.5).
//
// Vector blocks are row-interleaved: entry (i, j) at x[i * ld + j], ld a
// multiple of 4, so one thread handles one row and 4 consecutive columns with
// one 16-byte (float32) or 32-byte (float64) load per nonzero.
#include "kernels.cuh"

namespace samg {

template <typename T> struct V4 { T a[4]; };

__device__ __forceinline__ V4<float> ld4(const float *p) {
    float4 v = *reinterpret_cast<const float4 *>(p);
    return V4<float>{{v.x, v.y, v.z, v.w}};
}
__device__ __forceinline__ V4<double> ld4(const double *p) {
    double2 u = reinterpret_cast<const double2 *>(p)[0];
    double2 w = reinterpret_cast<const double2 *>(p)[1];
    return V4<double>{{u.x, u.y, w.x, w.y}};
}
__device__ __forceinline__ void st4(float *p, const V4<float> &v) {
    *reinterpret_cast<float4 *>(p) = make_float4(v.a[0], v.a[1], v.a[2], v.a[3]);
}
__device__ __forceinline__ void st4(double *p, const V4<double> &v) {
    reinterpret_cast<double2 *>(p)[0] = make_double2(v.a[0], v.a[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2(v.a[2], v.a[3]);
}
// bfloat16 storage: 4 values in 8 bytes, arithmetic in float32
__device__ __forceinline__ V4<float> ld4(const bf16 *p) {
    const uint2 w = *reinterpret_cast<const uint2 *>(p);
    const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&w.x));
    const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&w.y));
    return V4<float>{{a.x, a.y, b.x, b.y}};
}
__device__ __forceinline__ void st4(bf16 *p, const V4<float> &v) {
    const __nv_bfloat162 a = __floats2bfloat162_rn(v.a[0], v.a[1]);
    const __nv_bfloat162 b = __floats2bfloat162_rn(v.a[2], v.a[3]);
    uint2 w;
    w.x = *reinterpret_cast<const unsigned *>(&a);
    w.y = *reinterpret_cast<const unsigned *>(&b);
    *reinterpret_cast<uint2 *>(p) = w;
}
template <typename TO, typename C> __device__ __forceinline__ V4<typename Acc<TO>::T> cvt4(const V4<C> &v) {
    V4<typename Acc<TO>::T> o;
#pragma unroll
    for (int k = 0; k < 4; ++k) o.a[k] = (typename Acc<TO>::T)v.a[k];
    return o;
}

// (M x)_i for 4 columns; identity when M.rp is null.  S: storage type of x,
// T: arithmetic and coefficient type.
template <typename T, typename S>
__device__ __forceinline__ V4<T> row_apply(const CsrView<T> &M, const S *x, int i, int ld,
                                           int c0) {
    V4<T> r{{T(0), T(0), T(0), T(0)}};
    if (M.rp == nullptr) return ld4(x + (size_t)i * ld + c0);
    int e0 = M.rp[i], e1 = M.rp[i + 1];
    for (int e = e0; e < e1; ++e) {
        T w = M.v[e];
        V4<T> xv = ld4(x + (size_t)M.ci[e] * ld + c0);
#pragma unroll
        for (int k = 0; k < 4; ++k) r.a[k] = fma(w, xv.a[k], r.a[k]);
    }
    return r;
}

template <typename TI>
struct TermD {
    CsrView<typename Acc<TI>::T> M;
    const TI *x;
    typename Acc<TI>::T c;
    int sig;
};

template <typename TI, typename TO>
__global__ void k_combine(int rows, int ld, const TI *__restrict__ in0, typename Acc<TI>::T a0,
                          TermD<TI> t1, TermD<TI> t2, const double *__restrict__ sigma,
                          TO *__restrict__ out) {
    using C = typename Acc<TI>::T;
    const int q4 = ld >> 2;
    int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= (int64_t)rows * q4) return;
    int i = (int)(tid / q4);
    int c0 = (int)(tid % q4) * 4;
    V4<C> acc{{C(0), C(0), C(0), C(0)}};
    if (in0) {
        V4<C> a = ld4(in0 + (size_t)i * ld + c0);
#pragma unroll
        for (int k = 0; k < 4; ++k) acc.a[k] = a0 * a.a[k];
    }
    if (t1.x) {
        V4<C> r = row_apply(t1.M, t1.x, i, ld, c0);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            C sc = t1.sig ? t1.c * (C)sigma[c0 + k] : t1.c;
            acc.a[k] = fma(sc, r.a[k], acc.a[k]);
        }
    }
    if (t2.x) {
        V4<C> r = row_apply(t2.M, t2.x, i, ld, c0);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            C sc = t2.sig ? t2.c * (C)sigma[c0 + k] : t2.c;
            acc.a[k] = fma(sc, r.a[k], acc.a[k]);
        }
    }
    st4(out + (size_t)i * ld + c0, cvt4<TO>(acc));
}

template <typename TI, typename TO>
void launch_combine(int rows, int ld, const TI *in0, double a0, const Term<TI> &t1,
                    const Term<TI> &t2, const double *sigma, TO *out, cudaStream_t s) {
    if (rows == 0) return;
    using C = typename Acc<TI>::T;
    TermD<TI> d1{t1.M, t1.x, (C)t1.c, t1.sig ? 1 : 0};
    TermD<TI> d2{t2.M, t2.x, (C)t2.c, t2.sig ? 1 : 0};
    int64_t n = (int64_t)rows * (ld / 4);
    int bs = 256;
    SAMG_COUNT_LAUNCH();
    k_combine<TI, TO><<<(unsigned)((n + bs - 1) / bs), bs, 0, s>>>(rows, ld, in0, (C)a0, d1, d2,
                                                                    sigma, out);
    SAMG_CUDA(cudaGetLastError());
}

template void launch_combine<float, float>(int, int, const float *, double, const Term<float> &,
                                           const Term<float> &, const double *, float *,
                                           cudaStream_t);
template void launch_combine<double, double>(int, int, const double *, double,
                                             const Term<double> &, const Term<double> &,
                                             const double *, double *, cudaStream_t);
template void launch_combine<double, float>(int, int, const double *, double,
                                            const Term<double> &, const Term<double> &,
                                            const double *, float *, cudaStream_t);
template void launch_combine<bf16, bf16>(int, int, const bf16 *, double, const Term<bf16> &,
                                         const Term<bf16> &, const double *, bf16 *, cudaStream_t);
template void launch_combine<double, bf16>(int, int, const double *, double,
                                           const Term<double> &, const Term<double> &,
                                           const double *, bf16 *, cudaStream_t);

// ------------------------------------------------------------------ Jacobi
template <typename S>
__global__ void k_jacobi(int rows, int ld, CsrView<typename Acc<S>::T> A, const S *__restrict__ y,
                         CsrView<typename Acc<S>::T> B, const typename Acc<S>::T *__restrict__ dB,
                         const S *__restrict__ x, const S *__restrict__ kappa,
                         const double *__restrict__ sigma, typename Acc<S>::T omega,
                         S *__restrict__ out) {
    using T = typename Acc<S>::T;
    const int q4 = ld >> 2;
    int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= (int64_t)rows * q4) return;
    int i = (int)(tid / q4);
    int c0 = (int)(tid % q4) * 4;
    V4<T> ay = row_apply(A, y, i, ld, c0);
    V4<T> bx = row_apply(B, x, i, ld, c0);
    V4<T> xi = ld4(x + (size_t)i * ld + c0);
    V4<T> ki{{T(0), T(0), T(0), T(0)}};
    if (kappa) ki = ld4(kappa + (size_t)i * ld + c0);
    T w = omega / (dB ? dB[i] : T(1));
    V4<T> o;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        T inv_s = T(1) / (T)sigma[c0 + k];
        o.a[k] = xi.a[k] - w * (bx.a[k] - (ay.a[k] - ki.a[k]) * inv_s);
    }
    st4(out + (size_t)i * ld + c0, cvt4<S>(o));
}

template <typename T>
void launch_jacobi(int rows, int ld, CsrView<typename Acc<T>::T> A, const T *y,
                   CsrView<typename Acc<T>::T> B, const typename Acc<T>::T *dB, const T *x,
                   const T *kappa, const double *sigma, double omega, T *out, cudaStream_t s) {
    if (rows == 0) return;
    int64_t n = (int64_t)rows * (ld / 4);
    int bs = 256;
    SAMG_COUNT_LAUNCH();
    k_jacobi<T><<<(unsigned)((n + bs - 1) / bs), bs, 0, s>>>(rows, ld, A, y, B, dB, x, kappa,
                                                             sigma, (typename Acc<T>::T)omega, out);
    SAMG_CUDA(cudaGetLastError());
}
template void launch_jacobi<float>(int, int, CsrView<float>, const float *, CsrView<float>,
                                   const float *, const float *, const float *, const double *,
                                   double, float *, cudaStream_t);
template void launch_jacobi<double>(int, int, CsrView<double>, const double *, CsrView<double>,
                                    const double *, const double *, const double *,
                                    const double *, double, double *, cudaStream_t);
template void launch_jacobi<bf16>(int, int, CsrView<float>, const bf16 *, CsrView<float>,
                                  const float *, const bf16 *, const bf16 *, const double *, double,
                                  bf16 *, cudaStream_t);

// ------------------------------------------------------------- elementwise
template <typename TA, typename TB>
__global__ void k_convert(size_t n, const TA *__restrict__ a, TB *__restrict__ b) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = from_acc<TB>((typename Acc<TB>::T)to_acc(a[i]));
}
template <typename TA, typename TB>
void launch_convert(size_t count, const TA *a, TB *b, cudaStream_t s) {
    if (!count) return;
    SAMG_COUNT_LAUNCH();
    k_convert<TA, TB><<<(unsigned)((count + 255) / 256), 256, 0, s>>>(count, a, b);
    SAMG_CUDA(cudaGetLastError());
}
template void launch_convert<double, float>(size_t, const double *, float *, cudaStream_t);
template void launch_convert<float, double>(size_t, const float *, double *, cudaStream_t);
template void launch_convert<double, bf16>(size_t, const double *, bf16 *, cudaStream_t);
template void launch_convert<bf16, double>(size_t, const bf16 *, double *, cudaStream_t);

template <typename TY>
__global__ void k_add_to(size_t n, double *__restrict__ x, const TY *__restrict__ y) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] += (double)to_acc(y[i]);
}
template <typename TY>
void launch_add_to(size_t count, double *x, const TY *y, cudaStream_t s) {
    if (!count) return;
    SAMG_COUNT_LAUNCH();
    k_add_to<TY><<<(unsigned)((count + 255) / 256), 256, 0, s>>>(count, x, y);
    SAMG_CUDA(cudaGetLastError());
}
template void launch_add_to<float>(size_t, double *, const float *, cudaStream_t);
template void launch_add_to<double>(size_t, double *, const double *, cudaStream_t);
template void launch_add_to<bf16>(size_t, double *, const bf16 *, cudaStream_t);

// ----------------------------------------------------------- column dots
// Column-wise x_j^t (M y)_j: per-block partial sums in a fixed order, then one
// block adds the partials in block order (deterministic).
template <typename T>
__global__ void k_coldot(int rows, int nb, int ld, const T *__restrict__ x, CsrView<T> M,
                         const T *__restrict__ y, double *__restrict__ part) {
    __shared__ double red[240][4];
    const int q4 = ld >> 2;
    double acc[4] = {0, 0, 0, 0};
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;  // multiple of q4 (blockDim = 240)
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int c0 = (int)(t0 % q4) * 4;
    for (int64_t tid = t0; tid < (int64_t)rows * q4; tid += stride) {
        const int i = (int)(tid / q4);
        V4<T> my = row_apply(M, y, i, ld, c0);
        V4<T> xi = ld4(x + (size_t)i * ld + c0);
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[k] += (double)xi.a[k] * (double)my.a[k];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) red[threadIdx.x][k] = acc[k];
    __syncthreads();
    if (threadIdx.x < nb) {  // column j: threads with c0 + k == j, in thread order
        const int jc = threadIdx.x;
        double s = 0.0;
        for (int t = 0; t < (int)blockDim.x; ++t)
            if ((t % q4) * 4 == (jc & ~3)) s += red[t][jc & 3];
        part[(size_t)blockIdx.x * 16 + jc] = s;
    }
}

__global__ void k_coldot_final(const double *part, int nblk, int nb, double *out) {
    const int j = threadIdx.x;
    if (j >= nb) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[(size_t)b * 16 + j];
    out[j] += s;
}

template <typename T>
void launch_coldot(int rows, int nb, int ld, const T *x, CsrView<T> M, const T *y, double *out,
                   cudaStream_t s) {
    if (rows == 0) return;
    int64_t n = (int64_t)rows * (ld / 4);
    int bs = 240;
    int64_t g = (n + bs - 1) / bs;
    if (g > 1216) g = 1216;
    DBuf<double> part((size_t)g * 16);
    SAMG_COUNT_LAUNCH();
    k_coldot<T><<<(unsigned)g, bs, 0, s>>>(rows, nb, ld, x, M, y, part.p);
    SAMG_COUNT_LAUNCH();
    k_coldot_final<<<1, 32, 0, s>>>(part.p, (int)g, nb, out);
    SAMG_CUDA(cudaGetLastError());
    SAMG_CUDA(cudaStreamSynchronize(s));  // part is released on return
}
template void launch_coldot<float>(int, int, int, const float *, CsrView<float>, const float *,
                                   double *, cudaStream_t);
template void launch_coldot<double>(int, int, int, const double *, CsrView<double>,
                                    const double *, double *, cudaStream_t);

template <typename T>
__global__ void k_scale_cols(int rows, int ld, T *x, const double *scale) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)rows * ld) return;
    x[t] = (T)((double)x[t] * scale[t % ld]);
}
template <typename T>
void launch_scale_cols(int rows, int ld, T *x, const double *scale, cudaStream_t s) {
    int64_t n = (int64_t)rows * ld;
    if (!n) return;
    SAMG_COUNT_LAUNCH();
    k_scale_cols<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(rows, ld, x, scale);
    SAMG_CUDA(cudaGetLastError());
}
template void launch_scale_cols<float>(int, int, float *, const double *, cudaStream_t);
template void launch_scale_cols<double>(int, int, double *, const double *, cudaStream_t);

template <typename T>
__global__ void k_gather_rows(int k, int ld, const int *idx, const T *x, const double *inv,
                              T *out) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)k * ld) return;
    int r = (int)(t / ld), j = (int)(t % ld);
    T v = x[(size_t)idx[r] * ld + j];
    out[t] = inv ? (T)((double)v / inv[j]) : v;
}
template <typename T>
void launch_gather_rows(int k, int ld, const int *idx, const T *x, const double *inv_colscale,
                        T *out, cudaStream_t s) {
    int64_t n = (int64_t)k * ld;
    if (!n) return;
    SAMG_COUNT_LAUNCH();
    k_gather_rows<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(k, ld, idx, x, inv_colscale, out);
    SAMG_CUDA(cudaGetLastError());
}
template void launch_gather_rows<float>(int, int, const int *, const float *, const double *,
                                        float *, cudaStream_t);
template void launch_gather_rows<double>(int, int, const int *, const double *, const double *,
                                         double *, cudaStream_t);

// ------------------------------------------------------------ row helpers
__global__ void k_inv_rownorm2(int m, const int *rp, const double *v, double *od, float *of) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    double s = 0.0;
    for (int e = rp[i]; e < rp[i + 1]; ++e) s += v[e] * v[e];
    double r = s > 0.0 ? 1.0 / s : 0.0;
    od[i] = r;
    of[i] = (float)r;
}
void launch_inv_rownorm2(const DCsr &a, DBuf<double> &outd, DBuf<float> &outf, cudaStream_t s) {
    outd.alloc(a.m);
    outf.alloc(a.m);
    if (!a.m) return;
    SAMG_COUNT_LAUNCH();
    k_inv_rownorm2<<<(a.m + 255) / 256, 256, 0, s>>>(a.m, a.rp.p, a.vd.p, outd.p, outf.p);
    SAMG_CUDA(cudaGetLastError());
}

__global__ void k_diagonal(int m, const int *rp, const int *ci, const double *v, double *od,
                           float *of) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    double d = 0.0;
    for (int e = rp[i]; e < rp[i + 1]; ++e)
        if (ci[e] == i) d = v[e];
    od[i] = d;
    of[i] = (float)d;
}
void launch_diagonal(const DCsr &a, DBuf<double> &outd, DBuf<float> &outf, cudaStream_t s) {
    outd.alloc(a.m);
    outf.alloc(a.m);
    if (!a.m) return;
    SAMG_COUNT_LAUNCH();
    k_diagonal<<<(a.m + 255) / 256, 256, 0, s>>>(a.m, a.rp.p, a.ci.p, a.vd.p, outd.p, outf.p);
    SAMG_CUDA(cudaGetLastError());
}

}  // namespace samg
