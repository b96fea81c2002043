// coloured.cu -- coloured-order Kaczmarz smoothing (a variant of the natural
// order of Sec. 5.3; see coloured.cuh): host colouring and program
// assembly, and the per-class kernel.
#include <algorithm>
#include <cstring>

#include "coloured.cuh"

namespace samg {

int greedy_row_colours(int rows, int cols, const std::vector<int64_t> &rp,
                       const std::vector<int> &ci, std::vector<int> &colour) {
    // per column: the colours of the earlier rows touching it, 64 per word
    std::vector<std::vector<uint64_t>> used(cols);
    colour.assign(rows, 0);
    int ncol = 0;
    std::vector<uint64_t> forbid;
    for (int i = 0; i < rows; ++i) {
        forbid.assign((ncol + 64) / 64, 0ull);
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
            const std::vector<uint64_t> &u = used[ci[e]];
            for (size_t w = 0; w < u.size() && w < forbid.size(); ++w) forbid[w] |= u[w];
        }
        int c = 0;
        while ((size_t)(c / 64) < forbid.size() && ((forbid[c / 64] >> (c % 64)) & 1u)) ++c;
        colour[i] = c;
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
            std::vector<uint64_t> &u = used[ci[e]];
            if (u.size() <= (size_t)(c / 64)) u.resize(c / 64 + 1, 0ull);
            u[c / 64] |= 1ull << (c % 64);
        }
        ncol = std::max(ncol, c + 1);
    }
    return ncol;
}

namespace {

struct CRows {  // a program's rows before upload
    std::vector<int64_t> rp{0};
    std::vector<int> ci, rrow;
    std::vector<double> a, b, inv;
    std::vector<int> class_off{0}, class_lg;
    int ncolour_max = 0;
};

// Appends one sweep: the rows of `src` grouped by colour (natural order in a
// colour).  row(i, push) emits row i's entries; rhs_row(i) its right-hand
// side row.
template <typename RowFn>
void append_sweep(CRows &P, int rows, const std::vector<int> &colour, int ncolour, RowFn row,
                  int rhs_off) {
    std::vector<std::vector<int>> by(ncolour);
    for (int i = 0; i < rows; ++i) by[colour[i]].push_back(i);
    for (int c = 0; c < ncolour; ++c) {
        if (by[c].empty()) continue;
        int maxe = 0;
        for (int i : by[c]) {
            const size_t e0 = P.ci.size();
            double n2 = 0.0;
            row(i, [&](int col, double a, double b) {
                P.ci.push_back(col);
                P.a.push_back(a);
                P.b.push_back(b);
                n2 += a * a;
            });
            P.rp.push_back((int64_t)P.ci.size());
            P.rrow.push_back(rhs_off + i);
            P.inv.push_back(n2 > 0.0 ? 1.0 / n2 : 0.0);
            maxe = std::max(maxe, (int)(P.ci.size() - e0));
        }
        int lg = 0;
        while (lg < 5 && (1 << lg) < maxe) ++lg;
        P.class_off.push_back((int)P.rrow.size());
        P.class_lg.push_back(lg);
    }
    P.ncolour_max = std::max(P.ncolour_max, ncolour);
}

void upload(const CRows &P, int cols, int mode, CSched &cs, cudaStream_t s) {
    cs.rows = (int)P.rrow.size();
    cs.cols = cols;
    cs.mode = mode;
    cs.nent = (int64_t)P.ci.size();
    cs.class_off = P.class_off;
    cs.class_lg = P.class_lg;
    cs.ncolour_max = P.ncolour_max;
    cs.max_class_threads = 0;
    for (size_t k = 0; k + 1 < P.class_off.size(); ++k)
        cs.max_class_threads = std::max(cs.max_class_threads,
                                        (P.class_off[k + 1] - P.class_off[k]) << P.class_lg[k]);
    cs.d_class_off.upload(P.class_off.data(), P.class_off.size(), s);
    cs.d_class_lg.upload(P.class_lg.data(), P.class_lg.size(), s);
    SAMG_CHECK(cs.nent < (int64_t)1 << 31, SAMG_E_INVALID, "coloured sweep: too many entries");
    std::vector<int> rp32(P.rp.begin(), P.rp.end());
    cs.rp.upload(rp32.data(), rp32.size(), s);
    cs.ci.upload(P.ci.data(), P.ci.size(), s);
    cs.rrow.upload(P.rrow.data(), P.rrow.size(), s);
    cs.ad.upload(P.a.data(), P.a.size(), s);
    cs.bd.upload(P.b.data(), P.b.size(), s);
    cs.invd.upload(P.inv.data(), P.inv.size(), s);
    std::vector<float> f(P.a.begin(), P.a.end());
    cs.af.upload(f.data(), f.size(), s);
    f.assign(P.b.begin(), P.b.end());
    cs.bf.upload(f.data(), f.size(), s);
    f.assign(P.inv.begin(), P.inv.end());
    cs.invf.upload(f.data(), f.size(), s);
    SAMG_CUDA(cudaStreamSynchronize(s));
}

}  // namespace

void build_cschedule_fused(const HCsr &A, const HCsr &At, const HCsr &B, const HCsr &C, int count,
                           CSched &cs, cudaStream_t s) {
    const int m = A.m, n = A.n;
    std::vector<int> colA, colAt;
    // rows of A update v (columns of A); rows of A^t update u
    const int kA = greedy_row_colours(m, n, A.rp, A.ci, colA);
    const int kAt = greedy_row_colours(n, m, At.rp, At.ci, colAt);
    CRows P;
    for (int k = 0; k < count; ++k) {
        // a_i . v - s_j (B u)_i = kappa_i: v entries (a), then u entries (b)
        append_sweep(P, m, colA, kA, [&](int i, auto push) {
            for (int64_t e = A.rp[i]; e < A.rp[i + 1]; ++e) push(A.ci[e], A.v[e], 0.0);
            for (int64_t e = B.rp[i]; e < B.rp[i + 1]; ++e) push(n + B.ci[e], 0.0, B.v[e]);
        }, 0);
        // a^t_j . u - s_j (C v)_j = tau_j: v entries (b), then u entries (a)
        append_sweep(P, n, colAt, kAt, [&](int j, auto push) {
            for (int64_t e = C.rp[j]; e < C.rp[j + 1]; ++e) push(C.ci[e], 0.0, C.v[e]);
            for (int64_t e = At.rp[j]; e < At.rp[j + 1]; ++e) push(n + At.ci[e], At.v[e], 0.0);
        }, m);
    }
    upload(P, n + m, 2, cs, s);
}

void build_cschedule_stacked(const HCsr &A, const HCsr &B, int count, CSched &cs, cudaStream_t s) {
    const int n = A.m;
    // rows of A - s B update every column of the union pattern
    HCsr U;
    U.m = U.n = n;
    U.rp.assign(1, 0);
    std::vector<double> ua, ub;
    for (int i = 0; i < n; ++i) {
        int64_t e = A.rp[i], ee = A.rp[i + 1], f = B.rp[i], fe = B.rp[i + 1];
        while (e < ee || f < fe) {
            if (f >= fe || (e < ee && A.ci[e] < B.ci[f])) {
                U.ci.push_back(A.ci[e]); ua.push_back(A.v[e]); ub.push_back(0.0); ++e;
            } else if (e >= ee || B.ci[f] < A.ci[e]) {
                U.ci.push_back(B.ci[f]); ua.push_back(0.0); ub.push_back(B.v[f]); ++f;
            } else {
                U.ci.push_back(A.ci[e]); ua.push_back(A.v[e]); ub.push_back(B.v[f]); ++e; ++f;
            }
        }
        U.rp.push_back((int64_t)U.ci.size());
    }
    std::vector<int> col;
    const int k = greedy_row_colours(n, n, U.rp, U.ci, col);
    CRows P;
    for (int c = 0; c < count; ++c)
        append_sweep(P, n, col, k, [&](int i, auto push) {
            for (int64_t e = U.rp[i]; e < U.rp[i + 1]; ++e) push(U.ci[e], ua[e], ub[e]);
        }, 0);
    upload(P, n, 1, cs, s);
}

namespace {

// A row of LD stored values S read into / written from the arithmetic type
// T (bfloat16 storage: 8-byte pieces of 4 values, converted to float32).
template <typename T, typename S, int LD>
__device__ __forceinline__ void cld(T (&v)[LD], const S *p) {
    if constexpr (sizeof(S) == 4 && sizeof(T) == 4) {
#pragma unroll
        for (int i = 0; i < LD / 4; ++i) {
            const float4 t = reinterpret_cast<const float4 *>(p)[i];
            v[4 * i] = t.x; v[4 * i + 1] = t.y; v[4 * i + 2] = t.z; v[4 * i + 3] = t.w;
        }
    } else if constexpr (sizeof(S) == 8) {
#pragma unroll
        for (int i = 0; i < LD / 2; ++i) {
            const double2 t = reinterpret_cast<const double2 *>(p)[i];
            v[2 * i] = t.x; v[2 * i + 1] = t.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < LD / 4; ++i) {
            const uint2 w = reinterpret_cast<const uint2 *>(p)[i];
            const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&w.x));
            const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&w.y));
            v[4 * i] = a.x; v[4 * i + 1] = a.y; v[4 * i + 2] = b.x; v[4 * i + 3] = b.y;
        }
    }
}
template <typename T, typename S, int LD>
__device__ __forceinline__ void cst(S *p, const T (&v)[LD]) {
    if constexpr (sizeof(S) == 4 && sizeof(T) == 4) {
#pragma unroll
        for (int i = 0; i < LD / 4; ++i)
            reinterpret_cast<float4 *>(p)[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
    } else if constexpr (sizeof(S) == 8) {
#pragma unroll
        for (int i = 0; i < LD / 2; ++i)
            reinterpret_cast<double2 *>(p)[i] = make_double2(v[2 * i], v[2 * i + 1]);
    } else {
#pragma unroll
        for (int i = 0; i < LD / 4; ++i) {
            const __nv_bfloat162 a = __floats2bfloat162_rn(v[4 * i], v[4 * i + 1]);
            const __nv_bfloat162 b = __floats2bfloat162_rn(v[4 * i + 2], v[4 * i + 3]);
            uint2 w;
            w.x = *reinterpret_cast<const unsigned *>(&a);
            w.y = *reinterpret_cast<const unsigned *>(&b);
            reinterpret_cast<uint2 *>(p)[i] = w;
        }
    }
}

// The rows [r0, r1) of one colour class, G = 2^lg lanes per row (aligned
// groups inside a warp; a lane takes entries lg, lg + G, ...), rows handed
// out to groups from `first` in steps of `groups`.  Every lane of a warp
// calls (the row sums shuffle within the group).
// MODE 1: coefficients a - s_j b for the row sums, the norms and the update.
// MODE 2: a - s_j b for the row sums, a for the update (b entries belong to
// the other unknown and are not written), norms given.
template <typename T, typename S, int LD, int MODE>
__device__ __forceinline__ void class_rows(int r0, int r1, int lg, long long first, long long groups,
                                           const int *__restrict__ rp, const int *__restrict__ ci,
                                           const int *__restrict__ rrow, const T *__restrict__ av,
                                           const T *__restrict__ bv, const T *__restrict__ inv,
                                           const S *__restrict__ rhs, S *x, const T (&sh)[LD]) {
    const int G = 1 << lg;
    const int lgi = (threadIdx.x & 31) & (G - 1);
    for (long long g = first;; g += groups) {
        const long long r = r0 + g;
        const bool act = r < r1;
        if (!__any_sync(0xffffffffu, act)) break;
        T acc[LD], nrm[LD], fv[LD];
#pragma unroll
        for (int q = 0; q < LD; ++q) { acc[q] = T(0); nrm[q] = T(0); fv[q] = T(0); }
        int e0 = 0, e1 = 0, fcol = 0;
        T fa = T(0), fb = T(0);
        if (act) {
            e0 = rp[r];
            e1 = rp[r + 1];
            for (int e = e0 + lgi; e < e1; e += G) {
                const int col = ci[e];
                const T a = av[e], b = MODE != 0 ? bv[e] : T(0);
                T val[LD];
                cld<T, S, LD>(val, x + (size_t)col * LD);
                if (e == e0 + lgi) {  // the lane's first entry stays in registers
                    fcol = col; fa = a; fb = b;
#pragma unroll
                    for (int q = 0; q < LD; ++q) fv[q] = val[q];
                }
#pragma unroll
                for (int q = 0; q < LD; ++q) {
                    const T coef = MODE != 0 ? a - sh[q] * b : a;
                    acc[q] = fma(coef, val[q], acc[q]);
                    if (MODE == 1) nrm[q] = fma(coef, coef, nrm[q]);
                }
            }
        }
        for (int o = 1; o < G; o <<= 1) {
#pragma unroll
            for (int q = 0; q < LD; ++q) {
                acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
                if (MODE == 1) nrm[q] += __shfl_xor_sync(0xffffffffu, nrm[q], o);
            }
        }
        if (!act) continue;
        T d[LD];
        const S *bq = rhs ? rhs + (size_t)rrow[r] * LD : nullptr;
        const T iv = MODE == 1 ? T(0) : inv[r];
#pragma unroll
        for (int q = 0; q < LD; ++q) {
            const T bi = bq ? (T)to_acc(bq[q]) : T(0);
            d[q] = MODE == 1 ? (nrm[q] > T(0) ? (bi - acc[q]) / nrm[q] : T(0)) : (bi - acc[q]) * iv;
        }
        for (int e = e0 + lgi; e < e1; e += G) {
            int col;
            T a, b, val[LD];
            if (e == e0 + lgi) {
                col = fcol; a = fa; b = fb;
#pragma unroll
                for (int q = 0; q < LD; ++q) val[q] = fv[q];
            } else {
                col = ci[e];
                a = av[e];
                b = MODE != 0 ? bv[e] : T(0);
                cld<T, S, LD>(val, x + (size_t)col * LD);
            }
            if (MODE == 2 && a == T(0)) continue;  // an entry of the other unknown
#pragma unroll
            for (int q = 0; q < LD; ++q) {
                const T coef = MODE == 1 ? a - sh[q] * b : a;
                val[q] = fma(d[q], coef, val[q]);
            }
            cst<T, S, LD>(x + (size_t)col * LD, val);
        }
    }
}

// One colour class on a grid.
template <typename T, typename S, int LD, int MODE>
__global__ void __launch_bounds__(256)
    k_kz_class(int r0, int r1, int lg, const int *__restrict__ rp, const int *__restrict__ ci,
               const int *__restrict__ rrow, const T *__restrict__ av, const T *__restrict__ bv,
               const T *__restrict__ inv, const S *__restrict__ rhs, S *x,
               const double *__restrict__ shift) {
    T sh[LD];
#pragma unroll
    for (int q = 0; q < LD; ++q) sh[q] = MODE != 0 ? (T)shift[q] : T(0);
    class_rows<T, S, LD, MODE>(r0, r1, lg, ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> lg,
                            (long long)gridDim.x * (blockDim.x >> lg), rp, ci, rrow, av, bv, inv,
                            rhs, x, sh);
}

// A whole program of small classes in one CTA: the classes in order, a CTA
// barrier between them (it orders the global stores of one class before the
// loads of the next for every thread of the CTA).
constexpr int COLOURED_CTA = 512;
constexpr int COLOURED_CTA_ROWS = 4 * COLOURED_CTA;
template <typename T, typename S, int LD, int MODE>
__global__ void __launch_bounds__(COLOURED_CTA)
    k_kz_classes_cta(int nclass, const int *__restrict__ class_off, const int *__restrict__ class_lg,
                     const int *__restrict__ rp, const int *__restrict__ ci,
                     const int *__restrict__ rrow, const T *__restrict__ av,
                     const T *__restrict__ bv, const T *__restrict__ inv,
                     const S *__restrict__ rhs, S *x, const double *__restrict__ shift) {
    T sh[LD];
#pragma unroll
    for (int q = 0; q < LD; ++q) sh[q] = MODE != 0 ? (T)shift[q] : T(0);
    for (int k = 0; k < nclass; ++k) {
        const int lg = class_lg[k];
        class_rows<T, S, LD, MODE>(class_off[k], class_off[k + 1], lg, (long long)threadIdx.x >> lg,
                                (long long)(blockDim.x >> lg), rp, ci, rrow, av, bv, inv, rhs, x, sh);
        __syncthreads();
    }
}

template <typename T> const T *pick(const DBuf<double> &d, const DBuf<float> &f);
template <> const double *pick<double>(const DBuf<double> &d, const DBuf<float> &) { return d.p; }
template <> const float *pick<float>(const DBuf<double> &, const DBuf<float> &f) { return f.p; }

template <typename S, int LD, int MODE>
void run(const CSched &cs, const S *rhs, S *x, const double *shift, cudaStream_t s) {
    using T = typename Acc<S>::T;
    static int nsm = 0;
    if (!nsm) {
        int dev = 0;
        SAMG_CUDA(cudaGetDevice(&dev));
        SAMG_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    }
    const T *a = pick<T>(cs.ad, cs.af), *b = pick<T>(cs.bd, cs.bf), *inv = pick<T>(cs.invd, cs.invf);
    const int nclass = (int)cs.class_off.size() - 1;
    if (cs.max_class_threads <= COLOURED_CTA_ROWS) {
        SAMG_COUNT_LAUNCH();
        k_kz_classes_cta<T, S, LD, MODE><<<1, COLOURED_CTA, 0, s>>>(
            nclass, cs.d_class_off.p, cs.d_class_lg.p, cs.rp.p, cs.ci.p, cs.rrow.p, a, b, inv, rhs,
            x, shift);
        SAMG_CUDA(cudaGetLastError());
        return;
    }
    for (int k = 0; k < nclass; ++k) {
        const int r0 = cs.class_off[k], r1 = cs.class_off[k + 1];
        const int lg = cs.class_lg[k];
        const long long threads = (long long)(r1 - r0) << lg;
        const int grid = (int)std::min<long long>((threads + 255) / 256, (long long)nsm * 8);
        SAMG_COUNT_LAUNCH();
        k_kz_class<T, S, LD, MODE><<<std::max(grid, 1), 256, 0, s>>>(
            r0, r1, lg, cs.rp.p, cs.ci.p, cs.rrow.p, a, b, inv, rhs, x, shift);
    }
    SAMG_CUDA(cudaGetLastError());
}

template <typename T>
void dispatch(const CSched &cs, int ld, const T *rhs, T *x, const double *shift, cudaStream_t s) {
    SAMG_CHECK(cs.mode == 1 || cs.mode == 2, SAMG_E_INVALID, "coloured sweep: bad mode");
    const uintptr_t al = ((size_t)ld * sizeof(T)) % 16 == 0 ? 16 : 8;
    SAMG_CHECK(((uintptr_t)x % al) == 0 && ((uintptr_t)rhs % al) == 0, SAMG_E_INVALID,
               "coloured sweep: vector blocks must be aligned to their row pieces");
#define CZ_CASE(L)                                                       \
    case L:                                                              \
        if (cs.mode == 1) run<T, L, 1>(cs, rhs, x, shift, s);            \
        else run<T, L, 2>(cs, rhs, x, shift, s);                         \
        break;
    switch (ld) {
        CZ_CASE(4)
        CZ_CASE(8)
        CZ_CASE(12)
        CZ_CASE(16)
        default:
            throw Error(SAMG_E_INVALID, "coloured sweep: unsupported block width");
    }
#undef CZ_CASE
}

}  // namespace

template <>
void launch_coloured<float>(const CSched &cs, int ld, const float *rhs, float *x,
                            const double *shift, cudaStream_t s) {
    if (cs.rows) dispatch<float>(cs, ld, rhs, x, shift, s);
}
template <>
void launch_coloured<double>(const CSched &cs, int ld, const double *rhs, double *x,
                             const double *shift, cudaStream_t s) {
    if (cs.rows) dispatch<double>(cs, ld, rhs, x, shift, s);
}
template <>
void launch_coloured<bf16>(const CSched &cs, int ld, const bf16 *rhs, bf16 *x, const double *shift,
                           cudaStream_t s) {
    if (cs.rows) dispatch<bf16>(cs, ld, rhs, x, shift, s);
}

}  // namespace samg
