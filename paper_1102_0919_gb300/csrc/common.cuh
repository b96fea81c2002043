// common.cuh -- shared device/host helpers of the GB300 SAMG library.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/samg.h"

namespace samg {

// A CUDA or argument failure inside the library; converted to a status at the
// C ABI boundary.
struct Error : public std::runtime_error {
    samg_status status;
    Error(samg_status s, const std::string &msg) : std::runtime_error(msg), status(s) {}
};

#define SAMG_CUDA(call)                                                                   \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            throw ::samg::Error(SAMG_E_CUDA, std::string(#call " failed: ") +             \
                                                 cudaGetErrorString(e_) + " at " +        \
                                                 __FILE__ + ":" + std::to_string(__LINE__)); \
    } while (0)

#define SAMG_CHECK(cond, status, msg)                          \
    do {                                                       \
        if (!(cond)) throw ::samg::Error((status), (msg));     \
    } while (0)

// Vector storage types of the V-cycle and the arithmetic each computes in:
// float64 and float32 compute in themselves; bfloat16 storage (16-bit
// vectors in HBM) computes in float32, with float32 matrix coefficients.
using bf16 = __nv_bfloat16;
template <typename S> struct Acc { using T = S; };
template <> struct Acc<bf16> { using T = float; };

__host__ __device__ inline float to_acc(bf16 v) { return __bfloat162float(v); }
__host__ __device__ inline float to_acc(float v) { return v; }
__host__ __device__ inline double to_acc(double v) { return v; }
template <typename S> __host__ __device__ inline S from_acc(typename Acc<S>::T v) { return (S)v; }
template <> __host__ __device__ inline bf16 from_acc<bf16>(float v) { return __float2bfloat16_rn(v); }

// Device buffer owned by value (move-only).
template <typename T>
struct DBuf {
    T *p = nullptr;
    size_t n = 0;
    DBuf() = default;
    explicit DBuf(size_t count) { alloc(count); }
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    DBuf(DBuf &&o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
    DBuf &operator=(DBuf &&o) noexcept {
        if (this != &o) { release(); p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
        return *this;
    }
    ~DBuf() { release(); }
    void alloc(size_t count) {
        release();
        if (count == 0) return;
        cudaError_t e = cudaMalloc(&p, count * sizeof(T));
        if (e != cudaSuccess) {
            p = nullptr;
            throw Error(e == cudaErrorMemoryAllocation ? SAMG_E_NOMEM : SAMG_E_CUDA,
                        std::string("cudaMalloc: ") + cudaGetErrorString(e));
        }
        n = count;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    void zero(cudaStream_t s) {
        if (n) SAMG_CUDA(cudaMemsetAsync(p, 0, n * sizeof(T), s));
    }
    void upload(const T *h, size_t count, cudaStream_t s) {
        if (count > n) alloc(count);
        if (count) SAMG_CUDA(cudaMemcpyAsync(p, h, count * sizeof(T), cudaMemcpyHostToDevice, s));
    }
    void download(T *h, size_t count, cudaStream_t s) const {
        if (count) SAMG_CUDA(cudaMemcpyAsync(h, p, count * sizeof(T), cudaMemcpyDeviceToHost, s));
    }
};

// Device CSR with int32 indices; float64 values and an optional float32 copy.
struct DCsr {
    int m = 0, n = 0;
    int64_t nnz = 0;
    DBuf<int> rp, ci;
    DBuf<double> vd;
    DBuf<float> vf;
    bool empty() const { return m == 0; }
};

// Plain view passed to kernels.
template <typename T>
struct CsrView {
    int m, n;
    const int *rp;
    const int *ci;
    const T *v;
};

template <typename T> inline CsrView<T> view(const DCsr &a);
template <> inline CsrView<double> view<double>(const DCsr &a) {
    return CsrView<double>{a.m, a.n, a.rp.p, a.ci.p, a.vd.p};
}
template <> inline CsrView<float> view<float>(const DCsr &a) {
    return CsrView<float>{a.m, a.n, a.rp.p, a.ci.p, a.vf.p};
}

// Host CSR (library side).
struct HCsr {
    int m = 0, n = 0;
    std::vector<int64_t> rp;
    std::vector<int> ci;
    std::vector<double> v;
    int64_t nnz() const { return rp.empty() ? 0 : rp.back(); }
};

inline int round_up(int x, int k) { return (x + k - 1) / k * k; }

// Count of kernel launches issued by the library (samg_launch_count); atomic,
// since contexts may be driven from several host threads.
std::atomic<uint64_t> &launch_counter();
#define SAMG_COUNT_LAUNCH() (++::samg::launch_counter())

// Columns of a device vector block: n_b padded to a multiple of 4 (16-byte rows
// in float32, 32-byte rows in float64); padding columns are kept at zero.
inline int block_ld(int nb) { return round_up(nb, 4); }

}  // namespace samg
