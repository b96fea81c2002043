// sparse_build.cu -- device construction of sparse operators: transposes and
// the Galerkin triple products A_c = P^t A Q, B_c = P^t B P, C_c = Q^t C Q
// (Eq. coarseOp), built once per hierarchy.
//
// C = A B: the column pattern of each row is collected in a per-row
// open-addressing hash table in global memory (sized 2 * upper bound, power of
// two) and written in increasing column order; the values are then summed by
// one thread per row in a fixed order, so the product is deterministic.
#include <cmath>

#include "kernels.cuh"

namespace samg {

// ------------------------------------------------------------------ scan
// Exclusive scan of n int64 values (n <= 4096 * 4096), two levels.
static constexpr int SCAN_T = 1024, SCAN_I = 4, SCAN_B = SCAN_T * SCAN_I;

__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t *sh, int64_t *total) {
    // Hillis-Steele over the warp, then over warp sums
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int64_t w = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        sh[lane] = w;
    }
    __syncthreads();
    int64_t base = warp ? sh[warp - 1] : 0;
    if (total) *total = sh[(blockDim.x >> 5) - 1];
    return base + x - v;
}

__global__ void k_scan_blocks(const int64_t *in, int64_t *out, int64_t *bsum, int n) {
    __shared__ int64_t sh[32];
    int base = blockIdx.x * SCAN_B + threadIdx.x * SCAN_I;
    int64_t loc[SCAN_I], s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_I; ++k) {
        loc[k] = (base + k < n) ? in[base + k] : 0;
        s += loc[k];
    }
    int64_t tot;
    int64_t ex = block_exclusive_scan(s, sh, &tot);
#pragma unroll
    for (int k = 0; k < SCAN_I; ++k) {
        if (base + k < n) out[base + k] = ex;
        ex += loc[k];
    }
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void k_scan_add(int64_t *out, const int64_t *bscan, int n) {
    int i = blockIdx.x * SCAN_B + threadIdx.x * SCAN_I;
#pragma unroll
    for (int k = 0; k < SCAN_I; ++k)
        if (i + k < n) out[i + k] += bscan[blockIdx.x];
}

void exclusive_scan(const int64_t *in, int64_t *out, int n, cudaStream_t s) {
    if (n == 0) {
        SAMG_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), s));
        return;
    }
    int nb = (n + SCAN_B - 1) / SCAN_B;
    SAMG_CHECK(nb <= SCAN_B, SAMG_E_INVALID, "exclusive_scan: too many elements");
    DBuf<int64_t> bsum(nb + 1), bscan(nb + 1);
    SAMG_COUNT_LAUNCH();
    k_scan_blocks<<<nb, SCAN_T, 0, s>>>(in, out, bsum.p, n);
    SAMG_COUNT_LAUNCH();
    k_scan_blocks<<<1, SCAN_T, 0, s>>>(bsum.p, bscan.p, bsum.p + nb, nb);
    SAMG_COUNT_LAUNCH();
    k_scan_add<<<nb, SCAN_T, 0, s>>>(out, bscan.p, n);
    SAMG_CUDA(cudaGetLastError());
    // out[n] = total = sum of the block sums
    SAMG_CUDA(cudaMemcpyAsync(out + n, bsum.p + nb, sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    SAMG_CUDA(cudaStreamSynchronize(s));  // bsum/bscan are released on return
}

// --------------------------------------------------------- host <-> device
__global__ void k_i64_to_i32(int n, const int64_t *a, int *b) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (int)a[i];
}

void refresh_float(DCsr &A, cudaStream_t s) {
    A.vf.alloc(A.nnz ? A.nnz : 1);
    launch_convert<double, float>((size_t)A.nnz, A.vd.p, A.vf.p, s);
}

void validate_csr(const samg_csr &h) {
    SAMG_CHECK(h.m >= 0 && h.n >= 0 && h.nnz >= 0, SAMG_E_INVALID, "csr: negative size");
    SAMG_CHECK(h.nnz < ((int64_t)1 << 31), SAMG_E_INVALID, "csr: nnz >= 2^31");
    SAMG_CHECK(h.row_ptr != nullptr, SAMG_E_INVALID, "csr: null row_ptr");
    SAMG_CHECK(h.nnz == 0 || (h.col != nullptr && h.val != nullptr), SAMG_E_INVALID,
               "csr: null col or val");
    SAMG_CHECK(h.row_ptr[0] == 0 && h.row_ptr[h.m] == h.nnz, SAMG_E_INVALID,
               "csr: row_ptr[0] != 0 or row_ptr[m] != nnz");
    for (int i = 0; i < h.m; ++i) {
        SAMG_CHECK(h.row_ptr[i + 1] >= h.row_ptr[i] && h.row_ptr[i + 1] <= h.nnz, SAMG_E_INVALID,
                   "csr: row_ptr decreasing");
        for (int64_t e = h.row_ptr[i]; e < h.row_ptr[i + 1]; ++e) {
            SAMG_CHECK(h.col[e] >= 0 && h.col[e] < h.n, SAMG_E_INVALID, "csr: column out of range");
            SAMG_CHECK(e == h.row_ptr[i] || h.col[e] > h.col[e - 1], SAMG_E_INVALID,
                       "csr: columns not strictly increasing in a row");
            SAMG_CHECK(std::isfinite(h.val[e]), SAMG_E_INVALID, "csr: non-finite value");
        }
    }
}

void upload_csr(const samg_csr &h, DCsr &d, cudaStream_t s) {
    validate_csr(h);
    d.m = h.m;
    d.n = h.n;
    d.nnz = h.nnz;
    std::vector<int> rp(h.m + 1);
    for (int i = 0; i <= h.m; ++i) rp[i] = (int)h.row_ptr[i];
    d.rp.upload(rp.data(), rp.size(), s);
    d.ci.alloc(h.nnz ? h.nnz : 1);
    d.vd.alloc(h.nnz ? h.nnz : 1);
    if (h.nnz) {
        SAMG_CUDA(cudaMemcpyAsync(d.ci.p, h.col, h.nnz * sizeof(int), cudaMemcpyHostToDevice, s));
        SAMG_CUDA(cudaMemcpyAsync(d.vd.p, h.val, h.nnz * sizeof(double), cudaMemcpyHostToDevice, s));
    }
    refresh_float(d, s);
    SAMG_CUDA(cudaStreamSynchronize(s));
}

void upload_csr(const HCsr &h, DCsr &d, cudaStream_t s) {
    samg_csr c{h.m, h.n, h.nnz(), h.rp.data(), h.ci.data(), h.v.data()};
    upload_csr(c, d, s);
}

void download_csr(const DCsr &d, HCsr &h, cudaStream_t s) {
    h.m = d.m;
    h.n = d.n;
    std::vector<int> rp(d.m + 1);
    d.rp.download(rp.data(), rp.size(), s);
    h.ci.resize(d.nnz);
    h.v.resize(d.nnz);
    d.ci.download(h.ci.data(), d.nnz, s);
    d.vd.download(h.v.data(), d.nnz, s);
    SAMG_CUDA(cudaStreamSynchronize(s));
    h.rp.assign(rp.begin(), rp.end());
}

// ------------------------------------------------------------ transpose
__global__ void k_count_cols(int64_t nnz, const int *ci, int64_t *cnt) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < nnz) atomicAdd((unsigned long long *)&cnt[ci[e]], 1ull);
}

__global__ void k_scatter_t(int m, const int *rp, const int *ci, const double *v,
                            const int64_t *off, int *fill, int *cit, double *vt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
        int c = ci[e];
        int pos = (int)off[c] + atomicAdd(&fill[c], 1);
        cit[pos] = i;
        vt[pos] = v[e];
    }
}

// Sort each row of (ci, v) by ci with a rank placement (keys distinct per row);
// one warp per row, result written to (co, vo).
__global__ void k_rank_sort_rows(int m, const int *rp, const int *ci, const double *v, int *co,
                                 double *vo) {
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (warp >= m) return;
    int e0 = rp[warp], e1 = rp[warp + 1];
    for (int e = e0 + lane; e < e1; e += 32) {
        int key = ci[e];
        int rank = 0;
        for (int f = e0; f < e1; ++f) rank += (ci[f] < key);
        co[e0 + rank] = key;
        vo[e0 + rank] = v[e];
    }
}

void transpose(const DCsr &A, DCsr &C, cudaStream_t s) {
    C.m = A.n;
    C.n = A.m;
    C.nnz = A.nnz;
    DBuf<int64_t> cnt(A.n + 1), off(A.n + 1);
    cnt.zero(s);
    if (A.nnz) {
        SAMG_COUNT_LAUNCH();
        k_count_cols<<<(unsigned)((A.nnz + 255) / 256), 256, 0, s>>>(A.nnz, A.ci.p, cnt.p);
    }
    exclusive_scan(cnt.p, off.p, A.n, s);
    C.rp.alloc(A.n + 1);
    SAMG_COUNT_LAUNCH();
    k_i64_to_i32<<<(A.n + 1 + 255) / 256, 256, 0, s>>>(A.n + 1, off.p, C.rp.p);
    DBuf<int> fill(A.n > 0 ? A.n : 1);
    fill.zero(s);
    DBuf<int> ctmp(A.nnz ? A.nnz : 1);
    DBuf<double> vtmp(A.nnz ? A.nnz : 1);
    if (A.m) {
        SAMG_COUNT_LAUNCH();
        k_scatter_t<<<(A.m + 255) / 256, 256, 0, s>>>(A.m, A.rp.p, A.ci.p, A.vd.p, off.p, fill.p,
                                                     ctmp.p, vtmp.p);
    }
    C.ci.alloc(A.nnz ? A.nnz : 1);
    C.vd.alloc(A.nnz ? A.nnz : 1);
    if (C.m) {
        SAMG_COUNT_LAUNCH();
        k_rank_sort_rows<<<(unsigned)(((int64_t)C.m * 32 + 255) / 256), 256, 0, s>>>(
            C.m, C.rp.p, ctmp.p, vtmp.p, C.ci.p, C.vd.p);
    }
    SAMG_CUDA(cudaGetLastError());
    refresh_float(C, s);
    SAMG_CUDA(cudaStreamSynchronize(s));
}

// --------------------------------------------------------------- SpGEMM
__global__ void k_row_bounds(int m, const int *arp, const int *aci, const int *brp,
                             int64_t *ub, int64_t *hs) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    int64_t u = 0;
    for (int e = arp[i]; e < arp[i + 1]; ++e) {
        int k = aci[e];
        u += brp[k + 1] - brp[k];
    }
    ub[i] = u;
    int64_t h = 0;
    if (u > 0) {
        h = 16;
        while (h < 2 * u) h <<= 1;
    }
    hs[i] = h;
}

__device__ __forceinline__ unsigned hash_col(int c) { return (unsigned)c * 2654435761u; }

__global__ void k_hash_insert(int m, const int *arp, const int *aci, const int *brp,
                              const int *bci, const int64_t *hoff, int *keys) {
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (warp >= m) return;
    int64_t h0 = hoff[warp];
    unsigned mask = (unsigned)(hoff[warp + 1] - h0) - 1u;
    if (hoff[warp + 1] == h0) return;
    for (int e = arp[warp] + lane; e < arp[warp + 1]; e += 32) {
        int k = aci[e];
        for (int f = brp[k]; f < brp[k + 1]; ++f) {
            int c = bci[f];
            unsigned h = hash_col(c) & mask;
            for (;;) {
                int old = atomicCAS(&keys[h0 + h], -1, c);
                if (old == -1 || old == c) break;
                h = (h + 1) & mask;
            }
        }
    }
}

// Values of C = A B, one thread per row, products accumulated in the order of
// A's row and B's rows (deterministic); the sorted column list of the row is
// searched by bisection.
__global__ void k_spgemm_values(int m, const int *arp, const int *aci, const double *av,
                                const int *brp, const int *bci, const double *bv,
                                const int64_t *crp, const int *cci, double *cv) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const int64_t c0 = crp[i], c1 = crp[i + 1];
    for (int64_t q = c0; q < c1; ++q) cv[q] = 0.0;
    for (int e = arp[i]; e < arp[i + 1]; ++e) {
        const int k = aci[e];
        const double a = av[e];
        for (int f = brp[k]; f < brp[k + 1]; ++f) {
            const int c = bci[f];
            int64_t lo = c0, hi = c1 - 1;
            while (lo < hi) {
                int64_t mid = (lo + hi) >> 1;
                if (cci[mid] < c) lo = mid + 1;
                else hi = mid;
            }
            cv[lo] += a * bv[f];
        }
    }
}

__global__ void k_hash_count(int m, const int64_t *hoff, const int *keys, int64_t *cnt) {
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (warp >= m) return;
    int c = 0;
    for (int64_t h = hoff[warp] + lane; h < hoff[warp + 1]; h += 32) c += (keys[h] >= 0);
    for (int o = 16; o; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if (lane == 0) cnt[warp] = c;
}

__global__ void k_hash_compact(int m, const int64_t *hoff, const int *keys, const int64_t *rp,
                               int *ci) {
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (warp >= m) return;
    int64_t h0 = hoff[warp], h1 = hoff[warp + 1];
    int64_t base = rp[warp];
    for (int64_t h = h0 + lane; h < h1; h += 32) {
        int key = keys[h];
        if (key < 0) continue;
        int rank = 0;
        for (int64_t g = h0; g < h1; ++g) {
            int k2 = keys[g];
            rank += (k2 >= 0 && k2 < key);
        }
        ci[base + rank] = key;
    }
}

void spgemm(const DCsr &A, const DCsr &B, DCsr &C, cudaStream_t s) {
    SAMG_CHECK(A.n == B.m, SAMG_E_INVALID, "spgemm: inner dimensions differ");
    int m = A.m;
    C.m = m;
    C.n = B.n;
    DBuf<int64_t> ub(m + 1), hs(m + 1), hoff(m + 1);
    if (m) {
        SAMG_COUNT_LAUNCH();
        k_row_bounds<<<(m + 255) / 256, 256, 0, s>>>(m, A.rp.p, A.ci.p, B.rp.p, ub.p, hs.p);
    }
    exclusive_scan(hs.p, hoff.p, m, s);
    int64_t H = 0;
    SAMG_CUDA(cudaMemcpyAsync(&H, hoff.p + m, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    SAMG_CUDA(cudaStreamSynchronize(s));
    DBuf<int> keys(H ? H : 1);
    SAMG_CUDA(cudaMemsetAsync(keys.p, 0xff, keys.n * sizeof(int), s));
    unsigned wb = (unsigned)(((int64_t)m * 32 + 255) / 256);
    if (m) {
        SAMG_COUNT_LAUNCH();
        k_hash_insert<<<wb, 256, 0, s>>>(m, A.rp.p, A.ci.p, B.rp.p, B.ci.p, hoff.p, keys.p);
        SAMG_COUNT_LAUNCH();
        k_hash_count<<<wb, 256, 0, s>>>(m, hoff.p, keys.p, ub.p);
    }
    DBuf<int64_t> rp64(m + 1);
    exclusive_scan(ub.p, rp64.p, m, s);
    int64_t nnz = 0;
    SAMG_CUDA(cudaMemcpyAsync(&nnz, rp64.p + m, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    SAMG_CUDA(cudaStreamSynchronize(s));
    SAMG_CHECK(nnz < ((int64_t)1 << 31), SAMG_E_INVALID, "spgemm: result nnz >= 2^31");
    C.nnz = nnz;
    C.rp.alloc(m + 1);
    SAMG_COUNT_LAUNCH();
    k_i64_to_i32<<<(m + 1 + 255) / 256, 256, 0, s>>>(m + 1, rp64.p, C.rp.p);
    C.ci.alloc(nnz ? nnz : 1);
    C.vd.alloc(nnz ? nnz : 1);
    if (m) {
        SAMG_COUNT_LAUNCH();
        k_hash_compact<<<wb, 256, 0, s>>>(m, hoff.p, keys.p, rp64.p, C.ci.p);
        SAMG_COUNT_LAUNCH();
        k_spgemm_values<<<(m + 127) / 128, 128, 0, s>>>(m, A.rp.p, A.ci.p, A.vd.p, B.rp.p, B.ci.p,
                                                        B.vd.p, rp64.p, C.ci.p, C.vd.p);
    }
    SAMG_CUDA(cudaGetLastError());
    refresh_float(C, s);
    SAMG_CUDA(cudaStreamSynchronize(s));
}

}  // namespace samg
