// kaczmarz.cu -- schedule builder (host) and sweep kernel (device) for the
// exact-order Kaczmarz relaxation of Sec. 5.3 (see kaczmarz.cuh).
#include <algorithm>
#include <cstring>

#include "kaczmarz.cuh"

namespace samg {

namespace {

constexpr int KZ_THREADS = 512;
constexpr int KZ_COMPUTE = 480;    // compute threads (15 warps); warp 15 communicates
constexpr int KZ_NBUF = 3;          // staging buffers: schedule two chunks ahead, values one
constexpr int KZ_PUB = 8;           // publish granularity (levels)
constexpr int TARGET_PAR = 32;       // wanted rows per level inside a band
constexpr int MAX_BAND_ROWS = 1 << 17;
constexpr int SLOT_CAP = 512;        // window slots: 512 * 16 cols * 8 B = 64 KiB
// staging chunk limits: levels, rows, entries, staged first values
constexpr int KZ_CHL = 32, KZ_CHR = 256, KZ_CHE = 1024, KZ_CHX = 256;
constexpr unsigned long long WAIT_NS = 2000000000ull;  // 2 s bound on any wait

struct Pattern {                      // merged rows: a (and b) coefficients
    int rows = 0, cols = 0;
    std::vector<int64_t> rp;
    std::vector<int> ci;
    std::vector<double> a, b;
};

Pattern merge_pattern(const HCsr &A, const HCsr *B) {
    Pattern p;
    p.rows = A.m;
    p.cols = A.n;
    p.rp.assign(A.m + 1, 0);
    if (!B) {
        p.rp = A.rp;
        p.ci = A.ci;
        p.a = A.v;
        return p;
    }
    p.ci.reserve(A.ci.size() + B->ci.size());
    for (int i = 0; i < A.m; ++i) {
        int64_t e = A.rp[i], ee = A.rp[i + 1], f = B->rp[i], fe = B->rp[i + 1];
        while (e < ee || f < fe) {
            if (f >= fe || (e < ee && A.ci[e] < B->ci[f])) {
                p.ci.push_back(A.ci[e]); p.a.push_back(A.v[e]); p.b.push_back(0.0); ++e;
            } else if (e >= ee || B->ci[f] < A.ci[e]) {
                p.ci.push_back(B->ci[f]); p.a.push_back(0.0); p.b.push_back(B->v[f]); ++f;
            } else {
                p.ci.push_back(A.ci[e]); p.a.push_back(A.v[e]); p.b.push_back(B->v[f]); ++e; ++f;
            }
        }
        p.rp[i + 1] = (int64_t)p.ci.size();
    }
    return p;
}

// Scratch over columns with stamps, so analysing a band costs O(nnz(band)).
struct BandWork {
    std::vector<int> stamp, firstlv, lastlv, cnt, touched, rowlv;
    int id = 0;
    explicit BandWork(int cols) : stamp(cols, -1), firstlv(cols), lastlv(cols), cnt(cols) {}
};

// Levels and window slots of rows [r0, r1).  Returns levels; *slots = peak
// number of columns live (touched >= 2 times) at one level.
int analyze_band(const Pattern &p, int r0, int r1, BandWork &w, int *slots) {
    const int id = ++w.id;
    w.touched.clear();
    w.rowlv.resize(r1 - r0);
    int nlev = 0;
    for (int r = r0; r < r1; ++r) {
        int lv = 0;
        for (int64_t e = p.rp[r]; e < p.rp[r + 1]; ++e) {
            int c = p.ci[e];
            if (w.stamp[c] == id) lv = std::max(lv, w.lastlv[c] + 1);
        }
        for (int64_t e = p.rp[r]; e < p.rp[r + 1]; ++e) {
            int c = p.ci[e];
            if (w.stamp[c] != id) {
                w.stamp[c] = id;
                w.firstlv[c] = lv;
                w.cnt[c] = 0;
                w.touched.push_back(c);
            }
            w.lastlv[c] = lv;
            w.cnt[c]++;
        }
        w.rowlv[r - r0] = lv;
        nlev = std::max(nlev, lv + 1);
    }
    std::vector<int> diff(nlev + 2, 0);
    for (int c : w.touched)
        if (w.cnt[c] >= 2) {
            diff[w.firstlv[c]]++;
            diff[w.lastlv[c] + 1]--;
        }
    int cur = 0, peak = 0;
    for (int l = 0; l <= nlev; ++l) {
        cur += diff[l];
        peak = std::max(peak, cur);
    }
    *slots = peak;
    return nlev;
}

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(unsigned long long *p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// asynchronous global -> shared copies (sizes 4, 8 or 16 bytes, both aligned)
template <int S>
__device__ __forceinline__ void cp_async(void *dst, const void *src) {
    unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    if (S == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d), "l"(src), "n"(S)
                     : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// 16-byte vector moves of one n_b-wide row (LD a multiple of 4; both
// pointers 16-byte aligned): shared memory (generic) and global (L2 only).
template <typename T, int LD>
__device__ __forceinline__ void vld(T (&v)[LD], const T *p) {
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int i = 0; i < LD / 4; ++i) {
            const float4 t = reinterpret_cast<const float4 *>(p)[i];
            v[4 * i] = t.x; v[4 * i + 1] = t.y; v[4 * i + 2] = t.z; v[4 * i + 3] = t.w;
        }
    } else {
#pragma unroll
        for (int i = 0; i < LD / 2; ++i) {
            const double2 t = reinterpret_cast<const double2 *>(p)[i];
            v[2 * i] = t.x; v[2 * i + 1] = t.y;
        }
    }
}
template <typename T, int LD>
__device__ __forceinline__ void vld_cg(T (&v)[LD], const T *p) {
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int i = 0; i < LD / 4; ++i) {
            const float4 t = __ldcg(reinterpret_cast<const float4 *>(p) + i);
            v[4 * i] = t.x; v[4 * i + 1] = t.y; v[4 * i + 2] = t.z; v[4 * i + 3] = t.w;
        }
    } else {
#pragma unroll
        for (int i = 0; i < LD / 2; ++i) {
            const double2 t = __ldcg(reinterpret_cast<const double2 *>(p) + i);
            v[2 * i] = t.x; v[2 * i + 1] = t.y;
        }
    }
}
template <typename T, int LD>
__device__ __forceinline__ void vst(T *p, const T (&v)[LD]) {
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int i = 0; i < LD / 4; ++i)
            reinterpret_cast<float4 *>(p)[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
    } else {
#pragma unroll
        for (int i = 0; i < LD / 2; ++i)
            reinterpret_cast<double2 *>(p)[i] = make_double2(v[2 * i], v[2 * i + 1]);
    }
}
template <typename T, int LD>
__device__ __forceinline__ void vst_cg(T *p, const T (&v)[LD]) {
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int i = 0; i < LD / 4; ++i)
            __stcg(reinterpret_cast<float4 *>(p) + i, make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]));
    } else {
#pragma unroll
        for (int i = 0; i < LD / 2; ++i)
            __stcg(reinterpret_cast<double2 *>(p) + i, make_double2(v[2 * i], v[2 * i + 1]));
    }
}

__host__ __device__ constexpr int ilog2(int v) { return v <= 1 ? 0 : 1 + ilog2(v / 2); }
__host__ __device__ constexpr bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }
__device__ __forceinline__ int brev_low(int v, int nbits) {  // reverse the low nbits
    return nbits ? (int)(__brev((unsigned)v) >> (32 - nbits)) : 0;
}

// Row sums over the G = 2^lgG lanes of a row group (groups aligned in the
// warp; every lane of the warp calls).  Reduce-scatter: at step s each lane
// keeps the half of its columns selected by bit s of its lane index and adds
// the partner's copy of that half, so after log2(LD) steps lane l holds the
// sum of column brev(l mod LD); the remaining steps add across the lanes that
// hold the same column.  Needs G >= LD, LD a power of two.
template <typename T, int LD>
__device__ __forceinline__ T group_reduce_scatter(T (&v)[LD], int lane, int lgG) {
#pragma unroll
    for (int s = 0; (LD >> s) > 1; ++s) {
        const int h = (LD >> s) / 2;
        const bool up = (lane >> s) & 1;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const T keep = up ? v[h + i] : v[i];
            const T send = up ? v[i] : v[h + i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 1 << s);
        }
    }
    T r = v[0];
    for (int s = ilog2(LD); s < lgG; ++s) r += __shfl_xor_sync(0xffffffffu, r, 1 << s);
    return r;
}
template <typename T, int LD>
__device__ __forceinline__ void group_allreduce(T (&v)[LD], int lgG) {
    for (int s = 0; s < lgG; ++s) {
#pragma unroll
        for (int q = 0; q < LD; ++q) v[q] += __shfl_xor_sync(0xffffffffu, v[q], 1 << s);
    }
}

struct KView {
    int *err;
    int nbands;
    const int *band_chunk;   // nbands + 1
    const int4 *chunk;       // 2 per chunk: {L0, L1, R0, R1}, {E0, E1, X0, X1}
    const int4 *lvl;         // {first row, first req, publish, log2 lanes per row} + sentinel
    const int2 *rinfo;       // {original row, first entry}
    const int2 *ent;         // {column, flags}
    const int *xsc;          // columns staged per chunk
    const int2 *req;
    unsigned long long *progress;
    KCtl *ctl;
};

// Shared-memory layout of one staging buffer (byte offsets, 16-byte aligned).
constexpr size_t al16(size_t x) { return (x + 15) / 16 * 16; }
template <typename T, int LD, bool SHIFT>
struct Stage {
    static constexpr int VB = LD * (int)sizeof(T);          // bytes of one vector row
    static constexpr bool VALS = VB <= 64;                   // stage rhs / first values
    static constexpr size_t o_lv = 0;
    static constexpr size_t o_ri = al16(o_lv + 16 * (KZ_CHL + 1));
    static constexpr size_t o_inv = al16(o_ri + 8 * (KZ_CHR + 1));
    static constexpr size_t o_ent = al16(o_inv + 8 * KZ_CHR);
    static constexpr size_t o_a = al16(o_ent + 8 * KZ_CHE);
    static constexpr size_t o_b = al16(o_a + sizeof(T) * KZ_CHE);
    static constexpr size_t o_xc = al16(o_b + (SHIFT ? sizeof(T) * KZ_CHE : 0));
    static constexpr size_t o_rhs = al16(o_xc + 4 * KZ_CHX);
    static constexpr size_t o_xs = al16(o_rhs + (VALS ? (size_t)VB * KZ_CHR : 0));
    static constexpr size_t bytes = al16(o_xs + (VALS ? (size_t)VB * KZ_CHX : 0));
    static constexpr size_t stride = (bytes + 127) / 128 * 128;
};

__device__ __forceinline__ void bar_compute() {  // named barrier of the compute warps
    asm volatile("bar.sync 1, %0;" ::"n"(KZ_COMPUTE) : "memory");
}
__device__ __forceinline__ int ld_acq_cta(const int *p) {
    int v;
    asm volatile("ld.acquire.cta.shared.s32 %0, [%1];" : "=r"(v) : "r"((unsigned)__cvta_generic_to_shared(p)) : "memory");
    return v;
}
__device__ __forceinline__ void st_rel_cta(int *p, int v) {
    asm volatile("st.release.cta.shared.s32 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(p)), "r"(v) : "memory");
}

// Warps 0 .. KZ_COMPUTE/32 - 1 compute; the last warp polls (acquire) the
// progress that upcoming levels require from earlier bands, so that the
// compute warps only wait on a shared-memory flag.  Thread 0 publishes the
// band's progress (release) at most every KZ_PUB levels when a later band
// waits on it, and at the end of the band.
template <typename T, int LD, bool SHIFT>
__global__ void __launch_bounds__(KZ_THREADS)
    k_kaczmarz(KView kv, const T *__restrict__ ea, const T *__restrict__ eb,
               const T *__restrict__ inv, const T *__restrict__ rhs, T *x,
               const double *__restrict__ shift, int window_slots) {
    using SG = Stage<T, LD, SHIFT>;
    extern __shared__ __align__(128) unsigned char smraw[];
    T *win = reinterpret_cast<T *>(smraw);
    unsigned char *bufs = smraw + ((size_t)window_slots * LD * sizeof(T) + 127) / 128 * 128;
    __shared__ int s_band;
    __shared__ int s_abort;
    __shared__ int s_done;   // band-local levels completed by the compute warps
    __shared__ int s_ready;  // band-local levels whose requirements are met
    __shared__ unsigned long long s_pc[64];  // comm warp: band << 32 | observed level
    const bool comm = threadIdx.x >= KZ_COMPUTE;
    T sh[SHIFT ? LD : 1];
#pragma unroll
    for (int q = 0; q < (SHIFT ? LD : 1); ++q) sh[q] = SHIFT ? (T)shift[q] : T(0);
    const unsigned long long epoch = *((volatile unsigned long long *)&kv.ctl->epoch);
    if (threadIdx.x == 0) s_abort = 0;
    if (threadIdx.x < 64) s_pc[threadIdx.x] = ~0ull;

    auto load_sched = [&](int c, int bi) {
        unsigned char *B = bufs + (size_t)bi * SG::stride;
        const int4 c0 = kv.chunk[2 * c], c1 = kv.chunk[2 * c + 1];
        const int nl = c0.y - c0.x, nr = c0.w - c0.z, ne = c1.y - c1.x, nx = c1.w - c1.z;
        for (int q = threadIdx.x; q <= nl; q += KZ_COMPUTE)
            cp_async<16>(B + SG::o_lv + 16 * q, kv.lvl + c0.x + q);
        for (int q = threadIdx.x; q <= nr; q += KZ_COMPUTE)
            cp_async<8>(B + SG::o_ri + 8 * q, kv.rinfo + c0.z + q);
        for (int q = threadIdx.x; q < nr; q += KZ_COMPUTE)
            cp_async<sizeof(T)>(B + SG::o_inv + sizeof(T) * q, inv + c0.z + q);
        for (int q = threadIdx.x; q < ne; q += KZ_COMPUTE) {
            cp_async<8>(B + SG::o_ent + 8 * q, kv.ent + c1.x + q);
            cp_async<sizeof(T)>(B + SG::o_a + sizeof(T) * q, ea + c1.x + q);
            if (SHIFT) cp_async<sizeof(T)>(B + SG::o_b + sizeof(T) * q, eb + c1.x + q);
        }
        for (int q = threadIdx.x; q < nx; q += KZ_COMPUTE)
            cp_async<4>(B + SG::o_xc + 4 * q, kv.xsc + c1.z + q);
        cp_commit();
    };
    auto load_vals = [&](int c, int bi) {
        unsigned char *B = bufs + (size_t)bi * SG::stride;
        if (SG::VALS) {
            const int4 c0 = kv.chunk[2 * c], c1 = kv.chunk[2 * c + 1];
            const int nr = c0.w - c0.z, nx = c1.w - c1.z;
            const int2 *ri = reinterpret_cast<const int2 *>(B + SG::o_ri);
            const int *xc = reinterpret_cast<const int *>(B + SG::o_xc);
            constexpr int P = SG::VB / 16;
            if (rhs)
                for (int q = threadIdx.x; q < nr * P; q += KZ_COMPUTE) {
                    const int r = q / P, p = q % P;
                    cp_async<16>(B + SG::o_rhs + (size_t)SG::VB * r + 16 * p,
                                 reinterpret_cast<const unsigned char *>(rhs + (size_t)ri[r].x * LD) + 16 * p);
                }
            for (int q = threadIdx.x; q < nx * P; q += KZ_COMPUTE) {
                const int r = q / P, p = q % P;
                cp_async<16>(B + SG::o_xs + (size_t)SG::VB * r + 16 * p,
                             reinterpret_cast<const unsigned char *>(x + (size_t)xc[r] * LD) + 16 * p);
            }
        }
        cp_commit();
    };

    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            s_band = (int)atomicAdd(&kv.ctl->ticket, 1u);
            s_done = 0;
            s_ready = 0;
        }
        __syncthreads();
        const int b = s_band;
        if (b >= kv.nbands || s_abort) break;
        const int cb = kv.band_chunk[b], ce = kv.band_chunk[b + 1];
        const int Lband = kv.chunk[2 * cb].x;
        const int Lend = kv.chunk[2 * (ce - 1)].y;
        const int nlev = Lend - Lband;
        if (comm) {
            // ---------------------------------------------- communication warp
            const int lane = threadIdx.x & 31;
            int published = 0, ready = 0;
            unsigned long long t0 = gtimer();  // re-armed whenever something advances
            while (published < nlev) {
                bool aborted = *((volatile int *)&s_abort) != 0;
                if (!aborted && (*((volatile int *)kv.err) || gtimer() - t0 > WAIT_NS)) {
                    if (lane == 0) {
                        atomicExch(kv.err, 1);
                        s_abort = 1;
                    }
                    aborted = true;
                }
                if (aborted) {
                    if (lane == 0) st_rel_cta(&s_ready, nlev);  // release the compute warps
                    break;
                }
                // requirements of the next levels, a few at a time
                int adv = 0;
                while (ready < nlev && adv < 8) {
                    const int4 l0 = kv.lvl[Lband + ready], l1 = kv.lvl[Lband + ready + 1];
                    bool ok = true;
                    for (int q = l0.y + lane; q < l1.y; q += 32) {
                        const int2 rq = kv.req[q];
                        const unsigned long long key = s_pc[rq.x & 63];
                        if ((int)(key >> 32) == rq.x && (unsigned)key >= (unsigned)rq.y) continue;
                        const unsigned long long v = ld_acquire(&kv.progress[rq.x]);
                        if ((v >> 32) == epoch)
                            s_pc[rq.x & 63] = ((unsigned long long)(unsigned)rq.x << 32) | (v & 0xffffffffull);
                        ok = ok && (v >= ((epoch << 32) | (unsigned)rq.y));
                    }
                    ok = __all_sync(0xffffffffu, ok);
                    if (!ok) break;
                    ++ready;
                    ++adv;
                }
                if (adv && lane == 0) st_rel_cta(&s_ready, ready);
                if (adv) t0 = gtimer();
                // the compute warps publish; follow their progress to finish
                const int done = *((volatile int *)&s_done);
                if (done > published) {
                    published = done;
                    t0 = gtimer();
                }
                if (!adv && done == published) __nanosleep(20);
            }
        } else {
            // ---------------------------------------------- compute warps
            bool pend_pub = false;  // thread 0: a flagged level awaits publication
            // pipeline over chunks: schedule arrays two chunks ahead, right-hand
            // sides and first values one chunk ahead, so that only the chunk
            // being processed is waited for
            load_sched(cb, 0);
            cp_wait<0>();
            bar_compute();
            load_vals(cb, 0);
            if (cb + 1 < ce) load_sched(cb + 1, 1);
            else cp_commit();
            for (int c = cb; c < ce; ++c) {
                const int bi = (c - cb) % KZ_NBUF;
                unsigned char *B = bufs + (size_t)bi * SG::stride;
                // sched(c+1) and vals(c) were issued one step earlier
                cp_wait<0>();
                bar_compute();
                if (c + 1 < ce) load_vals(c + 1, (c + 1 - cb) % KZ_NBUF);
                else cp_commit();
                if (c + 2 < ce) load_sched(c + 2, (c + 2 - cb) % KZ_NBUF);
                else cp_commit();
                const int4 c0 = kv.chunk[2 * c], c1 = kv.chunk[2 * c + 1];
                const int4 *lv = reinterpret_cast<const int4 *>(B + SG::o_lv);
                const int2 *ri = reinterpret_cast<const int2 *>(B + SG::o_ri);
                const T *sinv = reinterpret_cast<const T *>(B + SG::o_inv);
                const int2 *se = reinterpret_cast<const int2 *>(B + SG::o_ent);
                const T *sa = reinterpret_cast<const T *>(B + SG::o_a);
                const T *sb = reinterpret_cast<const T *>(B + SG::o_b);
                const T *srhs = reinterpret_cast<const T *>(B + SG::o_rhs);
                const T *sxs = reinterpret_cast<const T *>(B + SG::o_xs);
                for (int L = 0; L < c0.y - c0.x; ++L) {
                    const int4 l0 = lv[L], l1 = lv[L + 1];
                    const int lb = c0.x + L - Lband;  // band-local level
                    if (l1.y > l0.y) {
                        // requirements of this level: wait for the comm warp,
                        // which releases every wait when it gives up.  The
                        // compute warps never leave the loop early, so every
                        // named barrier is reached by all of them.
                        const unsigned long long t0 = gtimer();
                        while (ld_acq_cta(&s_ready) <= lb) {
                            if (gtimer() - t0 > 2 * WAIT_NS) break;
                        }
                    }
                    {
                        // G = 2^lgG lanes per row (the smallest power of two not
                        // below the sub-level's longest row, at most 32); lane lg
                        // takes entries lg, lg + G, ... for all LD columns.  A
                        // warp holding no row of the level goes straight to the
                        // barrier.
                        const int lgG = l0.w;
                        const int G = 1 << lgG;
                        const int nrow = l1.x - l0.x;
                        const int lane = threadIdx.x & 31;
                        const int lg = threadIdx.x & (G - 1);
                        const int wrow = (threadIdx.x & ~31) >> lgG;
                        for (int pr = 0; pr + wrow < nrow; pr += KZ_COMPUTE >> lgG) {
                            const int r = pr + (threadIdx.x >> lgG);
                            const bool act = r < nrow;
                            const int k = l0.x - c0.z + r;
                            T acc[LD], nrm[SHIFT ? LD : 1];
#pragma unroll
                            for (int q = 0; q < LD; ++q) acc[q] = T(0);
#pragma unroll
                            for (int q = 0; q < (SHIFT ? LD : 1); ++q) nrm[q] = T(0);
                            // the lane's first entry stays in registers for the update
                            int2 fen = make_int2(0, 0);
                            T fa = T(0), fb = T(0), fv[LD];
                            int e1 = 0;
                            bool own = false;
                            if (act) {
                                const int e0 = ri[k].y - c1.x;
                                e1 = ri[k + 1].y - c1.x;
                                own = e0 + lg < e1;
                                for (int e = e0 + lg; e < e1; e += G) {
                                    const int2 en = se[e];
                                    const T a = sa[e];
                                    const T bq = SHIFT ? sb[e] : T(0);
                                    T val[LD];
                                    const int fl = en.y;
                                    if (!(fl & 1))
                                        vld<T, LD>(val, win + ((fl >> 3) & 0xfff) * LD);
                                    else if (SG::VALS && (fl & 4))
                                        vld<T, LD>(val, sxs + (fl >> 15) * LD);
                                    else
                                        vld_cg<T, LD>(val, x + (size_t)en.x * LD);
#pragma unroll
                                    for (int q = 0; q < LD; ++q) {
                                        const T coef = SHIFT ? a - sh[q] * bq : a;
                                        acc[q] = fma(coef, val[q], acc[q]);
                                        if (SHIFT) nrm[q] = fma(coef, coef, nrm[q]);
                                    }
                                    if (e == e0 + lg) {
                                        fen = en; fa = a; fb = bq;
#pragma unroll
                                        for (int q = 0; q < LD; ++q) fv[q] = val[q];
                                    }
                                }
                            }
                            // d_q = (b_i - <a_i, x_q>) / ||a_i||^2 for every column q
                            T d[LD];
                            if (pow2(LD) && G >= LD) {
                                const T sa_c = group_reduce_scatter<T, LD>(acc, lane, lgG);
                                const T sn_c = SHIFT ? group_reduce_scatter<T, (SHIFT ? LD : 1)>(nrm, lane, lgG) : T(0);
                                const int c = brev_low(lane & (LD - 1), ilog2(LD));
                                T dc = T(0);
                                if (act) {
                                    const T bi = rhs ? (SG::VALS ? srhs[k * LD + c] : rhs[(size_t)ri[k].x * LD + c]) : T(0);
                                    dc = SHIFT ? (sn_c > T(0) ? (bi - sa_c) / sn_c : T(0)) : (bi - sa_c) * sinv[k];
                                }
                                const int gb = lane & ~(G - 1);
#pragma unroll
                                for (int q = 0; q < LD; ++q)
                                    d[q] = __shfl_sync(0xffffffffu, dc, gb + brev_low(q, ilog2(LD)));
                            } else {
                                group_allreduce<T, LD>(acc, lgG);
                                if (SHIFT) group_allreduce<T, (SHIFT ? LD : 1)>(nrm, lgG);
#pragma unroll
                                for (int q = 0; q < LD; ++q) d[q] = T(0);
                                if (act) {
#pragma unroll
                                    for (int q = 0; q < LD; ++q) {
                                        const T bi = rhs ? (SG::VALS ? srhs[k * LD + q] : rhs[(size_t)ri[k].x * LD + q]) : T(0);
                                        const T nq = SHIFT ? nrm[q] : T(1);
                                        d[q] = SHIFT ? (nq > T(0) ? (bi - acc[q]) / nq : T(0)) : (bi - acc[q]) * sinv[k];
                                    }
                                }
                            }
                            // x_q += d_q a_i on the row's entries
                            if (own) {
                                const int e0 = ri[k].y - c1.x;
                                for (int e = e0 + lg; e < e1; e += G) {
                                    int2 en = fen;
                                    T a = fa, bq = fb, val[LD];
                                    if (e == e0 + lg) {
#pragma unroll
                                        for (int q = 0; q < LD; ++q) val[q] = fv[q];
                                    } else {
                                        en = se[e];
                                        a = sa[e];
                                        bq = SHIFT ? sb[e] : T(0);
                                        const int fl = en.y;
                                        if (!(fl & 1))
                                            vld<T, LD>(val, win + ((fl >> 3) & 0xfff) * LD);
                                        else if (SG::VALS && (fl & 4))
                                            vld<T, LD>(val, sxs + (fl >> 15) * LD);
                                        else
                                            vld_cg<T, LD>(val, x + (size_t)en.x * LD);
                                    }
#pragma unroll
                                    for (int q = 0; q < LD; ++q) {
                                        const T coef = SHIFT ? a - sh[q] * bq : a;
                                        val[q] = fma(d[q], coef, val[q]);
                                    }
                                    if (en.y & 2)
                                        vst_cg<T, LD>(x + (size_t)en.x * LD, val);
                                    else
                                        vst<T, LD>(win + ((en.y >> 3) & 0xfff) * LD, val);
                                }
                            }
                        }
                    }
                    bar_compute();
                    if (threadIdx.x == 0) {
                        pend_pub = pend_pub || l0.z;
                        // the release makes every compute thread's stores of the
                        // finished levels visible (cumulative over the barrier)
                        if (pend_pub && ((lb + 1) % KZ_PUB == 0 || lb + 1 == nlev)) {
                            st_release(&kv.progress[b], (epoch << 32) | (unsigned)(lb + 1));
                            pend_pub = false;
                        }
                        *((volatile int *)&s_done) = lb + 1;
                    }
                }
            }
            cp_wait<0>();
            bar_compute();
            if (threadIdx.x == 0) st_release(&kv.progress[b], (epoch << 32) | (unsigned)nlev);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned d = atomicAdd(&kv.ctl->done, 1u);
        if (d == gridDim.x - 1) {  // last CTA: reset for the next launch
            kv.ctl->ticket = 0;
            kv.ctl->done = 0;
            kv.ctl->epoch = epoch + 1;
            __threadfence();
        }
    }
}


template <typename T, int LD, bool SHIFT>
void launch_one(const KSched &ks, const T *ea, const T *eb, const T *inv, const T *rhs, T *x,
                const double *shift, cudaStream_t s) {
    using SG = Stage<T, LD, SHIFT>;
    auto kern = k_kaczmarz<T, LD, SHIFT>;
    const int slots = std::max(ks.max_slots, 1);
    const size_t smem = ((size_t)slots * LD * sizeof(T) + 127) / 128 * 128 + KZ_NBUF * SG::stride;
    // per kernel instance: the largest dynamic shared memory set so far, and
    // the SM count; per schedule and instance: the resident CTA count
    static size_t smem_set = 0;
    static int nsm = 0;
    if (smem > smem_set) {
        SAMG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        smem_set = smem;
    }
    if (!nsm) {
        int dev = 0;
        SAMG_CUDA(cudaGetDevice(&dev));
        SAMG_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    }
    const int key = (int)sizeof(T) * 64 + LD * 2 + (SHIFT ? 1 : 0);
    int &grid = ks.grid_cache[key & 255];
    if (!grid) {
        int bps = 0;
        SAMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, KZ_THREADS, smem));
        SAMG_CHECK(bps > 0, SAMG_E_CUDA, "kaczmarz: staging buffers do not fit in shared memory");
        grid = std::min(ks.nbands, nsm * bps);
    }
    KView kv{ks.err ? ks.err : &ks.ctl.p->err, ks.nbands, ks.band_chunk.p, ks.chunk.p, ks.lvl.p,
             ks.rinfo.p, ks.ent.p, ks.xsc.p, ks.req.p, ks.progress.p, ks.ctl.p};
    SAMG_COUNT_LAUNCH();
    kern<<<grid, KZ_THREADS, smem, s>>>(kv, ea, eb, inv, rhs, x, shift, slots);
    SAMG_CUDA(cudaGetLastError());
}

}  // namespace

void build_kschedule(const HCsr &A, const HCsr *B, KSched &ks, cudaStream_t s) {
    Pattern p = merge_pattern(A, B);
    const int rows = p.rows, cols = p.cols;
    ks.rows = rows;
    ks.cols = cols;
    ks.shifted = (B != nullptr);
    BandWork w(cols);
    // 1. bands: contiguous rows, grown until about TARGET_PAR rows per level
    std::vector<int> bstart;
    int slots = 0;
    for (int r0 = 0; r0 < rows;) {
        int R = std::min(256, rows - r0), good = 0;
        for (;;) {
            int nl = analyze_band(p, r0, r0 + R, w, &slots);
            if (slots > SLOT_CAP) {
                if (good) break;
                R = std::max(1, R / 2);
                if (R == 1) { good = 1; break; }
                continue;
            }
            good = R;
            if (r0 + R >= rows || R >= MAX_BAND_ROWS || (R / std::max(nl, 1)) >= TARGET_PAR) break;
            R = std::min(2 * R, rows - r0);
        }
        bstart.push_back(r0);
        r0 += good;
    }
    const int nb = (int)bstart.size();
    bstart.push_back(rows);
    ks.nbands = nb;
    // 2. per band: levels, window slots, sub-levels (<= chunk limits), chunks
    std::vector<int> band_chunk(nb + 1, 0);
    std::vector<int4> lvl, chunk;
    std::vector<int2> rinfo, ent, req;
    std::vector<int> xsc;
    std::vector<double> ea, eb, inv;
    std::vector<int> g_band(cols, -1), g_sub(cols, 0), slot(cols, 0), last_sub(cols, 0);
    std::vector<int> waited(nb, 0), waited_stamp(nb, -1);
    ent.reserve(p.ci.size());
    ea.reserve(p.ci.size());
    if (ks.shifted) eb.reserve(p.ci.size());
    int max_slots = 0;
    std::vector<std::vector<int>> pub(nb);  // per band: band-local sub-levels to publish
    std::vector<int> band_lvl0(nb + 1, 0);
    struct PendReq { int sub, band, need; };
    struct RowRec { int row, sub; };
    for (int b = 0; b < nb; ++b) {
        const int r0 = bstart[b], r1 = bstart[b + 1];
        int nl = analyze_band(p, r0, r1, w, &slots);
        max_slots = std::max(max_slots, slots);
        // rows grouped by level (ascending row order inside a level)
        std::vector<int> lcount(nl + 1, 0);
        for (int r = r0; r < r1; ++r) lcount[w.rowlv[r - r0] + 1]++;
        for (int l = 0; l < nl; ++l) lcount[l + 1] += lcount[l];
        std::vector<int> order(r1 - r0);
        {
            std::vector<int> fillp(lcount.begin(), lcount.end() - 1);
            for (int r = r0; r < r1; ++r) order[fillp[w.rowlv[r - r0]]++] = r;
        }
        // window slots by interval colouring over levels
        std::vector<std::vector<int>> starts(nl), ends(nl);
        for (int c : w.touched)
            if (w.cnt[c] >= 2) {
                starts[w.firstlv[c]].push_back(c);
                ends[w.lastlv[c]].push_back(c);
            }
        {
            std::vector<int> freel;
            int next = 0;
            for (int l = 0; l < nl; ++l) {
                for (int c : starts[l]) {
                    if (!freel.empty()) { slot[c] = freel.back(); freel.pop_back(); }
                    else slot[c] = next++;
                }
                for (int c : ends[l]) freel.push_back(slot[c]);
            }
        }
        // sub-levels: a level's independent rows split so that each piece fits
        // one staging chunk
        std::vector<RowRec> rr;
        std::vector<int> sub_rows, sub_ents, sub_xs, sub_maxe;  // per sub-level counts
        for (int l = 0; l < nl; ++l) {
            int cr = 0, ce = 0, cx = 0;
            bool open = false;
            for (int k = lcount[l]; k < lcount[l + 1]; ++k) {
                const int r = order[k];
                const int ne = (int)(p.rp[r + 1] - p.rp[r]);
                int nx = 0;
                for (int64_t e = p.rp[r]; e < p.rp[r + 1]; ++e) {
                    const int c = p.ci[e];
                    if (w.firstlv[c] == l && g_band[c] < 0) ++nx;
                }
                if (!open || cr + 1 > KZ_CHR || ce + ne > KZ_CHE || cx + nx > KZ_CHX) {
                    sub_rows.push_back(0); sub_ents.push_back(0); sub_xs.push_back(0);
                    sub_maxe.push_back(0);
                    cr = ce = cx = 0;
                    open = true;
                }
                SAMG_CHECK(ne <= KZ_CHE && nx <= KZ_CHX, SAMG_E_INVALID,
                           "kaczmarz: a row has more entries than a staging chunk holds");
                cr += 1; ce += ne; cx += nx;
                sub_rows.back() = cr; sub_ents.back() = ce; sub_xs.back() = cx;
                sub_maxe.back() = std::max(sub_maxe.back(), ne);
                rr.push_back({r, (int)sub_rows.size() - 1});
            }
        }
        const int nsub = (int)sub_rows.size();
        // chunks of consecutive sub-levels
        std::vector<int> sub_chunk(nsub), chunk_first_sub;
        {
            int cl = 0, cr = 0, ce = 0, cx = 0;
            for (int q = 0; q < nsub; ++q) {
                if (q == 0 || cl + 1 > KZ_CHL || cr + sub_rows[q] > KZ_CHR ||
                    ce + sub_ents[q] > KZ_CHE || cx + sub_xs[q] > KZ_CHX) {
                    chunk_first_sub.push_back(q);
                    cl = cr = ce = cx = 0;
                }
                cl += 1; cr += sub_rows[q]; ce += sub_ents[q]; cx += sub_xs[q];
                sub_chunk[q] = (int)chunk_first_sub.size() - 1;
            }
        }
        for (const RowRec &x : rr)
            for (int64_t e = p.rp[x.row]; e < p.rp[x.row + 1]; ++e)
                if (w.lastlv[p.ci[e]] == w.rowlv[x.row - r0]) last_sub[p.ci[e]] = x.sub;
        // emit levels, rows, entries, chunk records, requirements
        const int L0 = (int)lvl.size();
        band_lvl0[b] = L0;
        band_chunk[b] = (int)chunk.size() / 2;
        std::vector<PendReq> pend;
        size_t ri = 0;
        int cur_chunk = -1, xs_local = 0;
        int4 crec0{0, 0, 0, 0}, crec1{0, 0, 0, 0};
        auto close_chunk = [&]() {
            if (cur_chunk < 0) return;
            crec0.y = (int)lvl.size();
            crec0.w = (int)rinfo.size();
            crec1.y = (int)ent.size();
            crec1.w = (int)xsc.size();
            chunk.push_back(crec0);
            chunk.push_back(crec1);
        };
        for (int q = 0; q < nsub; ++q) {
            if (sub_chunk[q] != cur_chunk) {
                close_chunk();
                cur_chunk = sub_chunk[q];
                crec0 = int4{(int)lvl.size(), 0, (int)rinfo.size(), 0};
                crec1 = int4{(int)ent.size(), 0, (int)xsc.size(), 0};
                xs_local = 0;
            }
            // lanes per row: a power of two >= the longest row of the level
            // (at most 32; longer rows give a lane several entries)
            int lg = 0;
            while (lg < 5 && (1 << lg) < sub_maxe[q]) ++lg;
            int4 L4{(int)rinfo.size(), 0, 0, lg};
            lvl.push_back(L4);
            for (; ri < rr.size() && rr[ri].sub == q; ++ri) {
                const int r = rr[ri].row;
                const int lv = w.rowlv[r - r0];
                rinfo.push_back(make_int2(r, (int)ent.size()));
                double n2 = 0.0;
                for (int64_t e = p.rp[r]; e < p.rp[r + 1]; ++e) {
                    const int c = p.ci[e];
                    const int first = (w.firstlv[c] == lv), last = (w.lastlv[c] == lv);
                    const int sl = (w.cnt[c] >= 2) ? slot[c] : 0;
                    int staged = 0, xi = 0;
                    if (first && g_band[c] < 0) {
                        staged = 1;
                        xi = xs_local++;
                        xsc.push_back(c);
                    }
                    ent.push_back(make_int2(c, first | (last << 1) | (staged << 2) | (sl << 3) | (xi << 15)));
                    ea.push_back(p.a[e]);
                    if (ks.shifted) eb.push_back(p.b[e]);
                    n2 += p.a[e] * p.a[e];
                    if (first && g_band[c] >= 0) pend.push_back({q, g_band[c], g_sub[c] + 1});
                }
                inv.push_back(n2 > 0.0 ? 1.0 / n2 : 0.0);
            }
        }
        close_chunk();
        // per sub-level: max need per band, dropping needs already waited for
        std::sort(pend.begin(), pend.end(), [](const PendReq &a, const PendReq &b2) {
            return a.sub != b2.sub ? a.sub < b2.sub : (a.band != b2.band ? a.band < b2.band : a.need > b2.need);
        });
        size_t q = 0;
        for (int l = 0; l < nsub; ++l) {
            lvl[L0 + l].y = (int)req.size();
            while (q < pend.size() && pend[q].sub == l) {
                const PendReq &pr = pend[q];
                if (waited_stamp[pr.band] != b || waited[pr.band] < pr.need) {
                    waited_stamp[pr.band] = b;
                    waited[pr.band] = pr.need;
                    req.push_back(make_int2(pr.band, pr.need));
                    pub[pr.band].push_back(pr.need - 1);
                }
                const int bb = pr.band;
                while (q < pend.size() && pend[q].sub == l && pend[q].band == bb) ++q;
            }
        }
        for (int c : w.touched) {
            g_band[c] = b;
            g_sub[c] = last_sub[c];
        }
    }
    band_chunk[nb] = (int)chunk.size() / 2;
    band_lvl0[nb] = (int)lvl.size();
    for (int b = 0; b < nb; ++b)
        for (int l : pub[b]) lvl[band_lvl0[b] + l].z = 1;
    lvl.push_back(int4{(int)rinfo.size(), (int)req.size(), 0, 0});
    rinfo.push_back(make_int2(0, (int)ent.size()));
    ks.nlevels = (int)lvl.size() - 1;
    ks.max_slots = max_slots;
    ks.nent = (int64_t)ent.size();
    ks.nchunks = (int)chunk.size() / 2;
    // 3. upload
    ks.band_chunk.upload(band_chunk.data(), band_chunk.size(), s);
    ks.chunk.upload(chunk.data(), chunk.size(), s);
    ks.lvl.upload(lvl.data(), lvl.size(), s);
    ks.rinfo.upload(rinfo.data(), rinfo.size(), s);
    if (ent.empty()) ent.push_back(make_int2(0, 0));
    ks.ent.upload(ent.data(), ent.size(), s);
    ks.ea_d.upload(ea.data(), ea.size(), s);
    std::vector<float> f(ea.begin(), ea.end());
    ks.ea_f.upload(f.data(), f.size(), s);
    if (ks.shifted) {
        ks.eb_d.upload(eb.data(), eb.size(), s);
        std::vector<float> fb(eb.begin(), eb.end());
        ks.eb_f.upload(fb.data(), fb.size(), s);
    }
    ks.inv_d.upload(inv.data(), inv.size(), s);
    std::vector<float> fi(inv.begin(), inv.end());
    ks.inv_f.upload(fi.data(), fi.size(), s);
    if (xsc.empty()) xsc.push_back(0);
    ks.xsc.upload(xsc.data(), xsc.size(), s);
    if (req.empty()) req.push_back(make_int2(0, 0));
    ks.req.upload(req.data(), req.size(), s);
    ks.progress.alloc(std::max(nb, 1));
    ks.progress.zero(s);
    ks.ctl.alloc(1);
    KCtl c0;
    std::memset(&c0, 0, sizeof(c0));
    c0.epoch = 1;
    ks.ctl.upload(&c0, 1, s);
    SAMG_CUDA(cudaStreamSynchronize(s));
}

template <typename T>
static void dispatch(const KSched &ks, int ld, const T *ea, const T *eb, const T *inv,
                     const T *rhs, T *x, const double *shift, cudaStream_t s) {
    if (ks.rows == 0) return;
#define KZ_CASE(L)                                                                   \
    case L:                                                                          \
        if (ks.shifted) launch_one<T, L, true>(ks, ea, eb, inv, rhs, x, shift, s);   \
        else launch_one<T, L, false>(ks, ea, eb, inv, rhs, x, shift, s);             \
        break;
    switch (ld) {
        KZ_CASE(4)
        KZ_CASE(8)
        KZ_CASE(12)
        KZ_CASE(16)
        default:
            throw Error(SAMG_E_INVALID, "kaczmarz: unsupported block width");
    }
#undef KZ_CASE
}

template <>
void launch_kaczmarz<double>(const KSched &ks, int ld, const double *rhs, double *x,
                             const double *shift, cudaStream_t s) {
    dispatch<double>(ks, ld, ks.ea_d.p, ks.eb_d.p, ks.inv_d.p, rhs, x, shift, s);
}
template <>
void launch_kaczmarz<float>(const KSched &ks, int ld, const float *rhs, float *x,
                            const double *shift, cudaStream_t s) {
    dispatch<float>(ks, ld, ks.ea_f.p, ks.eb_f.p, ks.inv_f.p, rhs, x, shift, s);
}

void kaczmarz_check(const KSched &ks, cudaStream_t s) {
    if (ks.rows == 0) return;
    int e = 0;
    const int *p = ks.err ? ks.err : &ks.ctl.p->err;
    SAMG_CUDA(cudaMemcpyAsync(&e, p, sizeof(int), cudaMemcpyDeviceToHost, s));
    SAMG_CUDA(cudaStreamSynchronize(s));
    SAMG_CHECK(e == 0, SAMG_E_TIMEOUT, "kaczmarz: a cross-band wait timed out");
}

}  // namespace samg
