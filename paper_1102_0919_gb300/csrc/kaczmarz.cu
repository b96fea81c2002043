// kaczmarz.cu -- schedule builder (host) and sweep kernel (device) for the
// exact-order Kaczmarz relaxation of Sec. 5.3 (see kaczmarz.cuh).
#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <exception>
#include <memory>
#include <mutex>
#include <queue>
#include <thread>
#include <type_traits>

#include "kaczmarz.cuh"

namespace samg {

namespace {

constexpr int KZ_THREADS = 512;
constexpr int KZ_COMPUTE = 480;    // compute threads (15 warps); warp 15 stages, polls, publishes
constexpr int KZ_NBUF = 3;          // staging buffers (the producer runs up to 2 chunks ahead)
constexpr int TARGET_PAR = 32;       // wanted rows per level inside a band
constexpr int MAX_BAND_ROWS = 1 << 21;
constexpr int SLOT_CAP = 512;        // window slots: 512 * 16 cols * 8 B = 64 KiB
// staging chunk limits: levels, rows, entries, staged first values,
// cross-band requirements carried in the image
constexpr int KZ_CHL = 32, KZ_CHR = 256, KZ_CHE = 1024, KZ_CHX = 256, KZ_CHQ = 256;
constexpr unsigned long long WAIT_NS = 2000000000ull;  // 2 s bound on any wait
constexpr unsigned FULL = 0xffffffffu;

// Byte layout of one chunk image: the schedule of up to KZ_CHL levels, copied
// to shared memory by one bulk copy.  Every array starts on 16 bytes.
//   lv  int4 per level {first row, rows, log2 lanes per row,
//                       flags: 1 has requirements | 2 publish after it}
//   lq  int2 per level {first requirement in rq, count}; count < 0: the
//                      level's -count - 1 requirements are read from the
//                      schedule's global list at the first index instead
//   ri  int2 per row   {original row, first entry | entries << 16}
//   inv T per row      1 / ||a_i||^2 (unshifted form)
//   ent int2 per entry {column, 1 first | 2 last | 4 staged | (slot + 1) << 3 | xs << 15}
//   a, b T per entry   coefficients (b: shifted form only)
//   xc  int per staged first value: its column
//   rq  int2 per requirement {band, levels that band must have completed}
struct ImgLayout {
    unsigned lv, lq, ri, inv, ent, a, b, xc, rq, bytes;
};
__host__ __device__ constexpr unsigned al16u(unsigned v) { return (v + 15u) & ~15u; }
__host__ __device__ constexpr ImgLayout img_layout(int nl, int nr, int ne, int nx, int nq, int tsz,
                                                   bool shifted) {
    const unsigned lq = al16u(16u * nl);
    const unsigned ri = al16u(lq + 8u * nl);
    const unsigned inv = al16u(ri + 8u * nr);
    const unsigned ent = al16u(inv + (unsigned)tsz * nr);
    const unsigned a = al16u(ent + 8u * ne);
    const unsigned b = al16u(a + (unsigned)tsz * ne);
    const unsigned xc = al16u(b + (shifted ? (unsigned)tsz * ne : 0u));
    const unsigned rq = al16u(xc + 4u * nx);
    return ImgLayout{0u, lq, ri, inv, ent, a, b, xc, rq, al16u(rq + 8u * nq)};
}

struct Pattern {                      // rows of a sweep program: a (and b) coefficients
    int rows = 0, cols = 0;
    std::vector<int64_t> rp;
    std::vector<int> ci;
    std::vector<double> a, b;
    std::vector<int> rhs;             // right-hand-side row of each row (empty: its own)
    std::vector<int> seg;             // first rows of the program's sweeps after the first:
                                      // no band crosses one
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

// Dependency level of every row in natural order over the whole operator:
// 1 + the level of the latest earlier row that shares a column.
std::vector<int> global_levels(const Pattern &p) {
    std::vector<int> last(p.cols, -1), lv(p.rows, 0);
    for (int r = 0; r < p.rows; ++r) {
        int l = 0;
        for (int64_t e = p.rp[r]; e < p.rp[r + 1]; ++e) l = std::max(l, last[p.ci[e]] + 1);
        lv[r] = l;
        for (int64_t e = p.rp[r]; e < p.rp[r + 1]; ++e) last[p.ci[e]] = l;
    }
    return lv;
}

// Levels and window slots of rows [r0, r1).  A row's band level is the rank
// of its global level among the global levels present in the band, so every
// band steps through the same global wavefront and a band waits for an
// earlier band only as long as a true dependency requires.  Returns levels;
// *slots = peak number of columns live (touched >= 2 times) at one level.
int analyze_band(const Pattern &p, const std::vector<int> &glv, int r0, int r1, BandWork &w,
                 int *slots) {
    const int id = ++w.id;
    w.touched.clear();
    w.rowlv.resize(r1 - r0);
    // ranks of the band's global levels
    std::vector<int> g(glv.begin() + r0, glv.begin() + r1);
    std::sort(g.begin(), g.end());
    g.erase(std::unique(g.begin(), g.end()), g.end());
    const int nlev = (int)g.size();
    for (int r = r0; r < r1; ++r) {
        const int lv = (int)(std::lower_bound(g.begin(), g.end(), glv[r]) - g.begin());
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
// asynchronous 16-byte global -> shared copy (both addresses 16-byte aligned)
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
// mbarriers: chunk images arrive by bulk copy (transaction count), gathered
// values by cp.async with one no-increment arrival per producer lane
__device__ __forceinline__ void mbar_init(unsigned long long *b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)),
                 "r"(bytes) : "memory");
}
// L2 policy for data read once per launch (chunk images, right-hand sides):
// evicted first, so that it does not displace the iterate's recently
// written rows, which other bands read next
__device__ __forceinline__ unsigned long long l2_evict_first() {
    unsigned long long pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
// bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned)
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes,
                                         unsigned long long *b, unsigned long long pol) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1], %2, [%3], %4;" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(b)), "l"(pol) : "memory");
}
// asynchronous 16-byte global -> shared copy with an L2 policy
__device__ __forceinline__ void cp_async16_hint(void *dst, const void *src, unsigned long long pol) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(d), "l"(src),
                 "l"(pol) : "memory");
}
__device__ __forceinline__ void cp_async_arrive(unsigned long long *b) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ bool mbar_test(unsigned long long *b, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}" : "=r"(ok) : "r"(smem_u32(b)), "r"(parity) : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_try(unsigned long long *b, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}" : "=r"(ok) : "r"(smem_u32(b)), "r"(parity) : "memory");
    return ok != 0;
}
// Wait for the phase of the given parity; false on abort (*abort set) or
// after WAIT_NS.
__device__ __noinline__ bool mbar_wait(unsigned long long *b, unsigned parity, const int *abort) {
    if (mbar_test(b, parity)) return true;
    const unsigned long long t0 = gtimer();
    for (;;) {
        if (mbar_try(b, parity)) return true;
        if (*((volatile const int *)abort) || gtimer() - t0 > WAIT_NS) return false;
    }
}

// Bounded wait that ignores aborts (draining copies in flight).
__device__ __noinline__ bool mbar_wait_bounded(unsigned long long *b, unsigned parity) {
    const unsigned long long t0 = gtimer();
    while (!mbar_try(b, parity))
        if (gtimer() - t0 > WAIT_NS) return false;
    return true;
}

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

// Rows of LD stored values S read into / written from LD values of the
// arithmetic type T (bfloat16 storage: 8-byte pieces of 4 values, converted
// to and from float32).  cg: global memory through L2 only.
template <typename T, typename S, int LD, bool CG>
__device__ __forceinline__ void sld(T (&v)[LD], const S *p) {
    if constexpr (std::is_same<S, T>::value) {
        if constexpr (CG) vld_cg<T, LD>(v, p);
        else vld<T, LD>(v, p);
    } else {
#pragma unroll
        for (int i = 0; i < LD / 4; ++i) {
            const uint2 w = CG ? __ldcg(reinterpret_cast<const uint2 *>(p) + i)
                               : reinterpret_cast<const uint2 *>(p)[i];
            const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&w.x));
            const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&w.y));
            v[4 * i] = a.x; v[4 * i + 1] = a.y; v[4 * i + 2] = b.x; v[4 * i + 3] = b.y;
        }
    }
}
template <typename T, typename S, int LD>
__device__ __forceinline__ void sst_cg(S *p, const T (&v)[LD]) {
    if constexpr (std::is_same<S, T>::value) {
        vst_cg<T, LD>(p, v);
    } else {
#pragma unroll
        for (int i = 0; i < LD / 4; ++i) {
            const __nv_bfloat162 a = __floats2bfloat162_rn(v[4 * i], v[4 * i + 1]);
            const __nv_bfloat162 b = __floats2bfloat162_rn(v[4 * i + 2], v[4 * i + 3]);
            uint2 w;
            w.x = *reinterpret_cast<const unsigned *>(&a);
            w.y = *reinterpret_cast<const unsigned *>(&b);
            __stcg(reinterpret_cast<uint2 *>(p) + i, w);
        }
    }
}
template <typename S>
__device__ __forceinline__ typename Acc<S>::T sval(const S *p) { return to_acc(*p); }

// asynchronous 8-byte global -> shared copy (bfloat16 rows of 4 or 12 values)
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
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

__device__ __forceinline__ void bar_compute() {  // named barrier of the compute warps
    asm volatile("bar.sync 1, %0;" ::"n"(KZ_COMPUTE) : "memory");
}
__device__ __forceinline__ int ld_acq_cta(const int *p) {
    int v;
    asm volatile("ld.acquire.cta.shared.s32 %0, [%1];" : "=r"(v) : "r"((unsigned)__cvta_generic_to_shared(p)) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_acq_cta64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.cta.shared.u64 %0, [%1];" : "=l"(v) : "r"((unsigned)__cvta_generic_to_shared(p)) : "memory");
    return v;
}
__device__ __forceinline__ void st_rel_cta64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.release.cta.shared.u64 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(p)), "l"(v) : "memory");
}
__device__ __forceinline__ void st_rel_cta(int *p, int v) {
    asm volatile("st.release.cta.shared.s32 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(p)), "r"(v) : "memory");
}


struct KView {
    int *err;
    int nbands;
    const int *band_chunk;     // nbands + 1: first chunk of each band
    const KChunk *chunk;
    const int4 *lvl;           // per level: {first req, requirement count, publish, 0}
    const unsigned char *img;  // chunk images with coefficients of the launch's precision
    const int2 *req;           // {band, levels that band must have completed}
    const int *order;          // ticket -> band (every band's requirements earlier)
    unsigned long long *progress;
    KCtl *ctl;
};

// One staging buffer: the chunk image (capacity of a full chunk), then the
// gathered right-hand-side rows and staged first values (when a row of LD
// values is at most 64 bytes; wider rows are read from global memory).
template <typename T, typename S, int LD, bool SHIFT>
struct Stage {
    static constexpr int VB = LD * (int)sizeof(S);  // bytes of one stored vector row
    static constexpr bool VALS = VB <= 64;
    static constexpr unsigned IMG = img_layout(KZ_CHL, KZ_CHR, KZ_CHE, KZ_CHX, KZ_CHQ, (int)sizeof(T), SHIFT).bytes;
    static constexpr unsigned o_rhs = IMG;
    static constexpr unsigned o_xs = o_rhs + (VALS ? (unsigned)VB * KZ_CHR : 0u);
    static constexpr unsigned bytes = o_xs + (VALS ? (unsigned)VB * KZ_CHX : 0u);
    static constexpr unsigned stride = (bytes + 127u) / 128u * 128u;
};

// Warps 0 .. KZ_COMPUTE/32 - 1 compute.  The last warp is the producer: it
// stages chunk images (bulk copies) and gathered values (cp.async) up to
// KZ_NBUF chunks ahead.  Cross-band handoffs involve no relay: after the
// barrier of a level the image flags as waited for by a later band (and
// after the band's last level), the last compute warp publishes (release)
// the band's progress; before a level with cross-band requirements, every
// compute warp that holds rows of it polls (acquire) the progress words of
// the bands the image lists.
// MODE 0: rows of A (norms given).  MODE 1: rows of A - s_j B (entries carry
// b; norms formed per column).  MODE 2: fused relaxations (entries carry b;
// the accumulation uses a - s_j b, the update only a; norms given).
template <typename S, int LD, int MODE>
__global__ void __launch_bounds__(KZ_THREADS, 1)
    k_kaczmarz(KView kv, const S *__restrict__ rhs, S *x, const double *__restrict__ shift,
               int window_slots) {
    using T = typename Acc<S>::T;      // arithmetic (and window) type
    constexpr bool SHIFT = MODE != 0;  // entries carry b
    constexpr bool NRM = MODE == 1;    // row norms formed per column
    using SG = Stage<T, S, LD, SHIFT>;
    extern __shared__ __align__(128) unsigned char smraw[];
    T *win = reinterpret_cast<T *>(smraw);
    unsigned char *bufs = smraw + ((size_t)window_slots * LD * sizeof(T) + 127) / 128 * 128;
    __shared__ __align__(8) unsigned long long mb_sched[KZ_NBUF], mb_vals[KZ_NBUF];
    __shared__ int s_band;
    __shared__ int s_abort;
    __shared__ int s_done;   // band-local levels completed by the compute warps
    // progress seen by this CTA: band << 32 | completed levels (slot band % 64)
    __shared__ unsigned long long s_pc[64];
    // producer: band-local first level and level count of the chunk in each buffer
    __shared__ int s_cl0[KZ_NBUF], s_cnl[KZ_NBUF];
    const bool comm = threadIdx.x >= KZ_COMPUTE;
    T sh[SHIFT ? LD : 1];
#pragma unroll
    for (int q = 0; q < (SHIFT ? LD : 1); ++q) sh[q] = SHIFT ? (T)shift[q] : T(0);
    const unsigned long long epoch = *((volatile unsigned long long *)&kv.ctl->epoch);
    if (threadIdx.x == 0) {
        s_abort = 0;
        for (int i = 0; i < KZ_NBUF; ++i) {
            mbar_init(&mb_sched[i], 1);
            mbar_init(&mb_vals[i], 32);
        }
        fence_mbar_init();
    }
    if (threadIdx.x < 64) s_pc[threadIdx.x] = ~0ull;
    int base = 0;  // chunks this CTA staged in earlier bands: chunk j uses buffer
                   // j % KZ_NBUF in phase (j / KZ_NBUF) & 1

    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const unsigned t = atomicAdd(&kv.ctl->ticket, 1u);
            s_band = t < (unsigned)kv.nbands ? kv.order[t] : kv.nbands;
            s_done = 0;
            for (int q = 0; q < KZ_NBUF; ++q) {  // no chunk of this band staged yet
                s_cl0[q] = -(1 << 30);
                s_cnl[q] = 0;
            }
        }
        __syncthreads();
        const int b = s_band;
        if (b >= kv.nbands || s_abort) break;
        const int cb = kv.band_chunk[b], ce = kv.band_chunk[b + 1];
        const int Lband = kv.chunk[cb].L0;
        if (comm) {
            // ------------------------------------------------------ producer warp
            const int lane = threadIdx.x & 31;
            const unsigned long long once = l2_evict_first();
            int sn = cb, vn = cb;
            bool aborted = false;
            unsigned long long t0 = gtimer();  // re-armed whenever something advances
            int idle = 0;
            for (;;) {
                // this CTA's abort flag every pass; the launch's error word (an
                // L2 read) only once the loop has idled for a while
                bool ab = *((volatile int *)&s_abort) != 0;
                if (!ab && idle >= 32) {
                    idle = 0;
                    ab = *((volatile int *)kv.err) != 0;
                }
                if (ab) {
                    // another warp or CTA gave up: stop staging
                    if (lane == 0) *((volatile int *)&s_abort) = 1;
                    aborted = true;
                }
                if (!aborted && gtimer() - t0 > 2 * WAIT_NS) {
                    if (lane == 0) {
                        atomicExch(kv.err, 1);
                        *((volatile int *)&s_abort) = 1;
                    }
                    aborted = true;
                }
                if (__any_sync(FULL, aborted)) {
                    aborted = true;
                    break;
                }
                bool adv = false;
                const int done = __shfl_sync(FULL, ld_acq_cta(&s_done), 0);
                // a. image of chunk sn, once the chunk that used its buffer
                // (its level range is kept in s_cl0 / s_cnl) is done
                if (sn < ce) {
                    const int j = base + (sn - cb);
                    const int bi = j % KZ_NBUF;
                    if (done >= s_cl0[bi] + s_cnl[bi]) {
                        __syncwarp();
                        if (lane == 0) {
                            const KChunk ck = kv.chunk[sn];
                            const unsigned bytes = sizeof(T) == 4 ? ck.bytes_f : ck.bytes_d;
                            const long long off = sizeof(T) == 4 ? ck.off_f : ck.off_d;
                            s_cl0[bi] = ck.L0 - Lband;
                            s_cnl[bi] = ck.nl;
                            // the compute warps' reads of the old chunk precede
                            // the asynchronous overwrite
                            fence_proxy_async();
                            mbar_expect_tx(&mb_sched[bi], bytes);
                            bulk_g2s(bufs + (size_t)bi * SG::stride, kv.img + off, bytes, &mb_sched[bi],
                                     once);
                        }
                        __syncwarp();
                        ++sn;
                        adv = true;
                    }
                }
                // b. right-hand sides and staged first values of chunk vn
                if (SG::VALS && vn < sn) {
                    const int j = base + (vn - cb);
                    const int bi = j % KZ_NBUF;
                    const unsigned par = (unsigned)(j / KZ_NBUF) & 1u;
                    const int landed = __shfl_sync(FULL, (int)mbar_test(&mb_sched[bi], par), 0);
                    if (landed) {
                        const KChunk ck = kv.chunk[vn];
                        unsigned char *B = bufs + (size_t)bi * SG::stride;
                        const ImgLayout IL = img_layout(ck.nl, ck.nr, ck.ne, ck.nx, ck.nq, (int)sizeof(T), SHIFT);
                        const int2 *ri = reinterpret_cast<const int2 *>(B + IL.ri);
                        const int *xc = reinterpret_cast<const int *>(B + IL.xc);
                        // 16-byte pieces, or 8-byte ones for rows of 8 or 24 bytes
                        constexpr int PB = SG::VB % 16 == 0 ? 16 : 8;
                        constexpr int P = SG::VB / PB;
                        auto piece = [&](unsigned char *d, const unsigned char *g) {
                            if constexpr (PB == 16) cp_async16(d, g);
                            else cp_async8(d, g);
                        };
                        if (rhs)
                            for (int q = lane; q < ck.nr * P; q += 32) {
                                const int r = q / P, p = q % P;
                                unsigned char *d = B + SG::o_rhs + (size_t)SG::VB * r + PB * p;
                                const unsigned char *g =
                                    reinterpret_cast<const unsigned char *>(rhs + (size_t)ri[r].x * LD) + PB * p;
                                if constexpr (PB == 16) cp_async16_hint(d, g, once);
                                else piece(d, g);
                            }
                        for (int q = lane; q < ck.nx * P; q += 32) {
                            const int r = q / P, p = q % P;
                            piece(B + SG::o_xs + (size_t)SG::VB * r + PB * p,
                                  reinterpret_cast<const unsigned char *>(x + (size_t)xc[r] * LD) + PB * p);
                        }
                        cp_async_arrive(&mb_vals[bi]);
                        ++vn;
                        adv = true;
                    }
                }
                // every chunk staged and its values requested: the compute
                // warps finish the band on their own
                if (sn >= ce && (!SG::VALS || vn >= ce)) break;
                if (adv) {
                    t0 = gtimer();
                    idle = 0;
                } else {
                    ++idle;
                    __nanosleep(20);
                }
            }
            if (aborted) {
                // copies issued by this warp land before the CTA moves on
                cp_async_wait_all();
                if (lane == 0)
                    for (int c = max(cb, sn - KZ_NBUF); c < sn; ++c) {
                        const int j = base + (c - cb);
                        mbar_wait_bounded(&mb_sched[j % KZ_NBUF], (unsigned)(j / KZ_NBUF) & 1u);
                    }
            }
        } else {
            // ------------------------------------------------------ compute warps
            bool aborted = false;
            // the last compute warp publishes (release) the band's progress after
            // the levels the image flags; its rows are the fewest, so its wait
            // for the release delays the next level the least
            const bool publisher = threadIdx.x == KZ_COMPUTE - 32;
            const bool mute = publisher && *((volatile int *)&kv.ctl->mute) == b;
            for (int c = cb; c < ce; ++c) {
                const int j = base + (c - cb);
                const int bi = j % KZ_NBUF;
                const unsigned par = (unsigned)(j / KZ_NBUF) & 1u;
                const KChunk ck = kv.chunk[c];
                if (!aborted) {
                    bool ok = mbar_wait(&mb_sched[bi], par, &s_abort);
                    if (ok && SG::VALS) ok = mbar_wait(&mb_vals[bi], par, &s_abort);
                    if (!ok) {
                        atomicExch(kv.err, 1);
                        *((volatile int *)&s_abort) = 1;
                    }
                    // warp-uniform, so that the row sums' shuffles see every lane
                    aborted = __any_sync(FULL, !ok);
                }
                unsigned char *B = bufs + (size_t)bi * SG::stride;
                const ImgLayout IL = img_layout(ck.nl, ck.nr, ck.ne, ck.nx, ck.nq, (int)sizeof(T), SHIFT);
                const int4 *lv = reinterpret_cast<const int4 *>(B + IL.lv);
                const int2 *lq = reinterpret_cast<const int2 *>(B + IL.lq);
                const int2 *srq = reinterpret_cast<const int2 *>(B + IL.rq);
                const int2 *ri = reinterpret_cast<const int2 *>(B + IL.ri);
                const T *sinv = reinterpret_cast<const T *>(B + IL.inv);
                const int2 *se = reinterpret_cast<const int2 *>(B + IL.ent);
                const T *sa = reinterpret_cast<const T *>(B + IL.a);
                const T *sb = reinterpret_cast<const T *>(B + IL.b);
                const S *srhs = reinterpret_cast<const S *>(B + SG::o_rhs);
                const S *sxs = reinterpret_cast<const S *>(B + SG::o_xs);
                for (int L = 0; L < ck.nl; ++L) {
                    const int lb = ck.L0 + L - Lband;  // band-local level
                    const int4 lr = lv[L];
                    if (!aborted) {
                        // G = 2^lgG lanes per row (the smallest power of two
                        // not below the level's longest row, at most 32);
                        // lane lg takes entries lg, lg + G, ... for all LD
                        // columns.  Rows of more than 16 entries (float32) or
                        // 32 entries (float64) take G = 2^(lr.z - 1) lanes, each
                        // loading its second entry together with its first,
                        // which keeps the row sums one shuffle step shorter.  A
                        // warp holding no row of the level goes straight to
                        // the barrier.
                        // (float64 keeps G = 32 for rows of 17-32 entries: the
                        // setup phase runs in float64, and its hierarchy
                        // should not depend on how float32 sweeps are tuned)
                        constexpr int TWO_FROM = sizeof(T) == 4 ? 5 : 6;
                        const bool two = lr.z >= TWO_FROM;
                        const int lgG = two ? lr.z - 1 : lr.z;
                        const int G = 1 << lgG;
                        const int nrow = lr.y;
                        const int lane = threadIdx.x & 31;
                        const int wrow = (threadIdx.x & ~31) >> lgG;
                        if ((lr.w & 1) && wrow < nrow) {
                            // cross-band requirements: the warp's lanes poll
                            // (acquire) the listed bands' progress words; a
                            // progress this CTA has already seen (s_pc, written
                            // with release after an acquire) needs no poll
                            const int2 q = lq[L];
                            const int cnt = q.y >= 0 ? q.y : -q.y - 1;
                            const int2 *rl = q.y >= 0 ? srq + q.x : kv.req + q.x;
                            bool bad = false;
                            for (int i = lane; i < cnt && !bad; i += 32) {
                                const int2 r = rl[i];
                                const unsigned long long key = ld_acq_cta64(&s_pc[r.x & 63]);
                                if ((int)(key >> 32) == r.x && (unsigned)key >= (unsigned)r.y) continue;
                                const unsigned long long want = (epoch << 32) | (unsigned)r.y;
                                unsigned long long v = ld_acquire(&kv.progress[r.x]);
                                if (v < want) {
                                    const unsigned long long t0 = gtimer();
                                    int k = 0;
                                    do {
                                        if ((++k & 15) == 0 && (*((volatile int *)&s_abort) ||
                                                                *((volatile int *)kv.err))) {
                                            bad = true;
                                            break;
                                        }
                                        if (gtimer() - t0 > WAIT_NS) {
                                            atomicExch(kv.err, 1);
                                            *((volatile int *)&s_abort) = 1;
                                            bad = true;
                                            break;
                                        }
                                        v = ld_acquire(&kv.progress[r.x]);
                                    } while (v < want);
                                }
                                if (!bad)
                                    st_rel_cta64(&s_pc[r.x & 63],
                                                 ((unsigned long long)(unsigned)r.x << 32) | (v & 0xffffffffull));
                            }
                            // the other lanes' loads follow the pollers' acquires
                            __syncwarp();
                            aborted = __any_sync(FULL, bad || *((volatile int *)&s_abort) != 0);
                        }
                        if (!aborted) {
                            const int lg = threadIdx.x & (G - 1);
                            for (int pr = 0; pr + wrow < nrow; pr += KZ_COMPUTE >> lgG) {
                                const int r = pr + (threadIdx.x >> lgG);
                                const bool act = r < nrow;
                                const int k = lr.x + r;
                                T acc[LD], nrm[NRM ? LD : 1];
#pragma unroll
                                for (int q = 0; q < LD; ++q) acc[q] = T(0);
#pragma unroll
                                for (int q = 0; q < (NRM ? LD : 1); ++q) nrm[q] = T(0);
                                // the lane's first (and second) entry stay in registers
                                // for the update
                                int2 fen = make_int2(0, 0), sen = make_int2(0, 0);
                                T fa = T(0), fb = T(0), fv[LD], sa2 = T(0), sb2 = T(0), sv[LD];
                                bool own = false, hb = false;
                                int2 rk = make_int2(0, 0);
                                int e0 = 0, e1 = 0;
                                auto load_val = [&](T (&val)[LD], int2 en) {
                                    const int fl = en.y;
                                    // first touches not staged come from global memory, the
                                    // rest from the staged values or the window
                                    if ((fl & 1) && !(SG::VALS && (fl & 4)))
                                        sld<T, S, LD, true>(val, x + (size_t)en.x * LD);
                                    else if (fl & 1)
                                        sld<T, S, LD, false>(val, sxs + (fl >> 15) * LD);
                                    else
                                        vld<T, LD>(val, win + ((fl >> 3) & 0xfff) * LD);
                                };
                                auto accumulate = [&](T a, T bq, const T (&val)[LD]) {
#pragma unroll
                                    for (int q = 0; q < LD; ++q) {
                                        const T coef = SHIFT ? a - sh[q] * bq : a;
                                        acc[q] = fma(coef, val[q], acc[q]);
                                        if (NRM) nrm[q] = fma(coef, coef, nrm[q]);
                                    }
                                };
                                if (act) {
                                    rk = ri[k];
                                    e0 = rk.y & 0xffff;
                                    e1 = e0 + (rk.y >> 16);
                                    const int ea = e0 + lg;
                                    own = ea < e1;
                                    if (own) {
                                        // the second entry's loads are issued with the first's;
                                        // a lane without one reloads its first (weight 0)
                                        hb = two && ea + G < e1;
                                        const int eb = hb ? ea + G : ea;
                                        fen = se[ea];
                                        fa = sa[ea];
                                        fb = SHIFT ? sb[ea] : T(0);
                                        if (two) {
                                            sen = se[eb];
                                            sa2 = hb ? sa[eb] : T(0);
                                            sb2 = (SHIFT && hb) ? sb[eb] : T(0);
                                        }
                                        load_val(fv, fen);
                                        if (two) load_val(sv, sen);
                                        accumulate(fa, fb, fv);
                                        if (two) accumulate(sa2, sb2, sv);
                                        for (int e = ea + (hb ? 2 : 1) * G; e < e1; e += G) {
                                            T val[LD];
                                            const int2 en = se[e];
                                            load_val(val, en);
                                            accumulate(sa[e], SHIFT ? sb[e] : T(0), val);
                                        }
                                    }
                                }
                                // d_q = (b_i - <a_i, x_q>) / ||a_i||^2 for every column q
                                T d[LD];
                                if (pow2(LD) && G >= LD) {
                                    const T sa_c = group_reduce_scatter<T, LD>(acc, lane, lgG);
                                    const T sn_c = NRM ? group_reduce_scatter<T, (NRM ? LD : 1)>(nrm, lane, lgG) : T(0);
                                    const int c = brev_low(lane & (LD - 1), ilog2(LD));
                                    T dc = T(0);
                                    if (act) {
                                        const T bi = rhs ? (SG::VALS ? sval(srhs + k * LD + c) : sval(rhs + (size_t)rk.x * LD + c)) : T(0);
                                        dc = NRM ? (sn_c > T(0) ? (bi - sa_c) / sn_c : T(0)) : (bi - sa_c) * sinv[k];
                                    }
                                    const int gb = lane & ~(G - 1);
#pragma unroll
                                    for (int q = 0; q < LD; ++q)
                                        d[q] = __shfl_sync(FULL, dc, gb + brev_low(q, ilog2(LD)));
                                } else {
                                    group_allreduce<T, LD>(acc, lgG);
                                    if (NRM) group_allreduce<T, (NRM ? LD : 1)>(nrm, lgG);
#pragma unroll
                                    for (int q = 0; q < LD; ++q) d[q] = T(0);
                                    if (act) {
#pragma unroll
                                        for (int q = 0; q < LD; ++q) {
                                            const T bi = rhs ? (SG::VALS ? sval(srhs + k * LD + q) : sval(rhs + (size_t)rk.x * LD + q)) : T(0);
                                            const T nq = NRM ? nrm[q] : T(1);
                                            d[q] = NRM ? (nq > T(0) ? (bi - acc[q]) / nq : T(0)) : (bi - acc[q]) * sinv[k];
                                        }
                                    }
                                }
                                // x_q += d_q a_i on the row's entries; every lane stores
                                // to its slot (slot 0: scratch), so the warp does not
                                // diverge; last touches also go to global memory
                                auto update = [&](int2 en, T a, T bq, T (&val)[LD]) {
#pragma unroll
                                    for (int q = 0; q < LD; ++q) {
                                        // fused relaxations update along a only: the
                                        // b entries belong to the other unknown
                                        const T coef = NRM ? a - sh[q] * bq : a;
                                        val[q] = fma(d[q], coef, val[q]);
                                    }
                                    vst<T, LD>(win + ((en.y >> 3) & 0xfff) * LD, val);
                                    if (en.y & 2) sst_cg<T, S, LD>(x + (size_t)en.x * LD, val);
                                };
                                if (own) {
                                    update(fen, fa, fb, fv);
                                    if (hb) update(sen, sa2, sb2, sv);
                                    for (int e = e0 + lg + (hb ? 2 : 1) * G; e < e1; e += G) {
                                        T val[LD];
                                        const int2 en = se[e];
                                        load_val(val, en);
                                        update(en, sa[e], SHIFT ? sb[e] : T(0), val);
                                    }
                                }
                            }
                        }
                    }
                    // every compute warp reaches every barrier, aborted or not
                    bar_compute();
                    if (threadIdx.x == 0) st_rel_cta(&s_done, lb + 1);
                    // the release covers every compute warp's stores, which
                    // precede the barrier
                    if (publisher && (lr.w & 2) && !mute && !aborted &&
                        !*((volatile int *)&s_abort))
                        st_release(&kv.progress[b], (epoch << 32) | (unsigned)(lb + 1));
                }
            }
        }
        base += ce - cb;
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

template <typename S, int LD, int MODE>
void launch_one(const KSched &ks, const S *rhs, S *x, const double *shift, cudaStream_t s) {
    using T = typename Acc<S>::T;
    using SG = Stage<T, S, LD, MODE != 0>;
    auto kern = k_kaczmarz<S, LD, MODE>;
    const int slots = ks.max_slots + 1;  // slot 0: scratch
    const size_t smem = ((size_t)slots * LD * sizeof(T) + 127) / 128 * 128 + (size_t)KZ_NBUF * SG::stride;
    // rows of 8 or 24 bytes (bfloat16, LD 4 or 12) move in 8-byte pieces
    constexpr uintptr_t AL = (LD * sizeof(S)) % 16 == 0 ? 16 : 8;
    SAMG_CHECK(((uintptr_t)x % AL) == 0 && ((uintptr_t)rhs % AL) == 0, SAMG_E_INVALID,
               "kaczmarz: vector blocks must be aligned to their row pieces");
    static_assert(LD % 4 == 0, "vector rows of a multiple of 4 values");
    // a window of more slots than a CTA's shared memory holds (a resident
    // schedule built for a narrower block or precision) is refused here
    SAMG_CHECK(smem <= 227u * 1024u, SAMG_E_INVALID,
               "kaczmarz: the schedule's window and staging buffers exceed 227 KB of shared memory "
               "at this block width and precision");
    // per kernel instance and device (a function attribute is set per
    // device): the largest dynamic shared memory set so far and the SM
    // count, under a lock since contexts may launch from several host
    // threads; per schedule and instance: the resident CTA count
    constexpr int MAXDEV = 64;
    static std::mutex mu;
    static size_t smem_set[MAXDEV] = {};
    static int nsm_of[MAXDEV] = {};
    int dev = 0;
    SAMG_CUDA(cudaGetDevice(&dev));
    SAMG_CHECK(dev >= 0 && dev < MAXDEV, SAMG_E_CUDA, "kaczmarz: device ordinal out of range");
    int nsm = 0;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (smem > smem_set[dev]) {
            SAMG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            smem_set[dev] = smem;
        }
        if (!nsm_of[dev])
            SAMG_CUDA(cudaDeviceGetAttribute(&nsm_of[dev], cudaDevAttrMultiProcessorCount, dev));
        nsm = nsm_of[dev];
    }
    const int key = (sizeof(S) == 2 ? 0 : sizeof(S) == 4 ? 1 : 2) * 64 + LD * 3 + MODE;
    int &grid = ks.grid_cache[key];
    if (!grid) {
        int bps = 0;
        SAMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, KZ_THREADS, smem));
        SAMG_CHECK(bps > 0, SAMG_E_CUDA, "kaczmarz: staging buffers do not fit in shared memory");
        grid = std::min(ks.nbands, nsm * bps);
    }
    const unsigned char *img = sizeof(T) == 4 ? ks.img_f.p : ks.img_d.p;
    KView kv{ks.err ? ks.err : &ks.ctl.p->err, ks.nbands, ks.band_chunk.p, ks.chunk.p, ks.lvl.p,
             img, ks.req.p, ks.order.p, ks.progress.p, ks.ctl.p};
    SAMG_COUNT_LAUNCH();
    kern<<<grid, KZ_THREADS, smem, s>>>(kv, rhs, x, shift, slots);
    SAMG_CUDA(cudaGetLastError());
}

// Appends the image of one chunk with coefficients of type T; returns its size.
template <typename T>
int write_image(std::vector<unsigned char> &img, bool shifted, const std::vector<int4> &lrec,
                const std::vector<int2> &qrec, const std::vector<int2> &rrec,
                const std::vector<double> &rinv, const std::vector<int2> &erec,
                const std::vector<double> &ca, const std::vector<double> &cb,
                const std::vector<int> &xc, const std::vector<int2> &rq) {
    const ImgLayout L = img_layout((int)lrec.size(), (int)rrec.size(), (int)erec.size(),
                                   (int)xc.size(), (int)rq.size(), (int)sizeof(T), shifted);
    const size_t base = img.size();
    img.resize(base + L.bytes, 0);
    unsigned char *p = img.data() + base;
    std::memcpy(p + L.lv, lrec.data(), 16 * lrec.size());
    std::memcpy(p + L.lq, qrec.data(), 8 * qrec.size());
    std::memcpy(p + L.rq, rq.data(), 8 * rq.size());
    std::memcpy(p + L.ri, rrec.data(), 8 * rrec.size());
    for (size_t i = 0; i < rinv.size(); ++i) {
        const T v = (T)rinv[i];
        std::memcpy(p + L.inv + sizeof(T) * i, &v, sizeof(T));
    }
    std::memcpy(p + L.ent, erec.data(), 8 * erec.size());
    for (size_t i = 0; i < ca.size(); ++i) {
        const T v = (T)ca[i];
        std::memcpy(p + L.a + sizeof(T) * i, &v, sizeof(T));
    }
    if (shifted)
        for (size_t i = 0; i < cb.size(); ++i) {
            const T v = (T)cb[i];
            std::memcpy(p + L.b + sizeof(T) * i, &v, sizeof(T));
        }
    std::memcpy(p + L.xc, xc.data(), 4 * xc.size());
    return (int)L.bytes;
}

}  // namespace

namespace {

// Runs fn(worker, b) for b in [0, n) on up to `threads` host threads (band
// b taken from a shared counter); the first exception is rethrown.
template <typename F>
void for_bands(int n, int threads, F &&fn) {
    threads = std::max(1, std::min(threads, n));
    std::atomic<int> next{0};
    std::exception_ptr err;
    std::mutex mu;
    auto work = [&](int t) {
        for (;;) {
            const int b = next.fetch_add(1);
            if (b >= n) return;
            try {
                fn(t, b);
            } catch (...) {
                std::lock_guard<std::mutex> lock(mu);
                if (!err) err = std::current_exception();
                next.store(n);
                return;
            }
        }
    };
    if (threads == 1) {
        work(0);
    } else {
        std::vector<std::thread> pool;
        for (int t = 1; t < threads; ++t) pool.emplace_back(work, t);
        work(0);
        for (std::thread &th : pool) th.join();
    }
    if (err) std::rethrow_exception(err);
}

// Host threads of the schedule builder: SAMG_HOST_THREADS when set (>= 1),
// else the hardware's, at most 16 (each holds five arrays over the columns).
int builder_threads() {
    if (const char *e = std::getenv("SAMG_HOST_THREADS")) {
        const int v = std::atoi(e);
        if (v >= 1) return std::min(v, 64);
    }
    const unsigned h = std::thread::hardware_concurrency();
    return (int)std::max(1u, std::min(h ? h : 1u, 16u));
}

// Contiguous bands of rows, each grown (doubling) until it has about
// `target` rows per level, at most MAX_BAND_ROWS rows, and at most slot_cap
// columns live at once.  Returns the first row of every band, then p.rows.
std::vector<int> form_bands_at(const Pattern &p, const std::vector<int> &glv, BandWork &w,
                               int slot_cap, int target, int from = 0, int to = -1) {
    std::vector<int> bstart;
    int slots = 0;
    size_t si = 0;
    if (to < 0) to = p.rows;
    for (int r0 = from; r0 < to;) {
        while (si < p.seg.size() && p.seg[si] <= r0) ++si;
        const int r_end = std::min(to, si < p.seg.size() ? p.seg[si] : p.rows);  // this sweep's end
        int R = std::min(256, r_end - r0), good = 0;
        for (;;) {
            int nl = analyze_band(p, glv, r0, r0 + R, w, &slots);
            if (slots > slot_cap) {
                if (good) break;
                R = std::max(1, R / 2);
                if (R == 1) { good = 1; break; }
                continue;
            }
            good = R;
            if (r0 + R >= r_end || R >= MAX_BAND_ROWS || (R / std::max(nl, 1)) >= target) break;
            R = std::min(2 * R, r_end - r0);
        }
        bstart.push_back(r0);
        r0 += good;
    }
    bstart.push_back(to);
    return bstart;
}

// The order in which the CTAs claim bands (ticket -> band).  Any order in
// which every band's required bands come earlier is free of deadlock: the
// unfinished band with the smallest ticket has all its required bands
// finished, so it always advances.  Program order is one such order, but
// a CTA that claims a band whose rows the wavefront reaches late holds its
// SM idle meanwhile, and with more bands than SMs the later sweeps of a
// fused program then start late.  Among the bands whose required bands are
// all placed, this takes the one that could start earliest: the start of
// its first level in a model with a CTA per band, levels of one unit and
// cross-band handoffs of two.
std::vector<int> claim_order(int nb, const std::vector<int> &band_lvl0,
                             const std::vector<int4> &lvl, const std::vector<int2> &req) {
    constexpr double HANDOFF = 2.0;
    std::vector<double> fin(lvl.size(), 0.0), est(nb, 0.0);
    std::vector<std::vector<int>> deps(nb);
    for (int b = 0; b < nb; ++b) {  // program order: required bands come first
        double t = 0.0;
        for (int L = band_lvl0[b]; L < band_lvl0[b + 1]; ++L) {
            for (int q = lvl[L].x; q < lvl[L].x + lvl[L].y; ++q) {
                const int bb = req[q].x;
                t = std::max(t, fin[band_lvl0[bb] + req[q].y - 1] + HANDOFF);
                deps[b].push_back(bb);
            }
            if (L == band_lvl0[b]) est[b] = t;
            t += 1.0;
            fin[L] = t;
        }
        std::sort(deps[b].begin(), deps[b].end());
        deps[b].erase(std::unique(deps[b].begin(), deps[b].end()), deps[b].end());
    }
    std::vector<std::vector<int>> users(nb);
    std::vector<int> left(nb);
    for (int b = 0; b < nb; ++b) {
        left[b] = (int)deps[b].size();
        for (int bb : deps[b]) users[bb].push_back(b);
    }
    using Item = std::pair<double, int>;
    std::priority_queue<Item, std::vector<Item>, std::greater<Item>> ready;
    for (int b = 0; b < nb; ++b)
        if (!left[b]) ready.push({est[b], b});
    std::vector<int> order;
    order.reserve(nb);
    while (!ready.empty()) {
        const int b = ready.top().second;
        ready.pop();
        order.push_back(b);
        for (int u : users[b])
            if (--left[u] == 0) ready.push({est[u], u});
    }
    SAMG_CHECK((int)order.size() == nb, SAMG_E_INVALID,
               "kaczmarz: band requirements are not acyclic");
    return order;
}

// resident_cap > 0: when the whole program keeps at most that many columns
// live, it is one band (every column resident in the window; no cross-band
// requirement and no first touch written by another band).  Otherwise bands
// of about band_rows rows per level (0: TARGET_PAR).
std::vector<int> form_bands(const Pattern &p, const std::vector<int> &glv, BandWork &w,
                            int resident_cap = 0, int slot_cap = SLOT_CAP, int band_rows = 0) {
    int slots = 0;
    if (resident_cap > 0 && p.rows > 0) {
        analyze_band(p, glv, 0, p.rows, w, &slots);
        if (slots <= resident_cap) return {0, p.rows};
    }
    const int target = band_rows > 0 ? band_rows : TARGET_PAR;
    if (p.seg.empty() || p.rows == 0) return form_bands_at(p, glv, w, slot_cap, target);
    // no band crosses a sweep: the sweeps are banded independently, each from
    // its first row, on several host threads
    std::vector<int> cut{0};
    for (int x : p.seg)
        if (x > cut.back() && x < p.rows) cut.push_back(x);
    cut.push_back(p.rows);
    const int nseg = (int)cut.size() - 1;
    std::vector<std::vector<int>> part(nseg);
    const int nthr = std::min(builder_threads(), nseg);
    std::vector<std::unique_ptr<BandWork>> works(nthr);
    for (auto &wp : works) wp.reset(new BandWork(p.cols));
    for_bands(nseg, nthr, [&](int t, int k) {
        part[k] = form_bands_at(p, glv, *works[t], slot_cap, target, cut[k], cut[k + 1]);
    });
    std::vector<int> bstart;
    for (int k = 0; k < nseg; ++k) bstart.insert(bstart.end(), part[k].begin(), part[k].end() - 1);
    bstart.push_back(p.rows);
    return bstart;
}

// Schedule of one sweep program (rows in program order).  mode: 0 plain rows
// of A; 1 rows of A - s B (norms formed per column); 2 a fused program of
// block Gauss-Seidel relaxations (b entries read the other unknown with
// coefficient -s_j and are not updated; norms from a).  The bands are
// analysed, given their requirements and written out on several host
// threads; every step that orders or numbers things across bands is a
// sequential pass, so the schedule does not depend on the thread count.
void build_host(const Pattern &p, int mode, HostSched &ks, int resident_cap = 0,
                int slot_cap = SLOT_CAP, int band_rows = 0) {
    const int rows = p.rows, cols = p.cols;
    ks.rows = rows;
    ks.cols = cols;
    ks.shifted = mode != 0;
    ks.mode = mode;
    const std::vector<int> glv = global_levels(p);
    // 1. bands: contiguous rows, grown until about band_rows rows per level
    std::vector<int> bstart;
    {
        BandWork w(cols);
        bstart = form_bands(p, glv, w, resident_cap, slot_cap, band_rows);
    }
    const int nb = (int)bstart.size() - 1;
    ks.nbands = nb;
    // per row its band; per entry the previous row touching the column (-1:
    // none); per column its first row
    std::vector<int> band_of(rows, 0), prev(p.ci.size(), -1), first_row(cols, -1);
    for (int b = 0; b < nb; ++b)
        for (int r = bstart[b]; r < bstart[b + 1]; ++r) band_of[r] = b;
    {
        std::vector<int> last(cols, -1);
        for (int r = 0; r < rows; ++r)
            for (int64_t e = p.rp[r]; e < p.rp[r + 1]; ++e) {
                const int c = p.ci[e];
                prev[e] = last[c];
                last[c] = r;
                if (first_row[c] < 0) first_row[c] = r;
            }
    }
    // a first touch in band b of a column no earlier band touched: its value
    // is final when the band starts (staged)
    auto fresh = [&](int c, int b) { return band_of[first_row[c]] == b; };
    const int nthr = builder_threads();
    std::vector<std::unique_ptr<BandWork>> works(std::min(nthr, std::max(nb, 1)));
    for (auto &wp : works) wp.reset(new BandWork(cols));
    struct RowRec { int row, sub; };
    struct Band {
        int nl = 0, slots = 0, nsub = 0;
        std::vector<RowRec> rr;                          // rows in sub-level order
        std::vector<int> sub_rows, sub_ents, sub_xs, sub_maxe;
        std::vector<int2> req;                           // requirements, sub-level order
        std::vector<int> sub_req0, sub_nreq;             // per sub-level: first, count
        std::vector<int2> pub;                           // {band, sub-level} to publish
        std::vector<KChunk> chunk;                       // offsets local to the band
        std::vector<int> lvl_chunk;                      // per sub-level: local chunk
        std::vector<unsigned char> img_f, img_d;
        int64_t nent = 0;
    };
    std::vector<Band> B(nb);
    std::vector<int> row_sub(rows, 0);
    // per worker: window slots by column
    std::vector<std::vector<int>> slot_of(works.size());
    // 2a. per band: levels, rows by level, sub-levels (<= chunk limits)
    for_bands(nb, (int)works.size(), [&](int t, int b) {
        BandWork &w = *works[t];
        Band &bd = B[b];
        const int r0 = bstart[b], r1 = bstart[b + 1];
        const int nl = analyze_band(p, glv, r0, r1, w, &bd.slots);
        bd.nl = nl;
        // rows grouped by level (ascending row order inside a level)
        std::vector<int> lcount(nl + 1, 0);
        for (int r = r0; r < r1; ++r) lcount[w.rowlv[r - r0] + 1]++;
        for (int l = 0; l < nl; ++l) lcount[l + 1] += lcount[l];
        std::vector<int> order(r1 - r0);
        {
            std::vector<int> fillp(lcount.begin(), lcount.end() - 1);
            for (int r = r0; r < r1; ++r) order[fillp[w.rowlv[r - r0]]++] = r;
        }
        // sub-levels: a level's independent rows split so that each piece
        // fits one staging chunk
        for (int l = 0; l < nl; ++l) {
            int cr = 0, ce = 0, cx = 0;
            bool open = false;
            for (int k = lcount[l]; k < lcount[l + 1]; ++k) {
                const int r = order[k];
                const int ne = (int)(p.rp[r + 1] - p.rp[r]);
                int nx = 0;
                for (int64_t e = p.rp[r]; e < p.rp[r + 1]; ++e) {
                    const int c = p.ci[e];
                    if (w.firstlv[c] == l && fresh(c, b)) ++nx;
                }
                if (!open || cr + 1 > KZ_CHR || ce + ne > KZ_CHE || cx + nx > KZ_CHX) {
                    bd.sub_rows.push_back(0); bd.sub_ents.push_back(0); bd.sub_xs.push_back(0);
                    bd.sub_maxe.push_back(0);
                    cr = ce = cx = 0;
                    open = true;
                }
                SAMG_CHECK(ne <= KZ_CHE && nx <= KZ_CHX, SAMG_E_INVALID,
                           "kaczmarz: a row has more entries than a staging chunk holds");
                cr += 1; ce += ne; cx += nx;
                bd.sub_rows.back() = cr; bd.sub_ents.back() = ce; bd.sub_xs.back() = cx;
                bd.sub_maxe.back() = std::max(bd.sub_maxe.back(), ne);
                const int sub = (int)bd.sub_rows.size() - 1;
                bd.rr.push_back({r, sub});
                row_sub[r] = sub;
            }
        }
        bd.nsub = (int)bd.sub_rows.size();
    });
    // 2b. per band: requirements.  A first touch of a column an earlier band
    // touched needs that band to have completed the sub-level of its last
    // touch, which is the previous touch of the column in program order.
    std::vector<std::vector<int>> waited(works.size()), waited_stamp(works.size());
    for (size_t t = 0; t < works.size(); ++t) {
        waited[t].assign(nb, 0);
        waited_stamp[t].assign(nb, -1);
    }
    for_bands(nb, (int)works.size(), [&](int t, int b) {
        BandWork &w = *works[t];
        Band &bd = B[b];
        const int r0 = bstart[b], r1 = bstart[b + 1];
        int slots = 0;
        analyze_band(p, glv, r0, r1, w, &slots);
        struct PendReq { int sub, band, need; };
        std::vector<PendReq> pend;
        for (const RowRec &x : bd.rr) {
            const int lv = w.rowlv[x.row - r0];
            for (int64_t e = p.rp[x.row]; e < p.rp[x.row + 1]; ++e) {
                const int c = p.ci[e];
                if (w.firstlv[c] == lv && prev[e] >= 0 && prev[e] < r0)
                    pend.push_back({x.sub, band_of[prev[e]], row_sub[prev[e]] + 1});
            }
        }
        // per sub-level: max need per band, dropping needs already waited for
        std::sort(pend.begin(), pend.end(), [](const PendReq &a, const PendReq &b2) {
            return a.sub != b2.sub ? a.sub < b2.sub : (a.band != b2.band ? a.band < b2.band : a.need > b2.need);
        });
        std::vector<int> &wt = waited[t], &ws = waited_stamp[t];
        bd.sub_req0.assign(bd.nsub, 0);
        bd.sub_nreq.assign(bd.nsub, 0);
        size_t q = 0;
        for (int l = 0; l < bd.nsub; ++l) {
            bd.sub_req0[l] = (int)bd.req.size();
            while (q < pend.size() && pend[q].sub == l) {
                const PendReq &pr = pend[q];
                if (ws[pr.band] != b || wt[pr.band] < pr.need) {
                    ws[pr.band] = b;
                    wt[pr.band] = pr.need;
                    bd.req.push_back(make_int2(pr.band, pr.need));
                    bd.pub.push_back(make_int2(pr.band, pr.need - 1));
                }
                const int bb = pr.band;
                while (q < pend.size() && pend[q].sub == l && pend[q].band == bb) ++q;
            }
            bd.sub_nreq[l] = (int)bd.req.size() - bd.sub_req0[l];
        }
    });
    // 2c. global level records and requirement list, in band order
    std::vector<int> band_lvl0(nb + 1, 0);
    std::vector<int4> lvl;  // per level: {first req, requirement count, publish, 0}
    std::vector<int2> req;
    int max_slots = 0;
    for (int b = 0; b < nb; ++b) {
        Band &bd = B[b];
        band_lvl0[b] = (int)lvl.size();
        const int base = (int)req.size();
        for (int l = 0; l < bd.nsub; ++l) lvl.push_back(make_int4(base + bd.sub_req0[l], bd.sub_nreq[l], 0, 0));
        req.insert(req.end(), bd.req.begin(), bd.req.end());
        max_slots = std::max(max_slots, bd.slots);
    }
    band_lvl0[nb] = (int)lvl.size();
    // 2d. per band: window slots, chunks and their images
    for (size_t t = 0; t < works.size(); ++t) slot_of[t].assign(cols, 0);
    for_bands(nb, (int)works.size(), [&](int t, int b) {
        BandWork &w = *works[t];
        std::vector<int> &slot = slot_of[t];
        Band &bd = B[b];
        const int r0 = bstart[b], r1 = bstart[b + 1];
        int slots = 0;
        const int nl = analyze_band(p, glv, r0, r1, w, &slots);
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
        const int L0 = band_lvl0[b];
        const int nsub = bd.nsub;
        // chunks of consecutive sub-levels; a sub-level's requirements travel
        // in its chunk's image unless they alone exceed KZ_CHQ (then the
        // kernel reads them from the global list)
        auto img_reqs = [&](int l) { return lvl[L0 + l].y <= KZ_CHQ ? lvl[L0 + l].y : 0; };
        std::vector<int> chunk_first_sub;
        {
            int cl = 0, cr = 0, ce = 0, cx = 0, cq = 0;
            for (int q = 0; q < nsub; ++q) {
                if (q == 0 || cl + 1 > KZ_CHL || cr + bd.sub_rows[q] > KZ_CHR ||
                    ce + bd.sub_ents[q] > KZ_CHE || cx + bd.sub_xs[q] > KZ_CHX ||
                    cq + img_reqs(q) > KZ_CHQ) {
                    chunk_first_sub.push_back(q);
                    cl = cr = ce = cx = cq = 0;
                }
                cl += 1; cr += bd.sub_rows[q]; ce += bd.sub_ents[q]; cx += bd.sub_xs[q]; cq += img_reqs(q);
            }
        }
        // one image per chunk (chunk-local row and entry numbers)
        size_t ri = 0;
        const int nch = (int)chunk_first_sub.size();
        std::vector<int4> lrec;
        std::vector<int2> qrec, rrec, erec, rqrec;
        std::vector<double> rinv, ca, cbv;
        std::vector<int> xc;
        for (int ch = 0; ch < nch; ++ch) {
            const int q0 = chunk_first_sub[ch];
            const int q1 = ch + 1 < nch ? chunk_first_sub[ch + 1] : nsub;
            lrec.clear(); qrec.clear(); rrec.clear(); erec.clear(); rinv.clear(); ca.clear();
            cbv.clear(); xc.clear(); rqrec.clear();
            for (int qq = q0; qq < q1; ++qq) {
                // lanes per row: a power of two >= the longest row of the level
                // (at most 32; 6 marks rows of more than 32 entries, whose lanes
                // take two or more entries)
                int lg = 0;
                while (lg < 6 && (1 << lg) < bd.sub_maxe[qq]) ++lg;
                const int row0 = (int)rrec.size();
                for (; ri < bd.rr.size() && bd.rr[ri].sub == qq; ++ri) {
                    const int r = bd.rr[ri].row;
                    const int lv = w.rowlv[r - r0];
                    const int e0 = (int)erec.size();
                    double n2 = 0.0;
                    for (int64_t e = p.rp[r]; e < p.rp[r + 1]; ++e) {
                        const int c = p.ci[e];
                        const int first = (w.firstlv[c] == lv), last = (w.lastlv[c] == lv);
                        // window slot + 1; slot 0 is scratch for columns touched once
                        const int sl = (w.cnt[c] >= 2) ? slot[c] + 1 : 0;
                        int staged = 0, xi = 0;
                        if (first && fresh(c, b)) {
                            staged = 1;
                            xi = (int)xc.size();
                            xc.push_back(c);
                        }
                        erec.push_back(make_int2(c, first | (last << 1) | (staged << 2) | (sl << 3) | (xi << 15)));
                        ca.push_back(p.a[e]);
                        if (ks.shifted) cbv.push_back(p.b[e]);
                        n2 += p.a[e] * p.a[e];
                    }
                    rrec.push_back(make_int2(p.rhs.empty() ? r : p.rhs[r], e0 | (((int)erec.size() - e0) << 16)));
                    rinv.push_back(n2 > 0.0 ? 1.0 / n2 : 0.0);
                }
                // flags: 1 requirements (the publish flag 2 is set once every
                // band's requirements are known)
                const int4 g = lvl[L0 + qq];
                lrec.push_back(make_int4(row0, (int)rrec.size() - row0, lg, g.y > 0 ? 1 : 0));
                if (g.y <= KZ_CHQ) {
                    qrec.push_back(make_int2((int)rqrec.size(), g.y));
                    for (int k = 0; k < g.y; ++k) rqrec.push_back(req[g.x + k]);
                } else {
                    qrec.push_back(make_int2(g.x, -g.y - 1));
                }
                bd.lvl_chunk.push_back((int)bd.chunk.size());
            }
            KChunk ck{};
            ck.L0 = L0 + q0;
            ck.nl = q1 - q0;
            ck.nr = (int)rrec.size();
            ck.ne = (int)erec.size();
            ck.nx = (int)xc.size();
            ck.nq = (int)rqrec.size();
            ck.off_f = (long long)bd.img_f.size();
            ck.off_d = (long long)bd.img_d.size();
            ck.bytes_f = write_image<float>(bd.img_f, ks.shifted, lrec, qrec, rrec, rinv, erec, ca, cbv, xc, rqrec);
            ck.bytes_d = write_image<double>(bd.img_d, ks.shifted, lrec, qrec, rrec, rinv, erec, ca, cbv, xc, rqrec);
            bd.chunk.push_back(ck);
            bd.nent += ck.ne;
        }
        bd.rr.clear();
        bd.rr.shrink_to_fit();
    });
    // 2e. concatenation in band order
    std::vector<int> band_chunk(nb + 1, 0);
    std::vector<KChunk> chunk;
    std::vector<int> lvl_chunk;  // per (global) level: its chunk
    std::vector<unsigned char> img_f, img_d;
    int64_t nent = 0;
    {
        size_t tf = 0, td = 0;
        for (const Band &bd : B) { tf += bd.img_f.size(); td += bd.img_d.size(); }
        img_f.reserve(tf);
        img_d.reserve(td);
    }
    for (int b = 0; b < nb; ++b) {
        Band &bd = B[b];
        band_chunk[b] = (int)chunk.size();
        const long long of = (long long)img_f.size(), od = (long long)img_d.size();
        for (KChunk ck : bd.chunk) {
            ck.off_f += of;
            ck.off_d += od;
            chunk.push_back(ck);
        }
        for (int lc : bd.lvl_chunk) lvl_chunk.push_back(band_chunk[b] + lc);
        img_f.insert(img_f.end(), bd.img_f.begin(), bd.img_f.end());
        img_d.insert(img_d.end(), bd.img_d.begin(), bd.img_d.end());
        std::vector<unsigned char>().swap(bd.img_f);
        std::vector<unsigned char>().swap(bd.img_d);
        nent += bd.nent;
    }
    band_chunk[nb] = (int)chunk.size();
    // publish flags: levels a later band waits for, and every band's last
    // level; set in the global records and in both images (flag 2 of the
    // level record, which sits at the image's offset 0)
    auto set_publish = [&](int L) {
        lvl[L].z = 1;
        const KChunk &ck = chunk[lvl_chunk[L]];
        const size_t at = 16u * (size_t)(L - ck.L0) + 12u;
        int f = 0;
        std::memcpy(&f, img_f.data() + ck.off_f + at, 4);
        f |= 2;
        std::memcpy(img_f.data() + ck.off_f + at, &f, 4);
        std::memcpy(&f, img_d.data() + ck.off_d + at, 4);
        f |= 2;
        std::memcpy(img_d.data() + ck.off_d + at, &f, 4);
    };
    for (int b = 0; b < nb; ++b) {
        for (const int2 &pb : B[b].pub) set_publish(band_lvl0[pb.x] + pb.y);
        set_publish(band_lvl0[b + 1] - 1);
    }
    ks.nlevels = (int)lvl.size();
    ks.max_slots = max_slots;
    ks.nent = nent;
    ks.nchunks = (int)chunk.size();
    ks.order = claim_order(nb, band_lvl0, lvl, req);
    if (req.empty()) req.push_back(make_int2(0, 0));
    ks.band_chunk = std::move(band_chunk);
    ks.chunk = std::move(chunk);
    ks.lvl = std::move(lvl);
    ks.img_f = std::move(img_f);
    ks.img_d = std::move(img_d);
    ks.req = std::move(req);
}

void build_from_pattern(const Pattern &p, int mode, KSched &ks, cudaStream_t s,
                        int slot_cap = SLOT_CAP, int band_rows = 0) {
    HostSched h;
    build_host(p, mode, h, 0, slot_cap, band_rows);
    ks.rows = h.rows;
    ks.cols = h.cols;
    ks.shifted = h.shifted;
    ks.mode = h.mode;
    ks.nbands = h.nbands;
    ks.nlevels = h.nlevels;
    ks.max_slots = h.max_slots;
    ks.nent = h.nent;
    ks.nchunks = h.nchunks;
    const int nb = h.nbands;
    // upload
    ks.band_chunk.upload(h.band_chunk.data(), h.band_chunk.size(), s);
    ks.chunk.upload(h.chunk.data(), h.chunk.size(), s);
    ks.lvl.upload(h.lvl.data(), h.lvl.size(), s);
    ks.img_f.upload(h.img_f.data(), h.img_f.size(), s);
    ks.img_d.upload(h.img_d.data(), h.img_d.size(), s);
    ks.req.upload(h.req.data(), h.req.size(), s);
    ks.order.upload(h.order.data(), h.order.size(), s);
    ks.progress.alloc(std::max(nb, 1));
    ks.progress.zero(s);
    ks.ctl.alloc(1);
    KCtl c0;
    std::memset(&c0, 0, sizeof(c0));
    c0.epoch = 1;
    c0.mute = -1;
    ks.ctl.upload(&c0, 1, s);
    SAMG_CUDA(cudaStreamSynchronize(s));
}

void append_row(Pattern &p, const HCsr &M, int i, int col_off, bool as_b) {
    for (int64_t e = M.rp[i]; e < M.rp[i + 1]; ++e) {
        p.ci.push_back(M.ci[e] + col_off);
        p.a.push_back(as_b ? 0.0 : M.v[e]);
        p.b.push_back(as_b ? M.v[e] : 0.0);
    }
}

}  // namespace

namespace {

// dynamic shared memory of one CTA: the window of `slots` rows (plus the
// scratch slot 0) in the arithmetic type, then the staging buffers
template <typename T, typename S, int LD, bool SHIFT>
constexpr size_t smem_bytes(int slots) {
    return ((size_t)(slots + 1) * LD * sizeof(T) + 127) / 128 * 128 +
           (size_t)KZ_NBUF * Stage<T, S, LD, SHIFT>::stride;
}
template <int LD, bool SHIFT>
int window_cap_ld(bool wide) {
    // the most window slots the launches of every storage type that uses the
    // schedule can hold in 227 KB, less 2 KB for the kernel's static shared
    // memory: float64 windows (wide), and float32 windows (float32 and
    // bfloat16 storage)
    constexpr size_t budget = 227u * 1024u - 2048u;
    int cap = 4095;
    auto fit = [&](size_t per_slot, size_t fixed) {
        const long long n = ((long long)budget - (long long)fixed - 128) / (long long)per_slot - 1;
        cap = std::min<long long>(cap, n);
    };
    if (wide)
        fit((size_t)LD * sizeof(double), smem_bytes<double, double, LD, SHIFT>(0) - LD * sizeof(double));
    fit((size_t)LD * sizeof(float), smem_bytes<float, float, LD, SHIFT>(0) - LD * sizeof(float));
    fit((size_t)LD * sizeof(float), smem_bytes<float, bf16, LD, SHIFT>(0) - LD * sizeof(float));
    return std::max(cap, SLOT_CAP);
}

}  // namespace

int kz_window_cap(int ld, int mode, bool wide) {
    const bool shift = mode != 0;
    switch (ld) {
        case 4: return shift ? window_cap_ld<4, true>(wide) : window_cap_ld<4, false>(wide);
        case 8: return shift ? window_cap_ld<8, true>(wide) : window_cap_ld<8, false>(wide);
        case 12: return shift ? window_cap_ld<12, true>(wide) : window_cap_ld<12, false>(wide);
        case 16: return shift ? window_cap_ld<16, true>(wide) : window_cap_ld<16, false>(wide);
        default: return SLOT_CAP;
    }
}


void build_kschedule(const HCsr &A, const HCsr *B, KSched &ks, cudaStream_t s) {
    build_from_pattern(merge_pattern(A, B), B ? 1 : 0, ks, s);
}

namespace {

// count sweeps over the rows of A - s B in sequence, as one program
Pattern stacked_pattern(const HCsr &A, const HCsr &B, int count) {
    const Pattern one = merge_pattern(A, &B);
    Pattern p;
    p.rows = one.rows * count;
    p.cols = one.cols;
    p.rp.assign(1, 0);
    for (int k = 0; k < count; ++k) {
        if (k > 0) p.seg.push_back(k * one.rows);
        for (int i = 0; i < one.rows; ++i) {
            for (int64_t e = one.rp[i]; e < one.rp[i + 1]; ++e) {
                p.ci.push_back(one.ci[e]);
                p.a.push_back(one.a[e]);
                p.b.push_back(one.b[e]);
            }
            p.rp.push_back((int64_t)p.ci.size());
            p.rhs.push_back(i);
        }
    }
    return p;
}

}  // namespace

void build_kschedule_stacked(const HCsr &A, const HCsr &B, int count, KSched &ks, cudaStream_t s,
                             int ld, bool wide, int band_rows) {
    build_from_pattern(stacked_pattern(A, B, count), 1, ks, s, kz_window_cap(ld, 1, wide),
                       band_rows);
}

namespace {

// count block Gauss-Seidel relaxations of the minimal SVD kind as one
// program over [v; u]
Pattern fused_pattern(const HCsr &A, const HCsr &At, const HCsr &B, const HCsr &C, int count) {
    const int m = A.m, n = A.n;
    Pattern p;
    p.rows = count * (m + n);
    p.cols = n + m;  // unknown [v; u]
    p.rp.assign(1, 0);
    for (int k = 0; k < count; ++k) {
        if (k > 0) p.seg.push_back(k * (m + n));
        p.seg.push_back(k * (m + n) + m);
        // rows of A for v: a_i . v - s_j (B u)_i = kappa_i (v columns, then u)
        for (int i = 0; i < m; ++i) {
            append_row(p, A, i, 0, false);
            append_row(p, B, i, n, true);
            p.rp.push_back((int64_t)p.ci.size());
            p.rhs.push_back(i);
        }
        // rows of A^t for u: a^t_j . u - s_j (C v)_j = tau_j (v columns, then u)
        for (int j = 0; j < n; ++j) {
            append_row(p, C, j, 0, true);
            append_row(p, At, j, n, false);
            p.rp.push_back((int64_t)p.ci.size());
            p.rhs.push_back(m + j);
        }
    }
    return p;
}

HCsr identity_csr(int k) {
    HCsr h;
    h.m = h.n = k;
    h.rp.resize(k + 1);
    h.ci.resize(k);
    h.v.assign(k, 1.0);
    for (int i = 0; i <= k; ++i) h.rp[i] = i;
    for (int i = 0; i < k; ++i) h.ci[i] = i;
    return h;
}

HCsr transpose_csr(const HCsr &A) {
    HCsr At;
    At.m = A.n;
    At.n = A.m;
    At.rp.assign(A.n + 1, 0);
    for (int64_t e = 0; e < A.nnz(); ++e) At.rp[A.ci[e] + 1]++;
    for (int j = 0; j < A.n; ++j) At.rp[j + 1] += At.rp[j];
    At.ci.resize(A.nnz());
    At.v.resize(A.nnz());
    std::vector<int64_t> fill(At.rp.begin(), At.rp.end() - 1);
    for (int i = 0; i < A.m; ++i)
        for (int64_t e = A.rp[i]; e < A.rp[i + 1]; ++e) {
            const int64_t f = fill[A.ci[e]]++;
            At.ci[f] = i;
            At.v[f] = A.v[e];
        }
    return At;
}

}  // namespace

void build_kschedule_fused(const HCsr &A, const HCsr &At, const HCsr &B, const HCsr &C, int count,
                           KSched &ks, cudaStream_t s, int ld, bool wide, int band_rows) {
    build_from_pattern(fused_pattern(A, At, B, C, count), 2, ks, s, kz_window_cap(ld, 2, wide),
                       band_rows);
}

namespace {

// The program of one sweep over the rows of A (fused_count 0), or of
// fused_count minimal-SVD relaxations with B = I, C = I, as the solve
// builds it with build_kschedule_fused.
Pattern sweep_pattern(const HCsr &A, int fused_count) {
    if (fused_count <= 0) return merge_pattern(A, nullptr);
    return fused_pattern(A, transpose_csr(A), identity_csr(A.m), identity_csr(A.n), fused_count);
}

}  // namespace

void host_schedule(const HCsr &A, const HCsr *B, const HCsr *C, int fused_count, bool spd,
                   HostSched &h, int resident_cap, int band_rows, int slot_cap) {
    SAMG_CHECK(resident_cap >= 0 && resident_cap <= 4095, SAMG_E_INVALID,
               "kaczmarz: resident window larger than the slot field (4095)");
    SAMG_CHECK(band_rows >= 0 && slot_cap >= 0 && slot_cap <= 4095, SAMG_E_INVALID,
               "kaczmarz: band_rows < 0, or a window outside the slot field (0..4095)");
    if (slot_cap == 0) slot_cap = SLOT_CAP;
    if (spd) {
        const HCsr I = B ? HCsr() : identity_csr(A.m);
        build_host(stacked_pattern(A, B ? *B : I, std::max(1, fused_count)), 1, h, resident_cap,
                   slot_cap, band_rows);
    } else if (fused_count <= 0) {
        build_host(merge_pattern(A, nullptr), 0, h, resident_cap, slot_cap, band_rows);
    } else {
        const HCsr Im = B ? HCsr() : identity_csr(A.m), In = C ? HCsr() : identity_csr(A.n);
        build_host(fused_pattern(A, transpose_csr(A), B ? *B : Im, C ? *C : In, fused_count), 2, h,
                   resident_cap, slot_cap, band_rows);
    }
}

void plan_sweep(const HCsr &A, int fused_count, std::vector<int> &levels, int *nbands) {
    const Pattern p = sweep_pattern(A, fused_count);
    levels = global_levels(p);
    BandWork w(p.cols);
    *nbands = (int)form_bands(p, levels, w).size() - 1;
}

template <typename T>
static void dispatch(const KSched &ks, int ld, const T *rhs, T *x, const double *shift,
                     cudaStream_t s) {
    if (ks.rows == 0) return;
#define KZ_CASE(L)                                                       \
    case L:                                                              \
        if (ks.mode == 1) launch_one<T, L, 1>(ks, rhs, x, shift, s);      \
        else if (ks.mode == 2) launch_one<T, L, 2>(ks, rhs, x, shift, s); \
        else launch_one<T, L, 0>(ks, rhs, x, shift, s);                   \
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
    dispatch<double>(ks, ld, rhs, x, shift, s);
}
template <>
void launch_kaczmarz<float>(const KSched &ks, int ld, const float *rhs, float *x,
                            const double *shift, cudaStream_t s) {
    dispatch<float>(ks, ld, rhs, x, shift, s);
}
template <>
void launch_kaczmarz<bf16>(const KSched &ks, int ld, const bf16 *rhs, bf16 *x,
                           const double *shift, cudaStream_t s) {
    dispatch<bf16>(ks, ld, rhs, x, shift, s);
}

void kaczmarz_mute_band(KSched &ks, int band, cudaStream_t s) {
    if (ks.rows == 0) return;
    SAMG_CHECK(band >= -1 && band < ks.nbands, SAMG_E_INVALID, "kaczmarz: band out of range");
    SAMG_CUDA(cudaMemcpyAsync(&ks.ctl.p->mute, &band, sizeof(int), cudaMemcpyHostToDevice, s));
    SAMG_CUDA(cudaStreamSynchronize(s));
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
