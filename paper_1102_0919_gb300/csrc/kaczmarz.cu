// kaczmarz.cu -- schedule builder (host) and sweep kernel (device) for the
// exact-order Kaczmarz relaxation of Sec. 5.3 (see kaczmarz.cuh).
#include <algorithm>
#include <cstring>

#include "kaczmarz.cuh"

namespace samg {

namespace {

constexpr int KZ_THREADS = 256;
constexpr int TARGET_PAR = 32;       // wanted rows per level inside a band
constexpr int MAX_BAND_ROWS = 1 << 17;
constexpr int SLOT_CAP = 1600;       // window slots: 1600 * 16 cols * 8 B = 200 KiB
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

struct KView {
    int *err;
    int nbands;
    const int *band_lvl;
    const int4 *lvl;
    const int *srow, *eoff, *ecol, *eslot;
    const int2 *req;
    unsigned long long *progress;
    KCtl *ctl;
};

template <typename T, int LD, bool SHIFT>
__global__ void __launch_bounds__(KZ_THREADS)
    k_kaczmarz(KView kv, const T *__restrict__ ea, const T *__restrict__ eb,
               const T *__restrict__ inv, const T *__restrict__ rhs, T *x,
               const double *__restrict__ shift) {
    extern __shared__ __align__(16) unsigned char smraw[];
    T *win = reinterpret_cast<T *>(smraw);
    __shared__ int s_band;
    __shared__ int s_abort;
    constexpr int RPP = KZ_THREADS / LD;  // rows per pass
    const int tr = threadIdx.x / LD;
    const int j = threadIdx.x % LD;
    const unsigned long long epoch = *((volatile unsigned long long *)&kv.ctl->epoch);
    if (threadIdx.x == 0) s_abort = 0;
    const T sh = SHIFT ? (T)shift[j] : T(0);
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_band = (int)atomicAdd(&kv.ctl->ticket, 1u);
        __syncthreads();
        const int b = s_band;
        if (b >= kv.nbands || s_abort) break;
        const int L0 = kv.band_lvl[b], L1 = kv.band_lvl[b + 1];
        for (int L = L0; L < L1; ++L) {
            const int4 lv = kv.lvl[L];
            const int4 ln = kv.lvl[L + 1];
            if (ln.y > lv.y) {  // cross-band requirements of this level
                for (int q = lv.y + threadIdx.x; q < ln.y; q += blockDim.x) {
                    const int2 rq = kv.req[q];
                    const unsigned long long target = (epoch << 32) | (unsigned)rq.y;
                    const unsigned long long t0 = gtimer();
                    while (ld_acquire(&kv.progress[rq.x]) < target) {
                        if (*((volatile int *)kv.err) || gtimer() - t0 > WAIT_NS) {
                            atomicExch(kv.err, 1);
                            s_abort = 1;
                            break;
                        }
                        __nanosleep(32);
                    }
                }
                __syncthreads();
                if (s_abort) break;
            }
            if (tr < RPP) {
                for (int k = lv.x + tr; k < ln.x; k += RPP) {
                    const int row = kv.srow[k];
                    const int e0 = kv.eoff[k], e1 = kv.eoff[k + 1];
                    T dot = T(0), nrm = T(0);
                    for (int e = e0; e < e1; ++e) {
                        const int sl = kv.eslot[e];
                        const T coef = SHIFT ? ea[e] - sh * eb[e] : ea[e];
                        const T val = (sl & 1) ? __ldcg(x + (size_t)kv.ecol[e] * LD + j)
                                               : win[(sl >> 2) * LD + j];
                        dot = fma(coef, val, dot);
                        if (SHIFT) nrm = fma(coef, coef, nrm);
                    }
                    T d = (rhs ? rhs[(size_t)row * LD + j] : T(0)) - dot;
                    if (SHIFT)
                        d = nrm > T(0) ? d / nrm : T(0);
                    else
                        d *= inv[k];
                    for (int e = e0; e < e1; ++e) {
                        const int sl = kv.eslot[e];
                        const T coef = SHIFT ? ea[e] - sh * eb[e] : ea[e];
                        T *gp = x + (size_t)kv.ecol[e] * LD + j;
                        const T val = (sl & 1) ? __ldcg(gp) : win[(sl >> 2) * LD + j];
                        const T nv = fma(d, coef, val);
                        if (sl & 2)
                            __stcg(gp, nv);
                        else
                            win[(sl >> 2) * LD + j] = nv;
                    }
                }
            }
            __syncthreads();
            if (lv.z && threadIdx.x == 0) {
                __threadfence();
                st_release(&kv.progress[b], (epoch << 32) | (unsigned)(L - L0 + 1));
            }
        }
        if (threadIdx.x == 0 && !s_abort) {
            __threadfence();
            st_release(&kv.progress[b], (epoch << 32) | (unsigned)(L1 - L0));
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
    size_t smem = (size_t)std::max(ks.max_slots, 1) * LD * sizeof(T);
    auto kern = k_kaczmarz<T, LD, SHIFT>;
    SAMG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int dev = 0, nsm = 0, bps = 0;
    SAMG_CUDA(cudaGetDevice(&dev));
    SAMG_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    SAMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, KZ_THREADS, smem));
    SAMG_CHECK(bps > 0, SAMG_E_CUDA, "kaczmarz: window does not fit in shared memory");
    int grid = std::min(ks.nbands, nsm * bps);
    KView kv{ks.err ? ks.err : &ks.ctl.p->err, ks.nbands, ks.band_lvl.p, ks.lvl.p, ks.srow.p, ks.eoff.p,
             ks.ecol.p, ks.eslot.p, ks.req.p, ks.progress.p, ks.ctl.p};
    SAMG_COUNT_LAUNCH();
    kern<<<grid, KZ_THREADS, smem, s>>>(kv, ea, eb, inv, rhs, x, shift);
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
    // 1. bands
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
    // 2. levels, slots, entries, requirements
    std::vector<int> band_lvl(nb + 1, 0);
    std::vector<int4> lvl;
    std::vector<int> srow, eoff, ecol, eslot;
    std::vector<double> ea, eb, inv;
    std::vector<int2> req;
    std::vector<int> g_band(cols, -1), g_lvl(cols, 0), slot(cols, 0);
    std::vector<int> waited(nb, 0), waited_stamp(nb, -1);
    ea.reserve(p.ci.size());
    ecol.reserve(p.ci.size());
    eslot.reserve(p.ci.size());
    if (ks.shifted) eb.reserve(p.ci.size());
    int max_slots = 0;
    std::vector<std::vector<int>> pub;  // per band: levels to publish
    pub.resize(nb);
    struct PendReq { int lvl, band, need; };
    for (int b = 0; b < nb; ++b) {
        const int r0 = bstart[b], r1 = bstart[b + 1];
        int nl = analyze_band(p, r0, r1, w, &slots);
        max_slots = std::max(max_slots, slots);
        band_lvl[b] = (int)lvl.size();
        // rows grouped by level (ascending row order inside a level)
        std::vector<int> lcount(nl + 1, 0);
        for (int r = r0; r < r1; ++r) lcount[w.rowlv[r - r0] + 1]++;
        for (int l = 0; l < nl; ++l) lcount[l + 1] += lcount[l];
        std::vector<int> order(r1 - r0);
        {
            std::vector<int> fillp(lcount.begin(), lcount.end() - 1);
            for (int r = r0; r < r1; ++r) order[fillp[w.rowlv[r - r0]]++] = r;
        }
        // slot assignment by interval colouring over levels
        std::vector<std::vector<int>> starts(nl), ends(nl);
        for (int c : w.touched)
            if (w.cnt[c] >= 2) {
                starts[w.firstlv[c]].push_back(c);
                ends[w.lastlv[c]].push_back(c);
            }
        std::vector<int> freel;
        int next = 0;
        for (int l = 0; l < nl; ++l) {
            for (int c : starts[l]) {
                if (!freel.empty()) { slot[c] = freel.back(); freel.pop_back(); }
                else slot[c] = next++;
            }
            for (int c : ends[l]) freel.push_back(slot[c]);
        }
        // entries and requirements
        std::vector<PendReq> pend;
        for (int l = 0; l < nl; ++l) {
            int4 L4;
            L4.x = (int)srow.size();
            L4.y = 0; L4.z = 0; L4.w = 0;
            lvl.push_back(L4);
            for (int k = lcount[l]; k < lcount[l + 1]; ++k) {
                const int r = order[k];
                srow.push_back(r);
                eoff.push_back((int)ecol.size());
                double n2 = 0.0;
                for (int64_t e = p.rp[r]; e < p.rp[r + 1]; ++e) {
                    const int c = p.ci[e];
                    const int first = (w.firstlv[c] == l), last = (w.lastlv[c] == l);
                    const int sl = (w.cnt[c] >= 2) ? slot[c] : 0;
                    ecol.push_back(c);
                    eslot.push_back((sl << 2) | (first ? 1 : 0) | (last ? 2 : 0));
                    ea.push_back(p.a[e]);
                    if (ks.shifted) eb.push_back(p.b[e]);
                    n2 += p.a[e] * p.a[e];
                    if (first && g_band[c] >= 0) pend.push_back({l, g_band[c], g_lvl[c] + 1});
                }
                inv.push_back(n2 > 0.0 ? 1.0 / n2 : 0.0);
            }
        }
        // per level: max need per band, dropping needs already waited for
        std::sort(pend.begin(), pend.end(), [](const PendReq &a, const PendReq &b2) {
            return a.lvl != b2.lvl ? a.lvl < b2.lvl : (a.band != b2.band ? a.band < b2.band : a.need > b2.need);
        });
        size_t q = 0;
        for (int l = 0; l < nl; ++l) {
            lvl[band_lvl[b] + l].y = (int)req.size();
            while (q < pend.size() && pend[q].lvl == l) {
                const PendReq &pr = pend[q];
                if (waited_stamp[pr.band] != b || waited[pr.band] < pr.need) {
                    waited_stamp[pr.band] = b;
                    waited[pr.band] = pr.need;
                    req.push_back(make_int2(pr.band, pr.need));
                    pub[pr.band].push_back(pr.need - 1);
                }
                // skip the rest of this (level, band) group
                const int bb = pr.band;
                while (q < pend.size() && pend[q].lvl == l && pend[q].band == bb) ++q;
            }
        }
        for (int c : w.touched) {
            g_band[c] = b;
            g_lvl[c] = w.lastlv[c];
        }
    }
    band_lvl[nb] = (int)lvl.size();
    for (int b = 0; b < nb; ++b)
        for (int l : pub[b]) lvl[band_lvl[b] + l].z = 1;
    int4 sentinel;
    sentinel.x = (int)srow.size();
    sentinel.y = (int)req.size();
    sentinel.z = 0; sentinel.w = 0;
    lvl.push_back(sentinel);
    eoff.push_back((int)ecol.size());
    ks.nlevels = (int)lvl.size() - 1;
    ks.max_slots = max_slots;
    ks.nent = (int64_t)ecol.size();
    // 3. upload
    ks.band_lvl.upload(band_lvl.data(), band_lvl.size(), s);
    ks.lvl.upload(lvl.data(), lvl.size(), s);
    ks.srow.upload(srow.data(), srow.size(), s);
    ks.eoff.upload(eoff.data(), eoff.size(), s);
    ks.ecol.upload(ecol.data(), ecol.size(), s);
    ks.eslot.upload(eslot.data(), eslot.size(), s);
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
