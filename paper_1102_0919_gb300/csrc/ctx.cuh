// ctx.cuh -- the solver context: hierarchy on the device, the finest-level
// boot triplets, and the drivers of the additive V-cycle (Sec. 4) and of the
// Ritz step (Sec. 4.3).
#pragma once

#include <memory>
#include <string>
#include <vector>

#include "coloured.cuh"
#include "common.cuh"
#include "dense.cuh"
#include "kaczmarz.cuh"
#include "kernels.cuh"

namespace samg {

template <typename T>
struct Work {          // V-cycle vectors of one level in one precision (ld columns)
    DBuf<T> u, v;      // iterate (error) blocks: m x ld, n x ld
    DBuf<T> k, t;      // right-hand sides kappa, tau
    DBuf<T> r, s;      // residuals / Kaczmarz right-hand sides
    DBuf<T> tu, tv;    // Jacobi double buffers
    DBuf<T> z, kt;     // fused relaxations: unknown [v; u] and right-hand side [kappa; tau]
};

struct Level {
    int m = 0, n = 0;           // A_l is m x n (SPD kind: n x n)
    DCsr A, At, B, C;           // B, C empty on the finest level (identity)
    DCsr P, Pt, Q, Qt;          // empty on the coarsest level
    KSched kA, kAt;             // Kaczmarz schedules (minimal target)
    std::vector<KSched> kF;     // fused programs of `count` relaxations, by count
    std::vector<KSched> kF4;    // the same with float32-only windows (float32, bfloat16)
    std::vector<CSched> kC;     // their coloured-order variants, by count
    DBuf<double> dBd, dCd;      // diagonals of B, C (dominant target)
    DBuf<float> dBf, dCf;
    Work<float> wf;
    Work<double> wd;
    Work<bf16> wb;              // bfloat16 storage (allocated on first use)
};

// Launch timing with CUDA events on the context's stream (samg_profile).
struct Profiler {
    bool on = false;
    struct Rec { int cls; cudaEvent_t a, b; double bytes; int level; };
    int cur_level = -1;
    double lvl_ms[5][32] = {};
    int64_t lvl_n[5][32] = {};
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    int64_t launches[5] = {0, 0, 0, 0, 0};
    double ms[5] = {0, 0, 0, 0, 0}, bytes[5] = {0, 0, 0, 0, 0};
    cudaEvent_t get() {
        if (pool.empty()) {
            cudaEvent_t e;
            SAMG_CUDA(cudaEventCreate(&e));
            return e;
        }
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
    void begin(cudaStream_t s, int cls, double b, cudaEvent_t *out) {
        if (!on) return;
        *out = get();
        SAMG_CUDA(cudaEventRecord(*out, s));
        recs.push_back({cls, *out, nullptr, b, cur_level});
    }
    void end(cudaStream_t s) {
        if (!on) return;
        cudaEvent_t e = get();
        SAMG_CUDA(cudaEventRecord(e, s));
        recs.back().b = e;
    }
    void collect() {  // synchronizes on the recorded events
        for (auto &r : recs) {
            float t = 0.f;
            SAMG_CUDA(cudaEventSynchronize(r.b));
            SAMG_CUDA(cudaEventElapsedTime(&t, r.a, r.b));
            launches[r.cls]++;
            ms[r.cls] += t;
            bytes[r.cls] += r.bytes;
            if (r.level >= 0 && r.level < 32) {
                lvl_ms[r.cls][r.level] += t;
                lvl_n[r.cls][r.level]++;
            }
            pool.push_back(r.a);
            pool.push_back(r.b);
        }
        recs.clear();
    }
    ~Profiler() {
        for (auto &r : recs) { cudaEventDestroy(r.a); if (r.b) cudaEventDestroy(r.b); }
        for (auto e : pool) cudaEventDestroy(e);
    }
};

// RAII bracket of one launch
struct Prof {
    Profiler &p;
    cudaStream_t s;
    cudaEvent_t e = nullptr;
    Prof(Profiler &pp, cudaStream_t ss, int cls, double bytes) : p(pp), s(ss) { p.begin(s, cls, bytes, &e); }
    ~Prof() { if (e) p.end(s); }
};

struct Coarse {
    int M = 0, m1 = 0;
    DBuf<double> X, Y, lam, W, Wt, work;
    DBuf<int> status;
    DBuf<double> qwarm;  // per column: the pseudo-inverse's subspace basis of the last call
    DBuf<double> cbuf;   // generalized-eigen variant: coefficients W^t r (M x ld)
    bool warm = false;
};

}  // namespace samg

struct samg_ctx {
    cudaStream_t stream = nullptr;
    samg_kind kind = SAMG_SVD;
    samg_target target = SAMG_MINIMAL;
    samg_params prm{};
    int nb = 0, ld = 0;
    std::vector<samg::Level> L;
    samg::Coarse co;
    // finest-level boot triplets (float64, ld columns; padding columns 0, sigma 1)
    samg::DBuf<double> sigma, U, V, resid;
    // Ritz work
    samg::DBuf<double> AV, AtU, Un, Vn, GU, GV, H, TU, TV, gwork, partu, partv;
    samg::DBuf<int> rstat;
    samg::Profiler prof;
    // banding of the smoothing phases' sweep programs (samg_set_sweep_banding):
    // rows per level a band grows to (0: the per-level default), per-level
    // overrides, and whether float32 launches get programs with float32-only
    // windows
    int band_rows = 0;
    std::vector<int> band_rows_level;
    bool float_windows = false;
    // wall seconds of the setup phase's stages (samg_setup_times)
    double setup_s[SAMG_SETUP_STAGES] = {};
    // the setup phase's state (fine test vectors, finest coarsening), kept
    // after samg_setup when redo_tol > 0 for the redo of Sec. 6.3
    std::shared_ptr<void> setup_keep;
    std::string err;
    bool poisoned = false;
    bool spd() const { return kind == SAMG_SPD_EIG; }
    bool minimal() const { return target == SAMG_MINIMAL; }
    int nlev() const { return (int)L.size(); }
};

namespace samg {

// hierarchy completion after the interpolation operators are known
void build_galerkin(samg_ctx &c);
void finalize_hierarchy(samg_ctx &c);
void prepare_level(samg_ctx &c, int l);
void prepare_coarsest(samg_ctx &c);
void csr_identity(int n, HCsr &h);
void alloc_finest_state(samg_ctx &c);
void share_error_word(samg_ctx &c);

// triplets host <-> device (row-major nb columns on the host)
void put_block(samg_ctx &c, const double *h, int rows, DBuf<double> &d);
void get_block(samg_ctx &c, const DBuf<double> &d, int rows, double *h);

// V-cycle pieces in precision T on level l (vectors in L[l].w*)
template <typename T> Work<T> &work(Level &L);
// every level's work vectors in storage type T (allocated when missing)
template <typename T> void ensure_work(samg_ctx &c);
template <typename T> void relax(samg_ctx &c, int l);
template <typename T> void relax_phase(samg_ctx &c, int l, int count);
template <typename T> void residual_restrict(samg_ctx &c, int l);
template <typename T> void interpolate(samg_ctx &c, int l);
template <typename T> void coarse_solve(samg_ctx &c);
template <typename T> void vcycle(samg_ctx &c, int l);
template <typename T> void outer_vcycle(samg_ctx &c);   // defect form on (U, V)

// identity: residuals of the current triplets only; check: wait for the
// step's status and raise on linearly dependent boot vectors (false: the
// caller reads rstat[0] later)
void ritz(samg_ctx &c, bool identity, bool check = true);
void host_setup(samg_ctx &c, const samg_csr &A);  // multiplicative phase (setup.cu)
// Sec. 6.3: new interpolation operators by one downward sweep of the
// multiplicative phase, LS weights of the test vectors and of the converged
// boot vectors (conv[j] != 0) divided by 1000; the iterate is unchanged
void redo_interpolation(samg_ctx &c, const std::vector<char> &conv);
// The setup's host steps on their own (setup.cu): strength (Eq. strength) and
// Ruge-Stueben coarsening of N; weighted LS interpolation (Eq. LS) from the
// strong C-point influences, nf vectors per point (row-major yF, yC).
void host_coarsen(const HCsr &N, double theta, std::vector<char> &cf);
// strong influences of N = A A^t from A itself, without forming N
void host_strength_product(const HCsr &A, double theta, HCsr &S);
void host_ls_interp(const HCsr &N, double theta, const std::vector<char> &cf,
                    const std::vector<double> &yF, const std::vector<double> &yC,
                    const std::vector<double> &w, int nf, HCsr &P);

}  // namespace samg
