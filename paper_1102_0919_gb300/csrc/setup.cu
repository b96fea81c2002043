// setup.cu -- multiplicative (setup) phase of Sec. 3.3: bootstrap V-cycles
// that relax random test vectors, coarsen (Sec. 3.7), fit interpolation by
// weighted least squares (Sec. 3.8), build Galerkin operators on the GPU,
// solve the coarsest generalized SVD directly (Sec. 3.6), interpolate and
// relax the boot triplets on the way up, and finish each cycle with a Ritz
// step.  Strength, Ruge-Stueben coarsening and the small LS solves run on the
// host; relaxations, products, Galerkin operators and the Ritz step run on the
// GPU.
//
// Minimal SVD kind with m >= n: the row interpolation is induced from the
// column interpolation, P_0 = A Q_0 and P_l = Q_l below the finest level,
// where A_l = B_l; row test vectors are A v_t (finest) or v_t.  A^t A-type
// row coarsening cannot represent the minimal left singular vectors of
// gradient-like operators and Kaczmarz on A^t u = 0 drifts into null(A^t).
#include <algorithm>
#include <cmath>
#include <set>
#include <thread>

#include "ctx.cuh"

namespace samg {

namespace {

// ------------------------------------------------------------- test vectors
// SplitMix64 (Steele, Lea, Flood 2014) used as a counter-based generator:
// entry (row i, vector k) = 2 * (z >> 11) * 2^-53 - 1, z = mix(seed ^ (k << 40) ^ i).
__device__ __forceinline__ unsigned long long splitmix_out(unsigned long long st) {
    unsigned long long z = st + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void k_random_block(unsigned long long seed, int rows, int nvec, int ld, double *out) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)rows * ld) return;
    int i = (int)(t / ld), k = (int)(t % ld);
    double v = 0.0;
    if (k < nvec) {
        unsigned long long z = splitmix_out(seed ^ ((unsigned long long)k << 40) ^ (unsigned long long)i);
        v = 2.0 * ((double)(z >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
    }
    out[t] = v;
}

// ------------------------------------------------------------ host helpers
struct Strength {
    HCsr S;  // S_i = points that strongly influence i, values |n_ij|
};

// i is strongly influenced by j != i iff |n_ij| >= theta * sum_k |n_ik|
// (Eq. strength, sum over all k including the diagonal).
void strength_of(const HCsr &N, double theta, HCsr &S) {
    S.m = S.n = N.m;
    S.rp.assign(N.m + 1, 0);
    S.ci.clear();
    S.v.clear();
    for (int i = 0; i < N.m; ++i) {
        double tot = 0.0;
        for (int64_t e = N.rp[i]; e < N.rp[i + 1]; ++e) tot += std::fabs(N.v[e]);
        const double thr = theta * tot;
        for (int64_t e = N.rp[i]; e < N.rp[i + 1]; ++e) {
            const double a = std::fabs(N.v[e]);
            if (N.ci[e] != i && a > 0.0 && a >= thr) {
                S.ci.push_back(N.ci[e]);
                S.v.push_back(a);
            }
        }
        S.rp[i + 1] = (int64_t)S.ci.size();
    }
}

// Strong influences (Eq. strength) of N = A A^t without forming N.  Row i of
// N is the sum over the entries a_ic of row i of A of a_ic times row c of
// A^t (entries accumulated in that order into a dense per-thread row); the
// row sum of |n_ik| over every touched k (the diagonal included) sets the
// threshold, and only the strong j != i are kept, sorted by column.  Memory
// is that of S and one dense row per thread: the product of a
// term-document matrix can hold ~1e10 entries while its strong graph holds
// at most 1/theta per row.  The rows run on up to 16 host threads, each
// writing its own block of rows.
void strength_product(const HCsr &A, const HCsr &At, double theta, HCsr &S) {
    const int m = A.m;
    S.m = S.n = m;
    unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    if (m < 4096) nt = 1;
    const int chunk = (m + (int)nt - 1) / (int)nt;
    struct Part {
        std::vector<int64_t> cnt;
        std::vector<int> ci;
        std::vector<double> v;
    };
    std::vector<Part> part(nt);
    auto work = [&](unsigned t) {
        const int a = (int)t * chunk, b = std::min(m, a + chunk);
        if (a >= b) return;
        Part &out = part[t];
        out.cnt.assign(b - a, 0);
        std::vector<double> acc(m, 0.0);
        std::vector<int> mark(m, -1), touched;
        std::vector<std::pair<int, double>> keep;
        for (int i = a; i < b; ++i) {
            touched.clear();
            for (int64_t e = A.rp[i]; e < A.rp[i + 1]; ++e) {
                const int c = A.ci[e];
                const double aic = A.v[e];
                for (int64_t f = At.rp[c]; f < At.rp[c + 1]; ++f) {
                    const int j = At.ci[f];
                    if (mark[j] != i) {
                        mark[j] = i;
                        acc[j] = 0.0;
                        touched.push_back(j);
                    }
                    acc[j] += aic * At.v[f];
                }
            }
            double tot = 0.0;
            for (int j : touched) tot += std::fabs(acc[j]);
            const double thr = theta * tot;
            keep.clear();
            for (int j : touched) {
                const double x = std::fabs(acc[j]);
                if (j != i && x > 0.0 && x >= thr) keep.push_back({j, x});
            }
            std::sort(keep.begin(), keep.end());
            out.cnt[i - a] = (int64_t)keep.size();
            for (auto &kv : keep) {
                out.ci.push_back(kv.first);
                out.v.push_back(kv.second);
            }
        }
    };
    if (nt == 1) {
        work(0);
    } else {
        std::vector<std::thread> th;
        for (unsigned t = 0; t < nt; ++t) th.emplace_back(work, t);
        for (auto &x : th) x.join();
    }
    S.rp.assign(m + 1, 0);
    S.ci.clear();
    S.v.clear();
    for (unsigned t = 0; t < nt; ++t) {
        const int a = (int)t * chunk;
        for (size_t r = 0; r < part[t].cnt.size(); ++r) S.rp[a + r + 1] = part[t].cnt[r];
        S.ci.insert(S.ci.end(), part[t].ci.begin(), part[t].ci.end());
        S.v.insert(S.v.end(), part[t].v.begin(), part[t].v.end());
    }
    for (int i = 0; i < m; ++i) S.rp[i + 1] += S.rp[i];
}

// One-pass Ruge-Stueben coarsening (Algorithm "coarsening"): repeatedly take
// the undecided point with the largest lambda (lowest index on ties), make it
// C, make the undecided points it strongly influences F, and raise lambda of
// the undecided points that strongly influence those new F points.
std::vector<char> rs_split(const HCsr &S) {
    const int n = S.m;
    std::vector<int64_t> tp(n + 1, 0);
    for (int64_t e = 0; e < S.nnz(); ++e) tp[S.ci[e] + 1]++;
    for (int i = 0; i < n; ++i) tp[i + 1] += tp[i];
    std::vector<int> tc(S.nnz());
    {
        std::vector<int64_t> f(tp.begin(), tp.end() - 1);
        for (int i = 0; i < n; ++i)
            for (int64_t e = S.rp[i]; e < S.rp[i + 1]; ++e) tc[f[S.ci[e]]++] = i;
    }
    std::vector<int64_t> lam(n);
    std::set<std::pair<int64_t, int>> open;  // (-lambda, index)
    for (int i = 0; i < n; ++i) {
        lam[i] = tp[i + 1] - tp[i];
        open.insert({-lam[i], i});
    }
    std::vector<char> st(n, 0);  // 0 undecided, 1 C, 2 F
    std::vector<int> fresh;
    while (!open.empty()) {
        const int i = open.begin()->second;
        open.erase(open.begin());
        st[i] = 1;
        fresh.clear();
        for (int64_t e = tp[i]; e < tp[i + 1]; ++e) {
            const int j = tc[e];
            if (st[j] != 0) continue;
            st[j] = 2;
            open.erase({-lam[j], j});
            fresh.push_back(j);
        }
        for (int j : fresh)
            for (int64_t e = S.rp[j]; e < S.rp[j + 1]; ++e) {
                const int k = S.ci[e];
                if (st[k] != 0) continue;
                open.erase({-lam[k], k});
                lam[k]++;
                open.insert({-lam[k], k});
            }
    }
    std::vector<char> cf(n);
    for (int i = 0; i < n; ++i) cf[i] = (st[i] == 1);
    return cf;
}

template <typename F>
void parallel_rows(int n, F &&f) {
    unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    if (n < 4096) nt = 1;
    std::vector<std::thread> th;
    const int chunk = (n + (int)nt - 1) / (int)nt;
    for (unsigned t = 0; t < nt; ++t) {
        const int a = (int)t * chunk, b = std::min(n, a + chunk);
        if (a >= b) break;
        th.emplace_back([&f, a, b] { f(a, b); });
    }
    for (auto &x : th) x.join();
}

// Weighted LS interpolation (Eq. LS): C rows carry 1 at alpha(i); F rows fit
// yF[i] ~ sum_{j in C^i} p_j yC[j] with weights w (multiplying the squared
// residuals) by the normal equations and a Cholesky factorization.  C^i = the
// strongest (ties: lowest index) C-point influences, at most nf - 1 of them;
// when a pivot is not positive the weakest member is dropped and the fit
// repeated.
void ls_interp(const HCsr &S, const std::vector<char> &cf, const std::vector<double> &yF,
               const std::vector<double> &yC, const std::vector<double> &w, int nf, HCsr &P) {
    const int n = S.m;
    std::vector<int> alpha(n, -1);
    int nc = 0;
    for (int i = 0; i < n; ++i)
        if (cf[i]) alpha[i] = nc++;
    std::vector<std::vector<std::pair<int, double>>> rows(n);
    parallel_rows(n, [&](int a, int b) {
        std::vector<std::pair<double, int>> cand;
        std::vector<double> N, r, x;
        for (int i = a; i < b; ++i) {
            if (cf[i]) {
                rows[i].push_back({alpha[i], 1.0});
                continue;
            }
            cand.clear();
            for (int64_t e = S.rp[i]; e < S.rp[i + 1]; ++e)
                if (cf[S.ci[e]]) cand.push_back({-S.v[e], S.ci[e]});
            std::sort(cand.begin(), cand.end());
            int len = std::min<int>((int)cand.size(), std::max(nf - 1, 1));
            while (len > 0) {
                N.assign((size_t)len * len, 0.0);
                r.assign(len, 0.0);
                for (int p = 0; p < len; ++p) {
                    const double *cp = &yC[(size_t)cand[p].second * nf];
                    for (int q = 0; q <= p; ++q) {
                        const double *cq = &yC[(size_t)cand[q].second * nf];
                        double acc = 0.0;
                        for (int k = 0; k < nf; ++k) acc += w[k] * cp[k] * cq[k];
                        N[(size_t)p * len + q] = acc;
                    }
                    double acc = 0.0;
                    const double *fi = &yF[(size_t)i * nf];
                    for (int k = 0; k < nf; ++k) acc += w[k] * cp[k] * fi[k];
                    r[p] = acc;
                }
                bool ok = true;  // lower Cholesky in place
                for (int p = 0; p < len && ok; ++p) {
                    for (int q = 0; q <= p; ++q) {
                        double v = N[(size_t)p * len + q];
                        for (int k = 0; k < q; ++k) v -= N[(size_t)p * len + k] * N[(size_t)q * len + k];
                        if (p == q) {
                            if (!(v > 0.0)) { ok = false; break; }
                            N[(size_t)p * len + p] = std::sqrt(v);
                        } else {
                            N[(size_t)p * len + q] = v / N[(size_t)q * len + q];
                        }
                    }
                }
                if (!ok) { --len; continue; }
                x.assign(len, 0.0);
                for (int p = 0; p < len; ++p) {
                    double v = r[p];
                    for (int k = 0; k < p; ++k) v -= N[(size_t)p * len + k] * x[k];
                    x[p] = v / N[(size_t)p * len + p];
                }
                for (int p = len - 1; p >= 0; --p) {
                    double v = x[p];
                    for (int k = p + 1; k < len; ++k) v -= N[(size_t)k * len + p] * x[k];
                    x[p] = v / N[(size_t)p * len + p];
                }
                for (int p = 0; p < len; ++p) rows[i].push_back({alpha[cand[p].second], x[p]});
                break;
            }
            std::sort(rows[i].begin(), rows[i].end());
        }
    });
    P.m = n;
    P.n = nc;
    P.rp.assign(n + 1, 0);
    P.ci.clear();
    P.v.clear();
    for (int i = 0; i < n; ++i) {
        for (auto &pr : rows[i]) {
            P.ci.push_back(pr.first);
            P.v.push_back(pr.second);
        }
        P.rp[i + 1] = (int64_t)P.ci.size();
    }
}

// y = x - om * D^-1 N x on the host (row-major blocks of nf columns)
void jacobi_host(const HCsr &N, const std::vector<double> &x, int nf, double om,
                 std::vector<double> &y) {
    y.resize(x.size());
    parallel_rows(N.m, [&](int a, int b) {
        std::vector<double> acc(nf);
        for (int i = a; i < b; ++i) {
            double d = 0.0;
            std::fill(acc.begin(), acc.end(), 0.0);
            for (int64_t e = N.rp[i]; e < N.rp[i + 1]; ++e) {
                if (N.ci[e] == i) d = N.v[e];
                const double *xc = &x[(size_t)N.ci[e] * nf];
                for (int k = 0; k < nf; ++k) acc[k] += N.v[e] * xc[k];
            }
            for (int k = 0; k < nf; ++k)
                y[(size_t)i * nf + k] = x[(size_t)i * nf + k] - (d != 0.0 ? om * acc[k] / d : 0.0);
        }
    });
}

double gershgorin(const HCsr &N) {
    double g = 0.0;
    for (int i = 0; i < N.m; ++i) {
        double d = 0.0, s = 0.0;
        for (int64_t e = N.rp[i]; e < N.rp[i + 1]; ++e) {
            s += std::fabs(N.v[e]);
            if (N.ci[e] == i) d = std::fabs(N.v[e]);
        }
        if (d > 0.0) g = std::max(g, s / d);
    }
    return g > 0.0 ? g : 2.0;
}

// download the first nvec columns of a device block (rows x ld) to host rows x nvec
void fetch(cudaStream_t s, const double *d, int rows, int ld, int nvec, double *h, int hld, int off) {
    if (!rows) return;
    SAMG_CUDA(cudaMemcpy2DAsync(h + off, hld * sizeof(double), d, ld * sizeof(double),
                                nvec * sizeof(double), rows, cudaMemcpyDeviceToHost, s));
}

// Charges the wall time since the previous mark to one setup stage, after
// the stream has drained (samg_setup_times).
struct StageClock {
    samg_ctx &c;
    std::chrono::steady_clock::time_point t;
    explicit StageClock(samg_ctx &cx, bool reset = true) : c(cx), t(std::chrono::steady_clock::now()) {
        if (reset)
            for (double &x : c.setup_s) x = 0.0;
    }
    void mark(int stage) {
        SAMG_CUDA(cudaStreamSynchronize(c.stream));
        const auto now = std::chrono::steady_clock::now();
        c.setup_s[stage] += std::chrono::duration<double>(now - t).count();
        t = now;
    }
};

struct SetupState {
    samg_ctx &c;
    cudaStream_t s;
    int nt, ldt;
    bool induced;
    int sq = 0;                     // square form in use (R23), 0 if none
    DBuf<double> Ut, Vt;            // fine test vectors (relaxed in place)
    std::vector<DBuf<double>> ut, vt;  // per level (coarse copies)
    DBuf<double> ones, dots, sgn;
    DBuf<int> idx;
    // cached finest-level coarsening (A_0 never changes)
    bool have0 = false;
    HCsr N0u, N0v, S0u, S0v;
    std::vector<char> cf0u, cf0v;
    explicit SetupState(samg_ctx &cc) : c(cc), s(cc.stream) {}
};

// column dots x_j^t M y_j (M null -> identity), nvec columns of a ld-wide block
std::vector<double> coldots(SetupState &st, int rows, int nvec, int ld, const double *x,
                            const DCsr *M, const double *y) {
    st.dots.alloc(16);
    st.dots.zero(st.s);
    CsrView<double> v{0, 0, nullptr, nullptr, nullptr};
    if (M && !M->empty()) v = view<double>(*M);
    launch_coldot<double>(rows, nvec, ld, x, v, y, st.dots.p, st.s);
    std::vector<double> h(16);
    st.dots.download(h.data(), 16, st.s);
    SAMG_CUDA(cudaStreamSynchronize(st.s));
    h.resize(nvec);
    return h;
}

void scale_columns(SetupState &st, int rows, int ld, double *x, const std::vector<double> &f) {
    std::vector<double> g(ld, 1.0);
    for (size_t j = 0; j < f.size(); ++j) g[j] = f[j];
    st.sgn.upload(g.data(), ld, st.s);
    launch_scale_cols<double>(rows, ld, x, st.sgn.p, st.s);
}

// Rayleigh quotients (Eq. Rayleigh) of the pairs (u_j, v_j) on level l
std::vector<double> rayleigh(SetupState &st, int l, int nvec, int ld, const double *u,
                             const double *v) {
    samg_ctx &c = st.c;
    Level &L = c.L[l];
    if (c.spd()) {
        auto num = coldots(st, L.n, nvec, ld, u, &L.A, u);
        auto den = coldots(st, L.n, nvec, ld, u, &L.B, u);
        for (int j = 0; j < nvec; ++j) num[j] /= den[j];
        return num;
    }
    auto num = coldots(st, L.m, nvec, ld, u, &L.A, v);
    auto bu = coldots(st, L.m, nvec, ld, u, &L.B, u);
    auto cv = coldots(st, L.n, nvec, ld, v, &L.C, v);
    for (int j = 0; j < nvec; ++j) num[j] /= std::sqrt(bu[j] * cv[j]);
    return num;
}

// mu_b boot relaxations on level l with kappa = tau = 0, sigma updated by the
// Rayleigh quotient after each; minimal SVD flips v_j when it is negative.
void relax_boot_rq(SetupState &st, int l) {
    samg_ctx &c = st.c;
    Level &L = c.L[l];
    for (int it = 0; it < c.prm.mu_b; ++it) {
        L.wd.k.zero(st.s);
        if (!c.spd()) L.wd.t.zero(st.s);
        relax<double>(c, l);
        auto rq = rayleigh(st, l, c.nb, c.ld, L.wd.u.p, c.spd() ? L.wd.u.p : L.wd.v.p);
        if (c.minimal() && !c.spd()) {
            std::vector<double> f(c.nb, 1.0);
            bool any = false;
            for (int j = 0; j < c.nb; ++j)
                if (rq[j] < 0) { f[j] = -1.0; rq[j] = -rq[j]; any = true; }
            if (any) scale_columns(st, L.n, c.ld, L.wd.v.p, f);
        }
        std::vector<double> sg(c.ld, 1.0);
        for (int j = 0; j < c.nb; ++j) sg[j] = rq[j];
        c.sigma.upload(sg.data(), c.ld, st.s);
    }
}

// mu_t relaxations of the test vectors on level l
void relax_test(SetupState &st, int l, double *u, double *v) {
    samg_ctx &c = st.c;
    Level &L = c.L[l];
    const int ld = st.ldt, nt = st.nt;
    const double om = c.prm.omega_J;
    if (c.minimal()) {
        for (int it = 0; it < c.prm.mu_t; ++it) {
            if (c.spd()) {
                st.ones.zero(st.s);  // shift 0: rows of A
                launch_kaczmarz<double>(L.kA, ld, nullptr, u, st.ones.p, st.s);
            } else {
                launch_kaczmarz<double>(L.kA, ld, nullptr, v, nullptr, st.s);
                if (!st.induced) launch_kaczmarz<double>(L.kAt, ld, nullptr, u, nullptr, st.s);
            }
        }
        // unit B (C) norm after the block of relaxations
        if (c.spd()) {
            auto nn = coldots(st, L.n, nt, ld, u, &L.B, u);
            for (auto &x : nn) x = 1.0 / std::sqrt(x);
            scale_columns(st, L.n, ld, u, nn);
        } else {
            auto nv = coldots(st, L.n, nt, ld, v, &L.C, v);
            for (auto &x : nv) x = 1.0 / std::sqrt(x);
            scale_columns(st, L.n, ld, v, nv);
            if (!st.induced) {
                auto nu = coldots(st, L.m, nt, ld, u, &L.B, u);
                for (auto &x : nu) x = 1.0 / std::sqrt(x);
                scale_columns(st, L.m, ld, u, nu);
            }
        }
        return;
    }
    // dominant: power method with one weighted-Jacobi inner step (Sec. 3.4)
    std::vector<double> one(ld, 1.0);
    st.ones.upload(one.data(), ld, st.s);
    DBuf<double> tmp((size_t)std::max(L.m, L.n) * ld);
    auto bview = [](const DCsr &M) {
        return M.empty() ? CsrView<double>{0, 0, nullptr, nullptr, nullptr} : view<double>(M);
    };
    for (int it = 0; it < c.prm.mu_t; ++it) {
        if (c.spd()) {
            launch_jacobi<double>(L.n, ld, view<double>(L.A), u, bview(L.B), L.dBd.p, u, nullptr,
                                  st.ones.p, om, tmp.p, st.s);
            SAMG_CUDA(cudaMemcpyAsync(u, tmp.p, sizeof(double) * L.n * ld, cudaMemcpyDeviceToDevice, st.s));
            auto nn = coldots(st, L.n, nt, ld, u, &L.B, u);
            for (auto &x : nn) x = 1.0 / std::sqrt(x);
            scale_columns(st, L.n, ld, u, nn);
            continue;
        }
        launch_jacobi<double>(L.n, ld, view<double>(L.At), u, bview(L.C), L.dCd.p, v, nullptr,
                              st.ones.p, om, tmp.p, st.s);
        SAMG_CUDA(cudaMemcpyAsync(v, tmp.p, sizeof(double) * L.n * ld, cudaMemcpyDeviceToDevice, st.s));
        auto nv = coldots(st, L.n, nt, ld, v, &L.C, v);
        for (auto &x : nv) x = 1.0 / std::sqrt(x);
        scale_columns(st, L.n, ld, v, nv);
        launch_jacobi<double>(L.m, ld, view<double>(L.A), v, bview(L.B), L.dBd.p, u, nullptr,
                              st.ones.p, om, tmp.p, st.s);
        SAMG_CUDA(cudaMemcpyAsync(u, tmp.p, sizeof(double) * L.m * ld, cudaMemcpyDeviceToDevice, st.s));
        auto nu = coldots(st, L.m, nt, ld, u, &L.B, u);
        for (auto &x : nu) x = 1.0 / std::sqrt(x);
        scale_columns(st, L.m, ld, u, nu);
    }
}

void gather(SetupState &st, const std::vector<char> &cf, int ld, const double *x, double *out,
            const double *inv_colscale) {
    std::vector<int> id;
    for (int i = 0; i < (int)cf.size(); ++i)
        if (cf[i]) id.push_back(i);
    st.idx.upload(id.data(), id.size(), st.s);
    launch_gather_rows<double>((int)id.size(), ld, st.idx.p, x, inv_colscale, out, st.s);
    SAMG_CUDA(cudaStreamSynchronize(st.s));
}

// n_b extremal generalized singular triplets of the coarsest level from
// X W = Y W Lam (Thm genSVD): the l = min(m, n) largest eigenvalues are the
// s_j >= 0 with [u; v] = sqrt(2) w; SPD: the eigenpairs of (A, B).
void coarsest_boot(SetupState &st) {
    samg_ctx &c = st.c;
    prepare_coarsest(c);
    Level &Lc = c.L.back();
    const int M = c.co.M, nb = c.nb, ld = c.ld;
    std::vector<double> lam(M), W((size_t)M * M);
    c.co.lam.download(lam.data(), M, st.s);
    c.co.W.download(W.data(), (size_t)M * M, st.s);
    SAMG_CUDA(cudaStreamSynchronize(st.s));
    std::vector<int> desc(M);
    for (int i = 0; i < M; ++i) desc[i] = i;
    std::stable_sort(desc.begin(), desc.end(), [&](int a, int b) { return lam[a] > lam[b]; });
    std::vector<int> sel;
    if (c.spd()) {
        if (c.minimal()) for (int k = 0; k < nb; ++k) sel.push_back(desc[M - 1 - k]);
        else for (int k = 0; k < nb; ++k) sel.push_back(desc[k]);
    } else {
        const int l = std::min(Lc.m, Lc.n);
        if (c.minimal()) for (int k = 0; k < nb; ++k) sel.push_back(desc[l - 1 - k]);
        else for (int k = 0; k < nb; ++k) sel.push_back(desc[k]);
    }
    const double f = c.spd() ? 1.0 : std::sqrt(2.0);
    const int mu = c.spd() ? Lc.n : Lc.m;
    std::vector<double> hu((size_t)mu * ld, 0.0), hv(c.spd() ? 0 : (size_t)Lc.n * ld, 0.0);
    std::vector<double> sg(ld, 1.0);
    for (int j = 0; j < nb; ++j) {
        const int k = sel[j];
        sg[j] = lam[k];
        for (int i = 0; i < mu; ++i) hu[(size_t)i * ld + j] = f * W[(size_t)i * M + k];
        if (!c.spd())
            for (int i = 0; i < Lc.n; ++i) hv[(size_t)i * ld + j] = f * W[(size_t)(mu + i) * M + k];
    }
    c.sigma.upload(sg.data(), ld, st.s);
    Lc.wd.u.upload(hu.data(), hu.size(), st.s);
    if (!c.spd()) Lc.wd.v.upload(hv.data(), hv.size(), st.s);
    SAMG_CUDA(cudaStreamSynchronize(st.s));
}

// One downward sweep of a multiplicative cycle (Sec. 3.3): on each level
// coarsen, relax the test vectors (and, after the first cycle, copies of the
// finest boot triplets with Rayleigh-quotient updates of sigma), fit P and Q
// by weighted LS, form the Galerkin operators and inject the vectors.  The
// levels below the finest are rebuilt.  wscale (one factor per fitted
// vector, or null) multiplies the LS weights.
void down_sweep(SetupState &st, int cyc, const std::vector<double> *wscale, StageClock &clk) {
    samg_ctx &c = st.c;
    cudaStream_t s = c.stream;
    const samg_params &p = c.prm;
    const bool spd = c.spd();
    const int sq = st.sq;
    const int ldt = st.ldt;
    c.L.resize(1);
    int l = 0;
    double *ut = st.Ut.p, *vt = spd ? nullptr : st.Vt.p;
    st.ut.clear();
    st.vt.clear();
    if (cyc > 0) {
        Level &L0 = c.L[0];
        SAMG_CUDA(cudaMemcpyAsync(L0.wd.u.p, c.U.p, c.U.n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        if (!spd)
            SAMG_CUDA(cudaMemcpyAsync(L0.wd.v.p, c.V.p, c.V.n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    for (;;) {
        Level &L = c.L[l];
        if (std::max(L.m, L.n) <= p.coarsest_max || (int)c.L.size() >= p.max_levels) break;
        // coarsening depends on A_l only (cached on the finest level)
        HCsr Nu, Nv, Su, Sv;
        std::vector<char> cfu, cfv;
        if (l == 0 && st.have0) {
            Nu = st.N0u; Nv = st.N0v; Su = st.S0u; Sv = st.S0v; cfu = st.cf0u; cfv = st.cf0v;
        } else {
            DCsr Nd;
            if (sq) {
                // one C/F splitting and one strength graph (of A) for u and v;
                // R14's Jacobi step (minimal) still needs A A^t and A^t A
                HCsr hA;
                download_csr(L.A, hA, s);
                strength_of(hA, p.theta, Su);
                Sv = Su;
                if (c.minimal()) {
                    spgemm(L.A, L.At, Nd, s);
                    download_csr(Nd, Nu, s);
                    DCsr Nd2;
                    spgemm(L.At, L.A, Nd2, s);
                    download_csr(Nd2, Nv, s);
                }
            } else if (spd || (st.induced && l > 0)) {
                download_csr(L.A, Nv, s);
            } else if (st.induced) {
                spgemm(L.At, L.A, Nd, s);
                download_csr(Nd, Nv, s);
            } else if (c.minimal()) {
                // minimal SVD kind in the paper's form (Sec. 3.7): rows
                // coarsened on N_u = A A^t, columns on N_v = A^t A; both
                // products are formed, since R14's Jacobi step needs them
                spgemm(L.A, L.At, Nd, s);
                download_csr(Nd, Nu, s);
                DCsr Nd2;
                spgemm(L.At, L.A, Nd2, s);
                download_csr(Nd2, Nv, s);
                strength_of(Nu, p.theta, Su);
                strength_of(Nv, p.theta, Sv);
            } else {
                // dominant SVD kind: the strength graphs of A A^t and
                // A^t A come from A and A^t directly (the LS fits need
                // no N here, R14 being a minimal-kind step)
                HCsr hA, hAt;
                download_csr(L.A, hA, s);
                download_csr(L.At, hAt, s);
                strength_product(hA, hAt, p.theta, Su);
                strength_product(hAt, hA, p.theta, Sv);
            }
            if (spd || st.induced) strength_of(Nv, p.theta, Sv);
            cfv = rs_split(Sv);
            if (sq) cfu = cfv;
            else if (!spd && !st.induced) cfu = rs_split(Su);
            if (l == 0) {
                st.have0 = true;
                st.N0u = Nu; st.N0v = Nv; st.S0u = Su; st.S0v = Sv; st.cf0u = cfu; st.cf0v = cfv;
            }
        }
        clk.mark(0);
        int nc = 0, mc = 0;
        for (char x : cfv) nc += x;
        if (spd || st.induced) mc = nc;
        else for (char x : cfu) mc += x;
        const int64_t tot_f = spd ? L.n : (int64_t)L.m + L.n;
        const int64_t tot_c = spd ? nc : (int64_t)mc + nc;
        if (tot_c > 0.9 * tot_f || std::min(mc, nc) < 2 * c.nb) break;
        // relaxation of the test and boot vectors
        relax_test(st, l, ut, vt);
        clk.mark(1);
        if (st.induced) {
            if (l == 0)
                launch_combine<double, double>(L.m, ldt, nullptr, 0.0,
                                               Term<double>{view<double>(L.A), vt, 1.0, false},
                                               Term<double>{}, c.sigma.p, ut, s);
            else
                SAMG_CUDA(cudaMemcpyAsync(ut, vt, sizeof(double) * L.n * ldt, cudaMemcpyDeviceToDevice, s));
        }
        if (cyc > 0) relax_boot_rq(st, l);
        clk.mark(2);
        // LS fit on [test, boot]
        const int nf = p.n_t + (cyc > 0 ? c.nb : 0);
        std::vector<double> w(nf);
        {
            auto rq = rayleigh(st, l, p.n_t, ldt, ut, spd ? ut : vt);
            for (int k = 0; k < p.n_t; ++k) w[k] = rq[k];
            if (cyc > 0) {
                std::vector<double> sg(c.ld);
                c.sigma.download(sg.data(), c.ld, s);
                SAMG_CUDA(cudaStreamSynchronize(s));
                for (int j = 0; j < c.nb; ++j) w[p.n_t + j] = sg[j];
            }
            for (auto &x : w) {
                double a = std::max(std::fabs(x), 1e-300);
                x = c.minimal() ? 1.0 / a : a;
            }
            // the redo of Sec. 6.3 scales the weights of the test vectors and
            // of the converged boot vectors
            if (wscale)
                for (int k = 0; k < nf; ++k) w[k] *= (*wscale)[k];
        }
        auto fit_side = [&](const HCsr &N, const HCsr &S, const std::vector<char> &cf, int rows,
                            const double *test, const double *boot, HCsr &Pout) {
            std::vector<double> Y((size_t)rows * nf);
            fetch(s, test, rows, ldt, p.n_t, Y.data(), nf, 0);
            if (cyc > 0) fetch(s, boot, rows, c.ld, c.nb, Y.data(), nf, p.n_t);
            SAMG_CUDA(cudaStreamSynchronize(s));
            if (c.minimal()) {  // extra Jacobi step on the F values (R14 weight)
                std::vector<double> YF;
                jacobi_host(N, Y, nf, p.omega_J * 2.0 / gershgorin(N), YF);
                ls_interp(S, cf, YF, Y, w, nf, Pout);
            } else {
                ls_interp(S, cf, Y, Y, w, nf, Pout);
            }
        };
        HCsr hQ, hP;
        if (sq == 2) {
            // P = Q fitted to the u and the v vectors together (weights
            // repeated), so that B_c = C_c on every level
            std::vector<double> Y((size_t)L.n * 2 * nf), w2(2 * nf);
            fetch(s, ut, L.n, ldt, p.n_t, Y.data(), 2 * nf, 0);
            if (cyc > 0) fetch(s, L.wd.u.p, L.n, c.ld, c.nb, Y.data(), 2 * nf, p.n_t);
            fetch(s, vt, L.n, ldt, p.n_t, Y.data(), 2 * nf, nf);
            if (cyc > 0) fetch(s, L.wd.v.p, L.n, c.ld, c.nb, Y.data(), 2 * nf, nf + p.n_t);
            SAMG_CUDA(cudaStreamSynchronize(s));
            for (int k = 0; k < nf; ++k) w2[k] = w2[nf + k] = w[k];
            if (c.minimal()) {  // R14 on each side's F values with its own N
                std::vector<double> Yu((size_t)L.n * nf), Yv((size_t)L.n * nf), Fu, Fv;
                for (int i = 0; i < L.n; ++i)
                    for (int k = 0; k < nf; ++k) {
                        Yu[(size_t)i * nf + k] = Y[(size_t)i * 2 * nf + k];
                        Yv[(size_t)i * nf + k] = Y[(size_t)i * 2 * nf + nf + k];
                    }
                jacobi_host(Nu, Yu, nf, p.omega_J * 2.0 / gershgorin(Nu), Fu);
                jacobi_host(Nv, Yv, nf, p.omega_J * 2.0 / gershgorin(Nv), Fv);
                std::vector<double> YF(Y.size());
                for (int i = 0; i < L.n; ++i)
                    for (int k = 0; k < nf; ++k) {
                        YF[(size_t)i * 2 * nf + k] = Fu[(size_t)i * nf + k];
                        YF[(size_t)i * 2 * nf + nf + k] = Fv[(size_t)i * nf + k];
                    }
                ls_interp(Su, cfu, YF, Y, w2, 2 * nf, hP);
            } else {
                ls_interp(Su, cfu, Y, Y, w2, 2 * nf, hP);
            }
            upload_csr(hP, L.P, s);
            upload_csr(hP, L.Q, s);
        } else if (spd) {
            fit_side(Nv, Sv, cfv, L.n, ut, L.wd.u.p, hP);
            upload_csr(hP, L.P, s);
        } else if (st.induced) {
            fit_side(Nv, Sv, cfv, L.n, vt, L.wd.v.p, hQ);
            upload_csr(hQ, L.Q, s);
            if (l == 0) {
                spgemm(L.A, L.Q, L.P, s);
            } else {
                upload_csr(hQ, L.P, s);
            }
        } else {
            fit_side(Nu, Su, cfu, L.m, ut, L.wd.u.p, hP);
            fit_side(Nv, Sv, cfv, L.n, vt, L.wd.v.p, hQ);
            upload_csr(hP, L.P, s);
            upload_csr(hQ, L.Q, s);
        }
        clk.mark(3);
        // Galerkin operators of level l+1
        c.L.emplace_back();
        {
            Level &Lf = c.L[l];
            Level &Lc = c.L[l + 1];
            transpose(Lf.P, Lf.Pt, s);
            DCsr t1, t2, t3;
            if (spd) {
                spgemm(Lf.A, Lf.P, t1, s);
                spgemm(Lf.Pt, t1, Lc.A, s);
                if (Lf.B.empty()) spgemm(Lf.Pt, Lf.P, Lc.B, s);
                else { spgemm(Lf.B, Lf.P, t2, s); spgemm(Lf.Pt, t2, Lc.B, s); }
            } else {
                transpose(Lf.Q, Lf.Qt, s);
                spgemm(Lf.A, Lf.Q, t1, s);
                spgemm(Lf.Pt, t1, Lc.A, s);
                if (Lf.B.empty()) spgemm(Lf.Pt, Lf.P, Lc.B, s);
                else { spgemm(Lf.B, Lf.P, t2, s); spgemm(Lf.Pt, t2, Lc.B, s); }
                if (Lf.C.empty()) spgemm(Lf.Qt, Lf.Q, Lc.C, s);
                else { spgemm(Lf.C, Lf.Q, t3, s); spgemm(Lf.Qt, t3, Lc.C, s); }
            }
            Lc.m = Lc.A.m;
            Lc.n = Lc.A.n;
        }
        clk.mark(4);
        prepare_level(c, l + 1);
        clk.mark(5);
        // injection of test and boot vectors to level l+1
        Level &Lf = c.L[l];
        Level &Lc = c.L[l + 1];
        st.ut.emplace_back((size_t)(spd ? Lc.n : Lc.m) * ldt);
        double *utc = st.ut.back().p;
        double *vtc = nullptr;
        if (spd) {
            gather(st, cfv, ldt, ut, utc, nullptr);
            if (cyc > 0) gather(st, cfv, c.ld, Lf.wd.u.p, Lc.wd.u.p, nullptr);
        } else {
            st.vt.emplace_back((size_t)Lc.n * ldt);
            vtc = st.vt.back().p;
            gather(st, cfv, ldt, vt, vtc, nullptr);
            if (st.induced) {
                // row test vectors are recomputed from vtc on the next level
                if (cyc > 0) {
                    if (l == 0) gather(st, cfv, c.ld, Lf.wd.v.p, Lc.wd.u.p, c.sigma.p);
                    else gather(st, cfv, c.ld, Lf.wd.u.p, Lc.wd.u.p, nullptr);
                    gather(st, cfv, c.ld, Lf.wd.v.p, Lc.wd.v.p, nullptr);
                }
            } else {
                gather(st, cfu, ldt, ut, utc, nullptr);
                if (cyc > 0) {
                    gather(st, cfu, c.ld, Lf.wd.u.p, Lc.wd.u.p, nullptr);
                    gather(st, cfv, c.ld, Lf.wd.v.p, Lc.wd.v.p, nullptr);
                }
            }
        }
        ut = utc;
        vt = vtc;
        ++l;
    }
}

}  // namespace

void host_setup(samg_ctx &c, const samg_csr &Ah) {
    cudaStream_t s = c.stream;
    const samg_params &p = c.prm;
    const bool spd = c.spd();
    SAMG_CHECK(spd || !c.minimal() || Ah.m >= Ah.n, SAMG_E_INVALID,
               "minimal SVD kind needs m >= n (pass A^t for wide matrices)");
    StageClock clk(c);
    c.L.clear();
    c.L.reserve(p.max_levels + 2);
    c.L.emplace_back();
    upload_csr(Ah, c.L[0].A, s);
    c.L[0].m = Ah.m;
    c.L[0].n = Ah.n;
    alloc_finest_state(c);
    clk.mark(9);
    prepare_level(c, 0);
    clk.mark(5);
    auto keep = std::make_shared<SetupState>(c);
    SetupState &st = *keep;
    st.nt = p.n_t;
    st.ldt = block_ld(p.n_t);
    // square SVD kind, Sec. 5.1 (R23): splitting and patterns from A itself
    // (1), or one operator P = Q for both sides (2)
    const int sq = (!spd && Ah.m == Ah.n) ? p.square_form : 0;
    st.sq = sq;
    st.induced = !spd && c.minimal() && p.row_form == 0 && sq == 0;
    const int m = Ah.m, n = Ah.n, ldt = st.ldt;
    st.ones.alloc(16);
    // random test vectors (Sec. 3.3)
    const int mu0 = spd ? n : m;
    st.Ut.alloc((size_t)mu0 * ldt);
    SAMG_COUNT_LAUNCH();
    k_random_block<<<(unsigned)(((int64_t)mu0 * ldt + 255) / 256), 256, 0, s>>>(p.seed, mu0, p.n_t, ldt, st.Ut.p);
    if (!spd) {
        st.Vt.alloc((size_t)n * ldt);
        SAMG_COUNT_LAUNCH();
        k_random_block<<<(unsigned)(((int64_t)n * ldt + 255) / 256), 256, 0, s>>>(
            p.seed ^ (1ull << 63), n, p.n_t, ldt, st.Vt.p);
        if (st.induced)
            launch_combine<double, double>(m, ldt, nullptr, 0.0,
                                           Term<double>{view<double>(c.L[0].A), st.Vt.p, 1.0, false},
                                           Term<double>{}, c.sigma.p, st.Ut.p, s);
    }
    SAMG_CUDA(cudaGetLastError());
    // the fine-level test vectors need schedules of width ldt (same schedules)
    clk.mark(9);
    for (int cyc = 0; cyc < p.n_mult; ++cyc) {
        down_sweep(st, cyc, nullptr, clk);
        SAMG_CHECK(c.L.size() >= 2, SAMG_E_INVALID,
                   "setup produced a single level (problem already at the coarsest size)");
        // coarsest: new boot triplets by a direct solve
        clk.mark(9);
        coarsest_boot(st);
        clk.mark(6);
        // upward: interpolate (Eq. ranges) and relax with Rayleigh-quotient updates
        for (int k = (int)c.L.size() - 2; k >= 0; --k) {
            Level &L = c.L[k];
            Level &Lc = c.L[k + 1];
            launch_combine<double, double>(spd ? L.n : L.m, c.ld, nullptr, 0.0,
                                           Term<double>{view<double>(L.P), Lc.wd.u.p, 1.0, false},
                                           Term<double>{}, c.sigma.p, L.wd.u.p, s);
            if (!spd)
                launch_combine<double, double>(L.n, c.ld, nullptr, 0.0,
                                               Term<double>{view<double>(L.Q), Lc.wd.v.p, 1.0, false},
                                               Term<double>{}, c.sigma.p, L.wd.v.p, s);
            relax_boot_rq(st, k);
        }
        clk.mark(2);
        // Ritz step on the finest level
        Level &L0 = c.L[0];
        SAMG_CUDA(cudaMemcpyAsync(c.U.p, L0.wd.u.p, c.U.n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        if (!spd)
            SAMG_CUDA(cudaMemcpyAsync(c.V.p, L0.wd.v.p, c.V.n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        ritz(c, false);
        clk.mark(7);
    }
    // hierarchy of the last cycle: the cycle's per-level data are in place
    finalize_hierarchy(c);
    clk.mark(8);
    share_error_word(c);
    for (auto &L : c.L) {
        L.wd.u.zero(s);
        if (!spd) L.wd.v.zero(s);
    }
    ritz(c, true);
    clk.mark(7);
    SAMG_CUDA(cudaStreamSynchronize(s));
    st.ut.clear();
    st.vt.clear();
    if (p.redo_tol > 0.0) c.setup_keep = keep;
}

void redo_interpolation(samg_ctx &c, const std::vector<char> &conv) {
    SAMG_CHECK(c.setup_keep != nullptr, SAMG_E_INVALID,
               "redo needs the setup phase's state: set redo_tol > 0 before samg_setup "
               "(an imported hierarchy has none)");
    SetupState &st = *static_cast<SetupState *>(c.setup_keep.get());
    cudaStream_t s = c.stream;
    const int nt = c.prm.n_t;
    std::vector<double> ws(nt + c.nb, 1.0);
    for (int k = 0; k < nt; ++k) ws[k] = 1e-3;
    for (int j = 0; j < c.nb; ++j)
        if (conv[j]) ws[nt + j] = 1e-3;
    // the sweep relaxes copies of the boot triplets and updates sigma: the
    // additive iterate's sigma is restored afterwards
    std::vector<double> sg(c.ld);
    c.sigma.download(sg.data(), c.ld, s);
    SAMG_CUDA(cudaStreamSynchronize(s));
    StageClock clk(c, false);
    down_sweep(st, 1, &ws, clk);
    SAMG_CHECK(c.L.size() >= 2, SAMG_E_INVALID, "redo produced a single level");
    c.sigma.upload(sg.data(), c.ld, s);
    finalize_hierarchy(c);
    share_error_word(c);
    for (auto &L : c.L) {
        L.wd.u.zero(s);
        if (!c.spd()) L.wd.v.zero(s);
    }
    st.ut.clear();
    st.vt.clear();
    SAMG_CUDA(cudaStreamSynchronize(s));
}

void host_coarsen(const HCsr &N, double theta, std::vector<char> &cf) {
    HCsr S;
    strength_of(N, theta, S);
    cf = rs_split(S);
}

void host_strength_product(const HCsr &A, double theta, HCsr &S) {
    HCsr At;
    At.m = A.n;
    At.n = A.m;
    At.rp.assign(A.n + 1, 0);
    for (int64_t e = 0; e < A.nnz(); ++e) At.rp[A.ci[e] + 1]++;
    for (int j = 0; j < A.n; ++j) At.rp[j + 1] += At.rp[j];
    At.ci.resize(A.nnz());
    At.v.resize(A.nnz());
    std::vector<int64_t> f(At.rp.begin(), At.rp.end() - 1);
    for (int i = 0; i < A.m; ++i)
        for (int64_t e = A.rp[i]; e < A.rp[i + 1]; ++e) {
            At.ci[f[A.ci[e]]] = i;
            At.v[f[A.ci[e]]++] = A.v[e];
        }
    strength_product(A, At, theta, S);
}

void host_ls_interp(const HCsr &N, double theta, const std::vector<char> &cf,
                    const std::vector<double> &yF, const std::vector<double> &yC,
                    const std::vector<double> &w, int nf, HCsr &P) {
    HCsr S;
    strength_of(N, theta, S);
    ls_interp(S, cf, yF, yC, w, nf, P);
}

}  // namespace samg
