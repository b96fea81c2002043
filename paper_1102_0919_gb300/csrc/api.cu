// api.cu -- the C ABI (include/samg.h): context creation from a hierarchy or
// by the setup phase, the solve loop, and single-step entry points.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <dlfcn.h>
#include <mutex>
#include <string>

#include "ctx.cuh"
#include "hierfile.cuh"

using namespace samg;

namespace {

samg_status fail(samg_ctx *c, samg_status st, const std::string &msg) {
    if (c) {
        c->err = msg;
        if (st == SAMG_E_CUDA || st == SAMG_E_TIMEOUT) c->poisoned = true;
    }
    return st;
}

template <typename F>
samg_status guarded(samg_ctx *c, F &&f) {
    if (c && c->poisoned) return fail(c, SAMG_E_INVALID, "context is poisoned by an earlier error");
    try {
        f();
        return SAMG_OK;
    } catch (const Error &e) {
        return fail(c, e.status, e.what());
    } catch (const std::bad_alloc &) {
        return fail(c, SAMG_E_NOMEM, "host allocation failed");
    } catch (const std::exception &e) {
        return fail(c, SAMG_E_INVALID, e.what());
    }
}

thread_local std::string g_create_error;

void check_device() {
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    SAMG_CHECK(e == cudaSuccess && n > 0, SAMG_E_CUDA, "no CUDA device available");
    int dev = 0;
    SAMG_CUDA(cudaGetDevice(&dev));
    cudaDeviceProp p;
    SAMG_CUDA(cudaGetDeviceProperties(&p, dev));
    SAMG_CHECK(p.major == 10 && p.minor == 3, SAMG_E_CUDA,
               "this library is built for sm_103a (GB300) only");
}

void check_common(int n_b, const samg_params *prm) {
    SAMG_CHECK(n_b >= 1 && n_b <= 16, SAMG_E_INVALID, "n_b must be in [1, 16]");
    SAMG_CHECK(prm != nullptr, SAMG_E_INVALID, "params is NULL");
    SAMG_CHECK(prm->mu_b >= 0 && prm->mu_t >= 0, SAMG_E_INVALID, "negative relaxation count");
    SAMG_CHECK(prm->prec == SAMG_FP64 || prm->prec == SAMG_FP32 || prm->prec == SAMG_BF16_STORE,
               SAMG_E_INVALID, "bad precision");
    SAMG_CHECK(prm->coarse_pinv == 0 || prm->coarse_pinv == 1, SAMG_E_INVALID,
               "coarse_pinv must be 0 (SVD pseudo-inverse) or 1 (generalized-eigen variant)");
    SAMG_CHECK(prm->row_form == 0 || prm->row_form == 1, SAMG_E_INVALID,
               "row_form must be 0 (rows from A) or 1 (the paper's A A^t coarsening)");
    SAMG_CHECK(prm->relax_order == 0 || prm->relax_order == 1, SAMG_E_INVALID,
               "relax_order must be 0 (natural, the paper's) or 1 (coloured variant)");
    SAMG_CHECK(prm->square_form >= 0 && prm->square_form <= 2, SAMG_E_INVALID,
               "square_form must be 0, 1 (splitting from A) or 2 (shared P = Q)");
    SAMG_CHECK(prm->redo_tol >= 0.0 && std::isfinite(prm->redo_tol), SAMG_E_INVALID,
               "redo_tol must be finite and >= 0");
}

template <typename T>
void put_level(samg_ctx &c, const double *h, int rows, DBuf<T> &d);
template <>
void put_level<double>(samg_ctx &c, const double *h, int rows, DBuf<double> &d) {
    if (h) put_block(c, h, rows, d);
    else d.zero(c.stream);
}
template <typename S>
void put_level_conv(samg_ctx &c, const double *h, int rows, DBuf<S> &d) {
    if (!h) { d.zero(c.stream); return; }
    DBuf<double> tmp((size_t)std::max(rows, 1) * c.ld);
    tmp.zero(c.stream);
    put_block(c, h, rows, tmp);
    launch_convert<double, S>((size_t)rows * c.ld, tmp.p, d.p, c.stream);
    SAMG_CUDA(cudaStreamSynchronize(c.stream));
}
template <>
void put_level<float>(samg_ctx &c, const double *h, int rows, DBuf<float> &d) {
    put_level_conv<float>(c, h, rows, d);
}
template <>
void put_level<bf16>(samg_ctx &c, const double *h, int rows, DBuf<bf16> &d) {
    put_level_conv<bf16>(c, h, rows, d);
}
template <typename T>
void get_level(samg_ctx &c, const DBuf<T> &d, int rows, double *h);
template <>
void get_level<double>(samg_ctx &c, const DBuf<double> &d, int rows, double *h) {
    if (!h) return;
    get_block(c, d, rows, h);
    SAMG_CUDA(cudaStreamSynchronize(c.stream));
}
template <typename S>
void get_level_conv(samg_ctx &c, const DBuf<S> &d, int rows, double *h) {
    if (!h) return;
    DBuf<double> tmp((size_t)std::max(rows, 1) * c.ld);
    launch_convert<S, double>((size_t)rows * c.ld, d.p, tmp.p, c.stream);
    get_block(c, tmp, rows, h);
    SAMG_CUDA(cudaStreamSynchronize(c.stream));
}
template <>
void get_level<float>(samg_ctx &c, const DBuf<float> &d, int rows, double *h) {
    get_level_conv<float>(c, d, rows, h);
}
template <>
void get_level<bf16>(samg_ctx &c, const DBuf<bf16> &d, int rows, double *h) {
    get_level_conv<bf16>(c, d, rows, h);
}

void set_sigma(samg_ctx &c, const double *sigma) {
    SAMG_CHECK(sigma != nullptr, SAMG_E_INVALID, "sigma is NULL");
    std::vector<double> sg(c.ld, 1.0);
    for (int j = 0; j < c.nb; ++j) sg[j] = sigma[j];
    c.sigma.upload(sg.data(), c.ld, c.stream);
}

int urows(const samg_ctx &c, int l) { return c.spd() ? c.L[l].n : c.L[l].m; }

void check_level(const samg_ctx &c, int l, bool need_coarser) {
    SAMG_CHECK(l >= 0 && l < c.nlev(), SAMG_E_INVALID, "level out of range");
    SAMG_CHECK(!need_coarser || l + 1 < c.nlev(), SAMG_E_INVALID, "level has no coarser level");
}

// Calls f with a value of the context's vector storage type (float64,
// float32 or bfloat16), after making sure every level has its work vectors
// in that type.
template <typename F>
void by_prec(samg_ctx &c, F f) {
    switch (c.prm.prec) {
        case SAMG_FP32: ensure_work<float>(c); f(float{}); break;
        case SAMG_BF16_STORE: ensure_work<bf16>(c); f(bf16{}); break;
        default: ensure_work<double>(c); f(double{}); break;
    }
}

template <typename T>
void step_relax(samg_ctx &c, int l, int count, double *U, double *V, const double *K,
                const double *Tt) {
    Level &L = c.L[l];
    Work<T> &w = work<T>(L);
    put_level<T>(c, U, urows(c, l), w.u);
    put_level<T>(c, K, urows(c, l), w.k);
    if (!c.spd()) {
        put_level<T>(c, V, L.n, w.v);
        put_level<T>(c, Tt, L.n, w.t);
    }
    relax_phase<T>(c, l, count);
    get_level<T>(c, w.u, urows(c, l), U);
    if (!c.spd()) get_level<T>(c, w.v, L.n, V);
}

template <typename T>
void step_restrict(samg_ctx &c, int l, const double *U, const double *V, const double *K,
                   const double *Tt, double *Kc, double *Tc) {
    Level &L = c.L[l];
    Work<T> &w = work<T>(L);
    put_level<T>(c, U, urows(c, l), w.u);
    put_level<T>(c, K, urows(c, l), w.k);
    if (!c.spd()) {
        put_level<T>(c, V, L.n, w.v);
        put_level<T>(c, Tt, L.n, w.t);
    }
    residual_restrict<T>(c, l);
    Work<T> &wc = work<T>(c.L[l + 1]);
    get_level<T>(c, wc.k, urows(c, l + 1), Kc);
    if (!c.spd()) get_level<T>(c, wc.t, c.L[l + 1].n, Tc);
}

template <typename T>
void step_interp(samg_ctx &c, int l, double *U, double *V, const double *Uc, const double *Vc) {
    Level &L = c.L[l];
    Work<T> &w = work<T>(L);
    Work<T> &wc = work<T>(c.L[l + 1]);
    put_level<T>(c, U, urows(c, l), w.u);
    put_level<T>(c, Uc, urows(c, l + 1), wc.u);
    if (!c.spd()) {
        put_level<T>(c, V, L.n, w.v);
        put_level<T>(c, Vc, c.L[l + 1].n, wc.v);
    }
    interpolate<T>(c, l);
    get_level<T>(c, w.u, urows(c, l), U);
    if (!c.spd()) get_level<T>(c, w.v, L.n, V);
}

template <typename T>
void step_coarse(samg_ctx &c, const double *K, const double *Tt, double *U, double *V) {
    int l = c.nlev() - 1;
    Work<T> &w = work<T>(c.L[l]);
    put_level<T>(c, K, urows(c, l), w.k);
    if (!c.spd()) put_level<T>(c, Tt, c.L[l].n, w.t);
    coarse_solve<T>(c);
    get_level<T>(c, w.u, urows(c, l), U);
    if (!c.spd()) get_level<T>(c, w.v, c.L[l].n, V);
}

void set_triplets_impl(samg_ctx &c, const double *sigma, const double *U, const double *V) {
    SAMG_CHECK(U != nullptr && (c.spd() || V != nullptr), SAMG_E_INVALID, "U or V is NULL");
    set_sigma(c, sigma);
    c.U.zero(c.stream);
    put_block(c, U, urows(c, 0), c.U);
    if (!c.spd()) {
        c.V.zero(c.stream);
        put_block(c, V, c.L[0].n, c.V);
    }
    ritz(c, true);
    SAMG_CUDA(cudaStreamSynchronize(c.stream));
}

}  // namespace

namespace samg {
// All Kaczmarz schedules of a context report timeouts in rstat[1].
void share_error_word(samg_ctx &c) {
    for (auto &L : c.L) {
        L.kA.err = c.rstat.p + 1;
        L.kAt.err = c.rstat.p + 1;
    }
}
}  // namespace samg

namespace {

void check_kaczmarz(samg_ctx &c) {
    int e = 0;
    SAMG_CUDA(cudaMemcpyAsync(&e, c.rstat.p + 1, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
    SAMG_CUDA(cudaStreamSynchronize(c.stream));
    SAMG_CHECK(e == 0, SAMG_E_TIMEOUT, "Kaczmarz sweep: a cross-band wait timed out");
}

}  // namespace

namespace samg {
std::atomic<uint64_t> &launch_counter() {
    static std::atomic<uint64_t> n{0};
    return n;
}
}  // namespace samg

extern "C" {

uint64_t samg_launch_count(void) { return samg::launch_counter().load(); }

void samg_default_params(samg_params *p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->n_t = 8;
    p->theta = 0.06;
    p->mu_t = 8;
    p->mu_b = 4;
    p->mu_tJ = 1;
    p->mu_bJ = 1;
    p->omega_J = 0.7;
    p->n_mult = 10;
    p->coarsest_max = 100;
    p->max_levels = 30;
    p->seed = 20110204ull;
    p->prec = SAMG_FP32;
    p->n_conv = 0;
    p->coarse_pinv = 0;
    p->row_form = 0;
    p->relax_order = 0;
    p->square_form = 0;
    p->redo_tol = 0.0;
}

const char *samg_last_error(const samg_ctx *ctx) {
    return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

void samg_destroy(samg_ctx *ctx) {
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    delete ctx;
}

samg_status samg_import(const samg_csr *A, int n_levels, const samg_csr *P, const samg_csr *Q,
                        int n_b, samg_target target, samg_kind kind, const samg_params *params,
                        const double *sigma, const double *U, const double *V, void *cuda_stream,
                        samg_ctx **out) {
    if (!out) return SAMG_E_INVALID;
    *out = nullptr;
    samg_ctx *c = new (std::nothrow) samg_ctx();
    if (!c) return SAMG_E_NOMEM;
    samg_status st = guarded(c, [&] {
        // argument checks first: they need no device
        check_common(n_b, params);
        SAMG_CHECK(!params || params->redo_tol == 0.0, SAMG_E_INVALID,
                   "redo_tol needs the setup phase's test vectors, which an imported "
                   "hierarchy does not have");
        SAMG_CHECK(A != nullptr && n_levels >= 2 && P != nullptr, SAMG_E_INVALID,
                   "import needs A, P and at least two levels");
        SAMG_CHECK(kind == SAMG_SPD_EIG || Q != nullptr, SAMG_E_INVALID, "import: Q is NULL");
        SAMG_CHECK(kind == SAMG_SVD || kind == SAMG_SPD_EIG, SAMG_E_INVALID, "bad kind");
        SAMG_CHECK(target == SAMG_DOMINANT || target == SAMG_MINIMAL, SAMG_E_INVALID, "bad target");
        validate_csr(*A);
        SAMG_CHECK(kind != SAMG_SPD_EIG || A->m == A->n, SAMG_E_INVALID, "SPD_EIG needs square A");
        SAMG_CHECK(n_b <= std::min(A->m, A->n), SAMG_E_INVALID, "n_b > min(m, n)");
        for (int l = 0; l + 1 < n_levels; ++l) {
            validate_csr(P[l]);
            const int rows_u = l == 0 ? (kind == SAMG_SPD_EIG ? A->n : A->m) : P[l - 1].n;
            SAMG_CHECK(P[l].m == rows_u, SAMG_E_INVALID, "P_l has the wrong number of rows");
            if (kind != SAMG_SPD_EIG) {
                validate_csr(Q[l]);
                const int rows_v = l == 0 ? A->n : Q[l - 1].n;
                SAMG_CHECK(Q[l].m == rows_v, SAMG_E_INVALID, "Q_l has the wrong number of rows");
            }
        }
        check_device();
        c->stream = (cudaStream_t)cuda_stream;
        c->kind = kind;
        c->target = target;
        c->prm = *params;
        c->nb = n_b;
        c->ld = block_ld(n_b);
        c->L.resize(n_levels);
        upload_csr(*A, c->L[0].A, c->stream);
        for (int l = 0; l + 1 < n_levels; ++l) {
            upload_csr(P[l], c->L[l].P, c->stream);
            if (kind != SAMG_SPD_EIG) upload_csr(Q[l], c->L[l].Q, c->stream);
        }
        build_galerkin(*c);
        finalize_hierarchy(*c);
        alloc_finest_state(*c);
        share_error_word(*c);
        set_triplets_impl(*c, sigma, U, V);
    });
    if (st != SAMG_OK) {
        g_create_error = c->err;
        delete c;
        return st;
    }
    *out = c;
    return SAMG_OK;
}

samg_status samg_setup(const samg_csr *A, int n_b, samg_target target, samg_kind kind,
                       const samg_params *params, void *cuda_stream, samg_ctx **out) {
    if (!out) return SAMG_E_INVALID;
    *out = nullptr;
    samg_ctx *c = new (std::nothrow) samg_ctx();
    if (!c) return SAMG_E_NOMEM;
    samg_status st = guarded(c, [&] {
        // argument checks first: they need no device
        check_common(n_b, params);
        SAMG_CHECK(A != nullptr, SAMG_E_INVALID, "A is NULL");
        SAMG_CHECK(kind == SAMG_SVD || kind == SAMG_SPD_EIG, SAMG_E_INVALID, "bad kind");
        SAMG_CHECK(target == SAMG_DOMINANT || target == SAMG_MINIMAL, SAMG_E_INVALID, "bad target");
        validate_csr(*A);
        SAMG_CHECK(kind != SAMG_SPD_EIG || A->m == A->n, SAMG_E_INVALID, "SPD_EIG needs square A");
        SAMG_CHECK(n_b <= std::min(A->m, A->n), SAMG_E_INVALID, "n_b > min(m, n)");
        SAMG_CHECK(params->n_t + n_b >= 2, SAMG_E_NT_TOO_SMALL, "n_t + n_b < 2");
        SAMG_CHECK(params->n_t >= 1 && params->n_t <= 16, SAMG_E_INVALID, "n_t must be in [1, 16]");
        check_device();
        c->stream = (cudaStream_t)cuda_stream;
        c->kind = kind;
        c->target = target;
        c->prm = *params;
        c->nb = n_b;
        c->ld = block_ld(n_b);
        host_setup(*c, *A);
    });
    if (st != SAMG_OK) {
        g_create_error = c->err;
        delete c;
        return st;
    }
    *out = c;
    return SAMG_OK;
}

struct samg_batch {
    std::vector<samg_ctx *> ctx;
    std::vector<cudaStream_t> streams;  // one per problem, owned by the batch
    cudaStream_t caller = nullptr;      // the stream given at setup
    std::string err;
};

void samg_batch_destroy(samg_batch *b) {
    if (!b) return;
    for (samg_ctx *c : b->ctx) samg_destroy(c);
    for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
    delete b;
}

samg_status samg_setup_batched(const samg_csr *const *A, int count, int n_b, samg_target target,
                               samg_kind kind, const samg_params *params, void *cuda_stream,
                               samg_batch **out) {
    if (!out) return SAMG_E_INVALID;
    *out = nullptr;
    try {
        // every problem's arguments are checked before any device call
        SAMG_CHECK(A != nullptr && count >= 1, SAMG_E_INVALID, "setup_batched: no problems");
        check_common(n_b, params);
        SAMG_CHECK(kind == SAMG_SVD || kind == SAMG_SPD_EIG, SAMG_E_INVALID, "bad kind");
        SAMG_CHECK(target == SAMG_DOMINANT || target == SAMG_MINIMAL, SAMG_E_INVALID, "bad target");
        for (int p = 0; p < count; ++p) {
            const std::string who = "setup_batched: problem " + std::to_string(p) + ": ";
            SAMG_CHECK(A[p] != nullptr, SAMG_E_INVALID, who + "A is NULL");
            try {
                validate_csr(*A[p]);
            } catch (const Error &e) {
                throw Error(e.status, who + e.what());
            }
            SAMG_CHECK(kind != SAMG_SPD_EIG || A[p]->m == A[p]->n, SAMG_E_INVALID,
                       who + "SPD_EIG needs square A");
            SAMG_CHECK(n_b <= std::min(A[p]->m, A[p]->n), SAMG_E_INVALID, who + "n_b > min(m, n)");
        }
    } catch (const Error &e) {
        g_create_error = e.what();
        return e.status;
    } catch (const std::bad_alloc &) {
        g_create_error = "setup_batched: host allocation failed";
        return SAMG_E_NOMEM;
    }
    samg_batch *b = new (std::nothrow) samg_batch();
    if (!b) return SAMG_E_NOMEM;
    try {
        b->ctx.reserve(count);  // push_back below cannot throw after this
        b->streams.reserve(count);
        for (int p = 0; p < count; ++p) {
            samg_ctx *c = nullptr;
            const samg_status st = samg_setup(A[p], n_b, target, kind, params, cuda_stream, &c);
            if (st != SAMG_OK) {
                const std::string msg = "setup_batched: problem " + std::to_string(p) + ": " + g_create_error;
                samg_batch_destroy(b);
                g_create_error = msg;
                return st;
            }
            b->ctx.push_back(c);
            // the problem's solve runs on a stream of its own, so that the
            // batch's problems overlap on the device
            cudaStream_t ps = nullptr;
            cudaError_t e = cudaStreamSynchronize(c->stream);
            if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ps, cudaStreamNonBlocking);
            if (e != cudaSuccess) {
                samg_batch_destroy(b);
                g_create_error = std::string("setup_batched: stream: ") + cudaGetErrorString(e);
                return SAMG_E_CUDA;
            }
            b->streams.push_back(ps);
            c->stream = ps;
        }
        b->caller = (cudaStream_t)cuda_stream;
    } catch (const std::bad_alloc &) {
        samg_batch_destroy(b);
        g_create_error = "setup_batched: host allocation failed";
        return SAMG_E_NOMEM;
    }
    *out = b;
    return SAMG_OK;
}

samg_status samg_solve_batched(samg_batch *b, double tol, int max_outer, int *outer_done) {
    if (!b) return SAMG_E_INVALID;
    b->err.clear();
    const int np = (int)b->ctx.size();
    bool redo = false;
    for (samg_ctx *c : b->ctx) redo = redo || c->prm.redo_tol > 0.0;
    if (redo || max_outer < 0 || !(tol > 0.0)) {
        // one problem after another (the redo of Sec. 6.3 rebuilds a
        // problem's hierarchy between its iterations)
        samg_status worst = SAMG_OK;
        for (int p = 0; p < np; ++p) {
            int done = 0;
            const samg_status st = samg_solve(b->ctx[p], tol, max_outer, &done);
            if (outer_done) outer_done[p] = done;
            if (st == SAMG_E_NOT_CONVERGED) {
                worst = SAMG_E_NOT_CONVERGED;
                b->err = "problem " + std::to_string(p) + " reached max_outer before the tolerance";
                continue;
            }
            if (st != SAMG_OK) {
                b->err = "problem " + std::to_string(p) + ": " + samg_last_error(b->ctx[p]);
                return st;
            }
        }
        return worst;
    }
    // Every problem advances one outer iteration per round on its own
    // stream; the host then reads all the rounds' residuals and Ritz
    // statuses (pinned copies) and drops the problems that converged.
    const int ld = b->ctx[0]->ld;
    const size_t per = (size_t)ld * sizeof(double) + 2 * sizeof(int);
    unsigned char *host = nullptr;
    if (cudaMallocHost(&host, per * np) != cudaSuccess) {
        b->err = "solve_batched: pinned host memory";
        return SAMG_E_NOMEM;
    }
    std::vector<int> done(np, 0);
    std::vector<char> state(np, 0);  // 0 running, 1 converged, 2 out of iterations, 3 failed
    samg_status fail = SAMG_OK;
    int failed_p = -1;
    cudaEvent_t ev = nullptr;
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ev, b->caller);
    for (int p = 0; p < np && e == cudaSuccess; ++p) e = cudaStreamWaitEvent(b->ctx[p]->stream, ev, 0);
    if (e != cudaSuccess) {
        fail = SAMG_E_CUDA;
        b->err = std::string("solve_batched: ") + cudaGetErrorString(e);
    }
    auto run = [&](int p, auto &&f) {
        const samg_status st = guarded(b->ctx[p], f);
        if (st != SAMG_OK && fail == SAMG_OK) {
            state[p] = 3;
            fail = st;
            failed_p = p;
        }
    };
    while (fail == SAMG_OK) {
        for (int p = 0; p < np; ++p)
            if (!state[p])
                run(p, [&] {
                    samg_ctx &c = *b->ctx[p];
                    unsigned char *h = host + per * p;
                    SAMG_CUDA(cudaMemcpyAsync(h, c.resid.p, (size_t)ld * sizeof(double),
                                              cudaMemcpyDeviceToHost, c.stream));
                    SAMG_CUDA(cudaMemcpyAsync(h + (size_t)ld * sizeof(double), c.rstat.p,
                                              2 * sizeof(int), cudaMemcpyDeviceToHost, c.stream));
                });
        bool any = false;
        for (int p = 0; p < np && fail == SAMG_OK; ++p) {
            if (state[p]) continue;
            run(p, [&] {
                samg_ctx &c = *b->ctx[p];
                SAMG_CUDA(cudaStreamSynchronize(c.stream));
                const unsigned char *h = host + per * p;
                const double *rs = reinterpret_cast<const double *>(h);
                int st2[2];
                std::memcpy(st2, h + (size_t)ld * sizeof(double), sizeof(st2));
                SAMG_CHECK(st2[1] == 0, SAMG_E_TIMEOUT, "Kaczmarz sweep: a cross-band wait timed out");
                SAMG_CHECK(done[p] == 0 || st2[0] != 1, SAMG_E_INVALID,
                           "ritz: boot vectors are linearly dependent");
                const int nconv = c.prm.n_conv > 0 && c.prm.n_conv < c.nb ? c.prm.n_conv : c.nb;
                double mx = 0.0;
                bool finite = true;
                for (int j = 0; j < c.nb; ++j) {
                    finite = finite && std::isfinite(rs[j]);
                    if (j < nconv) mx = std::max(mx, rs[j]);
                }
                SAMG_CHECK(finite, SAMG_E_INVALID, "non-finite residual");
                if (mx <= tol) { state[p] = 1; return; }
                if (done[p] >= max_outer) { state[p] = 2; return; }
                by_prec(c, [&](auto tag) { outer_vcycle<decltype(tag)>(c); });
                ritz(c, false, false);
                ++done[p];
                any = true;
            });
        }
        if (!any) break;
    }
    // the caller's stream continues after every problem's work
    for (int p = 0; p < np; ++p) {
        if (e == cudaSuccess) e = cudaEventRecord(ev, b->ctx[p]->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->caller, ev, 0);
    }
    if (ev) cudaEventDestroy(ev);
    cudaFreeHost(host);
    if (outer_done)
        for (int p = 0; p < np; ++p) outer_done[p] = done[p];
    if (fail != SAMG_OK) {
        b->err = failed_p >= 0 ? "problem " + std::to_string(failed_p) + ": " +
                                     samg_last_error(b->ctx[failed_p])
                               : b->err;
        return fail;
    }
    if (e != cudaSuccess) {
        b->err = std::string("solve_batched: ") + cudaGetErrorString(e);
        return SAMG_E_CUDA;
    }
    for (int p = 0; p < np; ++p)
        if (state[p] == 2) {
            b->err = "problem " + std::to_string(p) + " reached max_outer before the tolerance";
            return SAMG_E_NOT_CONVERGED;
        }
    return SAMG_OK;
}

samg_status samg_batch_problem(samg_batch *b, int problem, samg_ctx **ctx) {
    if (!b || !ctx || problem < 0 || problem >= (int)b->ctx.size()) return SAMG_E_INVALID;
    *ctx = b->ctx[problem];
    return SAMG_OK;
}

int samg_batch_size(const samg_batch *b) { return b ? (int)b->ctx.size() : 0; }

const char *samg_batch_last_error(const samg_batch *b) {
    return b ? b->err.c_str() : g_create_error.c_str();
}

samg_status samg_set_triplets_device(samg_ctx *ctx, const double *sigma, const double *U,
                                     const double *V) {
    if (!ctx) return SAMG_E_INVALID;
    return guarded(ctx, [&] {
        samg_ctx &c = *ctx;
        SAMG_CHECK(sigma && U && (c.spd() || V), SAMG_E_INVALID, "null device pointer");
        cudaStream_t s = c.stream;
        std::vector<double> one(c.ld, 1.0);
        c.sigma.upload(one.data(), c.ld, s);  // padding columns keep sigma = 1
        SAMG_CUDA(cudaMemcpyAsync(c.sigma.p, sigma, c.nb * sizeof(double), cudaMemcpyDeviceToDevice, s));
        const int mu = urows(c, 0);
        SAMG_CUDA(cudaMemcpy2DAsync(c.U.p, c.ld * sizeof(double), U, c.nb * sizeof(double),
                                    c.nb * sizeof(double), mu, cudaMemcpyDeviceToDevice, s));
        if (!c.spd())
            SAMG_CUDA(cudaMemcpy2DAsync(c.V.p, c.ld * sizeof(double), V, c.nb * sizeof(double),
                                        c.nb * sizeof(double), c.L[0].n, cudaMemcpyDeviceToDevice, s));
        ritz(c, true);
    });
}

samg_status samg_profile(samg_ctx *ctx, int enable) {
    if (!ctx) return SAMG_E_INVALID;
    return guarded(ctx, [&] { ctx->prof.on = enable != 0; });
}

samg_status samg_profile_read(samg_ctx *ctx, int kernel_class, int reset, int64_t *launches,
                              double *total_ms, double *alg_bytes) {
    if (!ctx) return SAMG_E_INVALID;
    return guarded(ctx, [&] {
        SAMG_CHECK(kernel_class >= 0 && kernel_class < 5, SAMG_E_INVALID, "kernel class 0..4");
        ctx->prof.collect();
        if (std::getenv("SAMG_PROFILE_LEVELS") && kernel_class == 0)
            for (int l = 0; l < ctx->nlev() && l < 32; ++l)
                fprintf(stderr, "[samg] level %d (%d x %d): kaczmarz %lld launches %.3f ms avg %.1f us"
                        " | A: bands %d levels %d chunks %d reqs %lld slots %d | At: bands %d levels %d chunks %d\n",
                        l, ctx->L[l].m, ctx->L[l].n, (long long)ctx->prof.lvl_n[0][l], ctx->prof.lvl_ms[0][l],
                        1e3 * ctx->prof.lvl_ms[0][l] / std::max<int64_t>(1, ctx->prof.lvl_n[0][l]),
                        ctx->L[l].kA.nbands, ctx->L[l].kA.nlevels, ctx->L[l].kA.nchunks,
                        (long long)ctx->L[l].kA.req.n, ctx->L[l].kA.max_slots, ctx->L[l].kAt.nbands,
                        ctx->L[l].kAt.nlevels, ctx->L[l].kAt.nchunks);
        if (std::getenv("SAMG_PROFILE_LEVELS") && kernel_class == 0)
            for (int l = 0; l < ctx->nlev(); ++l)
                for (int wide = 1; wide >= 0; --wide) {
                    const std::vector<KSched> &progs = wide ? ctx->L[l].kF : ctx->L[l].kF4;
                    for (size_t k = 0; k < progs.size(); ++k) {
                        const KSched &f = progs[k];
                        if (f.rows)
                            fprintf(stderr, "[samg] level %d fused program of %zu relaxations (%s"
                                    " windows): rows %d bands %d levels %d chunks %d reqs %lld"
                                    " slots %d\n",
                                    l, k, wide ? "float64" : "float32", f.rows, f.nbands, f.nlevels,
                                    f.nchunks, (long long)f.req.n, f.max_slots);
                    }
                }
        if (launches) *launches = ctx->prof.launches[kernel_class];
        if (total_ms) *total_ms = ctx->prof.ms[kernel_class];
        if (alg_bytes) *alg_bytes = ctx->prof.bytes[kernel_class];
        if (reset)
            for (int k = 0; k < 5; ++k) {
                for (int l = 0; l < 32; ++l) { ctx->prof.lvl_ms[k][l] = 0.0; ctx->prof.lvl_n[k][l] = 0; }
                ctx->prof.launches[k] = 0;
                ctx->prof.ms[k] = 0.0;
                ctx->prof.bytes[k] = 0.0;
            }
    });
}

samg_status samg_setup_times(const samg_ctx *ctx, double *seconds, int32_t count) {
    if (!ctx || !seconds || count < 0) return SAMG_E_INVALID;
    for (int k = 0; k < count && k < SAMG_SETUP_STAGES; ++k) seconds[k] = ctx->setup_s[k];
    return SAMG_OK;
}

samg_status samg_set_precision(samg_ctx *ctx, samg_precision prec) {
    if (!ctx) return SAMG_E_INVALID;
    return guarded(ctx, [&] {
        SAMG_CHECK(prec == SAMG_FP64 || prec == SAMG_FP32 || prec == SAMG_BF16_STORE,
                   SAMG_E_INVALID, "bad precision");
        ctx->prm.prec = prec;
    });
}

samg_status samg_set_relax_order(samg_ctx *ctx, int order) {
    if (!ctx) return SAMG_E_INVALID;
    return guarded(ctx, [&] {
        SAMG_CHECK(order == 0 || order == 1, SAMG_E_INVALID,
                   "relax_order must be 0 (natural, the paper's) or 1 (coloured variant)");
        ctx->prm.relax_order = order;
    });
}

samg_status samg_set_sweep_banding(samg_ctx *ctx, int band_rows, int float_windows) {
    if (!ctx) return SAMG_E_INVALID;
    return guarded(ctx, [&] {
        SAMG_CHECK(band_rows >= 0 && band_rows <= 4096 && (float_windows == 0 || float_windows == 1),
                   SAMG_E_INVALID, "sweep banding: band_rows in 0..4096, float_windows 0 or 1");
        ctx->band_rows = band_rows;
        ctx->band_rows_level.clear();
        ctx->float_windows = float_windows != 0;
        for (Level &L : ctx->L) {
            L.kF.clear();
            L.kF4.clear();
        }
    });
}

samg_status samg_set_sweep_banding_level(samg_ctx *ctx, int level, int band_rows) {
    if (!ctx) return SAMG_E_INVALID;
    return guarded(ctx, [&] {
        SAMG_CHECK(level >= 0 && level < ctx->nlev() && band_rows >= 0 && band_rows <= 4096,
                   SAMG_E_INVALID, "sweep banding: level out of range or band_rows not in 0..4096");
        if ((int)ctx->band_rows_level.size() <= level) ctx->band_rows_level.resize(level + 1, 0);
        ctx->band_rows_level[level] = band_rows;
        ctx->L[level].kF.clear();
        ctx->L[level].kF4.clear();
    });
}

samg_status samg_set_coarse_pinv(samg_ctx *ctx, int form) {
    if (!ctx) return SAMG_E_INVALID;
    return guarded(ctx, [&] {
        SAMG_CHECK(form == 0 || form == 1, SAMG_E_INVALID,
                   "coarse_pinv must be 0 (SVD pseudo-inverse) or 1 (generalized-eigen variant)");
        ctx->prm.coarse_pinv = form;
    });
}

samg_status samg_set_triplets(samg_ctx *ctx, const double *sigma, const double *U,
                              const double *V) {
    if (!ctx) return SAMG_E_INVALID;
    return guarded(ctx, [&] { set_triplets_impl(*ctx, sigma, U, V); });
}

samg_status samg_get_triplets(samg_ctx *ctx, double *sigma, double *U, double *V,
                              double *resid) {
    if (!ctx) return SAMG_E_INVALID;
    return guarded(ctx, [&] {
        samg_ctx &c = *ctx;
        std::vector<double> sg(c.ld), rs(c.ld);
        c.sigma.download(sg.data(), c.ld, c.stream);
        c.resid.download(rs.data(), c.ld, c.stream);
        if (U) get_block(c, c.U, urows(c, 0), U);
        if (V && !c.spd()) get_block(c, c.V, c.L[0].n, V);
        SAMG_CUDA(cudaStreamSynchronize(c.stream));
        if (sigma) std::copy(sg.begin(), sg.begin() + c.nb, sigma);
        if (resid) std::copy(rs.begin(), rs.begin() + c.nb, resid);
    });
}

samg_status samg_solve(samg_ctx *ctx, double tol, int max_outer, int *outer_done) {
    if (!ctx) return SAMG_E_INVALID;
    int done = 0;
    bool converged = false;
    samg_status st = guarded(ctx, [&] {
        samg_ctx &c = *ctx;
        SAMG_CHECK(max_outer >= 0 && tol > 0.0, SAMG_E_INVALID, "bad tol or max_outer");
        const int nconv = c.prm.n_conv > 0 && c.prm.n_conv < c.nb ? c.prm.n_conv : c.nb;
        std::vector<double> rs(c.ld);
        int nredo = 0;  // most triplets seen at rho_j <= redo_tol (Sec. 6.3)
        for (;;) {
            c.resid.download(rs.data(), c.ld, c.stream);
            SAMG_CUDA(cudaStreamSynchronize(c.stream));
            double mx = 0.0;
            bool finite = true;
            for (int j = 0; j < c.nb; ++j) {
                finite = finite && std::isfinite(rs[j]);
                if (j < nconv) mx = std::max(mx, rs[j]);
            }
            if (!finite) check_kaczmarz(c);
            SAMG_CHECK(finite, SAMG_E_INVALID, "non-finite residual");
            if (done > 0 && c.prm.redo_tol > 0.0) {
                std::vector<char> conv(c.nb);
                int k = 0;
                for (int j = 0; j < c.nb; ++j) k += (conv[j] = rs[j] <= c.prm.redo_tol);
                if (k > nredo && k < c.nb) redo_interpolation(c, conv);
                nredo = std::max(nredo, k);
            }
            if (mx <= tol) { converged = true; break; }
            if (done >= max_outer) break;
            by_prec(c, [&](auto tag) { outer_vcycle<decltype(tag)>(c); });
            ritz(c, false);
            ++done;
        }
        check_kaczmarz(c);
    });
    if (outer_done) *outer_done = done;
    if (st == SAMG_OK && !converged) {
        ctx->err = "max_outer reached before the tolerance";
        return SAMG_E_NOT_CONVERGED;
    }
    return st;
}

samg_status samg_redo_interpolation(samg_ctx *ctx, const int32_t *converged) {
    if (!ctx) return SAMG_E_INVALID;
    return guarded(ctx, [&] {
        SAMG_CHECK(converged != nullptr, SAMG_E_INVALID, "converged is NULL");
        std::vector<char> conv(ctx->nb);
        for (int j = 0; j < ctx->nb; ++j) conv[j] = converged[j] != 0;
        redo_interpolation(*ctx, conv);
    });
}

samg_status samg_get_hierarchy_info(const samg_ctx *ctx, int *n_levels, int32_t *m, int32_t *n,
                                    int64_t *nnz_A) {
    if (!ctx || !n_levels) return SAMG_E_INVALID;
    *n_levels = ctx->nlev();
    for (int l = 0; l < ctx->nlev(); ++l) {
        if (m) m[l] = ctx->L[l].m;
        if (n) n[l] = ctx->L[l].n;
        if (nnz_A) nnz_A[l] = ctx->L[l].A.nnz;
    }
    return SAMG_OK;
}

samg_status samg_get_level_matrix(const samg_ctx *ctx, int level, int which, int32_t *rows,
                                  int32_t *cols, int64_t *nnz, int64_t *row_ptr, int32_t *col,
                                  double *val) {
    if (!ctx) return SAMG_E_INVALID;
    samg_ctx *c = const_cast<samg_ctx *>(ctx);
    return guarded(c, [&] {
        check_level(*c, level, which >= 3);
        const Level &L = c->L[level];
        const DCsr *M = nullptr;
        switch (which) {
            case 0: M = &L.A; break;
            case 1: M = &L.B; break;
            case 2: M = &L.C; break;
            case 3: M = &L.P; break;
            case 4: M = c->spd() ? &L.P : &L.Q; break;
            default: throw Error(SAMG_E_INVALID, "which must be 0..4");
        }
        SAMG_CHECK(!M->empty(), SAMG_E_INVALID, "operator not stored (identity on level 0)");
        if (rows) *rows = M->m;
        if (cols) *cols = M->n;
        if (nnz) *nnz = M->nnz;
        if (!row_ptr) return;
        HCsr h;
        download_csr(*M, h, c->stream);
        std::copy(h.rp.begin(), h.rp.end(), row_ptr);
        std::copy(h.ci.begin(), h.ci.end(), col);
        std::copy(h.v.begin(), h.v.end(), val);
    });
}

samg_status samg_relax(samg_ctx *ctx, int level, int count, const double *sigma, double *U,
                       double *V, const double *kappa, const double *tau) {
    if (!ctx) return SAMG_E_INVALID;
    return guarded(ctx, [&] {
        check_level(*ctx, level, false);
        set_sigma(*ctx, sigma);
        by_prec(*ctx, [&](auto tag) {
            step_relax<decltype(tag)>(*ctx, level, count, U, V, kappa, tau);
        });
        check_kaczmarz(*ctx);
    });
}

samg_status samg_residual_restrict(samg_ctx *ctx, int level, const double *sigma,
                                   const double *U, const double *V, const double *kappa,
                                   const double *tau, double *kappa_c, double *tau_c) {
    if (!ctx) return SAMG_E_INVALID;
    return guarded(ctx, [&] {
        check_level(*ctx, level, true);
        set_sigma(*ctx, sigma);
        by_prec(*ctx, [&](auto tag) {
            step_restrict<decltype(tag)>(*ctx, level, U, V, kappa, tau, kappa_c, tau_c);
        });
    });
}

samg_status samg_interpolate(samg_ctx *ctx, int level, double *U, double *V, const double *Uc,
                             const double *Vc) {
    if (!ctx) return SAMG_E_INVALID;
    return guarded(ctx, [&] {
        check_level(*ctx, level, true);
        by_prec(*ctx, [&](auto tag) { step_interp<decltype(tag)>(*ctx, level, U, V, Uc, Vc); });
    });
}

samg_status samg_coarsest_solve(samg_ctx *ctx, const double *sigma, const double *kappa,
                                const double *tau, double *U, double *V) {
    if (!ctx) return SAMG_E_INVALID;
    return guarded(ctx, [&] {
        set_sigma(*ctx, sigma);
        by_prec(*ctx, [&](auto tag) { step_coarse<decltype(tag)>(*ctx, kappa, tau, U, V); });
    });
}

samg_status samg_vcycle(samg_ctx *ctx, const double *sigma, double *U, double *V) {
    if (!ctx) return SAMG_E_INVALID;
    return guarded(ctx, [&] {
        samg_ctx &c = *ctx;
        set_sigma(c, sigma);
        c.U.zero(c.stream);
        put_block(c, U, urows(c, 0), c.U);
        if (!c.spd()) {
            c.V.zero(c.stream);
            put_block(c, V, c.L[0].n, c.V);
        }
        by_prec(c, [&](auto tag) { outer_vcycle<decltype(tag)>(c); });
        get_block(c, c.U, urows(c, 0), U);
        if (!c.spd()) get_block(c, c.V, c.L[0].n, V);
        SAMG_CUDA(cudaStreamSynchronize(c.stream));
        check_kaczmarz(c);
    });
}

samg_status samg_ritz(samg_ctx *ctx, double *sigma, double *U, double *V, double *resid) {
    if (!ctx) return SAMG_E_INVALID;
    return guarded(ctx, [&] {
        samg_ctx &c = *ctx;
        std::vector<double> one(c.nb, 1.0);
        set_sigma(c, one.data());
        c.U.zero(c.stream);
        put_block(c, U, urows(c, 0), c.U);
        if (!c.spd()) {
            c.V.zero(c.stream);
            put_block(c, V, c.L[0].n, c.V);
        }
        ritz(c, false);
        std::vector<double> sg(c.ld), rs(c.ld);
        c.sigma.download(sg.data(), c.ld, c.stream);
        c.resid.download(rs.data(), c.ld, c.stream);
        get_block(c, c.U, urows(c, 0), U);
        if (!c.spd()) get_block(c, c.V, c.L[0].n, V);
        SAMG_CUDA(cudaStreamSynchronize(c.stream));
        if (sigma) std::copy(sg.begin(), sg.begin() + c.nb, sigma);
        if (resid) std::copy(rs.begin(), rs.begin() + c.nb, resid);
    });
}

// Host copy of a caller's CSR, validated (host-only entry points).
static HCsr host_copy(const samg_csr *A, bool square) {
    SAMG_CHECK(A && A->m > 0 && A->n > 0, SAMG_E_INVALID, "bad CSR");
    SAMG_CHECK(!square || A->m == A->n, SAMG_E_INVALID, "the matrix must be square");
    validate_csr(*A);
    HCsr h;
    h.m = A->m;
    h.n = A->n;
    h.rp.assign(A->row_ptr, A->row_ptr + A->m + 1);
    h.ci.assign(A->col, A->col + A->nnz);
    h.v.assign(A->val, A->val + A->nnz);
    return h;
}

samg_status samg_host_coarsen(const samg_csr *N, double theta, int8_t *cf) {
    try {
        SAMG_CHECK(cf && theta >= 0.0, SAMG_E_INVALID, "host_coarsen: bad arguments");
        const HCsr h = host_copy(N, true);
        std::vector<char> c;
        host_coarsen(h, theta, c);
        for (int i = 0; i < h.m; ++i) cf[i] = (int8_t)c[i];
        return SAMG_OK;
    } catch (const Error &e) {
        g_create_error = e.what();
        return e.status;
    } catch (...) {
        return SAMG_E_INVALID;
    }
}

samg_status samg_host_ls_interp(const samg_csr *N, double theta, const int8_t *cf, int nf,
                                const double *yF, const double *yC, const double *w,
                                int64_t *nnz, int64_t *row_ptr, int32_t *col, double *val) {
    try {
        SAMG_CHECK(cf && nf >= 1 && yF && yC && w && nnz && theta >= 0.0, SAMG_E_INVALID,
                   "host_ls_interp: bad arguments");
        const HCsr h = host_copy(N, true);
        std::vector<char> c(cf, cf + h.m);
        std::vector<double> f(yF, yF + (size_t)h.m * nf), cc(yC, yC + (size_t)h.m * nf),
            ww(w, w + nf);
        HCsr P;
        host_ls_interp(h, theta, c, f, cc, ww, nf, P);
        *nnz = P.nnz();
        if (row_ptr) {
            SAMG_CHECK(col && val, SAMG_E_INVALID, "host_ls_interp: output arrays missing");
            std::copy(P.rp.begin(), P.rp.end(), row_ptr);
            std::copy(P.ci.begin(), P.ci.end(), col);
            std::copy(P.v.begin(), P.v.end(), val);
        }
        return SAMG_OK;
    } catch (const Error &e) {
        g_create_error = e.what();
        return e.status;
    } catch (...) {
        return SAMG_E_INVALID;
    }
}

// host CSR -> caller-style view (arrays stay owned by h)
static samg_csr view_of(const HCsr &h) {
    return samg_csr{h.m, h.n, h.nnz(), h.rp.data(), h.ci.data(), h.v.data()};
}

samg_status samg_write_hierarchy(const char *path, const samg_csr *A, int n_levels,
                                 const samg_csr *P, const samg_csr *Q, int n_b, samg_target target,
                                 samg_kind kind, const double *sigma, const double *U,
                                 const double *V) {
    try {
        SAMG_CHECK(path && A && P && n_levels >= 2 && n_levels <= 64 && n_b >= 1 && n_b <= 16,
                   SAMG_E_INVALID, "write_hierarchy: bad arguments");
        SAMG_CHECK(kind == SAMG_SVD || kind == SAMG_SPD_EIG, SAMG_E_INVALID, "bad kind");
        SAMG_CHECK(target == SAMG_DOMINANT || target == SAMG_MINIMAL, SAMG_E_INVALID, "bad target");
        const bool spd = kind == SAMG_SPD_EIG;
        SAMG_CHECK(spd || Q, SAMG_E_INVALID, "write_hierarchy: Q is NULL");
        SAMG_CHECK(sigma && U && (spd || V), SAMG_E_INVALID, "write_hierarchy: triplets missing");
        HierFile h;
        h.kind = kind;
        h.target = target;
        h.nb = n_b;
        h.A = host_copy(A, spd);
        for (int l = 0; l + 1 < n_levels; ++l) {
            const int rows_u = l == 0 ? (spd ? A->n : A->m) : P[l - 1].n;
            SAMG_CHECK(P[l].m == rows_u, SAMG_E_INVALID, "P_l has the wrong number of rows");
            h.P.push_back(host_copy(&P[l], false));
            if (!spd) {
                const int rows_v = l == 0 ? A->n : Q[l - 1].n;
                SAMG_CHECK(Q[l].m == rows_v, SAMG_E_INVALID, "Q_l has the wrong number of rows");
                h.Q.push_back(host_copy(&Q[l], false));
            }
        }
        const size_t ru = (size_t)(spd ? A->n : A->m);
        h.sigma.assign(sigma, sigma + n_b);
        h.U.assign(U, U + ru * n_b);
        if (!spd) h.V.assign(V, V + (size_t)A->n * n_b);
        write_hierarchy_file(path, h);
        return SAMG_OK;
    } catch (const Error &e) {
        g_create_error = e.what();
        return e.status;
    } catch (const std::bad_alloc &) {
        g_create_error = "host allocation failed";
        return SAMG_E_NOMEM;
    } catch (...) {
        return SAMG_E_INVALID;
    }
}

samg_status samg_import_file(const char *path, const samg_params *params, void *cuda_stream,
                             samg_ctx **out) {
    if (!out) return SAMG_E_INVALID;
    *out = nullptr;
    HierFile h;
    try {
        SAMG_CHECK(path != nullptr, SAMG_E_INVALID, "import_file: path is NULL");
        read_hierarchy_file(path, h);
    } catch (const Error &e) {
        g_create_error = e.what();
        return e.status;
    } catch (const std::bad_alloc &) {
        g_create_error = "host allocation failed";
        return SAMG_E_NOMEM;
    } catch (...) {
        return SAMG_E_INVALID;
    }
    const samg_csr A = view_of(h.A);
    std::vector<samg_csr> P, Q;
    for (const HCsr &x : h.P) P.push_back(view_of(x));
    for (const HCsr &x : h.Q) Q.push_back(view_of(x));
    return samg_import(&A, (int)h.P.size() + 1, P.data(), Q.empty() ? nullptr : Q.data(), h.nb,
                       h.target, h.kind, params, h.sigma.data(), h.U.data(),
                       h.V.empty() ? nullptr : h.V.data(), cuda_stream, out);
}

samg_status samg_export(samg_ctx *ctx, const char *path) {
    if (!ctx) return SAMG_E_INVALID;
    return guarded(ctx, [&] {
        samg_ctx &c = *ctx;
        SAMG_CHECK(path != nullptr, SAMG_E_INVALID, "export: path is NULL");
        SAMG_CHECK(c.nlev() >= 2, SAMG_E_INVALID, "export: no hierarchy");
        HierFile h;
        h.kind = c.kind;
        h.target = c.target;
        h.nb = c.nb;
        download_csr(c.L[0].A, h.A, c.stream);
        h.P.resize(c.nlev() - 1);
        if (!c.spd()) h.Q.resize(c.nlev() - 1);
        for (int l = 0; l + 1 < c.nlev(); ++l) {
            download_csr(c.L[l].P, h.P[l], c.stream);
            if (!c.spd()) download_csr(c.L[l].Q, h.Q[l], c.stream);
        }
        std::vector<double> sg(c.ld);
        c.sigma.download(sg.data(), c.ld, c.stream);
        h.U.resize((size_t)urows(c, 0) * c.nb);
        get_block(c, c.U, urows(c, 0), h.U.data());
        if (!c.spd()) {
            h.V.resize((size_t)c.L[0].n * c.nb);
            get_block(c, c.V, c.L[0].n, h.V.data());
        }
        SAMG_CUDA(cudaStreamSynchronize(c.stream));
        h.sigma.assign(sg.begin(), sg.begin() + c.nb);
        write_hierarchy_file(path, h);
    });
}

samg_status samg_host_strength_product(const samg_csr *A, double theta, int64_t *nnz,
                                       int64_t *row_ptr, int32_t *col, double *val) {
    try {
        SAMG_CHECK(nnz && theta >= 0.0, SAMG_E_INVALID, "host_strength_product: bad arguments");
        const HCsr h = host_copy(A, false);
        HCsr S;
        host_strength_product(h, theta, S);
        *nnz = S.nnz();
        if (row_ptr) {
            SAMG_CHECK(col && val, SAMG_E_INVALID, "host_strength_product: output arrays missing");
            std::copy(S.rp.begin(), S.rp.end(), row_ptr);
            std::copy(S.ci.begin(), S.ci.end(), col);
            std::copy(S.v.begin(), S.v.end(), val);
        }
        return SAMG_OK;
    } catch (const Error &e) {
        g_create_error = e.what();
        return e.status;
    } catch (...) {
        return SAMG_E_INVALID;
    }
}

samg_status samg_sweep_plan(const samg_csr *A, int fused_count, int32_t *row_level,
                            int64_t capacity, int *depth, int *nbands) {
    try {
        SAMG_CHECK(fused_count >= 0 && depth && nbands, SAMG_E_INVALID, "sweep_plan: bad arguments");
        const HCsr h = host_copy(A, false);
        std::vector<int> lv;
        plan_sweep(h, fused_count, lv, nbands);
        int d = 0;
        for (int x : lv) d = std::max(d, x + 1);
        *depth = d;
        if (row_level) {
            SAMG_CHECK(capacity >= (int64_t)lv.size(), SAMG_E_INVALID,
                       "sweep_plan: row_level holds fewer entries than the program has rows");
            std::copy(lv.begin(), lv.end(), row_level);
        }
        return SAMG_OK;
    } catch (const Error &e) {
        g_create_error = e.what();
        return e.status;
    } catch (...) {
        return SAMG_E_INVALID;
    }
}

samg_status samg_row_colours(const samg_csr *A, int32_t *colour, int32_t *ncolour) {
    try {
        SAMG_CHECK(A && colour && ncolour, SAMG_E_INVALID, "row_colours: NULL argument");
        validate_csr(*A);
        std::vector<int64_t> rp(A->row_ptr, A->row_ptr + A->m + 1);
        std::vector<int> ci(A->col, A->col + A->nnz);
        std::vector<int> col;
        *ncolour = greedy_row_colours(A->m, A->n, rp, ci, col);
        std::copy(col.begin(), col.end(), colour);
        return SAMG_OK;
    } catch (const Error &e) {
        g_create_error = e.what();
        return e.status;
    } catch (const std::bad_alloc &) {
        g_create_error = "row_colours: host allocation failed";
        return SAMG_E_NOMEM;
    }
}

samg_status samg_sweep_schedule(const samg_csr *A, const samg_csr *B, const samg_csr *C,
                                int fused_count, int spd, int resident_slots, int band_rows,
                                int slot_cap, unsigned char *buf,
                                int64_t capacity, int64_t *size) {
    try {
        SAMG_CHECK(fused_count >= 0 && size && (capacity == 0 || buf), SAMG_E_INVALID,
                   "sweep_schedule: bad arguments");
        const HCsr h = host_copy(A, spd != 0);
        HCsr hb, hc;
        if (B) {
            hb = host_copy(B, true);
            SAMG_CHECK(hb.m == h.m, SAMG_E_INVALID, "sweep_schedule: B must be m x m");
        }
        if (C) {
            hc = host_copy(C, true);
            SAMG_CHECK(hc.m == h.n, SAMG_E_INVALID, "sweep_schedule: C must be n x n");
        }
        HostSched hs;
        host_schedule(h, B ? &hb : nullptr, C ? &hc : nullptr, fused_count, spd != 0, hs,
                      resident_slots, band_rows, slot_cap);
        std::vector<unsigned char> out;
        out.reserve(64 + 4 * hs.band_chunk.size() + 40 * hs.chunk.size() + 16 * hs.lvl.size() +
                    8 * hs.req.size() + hs.img_d.size());
        auto put32 = [&](int32_t v) {
            const unsigned char *q = reinterpret_cast<const unsigned char *>(&v);
            out.insert(out.end(), q, q + 4);
        };
        auto put64 = [&](int64_t v) {
            const unsigned char *q = reinterpret_cast<const unsigned char *>(&v);
            out.insert(out.end(), q, q + 8);
        };
        for (int32_t v : {hs.rows, hs.cols, hs.nbands, hs.nlevels, hs.nchunks, hs.max_slots,
                          hs.mode, (int32_t)hs.shifted})
            put32(v);
        put64((int64_t)hs.req.size());
        put64((int64_t)hs.img_d.size());
        for (int v : hs.band_chunk) put32(v);
        for (const KChunk &c : hs.chunk) {
            for (int32_t v : {c.L0, c.nl, c.nr, c.ne, c.nx, c.nq, c.bytes_d, 0}) put32(v);
            put64(c.off_d);
        }
        for (const int4 &l : hs.lvl)
            for (int32_t v : {l.x, l.y, l.z, l.w}) put32(v);
        for (const int2 &r : hs.req) {
            put32(r.x);
            put32(r.y);
        }
        out.insert(out.end(), hs.img_d.begin(), hs.img_d.end());
        for (int v : hs.order) put32(v);
        *size = (int64_t)out.size();
        if (buf) {
            SAMG_CHECK(capacity >= (int64_t)out.size(), SAMG_E_INVALID,
                       "sweep_schedule: buffer smaller than the schedule");
            std::copy(out.begin(), out.end(), buf);
        }
        return SAMG_OK;
    } catch (const Error &e) {
        g_create_error = e.what();
        return e.status;
    } catch (const std::bad_alloc &) {
        g_create_error = "host allocation failed";
        return SAMG_E_NOMEM;
    } catch (...) {
        return SAMG_E_INVALID;
    }
}

samg_status samg_debug_mute_band(samg_ctx *ctx, int level, int which, int band) {
    if (!ctx) return SAMG_E_INVALID;
    return guarded(ctx, [&] {
        SAMG_CHECK(level >= 0 && level < (int)ctx->L.size() && which >= 0 && which <= 2,
                   SAMG_E_INVALID, "debug_mute_band: bad level or operator");
        Level &L = ctx->L[level];
        if (which < 2) {
            kaczmarz_mute_band(which == 0 ? L.kA : L.kAt, band, ctx->stream);
        } else {
            for (auto *progs : {&L.kF, &L.kF4})
                for (KSched &k : *progs)
                    if (k.rows) kaczmarz_mute_band(k, band, ctx->stream);
        }
    });
}

samg_status samg_block_gram(const double *X, const double *Y, int64_t rows, int nb, int ld,
                            double *G, void *cuda_stream) {
    try {
        SAMG_CHECK(X && Y && G && rows >= 0 && nb >= 1 && nb <= 16 && ld >= nb, SAMG_E_INVALID,
                   "block_gram: bad arguments");
        check_device();
        cudaStream_t s = (cudaStream_t)cuda_stream;
        DBuf<double> work(gram_workspace(rows, nb));
        launch_gram(X, Y, rows, nb, ld, G, work.p, s);
        SAMG_CUDA(cudaStreamSynchronize(s));
        return SAMG_OK;
    } catch (const Error &e) {
        g_create_error = e.what();
        return e.status;
    } catch (...) {
        return SAMG_E_INVALID;
    }
}


}  // extern "C"

// ----------------------------------------------- allocation-free Gram product
// samg_block_gram_noalloc keeps the per-CTA partial sums of the Gram product
// in one fixed device array instead of a cudaMalloc'd workspace.
namespace {

constexpr size_t GRAM_STATIC_DOUBLES = 131072;  // 1 MiB of partial sums
__device__ __align__(256) double g_gram_static[GRAM_STATIC_DOUBLES];

// The scratch's device address belongs to a CUDA context: a device reset or a
// new primary context loads the module again, possibly elsewhere.  The cache
// is therefore keyed on the current context's process-unique id
// (cuCtxGetId), which a new context never repeats, unlike its handle.
struct ScratchAddr {
    unsigned long long ctx_id;
    double *addr;
};
std::vector<ScratchAddr> g_gram_static_addr;  // one entry per context seen
std::mutex g_gram_static_mu;

// Current context's unique id from the driver API, through the driver
// library the runtime has already loaded (the library links only the
// runtime).  0 when no context is current yet.
unsigned long long current_context_id() {
    using GetCurrent = int (*)(void **);
    using GetId = int (*)(void *, unsigned long long *);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static bool looked = false;
    if (!looked) {
        looked = true;
        void *h = dlopen("libcuda.so.1", RTLD_NOW | RTLD_LOCAL);
        if (h) {
            get_current = reinterpret_cast<GetCurrent>(dlsym(h, "cuCtxGetCurrent"));
            get_id = reinterpret_cast<GetId>(dlsym(h, "cuCtxGetId"));
        }
    }
    SAMG_CHECK(get_current && get_id, SAMG_E_CUDA,
               "block_gram_noalloc: the CUDA driver's context functions are unavailable");
    void *ctx = nullptr;
    SAMG_CHECK(get_current(&ctx) == 0, SAMG_E_CUDA, "block_gram_noalloc: cuCtxGetCurrent failed");
    if (!ctx) return 0;
    unsigned long long id = 0;
    SAMG_CHECK(get_id(ctx, &id) == 0, SAMG_E_CUDA, "block_gram_noalloc: cuCtxGetId failed");
    return id;
}

// Device address of g_gram_static in the current context.  The first call
// in a context asks the runtime once (cudaGetSymbolAddress, which also makes
// the device's primary context current) and caches the answer under the
// context's id; later calls in that context only read the cache.
double *gram_static_scratch() {
    std::lock_guard<std::mutex> lock(g_gram_static_mu);
    unsigned long long id = current_context_id();
    if (id != 0)
        for (const ScratchAddr &e : g_gram_static_addr)
            if (e.ctx_id == id) return e.addr;
    void *p = nullptr;
    SAMG_CUDA(cudaGetSymbolAddress(&p, g_gram_static));
    SAMG_CHECK(p != nullptr, SAMG_E_CUDA, "block_gram_noalloc: no address for the scratch");
    id = current_context_id();
    SAMG_CHECK(id != 0, SAMG_E_CUDA, "block_gram_noalloc: no current CUDA context");
    g_gram_static_addr.push_back({id, static_cast<double *>(p)});
    return static_cast<double *>(p);
}

}  // namespace

extern "C" {

samg_status samg_block_gram_noalloc(const double *X, const double *Y, int64_t rows, int nb,
                                    int ld, double *G, void *cuda_stream) {
    try {
        SAMG_CHECK(X && Y && G && rows >= 0 && nb >= 1 && nb <= 16 && ld >= nb, SAMG_E_INVALID,
                   "block_gram_noalloc: bad arguments");
        const size_t need = gram_workspace(rows, nb);
        SAMG_CHECK(need <= GRAM_STATIC_DOUBLES, SAMG_E_INVALID,
                   "block_gram_noalloc: ceil(rows / 4096) * nb * nb = " + std::to_string(need) +
                       " partial sums exceed the fixed scratch of " +
                       std::to_string(GRAM_STATIC_DOUBLES) + " doubles");
        check_device();
        // Every partial sum the final pass reads is written by the partial
        // pass of the same call, so the scratch needs no clearing.
        launch_gram(X, Y, rows, nb, ld, G, gram_static_scratch(), (cudaStream_t)cuda_stream);
        return SAMG_OK;
    } catch (const Error &e) {
        g_create_error = e.what();
        return e.status;
    } catch (...) {
        return SAMG_E_INVALID;
    }
}

}  // extern "C"
