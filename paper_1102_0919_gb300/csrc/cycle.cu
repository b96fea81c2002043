// cycle.cu -- additive V-cycle (Secs. 4.1-4.2) and Ritz step (Sec. 4.3)
// drivers, and completion of a hierarchy on the device (Eq. coarseOp).
#include <algorithm>
#include <cmath>

#include "ctx.cuh"

namespace samg {

template <> Work<float> &work<float>(Level &L) { return L.wf; }
template <> Work<double> &work<double>(Level &L) { return L.wd; }
template <> Work<bf16> &work<bf16>(Level &L) { return L.wb; }

// diagonals and matrix views in the arithmetic type of storage type T
template <typename T> static const typename Acc<T>::T *dgB(const Level &L);
template <> const float *dgB<float>(const Level &L) { return L.dBf.p; }
template <> const float *dgB<bf16>(const Level &L) { return L.dBf.p; }
template <> const double *dgB<double>(const Level &L) { return L.dBd.p; }
template <typename T> static const typename Acc<T>::T *dgC(const Level &L);
template <> const float *dgC<float>(const Level &L) { return L.dCf.p; }
template <> const float *dgC<bf16>(const Level &L) { return L.dCf.p; }
template <> const double *dgC<double>(const Level &L) { return L.dCd.p; }

template <typename T> static CsrView<typename Acc<T>::T> mview(const DCsr &a) {
    return view<typename Acc<T>::T>(a);
}
template <typename T> static CsrView<typename Acc<T>::T> opt_view(const DCsr &a) {
    if (a.empty()) return CsrView<typename Acc<T>::T>{0, 0, nullptr, nullptr, nullptr};
    return mview<T>(a);
}

// Algorithmic bytes of one pass (what the method must move, no credit for
// reuse): matrix values + column indices + row offsets, the right-hand side
// read, the iterate read and written; n_b columns counted (not the padding).
static double kz_bytes(const KSched &k, int nb, size_t s) {
    const double val = k.shifted ? 2.0 * s : (double)s;
    return (double)k.nent * (val + 4.0) + 4.0 * (k.rows + 1.0) + (double)k.rows * nb * s +
           2.0 * k.cols * nb * s;
}
static double spmv_bytes(const DCsr &M, int nb, size_t s) {  // y = M x
    if (M.empty()) return 0.0;
    return (double)M.nnz * (s + 4.0) + 4.0 * (M.m + 1.0) + (double)M.n * nb * s +
           (double)M.m * nb * s;
}

// ------------------------------------------------------------ relaxation
// One block Gauss-Seidel relaxation of A v - s B u = kappa,
// A^t u - s C v = tau (Eqs. genSVDresid1-2, add), sigma fixed per column.
template <typename T>
void relax(samg_ctx &c, int l) {
    c.prof.cur_level = l;
    Level &L = c.L[l];
    Work<T> &w = work<T>(L);
    const int ld = c.ld;
    cudaStream_t s = c.stream;
    const double *sig = c.sigma.p;
    if (c.minimal()) {
        const int nb = c.nb;
        const size_t sz = sizeof(T);
        if (c.spd()) {  // one sweep over the rows of A - s B (Sec. 5.3)
            Prof pr(c.prof, s, 0, kz_bytes(L.kA, nb, sz));
            launch_kaczmarz<T>(L.kA, ld, w.k.p, w.u.p, sig, s);
            return;
        }
        // v from the rows of A with rhs s B u + kappa
        Term<T> tb{opt_view<T>(L.B), w.u.p, 1.0, true};
        {
            Prof pr(c.prof, s, 1, spmv_bytes(L.B, nb, sz) + 2.0 * L.m * nb * sz);
            launch_combine<T, T>(L.m, ld, w.k.p, 1.0, tb, Term<T>{}, sig, w.r.p, s);
        }
        {
            Prof pr(c.prof, s, 0, kz_bytes(L.kA, nb, sz));
            launch_kaczmarz<T>(L.kA, ld, w.r.p, w.v.p, nullptr, s);
        }
        // u from the rows of A^t with rhs s C v + tau
        Term<T> tc{opt_view<T>(L.C), w.v.p, 1.0, true};
        {
            Prof pr(c.prof, s, 1, spmv_bytes(L.C, nb, sz) + 2.0 * L.n * nb * sz);
            launch_combine<T, T>(L.n, ld, w.t.p, 1.0, tc, Term<T>{}, sig, w.s.p, s);
        }
        {
            Prof pr(c.prof, s, 0, kz_bytes(L.kAt, nb, sz));
            launch_kaczmarz<T>(L.kAt, ld, w.s.p, w.u.p, nullptr, s);
        }
        return;
    }
    // dominant: weighted Jacobi for u from Eq. genSVDresid1, then v (Sec. 3.5)
    const double om = c.prm.omega_J;
    Prof pr(c.prof, s, 2,
            2.0 * (spmv_bytes(L.A, c.nb, sizeof(T)) + spmv_bytes(L.B, c.nb, sizeof(T))));
    if (c.spd()) {
        launch_jacobi<T>(L.n, ld, mview<T>(L.A), w.u.p, opt_view<T>(L.B), dgB<T>(L), w.u.p, w.k.p,
                         sig, om, w.tu.p, s);
        std::swap(w.u, w.tu);
        return;
    }
    launch_jacobi<T>(L.m, ld, mview<T>(L.A), w.v.p, opt_view<T>(L.B), dgB<T>(L), w.u.p, w.k.p, sig,
                     om, w.tu.p, s);
    std::swap(w.u, w.tu);
    launch_jacobi<T>(L.n, ld, mview<T>(L.At), w.u.p, opt_view<T>(L.C), dgC<T>(L), w.v.p, w.t.p,
                     sig, om, w.tv.p, s);
    std::swap(w.v, w.tv);
}

// The coloured-order variant of a smoothing phase (not the paper's order):
// the same relaxations with every sweep's rows visited colour by colour
// (coloured.cuh), on the same unknown [v; u] and right-hand side [kappa; tau]
// as the exact-order program.  The program is built on first use.
template <typename T>
static void relax_phase_coloured(samg_ctx &c, int l, int count) {
    Level &L = c.L[l];
    Work<T> &w = work<T>(L);
    cudaStream_t s = c.stream;
    const int ld = c.ld;
    if ((int)L.kC.size() <= count) L.kC.resize(count + 1);
    CSched &cs = L.kC[count];
    if (cs.rows == 0) {
        HCsr hA, hB;
        download_csr(L.A, hA, s);
        if (L.B.empty()) csr_identity(c.spd() ? L.n : L.m, hB);
        else download_csr(L.B, hB, s);
        if (c.spd()) {
            build_cschedule_stacked(hA, hB, count, cs, s);
        } else {
            HCsr hAt, hC;
            download_csr(L.At, hAt, s);
            if (L.C.empty()) csr_identity(L.n, hC);
            else download_csr(L.C, hC, s);
            build_cschedule_fused(hA, hAt, hB, hC, count, cs, s);
        }
    }
    const size_t sz = sizeof(T);
    const double bytes = (double)cs.nent * ((cs.mode == 1 ? 2.0 : 1.0) * sz + 4.0) +
                         4.0 * (cs.rows + 1.0) + (double)cs.rows * c.nb * sz +
                         2.0 * count * (double)(c.spd() ? L.n : L.m + L.n) * c.nb * sz;
    Prof pr(c.prof, s, 0, bytes);
    if (c.spd()) {
        launch_coloured<T>(cs, ld, w.k.p, w.u.p, c.sigma.p, s);
        return;
    }
    const size_t nv = (size_t)L.n * ld, nu = (size_t)L.m * ld;
    if (w.z.n != nu + nv) {
        w.z.alloc(nu + nv);
        w.kt.alloc(nu + nv);
    }
    SAMG_CUDA(cudaMemcpyAsync(w.z.p, w.v.p, nv * sizeof(T), cudaMemcpyDeviceToDevice, s));
    SAMG_CUDA(cudaMemcpyAsync(w.z.p + nv, w.u.p, nu * sizeof(T), cudaMemcpyDeviceToDevice, s));
    SAMG_CUDA(cudaMemcpyAsync(w.kt.p, w.k.p, nu * sizeof(T), cudaMemcpyDeviceToDevice, s));
    SAMG_CUDA(cudaMemcpyAsync(w.kt.p + nu, w.t.p, nv * sizeof(T), cudaMemcpyDeviceToDevice, s));
    launch_coloured<T>(cs, ld, w.kt.p, w.z.p, c.sigma.p, s);
    SAMG_CUDA(cudaMemcpyAsync(w.v.p, w.z.p, nv * sizeof(T), cudaMemcpyDeviceToDevice, s));
    SAMG_CUDA(cudaMemcpyAsync(w.u.p, w.z.p + nv, nu * sizeof(T), cudaMemcpyDeviceToDevice, s));
}

// count relaxations of the minimal kind as one fused sweep program (the
// schedule is built on first use for each count); other kinds relax one at a
// time.  The result is that of count calls of relax() up to the rounding
// order inside each row.
// Rows per dependency level a band of level l's smoothing programs grows to:
// a per-level override, else the context's setting, else the default.  The
// default follows measurements (mixed precision, the 1024^2 gradient's 13
// levels, every level timed at 1 to 32 rows per level, bands claimed in
// claim order): the finest level runs fastest at 32; on the Galerkin levels
// the best width falls with the level's size, about max(m, n) / 65536
// rows (8 at 524,288 unknowns, 4 at 262,143, 2 from about 65,000 down),
// narrower bands keeping more sweeps' wavefronts resident at once.
static int band_rows_for(const samg_ctx &c, int l) {
    if (l < (int)c.band_rows_level.size() && c.band_rows_level[l] > 0) return c.band_rows_level[l];
    if (c.band_rows > 0) return c.band_rows;
    if (l == 0) return 32;
    const int64_t size = std::max(c.L[l].m, c.L[l].n);
    int t = 2;  // max(m, n) / 65536 rounded to a power of two, within [2, 32]
    while (t < 32 && 2 * size >= (int64_t)3 * t * 65536) t *= 2;
    return t;
}

template <typename T>
void relax_phase(samg_ctx &c, int l, int count) {
    if (!c.minimal() || count <= 0) {
        for (int k = 0; k < count; ++k) relax<T>(c, l);
        return;
    }
    c.prof.cur_level = l;
    Level &L = c.L[l];
    Work<T> &w = work<T>(L);
    cudaStream_t s = c.stream;
    const int ld = c.ld;
    if (c.prm.relax_order == 1) {
        relax_phase_coloured<T>(c, l, count);
        return;
    }
    // float64 launches need float64 windows; float32 and bfloat16 storage
    // arithmetic in float32, whose windows hold twice the columns
    const bool wide = sizeof(typename Acc<T>::T) == 8 || !c.float_windows;
    std::vector<KSched> &progs = wide ? L.kF : L.kF4;
    if ((int)progs.size() <= count) progs.resize(count + 1);
    KSched &ks = progs[count];
    if (ks.rows == 0) {
        HCsr hA, hB;
        download_csr(L.A, hA, s);
        if (L.B.empty()) csr_identity(c.spd() ? L.n : L.m, hB);
        else download_csr(L.B, hB, s);
        if (c.spd()) {
            build_kschedule_stacked(hA, hB, count, ks, s, ld, wide, band_rows_for(c, l));
        } else {
            HCsr hAt, hC;
            download_csr(L.At, hAt, s);
            if (L.C.empty()) csr_identity(L.n, hC);
            else download_csr(L.C, hC, s);
            build_kschedule_fused(hA, hAt, hB, hC, count, ks, s, ld, wide, band_rows_for(c, l));
        }
        if (c.rstat.n >= 2) ks.err = c.rstat.p + 1;
    }
    Prof pr(c.prof, s, 0, kz_bytes(ks, c.nb, sizeof(T)));
    if (c.spd()) {
        launch_kaczmarz<T>(ks, ld, w.k.p, w.u.p, c.sigma.p, s);
        return;
    }
    const size_t nv = (size_t)L.n * ld, nu = (size_t)L.m * ld;
    if (w.z.n != nu + nv) {
        w.z.alloc(nu + nv);
        w.kt.alloc(nu + nv);
    }
    // unknown [v; u], right-hand side [kappa; tau]
    SAMG_CUDA(cudaMemcpyAsync(w.z.p, w.v.p, nv * sizeof(T), cudaMemcpyDeviceToDevice, s));
    SAMG_CUDA(cudaMemcpyAsync(w.z.p + nv, w.u.p, nu * sizeof(T), cudaMemcpyDeviceToDevice, s));
    SAMG_CUDA(cudaMemcpyAsync(w.kt.p, w.k.p, nu * sizeof(T), cudaMemcpyDeviceToDevice, s));
    SAMG_CUDA(cudaMemcpyAsync(w.kt.p + nu, w.t.p, nv * sizeof(T), cudaMemcpyDeviceToDevice, s));
    launch_kaczmarz<T>(ks, ld, w.kt.p, w.z.p, c.sigma.p, s);
    SAMG_CUDA(cudaMemcpyAsync(w.v.p, w.z.p, nv * sizeof(T), cudaMemcpyDeviceToDevice, s));
    SAMG_CUDA(cudaMemcpyAsync(w.u.p, w.z.p + nv, nu * sizeof(T), cudaMemcpyDeviceToDevice, s));
}
template void relax_phase<float>(samg_ctx &, int, int);
template void relax_phase<double>(samg_ctx &, int, int);
template void relax_phase<bf16>(samg_ctx &, int, int);

// r = kappa - (A v - s B u), s = tau - (A^t u - s C v); kappa_c = P^t r,
// tau_c = Q^t s into level l+1 (Eqs. add, addCoarse).
template <typename T>
void residual_restrict(samg_ctx &c, int l) {
    Level &L = c.L[l];
    Level &Lc = c.L[l + 1];
    Work<T> &w = work<T>(L);
    Work<T> &wc = work<T>(Lc);
    const int ld = c.ld;
    cudaStream_t s = c.stream;
    const double *sig = c.sigma.p;
    const size_t sz = sizeof(T);
    const int nb = c.nb;
    Prof pr(c.prof, s, 1,
            spmv_bytes(L.A, nb, sz) + spmv_bytes(L.B, nb, sz) + spmv_bytes(L.Pt, nb, sz) +
                (c.spd() ? 0.0 : spmv_bytes(L.At, nb, sz) + spmv_bytes(L.C, nb, sz) +
                                     spmv_bytes(L.Qt, nb, sz)));
    if (c.spd()) {
        Term<T> ta{mview<T>(L.A), w.u.p, -1.0, false};
        Term<T> tb{opt_view<T>(L.B), w.u.p, 1.0, true};
        launch_combine<T, T>(L.n, ld, w.k.p, 1.0, ta, tb, sig, w.r.p, s);
        launch_combine<T, T>(Lc.n, ld, (const T *)nullptr, 0.0,
                             Term<T>{mview<T>(L.Pt), w.r.p, 1.0, false}, Term<T>{}, sig, wc.k.p, s);
        return;
    }
    Term<T> ta{mview<T>(L.A), w.v.p, -1.0, false};
    Term<T> tb{opt_view<T>(L.B), w.u.p, 1.0, true};
    launch_combine<T, T>(L.m, ld, w.k.p, 1.0, ta, tb, sig, w.r.p, s);
    Term<T> tat{mview<T>(L.At), w.u.p, -1.0, false};
    Term<T> tc{opt_view<T>(L.C), w.v.p, 1.0, true};
    launch_combine<T, T>(L.n, ld, w.t.p, 1.0, tat, tc, sig, w.s.p, s);
    launch_combine<T, T>(Lc.m, ld, (const T *)nullptr, 0.0,
                         Term<T>{mview<T>(L.Pt), w.r.p, 1.0, false}, Term<T>{}, sig, wc.k.p, s);
    launch_combine<T, T>(Lc.n, ld, (const T *)nullptr, 0.0,
                         Term<T>{mview<T>(L.Qt), w.s.p, 1.0, false}, Term<T>{}, sig, wc.t.p, s);
}

// u += P u_c, v += Q v_c (Eq. corrAdd)
template <typename T>
void interpolate(samg_ctx &c, int l) {
    Level &L = c.L[l];
    Work<T> &w = work<T>(L);
    Work<T> &wc = work<T>(c.L[l + 1]);
    const int ld = c.ld;
    cudaStream_t s = c.stream;
    const double *sig = c.sigma.p;
    Prof pr(c.prof, s, 1,
            spmv_bytes(L.P, c.nb, sizeof(T)) + (double)L.P.m * c.nb * sizeof(T) +
                (c.spd() ? 0.0 : spmv_bytes(L.Q, c.nb, sizeof(T)) + (double)L.Q.m * c.nb * sizeof(T)));
    if (c.spd()) {
        launch_combine<T, T>(L.n, ld, w.u.p, 1.0, Term<T>{mview<T>(L.P), wc.u.p, 1.0, false},
                             Term<T>{}, sig, w.u.p, s);
        return;
    }
    launch_combine<T, T>(L.m, ld, w.u.p, 1.0, Term<T>{mview<T>(L.P), wc.u.p, 1.0, false},
                         Term<T>{}, sig, w.u.p, s);
    launch_combine<T, T>(L.n, ld, w.v.p, 1.0, Term<T>{mview<T>(L.Q), wc.v.p, 1.0, false},
                         Term<T>{}, sig, w.v.p, s);
}

// [u; v] = (X_L - s Y_L)^+ [kappa; tau] without the smallest singular value
template <typename T>
void coarse_solve(samg_ctx &c) {
    Level &L = c.L.back();
    Work<T> &w = work<T>(L);
    Prof pr(c.prof, c.stream, 3, 2.0 * (double)c.co.M * c.co.M * 8.0);
    if (c.prm.coarse_pinv == 1) {
        if (c.co.cbuf.n < (size_t)c.co.M * c.ld) c.co.cbuf.alloc((size_t)c.co.M * c.ld);
        launch_coarse_apply_geneig<T>(c.co.M, c.co.m1, c.ld, c.nb, c.co.lam.p, c.co.W.p, c.co.Wt.p,
                                      c.sigma.p, w.k.p, c.spd() ? w.k.p : w.t.p, w.u.p,
                                      c.spd() ? w.u.p : w.v.p, c.co.cbuf.p, c.stream);
        return;
    }
    const size_t nq = coarse_warm_size(c.co.M, c.nb);
    if (c.co.qwarm.n != nq) {
        c.co.qwarm.alloc(nq);
        c.co.warm = false;
    }
    launch_coarse_apply<T>(c.co.M, c.co.m1, c.ld, c.nb, c.co.lam.p, c.co.W.p, c.co.Wt.p,
                           c.sigma.p, w.k.p, c.spd() ? w.k.p : w.t.p, w.u.p,
                           c.spd() ? w.u.p : w.v.p, c.co.qwarm.p, c.co.warm ? 1 : 0, c.stream);
    c.co.warm = true;
}

template <typename T>
void vcycle(samg_ctx &c, int l) {
    if (l == c.nlev() - 1) {
        coarse_solve<T>(c);
        return;
    }
    relax_phase<T>(c, l, c.prm.mu_b);
    residual_restrict<T>(c, l);
    Work<T> &wc = work<T>(c.L[l + 1]);
    wc.u.zero(c.stream);
    if (!c.spd()) wc.v.zero(c.stream);
    vcycle<T>(c, l + 1);
    interpolate<T>(c, l);
    relax_phase<T>(c, l, c.prm.mu_b);
}

// Defect-correction form of one outer V-cycle: (r, s) = -(A V - s U,
// A^t U - s V) in float64, the whole cycle on the error equation with zero
// initial guess in precision T, then U += e_u, V += e_v in float64.  The
// relaxations are affine in (iterate, rhs), so this equals the V-cycle on the
// iterate itself.
template <typename T>
void outer_vcycle(samg_ctx &c) {
    Level &L0 = c.L[0];
    Work<T> &w = work<T>(L0);
    const int ld = c.ld;
    cudaStream_t s = c.stream;
    const double *sig = c.sigma.p;
    if (c.spd()) {
        Term<double> ta{view<double>(L0.A), c.U.p, -1.0, false};
        Term<double> tu{CsrView<double>{0, 0, nullptr, nullptr, nullptr}, c.U.p, 1.0, true};
        launch_combine<double, T>(L0.n, ld, nullptr, 0.0, ta, tu, sig, w.k.p, s);
        w.u.zero(s);
        vcycle<T>(c, 0);
        launch_add_to<T>((size_t)L0.n * ld, c.U.p, w.u.p, s);
        return;
    }
    Term<double> ta{view<double>(L0.A), c.V.p, -1.0, false};
    Term<double> tu{CsrView<double>{0, 0, nullptr, nullptr, nullptr}, c.U.p, 1.0, true};
    launch_combine<double, T>(L0.m, ld, nullptr, 0.0, ta, tu, sig, w.k.p, s);
    Term<double> tat{view<double>(L0.At), c.U.p, -1.0, false};
    Term<double> tv{CsrView<double>{0, 0, nullptr, nullptr, nullptr}, c.V.p, 1.0, true};
    launch_combine<double, T>(L0.n, ld, nullptr, 0.0, tat, tv, sig, w.t.p, s);
    w.u.zero(s);
    w.v.zero(s);
    vcycle<T>(c, 0);
    launch_add_to<T>((size_t)L0.m * ld, c.U.p, w.u.p, s);
    launch_add_to<T>((size_t)L0.n * ld, c.V.p, w.v.p, s);
}

template <typename T>
static void alloc_work(Work<T> &w, int m, int n, int ld, bool spd, cudaStream_t s);

template <typename T>
void ensure_work(samg_ctx &c) {
    for (int l = 0; l < c.nlev(); ++l) {
        Level &L = c.L[l];
        Work<T> &w = work<T>(L);
        const size_t want = (size_t)(c.spd() ? L.n : L.m) * c.ld;
        if (w.u.n != want) alloc_work(w, L.m, L.n, c.ld, c.spd(), c.stream);
    }
}
template void ensure_work<float>(samg_ctx &);
template void ensure_work<double>(samg_ctx &);
template void ensure_work<bf16>(samg_ctx &);

template void relax<float>(samg_ctx &, int);
template void relax<double>(samg_ctx &, int);
template void residual_restrict<float>(samg_ctx &, int);
template void residual_restrict<double>(samg_ctx &, int);
template void interpolate<float>(samg_ctx &, int);
template void interpolate<double>(samg_ctx &, int);
template void coarse_solve<float>(samg_ctx &);
template void coarse_solve<double>(samg_ctx &);
template void vcycle<float>(samg_ctx &, int);
template void vcycle<double>(samg_ctx &, int);
template void outer_vcycle<float>(samg_ctx &);
template void outer_vcycle<double>(samg_ctx &);
template void relax<bf16>(samg_ctx &, int);
template void residual_restrict<bf16>(samg_ctx &, int);
template void interpolate<bf16>(samg_ctx &, int);
template void coarse_solve<bf16>(samg_ctx &);
template void vcycle<bf16>(samg_ctx &, int);
template void outer_vcycle<bf16>(samg_ctx &);

// ------------------------------------------------------------------ Ritz
// Sec. 4.3 on the finest level (B = I, C = I): Gram matrices, M = U^t A V
// through Cholesky factors, its SVD, U <- U R_U^-1 Y, V <- V R_V^-1 Z, and
// rho_j from A V_new = (A V) R_V^-1 Z, A^t U_new = (A^t U) R_U^-1 Y.
// identity = true keeps the triplets and only evaluates rho_j.
__global__ void k_identity(int ld, double *T) {
    int q = threadIdx.x;
    if (q < ld * ld) T[q] = (q / ld == q % ld) ? 1.0 : 0.0;
}

void ritz(samg_ctx &c, bool identity, bool check) {
    Level &L0 = c.L[0];
    const int ld = c.ld, nb = c.nb;
    cudaStream_t s = c.stream;
    Prof pr(c.prof, s, 4,
            identity ? 0.0
                     : 10.0 * ((double)L0.m + L0.n) * nb * 8.0 + 12.0 * (double)L0.A.nnz);
    const int64_t n = L0.n;
    const int64_t mu = c.spd() ? L0.n : L0.m;
    Term<double> none{};
    const bool square_form = !c.spd() && L0.m == L0.n && c.prm.square_form != 0;
    if (!identity && c.minimal() && !c.spd() && L0.m >= L0.n && c.prm.row_form == 0 &&
        !square_form) {
        // left basis A V (Rayleigh-Ritz for A^t A on span V): excludes the
        // null(A^t) modes that no relaxation or correction can remove
        launch_combine<double, double>(L0.m, ld, nullptr, 0.0,
                                       Term<double>{view<double>(L0.A), c.V.p, 1.0, false}, none,
                                       c.sigma.p, c.U.p, s);
    }
    if (c.spd()) {
        launch_combine<double, double>(L0.n, ld, nullptr, 0.0,
                                       Term<double>{view<double>(L0.A), c.U.p, 1.0, false}, none,
                                       c.sigma.p, c.AV.p, s);
    } else {
        launch_combine<double, double>(L0.m, ld, nullptr, 0.0,
                                       Term<double>{view<double>(L0.A), c.V.p, 1.0, false}, none,
                                       c.sigma.p, c.AV.p, s);
        launch_combine<double, double>(L0.n, ld, nullptr, 0.0,
                                       Term<double>{view<double>(L0.At), c.U.p, 1.0, false}, none,
                                       c.sigma.p, c.AtU.p, s);
    }
    if (identity) {
        SAMG_COUNT_LAUNCH();
        k_identity<<<1, 256, 0, s>>>(ld, c.TU.p);
        SAMG_COUNT_LAUNCH();
        k_identity<<<1, 256, 0, s>>>(ld, c.TV.p);
    } else {
        launch_gram(c.U.p, c.U.p, mu, nb, ld, c.GU.p, c.gwork.p, s);
        if (!c.spd()) launch_gram(c.V.p, c.V.p, n, nb, ld, c.GV.p, c.gwork.p, s);
        launch_gram(c.U.p, c.AV.p, mu, nb, ld, c.H.p, c.gwork.p, s);
        launch_ritz_small(c.GU.p, c.spd() ? c.GU.p : c.GV.p, c.H.p, nb, ld, c.spd(),
                          !c.minimal(), c.sigma.p, c.TU.p, c.TV.p, c.rstat.p, s);
    }
    launch_ritz_update(c.U.p, c.AV.p, c.TU.p, c.spd() ? c.TU.p : c.TV.p, c.sigma.p, mu, nb, ld,
                       c.Un.p, c.partu.p, s);
    if (!c.spd())
        launch_ritz_update(c.V.p, c.AtU.p, c.TV.p, c.TU.p, c.sigma.p, n, nb, ld, c.Vn.p,
                           c.partv.p, s);
    launch_ritz_resid(c.partu.p, mu, c.spd() ? nullptr : c.partv.p, n, nb, c.sigma.p,
                      c.resid.p, s);
    std::swap(c.U, c.Un);
    if (!c.spd()) std::swap(c.V, c.Vn);
    if (!identity && check) {
        int st = 0;
        SAMG_CUDA(cudaMemcpyAsync(&st, c.rstat.p, sizeof(int), cudaMemcpyDeviceToHost, s));
        SAMG_CUDA(cudaStreamSynchronize(s));
        SAMG_CHECK(st != 1, SAMG_E_INVALID, "ritz: boot vectors are linearly dependent");
    }
}

// ------------------------------------------------------------ hierarchy
void csr_identity(int n, HCsr &h) {
    h.m = h.n = n;
    h.rp.resize(n + 1);
    h.ci.resize(n);
    h.v.assign(n, 1.0);
    for (int i = 0; i <= n; ++i) h.rp[i] = i;
    for (int i = 0; i < n; ++i) h.ci[i] = i;
}

// A_{l+1} = P^t A_l Q, B_{l+1} = P^t B_l P, C_{l+1} = Q^t C_l Q (Eq. coarseOp)
// for every level whose P (and Q) are set; transposes P^t, Q^t.
void build_galerkin(samg_ctx &c) {
    cudaStream_t s = c.stream;
    for (int l = 0; l + 1 < c.nlev(); ++l) {
        Level &L = c.L[l];
        Level &Lc = c.L[l + 1];
        transpose(L.P, L.Pt, s);
        DCsr tmp, tmp2;
        if (c.spd()) {
            spgemm(L.A, L.P, tmp, s);
            spgemm(L.Pt, tmp, Lc.A, s);
            if (L.B.empty()) {
                spgemm(L.Pt, L.P, Lc.B, s);
            } else {
                spgemm(L.B, L.P, tmp2, s);
                spgemm(L.Pt, tmp2, Lc.B, s);
            }
            Lc.m = Lc.n = Lc.A.m;
            continue;
        }
        transpose(L.Q, L.Qt, s);
        spgemm(L.A, L.Q, tmp, s);
        spgemm(L.Pt, tmp, Lc.A, s);
        if (L.B.empty()) {
            spgemm(L.Pt, L.P, Lc.B, s);
        } else {
            spgemm(L.B, L.P, tmp2, s);
            spgemm(L.Pt, tmp2, Lc.B, s);
        }
        DCsr tmp3;
        if (L.C.empty()) {
            spgemm(L.Qt, L.Q, Lc.C, s);
        } else {
            spgemm(L.C, L.Q, tmp3, s);
            spgemm(L.Qt, tmp3, Lc.C, s);
        }
        Lc.m = Lc.A.m;
        Lc.n = Lc.A.n;
    }
}

template <typename T>
static void alloc_work(Work<T> &w, int m, int n, int ld, bool spd, cudaStream_t s) {
    size_t mu = (size_t)(spd ? n : m) * ld, nv = (size_t)n * ld;
    w.u.alloc(mu); w.k.alloc(mu); w.r.alloc(mu); w.tu.alloc(mu);
    w.u.zero(s); w.k.zero(s); w.r.zero(s); w.tu.zero(s);
    if (!spd) {
        w.v.alloc(nv); w.t.alloc(nv); w.s.alloc(nv); w.tv.alloc(nv);
        w.v.zero(s); w.t.zero(s); w.s.zero(s); w.tv.zero(s);
    }
}

// Per-level data used by the cycle: A^t, Kaczmarz schedules (minimal) or
// diagonals of B, C (dominant), and the work vectors.  Schedules already built
// for the same operator are kept.
void prepare_level(samg_ctx &c, int l) {
    cudaStream_t s = c.stream;
    Level &L = c.L[l];
    L.m = L.A.m;
    L.n = L.A.n;
    if (!c.spd() && L.At.m != L.A.n) transpose(L.A, L.At, s);
    if (c.minimal()) {
        if (L.kA.nbands == 0) {
            HCsr hA;
            download_csr(L.A, hA, s);
            if (c.spd()) {
                HCsr hB;
                if (L.B.empty()) csr_identity(L.n, hB);
                else download_csr(L.B, hB, s);
                build_kschedule(hA, &hB, L.kA, s);
            } else {
                HCsr hAt;
                download_csr(L.At, hAt, s);
                build_kschedule(hA, nullptr, L.kA, s);
                build_kschedule(hAt, nullptr, L.kAt, s);
            }
        }
        if (c.rstat.n >= 2) {
            L.kA.err = c.rstat.p + 1;
            L.kAt.err = c.rstat.p + 1;
        }
    } else {
        if (!L.B.empty()) launch_diagonal(L.B, L.dBd, L.dBf, s);
        if (!c.spd() && !L.C.empty()) launch_diagonal(L.C, L.dCd, L.dCf, s);
    }
    const size_t want = (size_t)(c.spd() ? L.n : L.m) * c.ld;
    if (L.wd.u.n != want) {
        alloc_work(L.wf, L.m, L.n, c.ld, c.spd(), s);
        alloc_work(L.wd, L.m, L.n, c.ld, c.spd(), s);
    }
}

// Coarsest level: X = [[0, A], [A^t, 0]], Y = diag(B, C) (SPD: A, B) and its
// generalized eigendecomposition X W = Y W Lam, W^t Y W = I.
void prepare_coarsest(samg_ctx &c) {
    c.co.warm = false;  // a new coarsest operator: start the pseudo-inverse afresh
    cudaStream_t s = c.stream;
    Level &Lc = c.L.back();
    Coarse &co = c.co;
    co.m1 = c.spd() ? Lc.n : Lc.m;
    co.M = c.spd() ? Lc.n : Lc.m + Lc.n;
    SAMG_CHECK(co.M <= 1280, SAMG_E_INVALID, "coarsest level larger than 1280");
    const size_t MM = (size_t)co.M * co.M;
    co.X.alloc(MM); co.Y.alloc(MM); co.W.alloc(MM); co.Wt.alloc(MM);
    co.lam.alloc(co.M); co.work.alloc(2 * MM); co.status.alloc(1);
    co.X.zero(s);
    co.Y.zero(s);
    HCsr hI;
    DCsr dI;
    auto fill_mass = [&](const DCsr &Bm, int n, int off) {
        if (!Bm.empty()) {
            dense_fill(Bm, off, off, co.M, co.Y.p, false, s);
        } else {
            csr_identity(n, hI);
            upload_csr(hI, dI, s);
            dense_fill(dI, off, off, co.M, co.Y.p, false, s);
        }
    };
    if (c.spd()) {
        dense_fill(Lc.A, 0, 0, co.M, co.X.p, false, s);
        fill_mass(Lc.B, Lc.n, 0);
    } else {
        dense_fill(Lc.A, 0, Lc.m, co.M, co.X.p, false, s);
        dense_fill(Lc.A, 0, Lc.m, co.M, co.X.p, true, s);
        fill_mass(Lc.B, Lc.m, 0);
        fill_mass(Lc.C, Lc.n, Lc.m);
    }
    launch_coarse_geneig(co.M, co.X.p, co.Y.p, co.work.p, co.lam.p, co.W.p, co.Wt.p,
                         co.status.p, s);
    int st = 0;
    SAMG_CUDA(cudaMemcpyAsync(&st, co.status.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    SAMG_CUDA(cudaStreamSynchronize(s));
    SAMG_CHECK(st == 0, SAMG_E_INVALID, "coarsest level: Y is not positive definite");
}

void finalize_hierarchy(samg_ctx &c) {
    for (int l = 0; l < c.nlev(); ++l) prepare_level(c, l);
    prepare_coarsest(c);
}

void alloc_finest_state(samg_ctx &c) {
    Level &L0 = c.L[0];
    const int ld = c.ld, nb = c.nb;
    cudaStream_t s = c.stream;
    size_t mu = (size_t)(c.spd() ? L0.n : L0.m) * ld, nv = (size_t)L0.n * ld;
    c.sigma.alloc(ld);
    c.resid.alloc(ld);
    c.U.alloc(mu); c.Un.alloc(mu); c.AV.alloc(mu);
    c.U.zero(s); c.Un.zero(s); c.AV.zero(s);
    if (!c.spd()) {
        c.V.alloc(nv); c.Vn.alloc(nv); c.AtU.alloc(nv);
        c.V.zero(s); c.Vn.zero(s); c.AtU.zero(s);
    }
    c.GU.alloc(256); c.GV.alloc(256); c.H.alloc(256); c.TU.alloc(256); c.TV.alloc(256);
    int64_t rows = std::max<int64_t>(c.spd() ? L0.n : L0.m, L0.n);
    c.gwork.alloc(gram_workspace(rows, nb));
    c.partu.alloc(gram_workspace(rows, 1) * nb + nb);
    c.partv.alloc(gram_workspace(rows, 1) * nb + nb);
    c.rstat.alloc(2);
    c.rstat.zero(s);
    std::vector<double> one(ld, 1.0);
    c.sigma.upload(one.data(), ld, s);
}

void put_block(samg_ctx &c, const double *h, int rows, DBuf<double> &d) {
    if (rows == 0) return;
    SAMG_CUDA(cudaMemcpy2DAsync(d.p, c.ld * sizeof(double), h, c.nb * sizeof(double),
                                c.nb * sizeof(double), rows, cudaMemcpyHostToDevice, c.stream));
}

void get_block(samg_ctx &c, const DBuf<double> &d, int rows, double *h) {
    if (rows == 0) return;
    SAMG_CUDA(cudaMemcpy2DAsync(h, c.nb * sizeof(double), d.p, c.ld * sizeof(double),
                                c.nb * sizeof(double), rows, cudaMemcpyDeviceToHost, c.stream));
}

}  // namespace samg
