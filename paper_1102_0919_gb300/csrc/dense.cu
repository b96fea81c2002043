// dense.cu -- float64 dense kernels of the Ritz step (Sec. 4.3) and of the
// coarsest-level solves (Secs. 3.6, 4.2).
#include <cmath>

#include "dense.cuh"
#include "kernels.cuh"

namespace samg {

// ====================================================================== Gram
// One CTA per GRAM_ROWS rows writes the partial sums of its rows; the final
// pass adds the partials in chunk order (a fixed order: the result is
// reproducible).  FP64 FMA latency on this part is long, so a thread keeps
// GRAM_ACC independent accumulators and the CTA's threads split the rows
// into groups, one group per (g, h) pair copy.
static constexpr int GRAM_ROWS = 2048;  // rows per CTA partial
static constexpr int GRAM_TILE = 64;    // rows staged in shared memory at a time
static constexpr int GRAM_ACC = 4;

size_t gram_workspace(int64_t rows, int nb) {
    int64_t chunks = (rows + GRAM_ROWS - 1) / GRAM_ROWS;
    return (size_t)std::max<int64_t>(chunks, 1) * nb * nb;
}

// partial[c][g][h] = sum over the chunk's rows of X[i][g] * Y[i][h]
__global__ void __launch_bounds__(256)
    k_gram_partial(const double *__restrict__ X, const double *__restrict__ Y, int64_t rows,
                   int nb, int ld, double *__restrict__ part) {
    __shared__ double sx[GRAM_TILE][17], sy[GRAM_TILE][17];
    __shared__ double red[256];
    const int t = threadIdx.x;
    const int pairs = nb * nb;
    const int groups = 256 / pairs;  // row groups (nb <= 16: at least 1)
    const int pr = t % pairs, grp = t / pairs;
    const int g = pr / nb, h = pr % nb;
    const bool act = grp < groups;
    double acc[GRAM_ACC];
#pragma unroll
    for (int a = 0; a < GRAM_ACC; ++a) acc[a] = 0.0;
    const int64_t r0 = (int64_t)blockIdx.x * GRAM_ROWS;
    const int64_t r1 = min(rows, r0 + GRAM_ROWS);
    for (int64_t rt = r0; rt < r1; rt += GRAM_TILE) {
        __syncthreads();
        for (int q = t; q < GRAM_TILE * 16; q += blockDim.x) {
            const int rr = q / 16, cc = q % 16;
            const int64_t row = rt + rr;
            const bool ok = row < r1 && cc < nb;
            sx[rr][cc] = ok ? X[row * ld + cc] : 0.0;
            sy[rr][cc] = ok ? Y[row * ld + cc] : 0.0;
        }
        __syncthreads();
        if (act) {
            // rows grp, grp + groups, ...; GRAM_ACC chains over them
            int k = 0;
            for (int rr = grp; rr < GRAM_TILE; rr += groups, ++k)
                acc[k % GRAM_ACC] = fma(sx[rr][g], sy[rr][h], acc[k % GRAM_ACC]);
        }
    }
    double v = 0.0;
#pragma unroll
    for (int a = 0; a < GRAM_ACC; ++a) v += acc[a];
    red[t] = act ? v : 0.0;
    __syncthreads();
    if (t < pairs) {
        double sum = 0.0;
        for (int q = 0; q < groups; ++q) sum += red[q * pairs + t];
        part[(size_t)blockIdx.x * pairs + t] = sum;
    }
}

// G[e] = sum over chunks of partial[c][e], one warp per entry e (lanes
// stride over the chunks, then a fixed shuffle tree)
__global__ void k_gram_final(const double *__restrict__ part, int chunks, int nb,
                             double *__restrict__ G) {
    const int lane = threadIdx.x & 31;
    const int e = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    if (e >= nb * nb) return;
    double a0 = 0.0, a1 = 0.0;
    int c = lane;
    for (; c + 32 < chunks; c += 64) {
        a0 += part[(size_t)c * nb * nb + e];
        a1 += part[(size_t)(c + 32) * nb * nb + e];
    }
    if (c < chunks) a0 += part[(size_t)c * nb * nb + e];
    double sum = a0 + a1;
    for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) G[e] = sum;
}

void launch_gram(const double *X, const double *Y, int64_t rows, int nb, int ld, double *G,
                 double *work, cudaStream_t s) {
    int chunks = (int)((rows + GRAM_ROWS - 1) / GRAM_ROWS);
    if (chunks == 0) {
        SAMG_CUDA(cudaMemsetAsync(G, 0, sizeof(double) * nb * nb, s));
        return;
    }
    SAMG_COUNT_LAUNCH();
    k_gram_partial<<<chunks, 256, 0, s>>>(X, Y, rows, nb, ld, work);
    SAMG_COUNT_LAUNCH();
    k_gram_final<<<(nb * nb + 7) / 8, 256, 0, s>>>(work, chunks, nb, G);
    SAMG_CUDA(cudaGetLastError());
}

// ================================================================ Ritz (small)
// Single-thread dense kernels for n_b <= 16: Cholesky, triangular inverse,
// one-sided (Hestenes) Jacobi SVD, cyclic Jacobi eigensolver.
// G = R^t R.  shift is added to the diagonal (0 for the plain factorization).
__device__ bool chol_upper(double *R, const double *G, int n, double shift = 0.0) {
    for (int i = 0; i < n * n; ++i) R[i] = 0.0;
    for (int j = 0; j < n; ++j) {
        double d = G[j * n + j] + shift;
        for (int k = 0; k < j; ++k) d -= R[k * n + j] * R[k * n + j];
        if (!(d > 1e-13 * (G[j * n + j] + shift))) return false;
        d = sqrt(d);
        R[j * n + j] = d;
        for (int i = j + 1; i < n; ++i) {
            double v = G[j * n + i];
            for (int k = 0; k < j; ++k) v -= R[k * n + j] * R[k * n + i];
            R[j * n + i] = v / d;
        }
    }
    return true;
}

__device__ void inv_upper(double *Ri, const double *R, int n) {  // Ri = R^-1 (upper)
    for (int i = 0; i < n * n; ++i) Ri[i] = 0.0;
    for (int j = 0; j < n; ++j) {
        Ri[j * n + j] = 1.0 / R[j * n + j];
        for (int i = j - 1; i >= 0; --i) {
            double v = 0.0;
            for (int k = i + 1; k <= j; ++k) v += R[i * n + k] * Ri[k * n + j];
            Ri[i * n + j] = -v / R[i * n + i];
        }
    }
}

// One-sided Jacobi: W (n x n, row-major) -> W Z with orthogonal columns.
__device__ void hestenes(double *W, double *Z, int n) {
    for (int i = 0; i < n * n; ++i) Z[i] = (i / n == i % n) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                double a = 0, b = 0, c = 0;
                for (int i = 0; i < n; ++i) {
                    a += W[i * n + p] * W[i * n + p];
                    b += W[i * n + q] * W[i * n + q];
                    c += W[i * n + p] * W[i * n + q];
                }
                if (c == 0.0) continue;
                double sc = fabs(c) / sqrt(a * b);
                off = fmax(off, sc);
                if (sc < 1e-17) continue;
                double zeta = (b - a) / (2.0 * c);
                double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
                for (int i = 0; i < n; ++i) {
                    double wp = W[i * n + p], wq = W[i * n + q];
                    W[i * n + p] = cs * wp - sn * wq;
                    W[i * n + q] = sn * wp + cs * wq;
                    double zp = Z[i * n + p], zq = Z[i * n + q];
                    Z[i * n + p] = cs * zp - sn * zq;
                    Z[i * n + q] = sn * zp + cs * zq;
                }
            }
        if (off < 1e-16) break;
    }
}

// Cyclic two-sided Jacobi for symmetric S (n x n): S -> diag, V eigenvectors.
__device__ void jacobi_eig(double *S, double *V, int n) {
    for (int i = 0; i < n * n; ++i) V[i] = (i / n == i % n) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < n; ++i)
            for (int k = 0; k < n; ++k) {
                tot += S[i * n + k] * S[i * n + k];
                if (i != k) off += S[i * n + k] * S[i * n + k];
            }
        if (off <= 1e-32 * tot) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                double apq = S[p * n + q];
                if (apq == 0.0) continue;
                double theta = (S[q * n + q] - S[p * n + p]) / (2.0 * apq);
                double t = copysign(1.0, theta) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {  // columns p, q
                    double skp = S[k * n + p], skq = S[k * n + q];
                    S[k * n + p] = c * skp - s * skq;
                    S[k * n + q] = s * skp + c * skq;
                }
                for (int k = 0; k < n; ++k) {  // rows p, q
                    double spk = S[p * n + k], sqk = S[q * n + k];
                    S[p * n + k] = c * spk - s * sqk;
                    S[q * n + k] = s * spk + c * sqk;
                }
                for (int k = 0; k < n; ++k) {
                    double vkp = V[k * n + p], vkq = V[k * n + q];
                    V[k * n + p] = c * vkp - s * vkq;
                    V[k * n + q] = s * vkp + c * vkq;
                }
            }
    }
}

// Inputs (device, row-major nb x nb): GU = U^t U, GV = V^t V, H = U^t A V
// (SPD: GU = X^t X, H = X^t A X).  Outputs: sigma (ld entries, padding 1),
// TU = R_U^-1 Y, TV = R_V^-1 Z (ld x ld, padding 0).  status[0] = 0 ok,
// 1 = Gram matrix not positive definite.
__global__ void k_ritz_small(const double *GU, const double *GV, const double *H, int nb, int ld,
                             int spd, int dominant, double *sigma, double *TU, double *TV,
                             int *status) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double RU[256], RV[256], RUi[256], RVi[256], M[256], Z[256], T1[256];
    double sv[16];
    int ord[16];
    const int n = nb;
    status[0] = 0;
    // Boot vectors that (nearly) coincide -- two members of a degenerate
    // cluster relaxed onto the same vector -- make a Gram matrix singular.
    // The basis is then taken from the factor of G + delta I, delta = 1e-12
    // max_j G_jj, which keeps n_b directions (the added one is the amplified
    // remainder of the dependent column) for the projection to sort out.
    auto factor = [&](double *R, const double *G) {
        if (chol_upper(R, G, n)) return true;
        double dmax = 0.0;
        for (int j = 0; j < n; ++j) dmax = fmax(dmax, G[j * n + j]);
        status[0] = 2;
        return chol_upper(R, G, n, 1e-12 * dmax);
    };
    if (!factor(RU, GU) || (!spd && !factor(RV, GV))) {
        status[0] = 1;
        return;
    }
    inv_upper(RUi, RU, n);
    if (spd) {
        for (int i = 0; i < n * n; ++i) { RV[i] = RU[i]; RVi[i] = RUi[i]; }
    } else {
        inv_upper(RVi, RV, n);
    }
    // M = RU^-t H RV^-1
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k) {
            double v = 0.0;
            for (int l = 0; l < n; ++l) v += H[i * n + l] * RVi[l * n + k];
            T1[i * n + k] = v;
        }
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k) {
            double v = 0.0;
            for (int l = 0; l < n; ++l) v += RUi[l * n + i] * T1[l * n + k];
            M[i * n + k] = v;
        }
    double *Y = T1;
    if (spd) {
        for (int i = 0; i < n; ++i)
            for (int k = 0; k < i; ++k) {
                double a = 0.5 * (M[i * n + k] + M[k * n + i]);
                M[i * n + k] = a;
                M[k * n + i] = a;
            }
        jacobi_eig(M, Y, n);  // eigenvalues on the diagonal of M, vectors in Y
        for (int j = 0; j < n; ++j) sv[j] = M[j * n + j];
        for (int i = 0; i < n * n; ++i) Z[i] = Y[i];
    } else {
        hestenes(M, Z, n);  // M <- Y Sigma, Z right vectors
        for (int j = 0; j < n; ++j) {
            double s2 = 0.0;
            for (int i = 0; i < n; ++i) s2 += M[i * n + j] * M[i * n + j];
            sv[j] = sqrt(s2);
            for (int i = 0; i < n; ++i) Y[i * n + j] = sv[j] > 0.0 ? M[i * n + j] / sv[j] : 0.0;
        }
    }
    // order: descending for dominant, ascending for minimal (stable)
    for (int j = 0; j < n; ++j) ord[j] = j;
    for (int a = 1; a < n; ++a) {
        int key = ord[a];
        int b = a - 1;
        while (b >= 0 && (dominant ? sv[ord[b]] < sv[key] : sv[ord[b]] > sv[key])) {
            ord[b + 1] = ord[b];
            --b;
        }
        ord[b + 1] = key;
    }
    for (int i = 0; i < ld * ld; ++i) { TU[i] = 0.0; TV[i] = 0.0; }
    for (int j = 0; j < ld; ++j) sigma[j] = 1.0;
    for (int jj = 0; jj < n; ++jj) {
        int j = ord[jj];
        sigma[jj] = sv[j];
        for (int i = 0; i < n; ++i) {
            double a = 0.0, b = 0.0;
            for (int l = 0; l < n; ++l) {
                a += RUi[i * n + l] * Y[l * n + j];
                b += RVi[i * n + l] * Z[l * n + j];
            }
            TU[i * ld + jj] = a;
            TV[i * ld + jj] = b;
        }
    }
}

void launch_ritz_small(const double *GU, const double *GV, const double *H, int nb, int ld,
                       bool spd, bool dominant, double *sigma, double *TU, double *TV,
                       int *status, cudaStream_t s) {
    SAMG_COUNT_LAUNCH();
    k_ritz_small<<<1, 32, 0, s>>>(GU, GV, H, nb, ld, spd ? 1 : 0, dominant ? 1 : 0, sigma, TU,
                                  TV, status);
    SAMG_CUDA(cudaGetLastError());
}

// Ritz update of one side: Xn = X T, AXn = W T2 (W = A x old other side),
// res[c][j] partial of |AXn_j - s_j Xn_j|^2 (deterministic per chunk).  The
// CTA's threads are ld columns x (256 / ld) row lanes.
__global__ void __launch_bounds__(256)
    k_ritz_update(const double *__restrict__ X, const double *__restrict__ W,
                  const double *__restrict__ T, const double *__restrict__ T2,
                  const double *__restrict__ sigma, int64_t rows, int nb, int ld,
                  double *__restrict__ Xn, double *__restrict__ part) {
    __shared__ double sT[256], sT2[256];
    __shared__ double red[256];
    for (int q = threadIdx.x; q < ld * ld && q < 256; q += blockDim.x) {
        sT[q] = T[q];
        sT2[q] = T2[q];
    }
    __syncthreads();
    const int lanes = 256 / ld;  // row lanes
    const int j = threadIdx.x % ld;
    const int rsub = threadIdx.x / ld;
    double acc0 = 0.0, acc1 = 0.0;
    const int64_t r0 = (int64_t)blockIdx.x * GRAM_ROWS;
    const int64_t r1 = min(rows, r0 + GRAM_ROWS);
    if (rsub < lanes) {
        int k = 0;
        for (int64_t i = r0 + rsub; i < r1; i += lanes, ++k) {
            double xn = 0.0, axn = 0.0;
            for (int l = 0; l < nb; ++l) {
                xn = fma(X[i * ld + l], sT[l * ld + j], xn);
                axn = fma(W[i * ld + l], sT2[l * ld + j], axn);
            }
            Xn[i * ld + j] = xn;
            if (j < nb) {
                const double r = axn - sigma[j] * xn;
                if (k & 1) acc1 = fma(r, r, acc1);
                else acc0 = fma(r, r, acc0);
            }
        }
    }
    red[threadIdx.x] = rsub < lanes ? acc0 + acc1 : 0.0;
    __syncthreads();
    if (threadIdx.x < nb) {
        double s = 0.0;
        for (int q = 0; q < lanes; ++q) s += red[q * ld + threadIdx.x];
        part[(size_t)blockIdx.x * nb + threadIdx.x] = s;
    }
}

__global__ void k_ritz_resid(const double *pu, int cu, const double *pv, int cv, int nb,
                             const double *sigma, double *resid) {
    int j = threadIdx.x;
    if (j >= nb) return;
    double a = 0.0, b = 0.0;
    for (int c = 0; c < cu; ++c) a += pu[(size_t)c * nb + j];
    for (int c = 0; c < cv; ++c) b += pv[(size_t)c * nb + j];
    resid[j] = sqrt(a + b) / fabs(sigma[j]);
}

void launch_ritz_update(const double *X, const double *W, const double *T, const double *T2,
                        const double *sigma, int64_t rows, int nb, int ld, double *Xn,
                        double *part, cudaStream_t s) {
    int chunks = (int)((rows + GRAM_ROWS - 1) / GRAM_ROWS);
    if (!chunks) return;
    SAMG_COUNT_LAUNCH();
    k_ritz_update<<<chunks, 256, 0, s>>>(X, W, T, T2, sigma, rows, nb, ld, Xn, part);
    SAMG_CUDA(cudaGetLastError());
}

void launch_ritz_resid(const double *pu, int64_t rows_u, const double *pv, int64_t rows_v,
                       int nb, const double *sigma, double *resid, cudaStream_t s) {
    int cu = (int)((rows_u + GRAM_ROWS - 1) / GRAM_ROWS);
    int cv = pv ? (int)((rows_v + GRAM_ROWS - 1) / GRAM_ROWS) : 0;
    SAMG_COUNT_LAUNCH();
    k_ritz_resid<<<1, 32, 0, s>>>(pu, cu, pv, cv, nb, sigma, resid);
    SAMG_CUDA(cudaGetLastError());
}

// ============================================================= coarsest level
// Dense X = [[0, A], [A^t, 0]], Y = diag(B, C) (SPD kind: X = A, Y = B).
__global__ void k_dense_fill(int rows, const int *rp, const int *ci, const double *v, int r_off,
                             int c_off, int Mdim, double *D, int transpose) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows) return;
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
        int r = r_off + i, c = c_off + ci[e];
        if (transpose) { int t = r; r = c; c = t; }
        D[(size_t)r * Mdim + c] = v[e];
    }
}

void dense_fill(const DCsr &a, int r_off, int c_off, int Mdim, double *D, bool transpose,
                cudaStream_t s) {
    if (!a.m) return;
    SAMG_COUNT_LAUNCH();
    k_dense_fill<<<(a.m + 127) / 128, 128, 0, s>>>(a.m, a.rp.p, a.ci.p, a.vd.p, r_off, c_off, Mdim,
                                                  D, transpose ? 1 : 0);
    SAMG_CUDA(cudaGetLastError());
}

__device__ __forceinline__ void cta_sync() { __syncthreads(); }

// One CTA: Y = L L^t; G = L^-1 X L^-t; Jacobi eig G = V Lam V^t (parallel
// round-robin pairs); W = L^-t V.  work: 2 M^2 doubles.  Outputs lam (M),
// W (M x M row-major), Wt (transpose).  status: 0 ok, 1 Y not SPD.
__global__ void k_coarse_geneig(int M, const double *X, const double *Yd, double *work,
                                double *lam, double *W, double *Wt, int *status) {
    double *L = work;          // M x M lower
    double *G = work + (size_t)M * M;
    __shared__ int s_bad;
    __shared__ double s_c[1024], s_s[1024];  // npair <= 1024 for M <= 2048
    __shared__ int s_p[1024], s_q[1024];
    __shared__ double s_off, s_tot;
    const int t = threadIdx.x, nt = blockDim.x;
    if (t == 0) s_bad = 0;
    for (size_t q = t; q < (size_t)M * M; q += nt) L[q] = 0.0;
    cta_sync();
    // Cholesky (column by column)
    for (int j = 0; j < M; ++j) {
        if (t == 0) {
            double d = Yd[(size_t)j * M + j];
            for (int k = 0; k < j; ++k) d -= L[(size_t)j * M + k] * L[(size_t)j * M + k];
            if (!(d > 0.0)) s_bad = 1;
            L[(size_t)j * M + j] = d > 0.0 ? sqrt(d) : 1.0;
        }
        cta_sync();
        const double djj = L[(size_t)j * M + j];
        for (int i = j + 1 + t; i < M; i += nt) {
            double v = Yd[(size_t)i * M + j];
            for (int k = 0; k < j; ++k) v -= L[(size_t)i * M + k] * L[(size_t)j * M + k];
            L[(size_t)i * M + j] = v / djj;
        }
        cta_sync();
    }
    if (s_bad) {
        if (t == 0) status[0] = 1;
        return;
    }
    // G = L^-1 X: forward substitution per column c (threads over columns)
    for (int c = t; c < M; c += nt)
        for (int i = 0; i < M; ++i) {
            double v = X[(size_t)i * M + c];
            for (int k = 0; k < i; ++k) v -= L[(size_t)i * M + k] * G[(size_t)k * M + c];
            G[(size_t)i * M + c] = v / L[(size_t)i * M + i];
        }
    cta_sync();
    // G <- G L^-t, i.e. solve Z L^t = G by rows (threads over rows), in place
    for (int r = t; r < M; r += nt)
        for (int i = 0; i < M; ++i) {
            double v = G[(size_t)r * M + i];
            for (int k = 0; k < i; ++k) v -= G[(size_t)r * M + k] * L[(size_t)i * M + k];
            G[(size_t)r * M + i] = v / L[(size_t)i * M + i];
        }
    cta_sync();
    // symmetrize
    for (size_t q = t; q < (size_t)M * M; q += nt) {
        int i = (int)(q / M), k = (int)(q % M);
        if (i < k) {
            double a = 0.5 * (G[(size_t)i * M + k] + G[(size_t)k * M + i]);
            G[(size_t)i * M + k] = a;
            G[(size_t)k * M + i] = a;
        }
    }
    // V = I  (use W as V)
    for (size_t q = t; q < (size_t)M * M; q += nt) W[q] = ((q / M) == (q % M)) ? 1.0 : 0.0;
    cta_sync();
    // parallel cyclic Jacobi with round-robin pairing (M padded to even)
    const int Me = M + (M & 1);
    const int npair = Me / 2;
    for (int sweep = 0; sweep < 40; ++sweep) {
        if (t == 0) { s_off = 0.0; s_tot = 0.0; }
        cta_sync();
        double lo = 0.0, lt = 0.0;
        for (size_t q = t; q < (size_t)M * M; q += nt) {
            double g = G[q];
            lt += g * g;
            if (q / M != q % M) lo += g * g;
        }
        atomicAdd(&s_off, lo);
        atomicAdd(&s_tot, lt);
        cta_sync();
        if (s_off <= 1e-30 * s_tot) break;
        for (int round = 0; round < Me - 1; ++round) {
            for (int k = t; k < npair; k += nt) {
                // round-robin: positions 0..Me-1, position 0 fixed
                int a = (k == 0) ? 0 : ((k - 1 + round) % (Me - 1)) + 1;
                int b = ((Me - 2 - k + round) % (Me - 1)) + 1;
                int p = min(a, b), q = max(a, b);
                double c = 1.0, s = 0.0;
                if (q < M && p != q) {
                    double apq = G[(size_t)p * M + q];
                    if (apq != 0.0) {
                        double th = (G[(size_t)q * M + q] - G[(size_t)p * M + p]) / (2.0 * apq);
                        double tt = copysign(1.0, th) / (fabs(th) + sqrt(th * th + 1.0));
                        c = 1.0 / sqrt(tt * tt + 1.0);
                        s = tt * c;
                    }
                }
                s_p[k] = p; s_q[k] = q; s_c[k] = c; s_s[k] = s;
            }
            cta_sync();
            // columns: G[:, p], G[:, q] and V[:, p], V[:, q]
            for (size_t w = t; w < (size_t)npair * M; w += nt) {
                int k = (int)(w / M), r = (int)(w % M);
                int p = s_p[k], q = s_q[k];
                if (q >= M || p == q) continue;
                double c = s_c[k], s = s_s[k];
                double gp = G[(size_t)r * M + p], gq = G[(size_t)r * M + q];
                G[(size_t)r * M + p] = c * gp - s * gq;
                G[(size_t)r * M + q] = s * gp + c * gq;
                double vp = W[(size_t)r * M + p], vq = W[(size_t)r * M + q];
                W[(size_t)r * M + p] = c * vp - s * vq;
                W[(size_t)r * M + q] = s * vp + c * vq;
            }
            cta_sync();
            // rows: G[p, :], G[q, :]
            for (size_t w = t; w < (size_t)npair * M; w += nt) {
                int k = (int)(w / M), r = (int)(w % M);
                int p = s_p[k], q = s_q[k];
                if (q >= M || p == q) continue;
                double c = s_c[k], s = s_s[k];
                double gp = G[(size_t)p * M + r], gq = G[(size_t)q * M + r];
                G[(size_t)p * M + r] = c * gp - s * gq;
                G[(size_t)q * M + r] = s * gp + c * gq;
            }
            cta_sync();
        }
    }
    for (int i = t; i < M; i += nt) lam[i] = G[(size_t)i * M + i];
    cta_sync();
    // W <- L^-t V : solve L^t W = V column by column (threads over columns)
    for (int c = t; c < M; c += nt)
        for (int i = M - 1; i >= 0; --i) {
            double v = W[(size_t)i * M + c];
            for (int k = i + 1; k < M; ++k) v -= L[(size_t)k * M + i] * W[(size_t)k * M + c];
            W[(size_t)i * M + c] = v / L[(size_t)i * M + i];
        }
    cta_sync();
    for (size_t q = t; q < (size_t)M * M; q += nt) {
        int i = (int)(q / M), k = (int)(q % M);
        Wt[(size_t)k * M + i] = W[q];
    }
    if (t == 0) status[0] = 0;
}

void launch_coarse_geneig(int M, const double *X, const double *Y, double *work, double *lam,
                          double *W, double *Wt, int *status, cudaStream_t s) {
    SAMG_COUNT_LAUNCH();
    k_coarse_geneig<<<1, 256, 0, s>>>(M, X, Y, work, lam, W, Wt, status);
    SAMG_CUDA(cudaGetLastError());
}

// Per column j (one CTA each): z = (X - s_j Y)^+ rhs without the smallest
// singular value.  With X W = Y W Lam, W^t Y W = I: S^-1 = W (Lam - s)^-1 W^t.
// The dropped singular vector w of the symmetric S (eigenvector of smallest
// |mu|) is found by subspace iteration on S^-1 with KB vectors started from
// the generalized eigenvectors nearest s_j, followed by a Rayleigh-Ritz step,
// so that near-ties among the smallest |mu| (degenerate singular values) are
// resolved.  Then z = S^-1 (r - w w^t r), projected once more against w.
// rhs/out: the first m1 rows from/for the first block, the rest from/for the
// second (SVD kind: [kappa; tau] -> [u; v]).
constexpr int KB = 4;

__device__ void small_sym_eig(double *H, double *V, int n) {  // thread-local Jacobi
    for (int i = 0; i < n * n; ++i) V[i] = (i / n == i % n) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 30; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) off += H[p * n + q] * H[p * n + q];
        if (off < 1e-300) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                double apq = H[p * n + q];
                if (apq == 0.0) continue;
                double th = (H[q * n + q] - H[p * n + p]) / (2.0 * apq);
                double t = copysign(1.0, th) / (fabs(th) + sqrt(th * th + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
                for (int k = 0; k < n; ++k) {
                    double a = H[k * n + p], b = H[k * n + q];
                    H[k * n + p] = c * a - sn * b;
                    H[k * n + q] = sn * a + c * b;
                }
                for (int k = 0; k < n; ++k) {
                    double a = H[p * n + k], b = H[q * n + k];
                    H[p * n + k] = c * a - sn * b;
                    H[q * n + k] = sn * a + c * b;
                }
                for (int k = 0; k < n; ++k) {
                    double a = V[k * n + p], b = V[k * n + q];
                    V[k * n + p] = c * a - sn * b;
                    V[k * n + q] = sn * a + c * b;
                }
            }
    }
}

template <typename T>
__global__ void k_coarse_apply(int M, int m1, int ld, const double *__restrict__ lam,
                               const double *__restrict__ W, const double *__restrict__ Wt,
                               const double *__restrict__ sigma, const T *__restrict__ k1,
                               const T *__restrict__ k2, T *__restrict__ o1, T *__restrict__ o2,
                               int nb, double *__restrict__ qwarm, int warm) {
    const int j = blockIdx.x;
    if (j >= nb) return;
    extern __shared__ double sm[];
    double *d = sm;               // M
    double *Q = d + M;            // KB x M
    double *Z = Q + KB * M;       // KB x M
    double *r = Z + KB * M;       // M
    double *y = r + M;            // M
    double *tq = y + M;           // KB x M (coefficients in the W basis)
    __shared__ double red[32];
    __shared__ double s_val;
    __shared__ double sH[KB * KB], sV[KB * KB];
    __shared__ int s_sel[KB];
    const int t = threadIdx.x, nt = blockDim.x;
    const double sj = sigma[j];
    auto bsum = [&](double v) -> double {
        for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((t & 31) == 0) red[t >> 5] = v;
        __syncthreads();
        if (t < 32) {
            double u = (t < (nt >> 5)) ? red[t] : 0.0;
            for (int o = 16; o; o >>= 1) u += __shfl_down_sync(0xffffffffu, u, o);
            if (t == 0) s_val = u;
        }
        __syncthreads();
        double res = s_val;
        __syncthreads();
        return res;
    };
    auto dot = [&](const double *a, const double *b) {
        double v = 0.0;
        for (int i = t; i < M; i += nt) v = fma(a[i], b[i], v);
        return bsum(v);
    };
    // Z[b] = S^-1 Q[b] for nq vectors (one pass over W^t and W for all of them)
    auto apply_inv = [&](const double *src, double *dst, int nq) {
        for (int k = t; k < M; k += nt) {
            double acc[KB] = {0.0, 0.0, 0.0, 0.0};
            for (int i = 0; i < M; ++i) {
                const double w = Wt[(size_t)k * M + i];
                for (int b = 0; b < nq; ++b) acc[b] = fma(w, src[b * M + i], acc[b]);
            }
            for (int b = 0; b < nq; ++b) tq[b * M + k] = d[k] * acc[b];
        }
        __syncthreads();
        for (int i = t; i < M; i += nt) {
            double acc[KB] = {0.0, 0.0, 0.0, 0.0};
            for (int k = 0; k < M; ++k) {
                const double w = W[(size_t)i * M + k];
                for (int b = 0; b < nq; ++b) acc[b] = fma(w, tq[b * M + k], acc[b]);
            }
            for (int b = 0; b < nq; ++b) dst[b * M + i] = acc[b];
        }
        __syncthreads();
    };
    auto orthonormalize = [&](double *B, int nq) {  // modified Gram-Schmidt
        for (int a = 0; a < nq; ++a) {
            for (int b = 0; b < a; ++b) {
                double pr = dot(B + a * M, B + b * M);
                for (int i = t; i < M; i += nt) B[a * M + i] -= pr * B[b * M + i];
                __syncthreads();
            }
            double nr = sqrt(dot(B + a * M, B + a * M));
            for (int i = t; i < M; i += nt) B[a * M + i] = nr > 0.0 ? B[a * M + i] / nr : 0.0;
            __syncthreads();
        }
    };
    const int kb = M < KB ? M : KB;
    for (int k = t; k < M; k += nt) {
        double den = lam[k] - sj;
        d[k] = den != 0.0 ? 1.0 / den : 1e300;
    }
    __syncthreads();
    if (t == 0) {  // the kb generalized eigenvectors nearest sigma_j
        for (int b = 0; b < kb; ++b) {
            int best = -1;
            double bv = -1.0;
            for (int k = 0; k < M; ++k) {
                bool used = false;
                for (int c2 = 0; c2 < b; ++c2) used = used || (s_sel[c2] == k);
                double a = fabs(d[k]);
                if (!used && a > bv) { bv = a; best = k; }
            }
            s_sel[b] = best;
        }
    }
    __syncthreads();
    // warm start: the two leading Ritz vectors of this column's previous call
    // (sigma_j moves little between outer iterations) replace the first two of
    // the nearest generalized eigenvectors
    const int nwarm = warm ? (kb < 2 ? kb : 2) : 0;
    for (int i = t; i < M; i += nt) {
        for (int b = 0; b < kb; ++b)
            Q[b * M + i] = b < nwarm ? qwarm[((size_t)j * 2 + b) * M + i] : W[(size_t)i * M + s_sel[b - nwarm]];
        r[i] = (i < m1) ? (double)to_acc(k1[(size_t)i * ld + j])
                        : (double)to_acc(k2[(size_t)(i - m1) * ld + j]);
    }
    __syncthreads();
    orthonormalize(Q, kb);
    double prev = 0.0;
    for (int it = 0; it < 60; ++it) {
        apply_inv(Q, Z, kb);
        // Rayleigh quotient of the leading direction, for the stopping test
        double th = 0.0;
        for (int b = 0; b < kb; ++b) {
            double v = dot(Q + b * M, Z + b * M);
            th = fmax(th, fabs(v));
        }
        for (int i = t; i < kb * M; i += nt) Q[i] = Z[i];
        __syncthreads();
        orthonormalize(Q, kb);
        if (it > 1 && fabs(th - prev) <= 1e-15 * th) break;
        prev = th;
    }
    // Rayleigh-Ritz on span(Q): H = Q^t S^-1 Q, pick the largest |1/mu|
    apply_inv(Q, Z, kb);
    for (int a = 0; a < kb; ++a)
        for (int b = 0; b < kb; ++b) {
            double v = dot(Q + a * M, Z + b * M);
            if (t == 0) sH[a * kb + b] = v;
        }
    __syncthreads();
    if (t == 0) {
        for (int a = 0; a < kb; ++a)
            for (int b = 0; b < a; ++b) {
                double v = 0.5 * (sH[a * kb + b] + sH[b * kb + a]);
                sH[a * kb + b] = v;
                sH[b * kb + a] = v;
            }
        small_sym_eig(sH, sV, kb);
        // Ritz values by decreasing |1/mu|: s_sel[0] picks w, s_sel[1] the next
        for (int a = 0; a < kb; ++a) s_sel[a] = a;
        for (int a = 0; a < kb; ++a)
            for (int b = a + 1; b < kb; ++b)
                if (fabs(sH[s_sel[b] * kb + s_sel[b]]) > fabs(sH[s_sel[a] * kb + s_sel[a]])) {
                    const int tmp = s_sel[a];
                    s_sel[a] = s_sel[b];
                    s_sel[b] = tmp;
                }
    }
    __syncthreads();
    // keep the two leading Ritz vectors as the next call's starting basis
    for (int i = t; i < M; i += nt)
        for (int a = 0; a < (kb < 2 ? kb : 2); ++a) {
            double v = 0.0;
            for (int b = 0; b < kb; ++b) v += Q[b * M + i] * sV[b * kb + s_sel[a]];
            qwarm[((size_t)j * 2 + a) * M + i] = v;
        }
    const int bsel = s_sel[0];
    double *w = y;  // reuse: w = Q sV[:, bsel]
    for (int i = t; i < M; i += nt) {
        double v = 0.0;
        for (int a = 0; a < kb; ++a) v += Q[a * M + i] * sV[a * kb + bsel];
        w[i] = v;
    }
    __syncthreads();
    double nw = sqrt(dot(w, w));
    for (int i = t; i < M; i += nt) w[i] /= nw;
    __syncthreads();
    // r' = r - w (w^t r);  z = S^-1 r';  z -= w (w^t z)
    double wr = dot(w, r);
    for (int i = t; i < M; i += nt) r[i] -= wr * w[i];
    __syncthreads();
    apply_inv(r, Z, 1);
    double wz = dot(w, Z);
    for (int i = t; i < M; i += nt) {
        double z = Z[i] - wz * w[i];
        if (i < m1) o1[(size_t)i * ld + j] = from_acc<T>((typename Acc<T>::T)z);
        else o2[(size_t)(i - m1) * ld + j] = from_acc<T>((typename Acc<T>::T)z);
    }
}

template <typename T>
void launch_coarse_apply(int M, int m1, int ld, int nb, const double *lam, const double *W,
                         const double *Wt, const double *sigma, const T *k1, const T *k2, T *o1,
                         T *o2, double *qwarm, int warm, cudaStream_t s) {
    size_t smem = (size_t)(4 + 3 * KB) * M * sizeof(double);
    auto kern = k_coarse_apply<T>;
    if (smem > 48 * 1024)
        SAMG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    SAMG_COUNT_LAUNCH();
    kern<<<nb, 256, smem, s>>>(M, m1, ld, lam, W, Wt, sigma, k1, k2, o1, o2, nb, qwarm, warm);
    SAMG_CUDA(cudaGetLastError());
}
size_t coarse_warm_size(int M, int nb) { return (size_t)nb * 2 * M; }

// Pass 1 of the generalized-eigen coarsest solve: warp w of the CTA owns
// row k of W^t; its lanes split the M-long dot products for all nb columns,
// then c[k, j] = (W^t r_j)_k / (lam_k - s_j), zero at k = k*_j.  Every CTA
// finds k*_j itself (an argmin over M values per column).
constexpr int CG_WARPS = 8;
template <typename T>
__global__ void __launch_bounds__(CG_WARPS * 32)
    k_coarse_geneig_c(int M, int m1, int ld, int nb, const double *__restrict__ lam,
                      const double *__restrict__ Wt, const double *__restrict__ sigma,
                      const T *__restrict__ k1, const T *__restrict__ k2, double *__restrict__ cbuf) {
    __shared__ int s_kstar[16];
    __shared__ double s_best[CG_WARPS][16];
    __shared__ int s_bidx[CG_WARPS][16];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // k*_j: nearest lam_k to s_j, lowest k on ties
    for (int j = 0; j < nb; ++j) {
        const double sj = sigma[j];
        double best = INFINITY;
        int bi = 0x7fffffff;
        for (int k = threadIdx.x; k < M; k += blockDim.x) {
            const double d = fabs(lam[k] - sj);
            if (d < best || (d == best && k < bi)) { best = d; bi = k; }
        }
        for (int o = 16; o; o >>= 1) {
            const double ob = __shfl_down_sync(0xffffffffu, best, o);
            const int oi = __shfl_down_sync(0xffffffffu, bi, o);
            if (ob < best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (lane == 0) { s_best[warp][j] = best; s_bidx[warp][j] = bi; }
    }
    __syncthreads();
    if (threadIdx.x < nb) {
        const int j = threadIdx.x;
        double best = s_best[0][j];
        int bi = s_bidx[0][j];
        for (int w = 1; w < CG_WARPS; ++w)
            if (s_best[w][j] < best || (s_best[w][j] == best && s_bidx[w][j] < bi)) {
                best = s_best[w][j];
                bi = s_bidx[w][j];
            }
        s_kstar[j] = bi;
    }
    __syncthreads();
    const int k = blockIdx.x * CG_WARPS + warp;
    if (k >= M) return;
    double acc[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) acc[j] = 0.0;
    const double *wrow = Wt + (size_t)k * M;
    for (int i = lane; i < M; i += 32) {
        const double w = wrow[i];
        const T *r = i < m1 ? k1 + (size_t)i * ld : k2 + (size_t)(i - m1) * ld;
#pragma unroll
        for (int j = 0; j < 16; ++j)
            if (j < nb) acc[j] = fma(w, (double)to_acc(r[j]), acc[j]);
    }
#pragma unroll
    for (int j = 0; j < 16; ++j)
        for (int o = 16; o; o >>= 1) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], o);
    if (lane < nb) {
        double v = 0.0;
#pragma unroll
        for (int j = 0; j < 16; ++j)
            if (j == lane) v = acc[j];
        const double den = lam[k] - sigma[lane];
        cbuf[(size_t)k * ld + lane] = (k == s_kstar[lane] || den == 0.0) ? 0.0 : v / den;
    }
}

// Pass 2: z = W c, warp w of the CTA owns row i of W.
template <typename T>
__global__ void __launch_bounds__(CG_WARPS * 32)
    k_coarse_geneig_z(int M, int m1, int ld, int nb, const double *__restrict__ W,
                      const double *__restrict__ cbuf, T *__restrict__ o1, T *__restrict__ o2) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i = blockIdx.x * CG_WARPS + warp;
    if (i >= M) return;
    double acc[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) acc[j] = 0.0;
    const double *wrow = W + (size_t)i * M;
    for (int k = lane; k < M; k += 32) {
        const double w = wrow[k];
        const double *c = cbuf + (size_t)k * ld;
#pragma unroll
        for (int j = 0; j < 16; ++j)
            if (j < nb) acc[j] = fma(w, c[j], acc[j]);
    }
#pragma unroll
    for (int j = 0; j < 16; ++j)
        for (int o = 16; o; o >>= 1) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], o);
    if (lane < nb) {
        double v = 0.0;
#pragma unroll
        for (int j = 0; j < 16; ++j)
            if (j == lane) v = acc[j];
        if (i < m1) o1[(size_t)i * ld + lane] = from_acc<T>((typename Acc<T>::T)v);
        else o2[(size_t)(i - m1) * ld + lane] = from_acc<T>((typename Acc<T>::T)v);
    }
}

template <typename T>
void launch_coarse_apply_geneig(int M, int m1, int ld, int nb, const double *lam,
                                const double *W, const double *Wt, const double *sigma,
                                const T *k1, const T *k2, T *o1, T *o2, double *cbuf,
                                cudaStream_t s) {
    SAMG_CHECK(nb >= 1 && nb <= 16 && ld >= nb, SAMG_E_INVALID, "coarse geneig: bad block width");
    const unsigned grid = (unsigned)((M + CG_WARPS - 1) / CG_WARPS);
    SAMG_COUNT_LAUNCH();
    k_coarse_geneig_c<T><<<grid, CG_WARPS * 32, 0, s>>>(M, m1, ld, nb, lam, Wt, sigma, k1, k2, cbuf);
    SAMG_CUDA(cudaGetLastError());
    SAMG_COUNT_LAUNCH();
    k_coarse_geneig_z<T><<<grid, CG_WARPS * 32, 0, s>>>(M, m1, ld, nb, W, cbuf, o1, o2);
    SAMG_CUDA(cudaGetLastError());
}
template void launch_coarse_apply_geneig<float>(int, int, int, int, const double *,
                                                const double *, const double *, const double *,
                                                const float *, const float *, float *, float *,
                                                double *, cudaStream_t);
template void launch_coarse_apply_geneig<double>(int, int, int, int, const double *,
                                                 const double *, const double *, const double *,
                                                 const double *, const double *, double *,
                                                 double *, double *, cudaStream_t);
template void launch_coarse_apply_geneig<bf16>(int, int, int, int, const double *, const double *,
                                               const double *, const double *, const bf16 *,
                                               const bf16 *, bf16 *, bf16 *, double *,
                                               cudaStream_t);
template void launch_coarse_apply<float>(int, int, int, int, const double *, const double *,
                                         const double *, const double *, const float *,
                                         const float *, float *, float *, double *, int,
                                         cudaStream_t);
template void launch_coarse_apply<double>(int, int, int, int, const double *, const double *,
                                          const double *, const double *, const double *,
                                          const double *, double *, double *, double *, int,
                                          cudaStream_t);
template void launch_coarse_apply<bf16>(int, int, int, int, const double *, const double *,
                                        const double *, const double *, const bf16 *, const bf16 *,
                                        bf16 *, bf16 *, double *, int, cudaStream_t);

}  // namespace samg
