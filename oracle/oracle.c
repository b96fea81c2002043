/*
 * oracle.c -- plain, sequential FP64 loops of the CPU oracle for the
 * self-learning AMG triplet method (De Sterck, arXiv:1102.0919).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and
 * bench.py's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the GPU library.
 *
 * Every loop below runs in the paper's order, one row or point at a time,
 * with no blocking, reordering or fusion.  Vector blocks are row-major
 * (x[i*nb + j] is entry i of vector j).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------
 * SplitMix64 (Steele, Lea, Flood: "Fast splittable pseudorandom number
 * generators", OOPSLA 2014), used as a counter-based generator for the
 * random initial test vectors of Sec. 3.3.  Entry (row i, vector k) of a
 * block drawn with seed s is
 *     z = mix(s ^ (k << 40) ^ i)          (mix = one SplitMix64 output step)
 *     value = 2 * (z >> 11) * 2^-53 - 1   in [-1, 1).
 * ---------------------------------------------------------------------- */
static uint64_t splitmix64_output(uint64_t state)
{
    uint64_t z = state + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

void oracle_random_block(uint64_t seed, int64_t nrows, int32_t nvec, double *out)
{
    for (int64_t i = 0; i < nrows; ++i) {
        for (int32_t k = 0; k < nvec; ++k) {
            uint64_t z = splitmix64_output(seed ^ ((uint64_t)k << 40) ^ (uint64_t)i);
            double u01 = (double)(z >> 11) * (1.0 / 9007199254740992.0);
            out[i * nvec + k] = 2.0 * u01 - 1.0;
        }
    }
}

/* ------------------------------------------------------------------------
 * Kaczmarz sweep (Sec. 5.3; Tanabe's row-projection method) over the rows
 * of R_j = A - shift_j * B in natural order 0..nrows-1, for each of the nb
 * vectors independently:
 *     for i = 0..nrows-1:   d = (rhs_ij - r_i . x_j) / ||r_i||^2,
 *                           x_j += d * r_i^t
 * B (b_ptr == NULL means no B term) is merged with A row by row; both have
 * sorted column indices.  Rows with ||r_i|| = 0 are skipped.
 * ---------------------------------------------------------------------- */
void oracle_kaczmarz_sweep(int64_t nrows, int32_t nb,
                           const int64_t *a_ptr, const int32_t *a_col, const double *a_val,
                           const int64_t *b_ptr, const int32_t *b_col, const double *b_val,
                           const double *shift, const double *rhs, double *x)
{
    for (int64_t i = 0; i < nrows; ++i) {
        for (int32_t j = 0; j < nb; ++j) {
            double s = (b_ptr != NULL) ? shift[j] : 0.0;
            /* pass 1: r_i . x_j and ||r_i||^2 over the merged pattern */
            double dot = 0.0, nrm2 = 0.0;
            int64_t p = a_ptr[i], pe = a_ptr[i + 1];
            int64_t q = b_ptr ? b_ptr[i] : 0, qe = b_ptr ? b_ptr[i + 1] : 0;
            while (p < pe || q < qe) {
                int32_t c;
                double r = 0.0;
                if (q >= qe || (p < pe && a_col[p] < b_col[q])) {
                    c = a_col[p]; r = a_val[p]; ++p;
                } else if (p >= pe || b_col[q] < a_col[p]) {
                    c = b_col[q]; r = -s * b_val[q]; ++q;
                } else {
                    c = a_col[p]; r = a_val[p] - s * b_val[q]; ++p; ++q;
                }
                dot += r * x[(int64_t)c * nb + j];
                nrm2 += r * r;
            }
            if (nrm2 == 0.0)
                continue;
            double d = (rhs[i * nb + j] - dot) / nrm2;
            /* pass 2: x_j += d * r_i^t */
            p = a_ptr[i];
            q = b_ptr ? b_ptr[i] : 0;
            while (p < pe || q < qe) {
                int32_t c;
                double r = 0.0;
                if (q >= qe || (p < pe && a_col[p] < b_col[q])) {
                    c = a_col[p]; r = a_val[p]; ++p;
                } else if (p >= pe || b_col[q] < a_col[p]) {
                    c = b_col[q]; r = -s * b_val[q]; ++q;
                } else {
                    c = a_col[p]; r = a_val[p] - s * b_val[q]; ++p; ++q;
                }
                x[(int64_t)c * nb + j] += d * r;
            }
        }
    }
}

/* ------------------------------------------------------------------------
 * One-pass Ruge-Stueben coarsening (Sec. 3.7, Algorithm "coarsening").
 * Input: S_i = points that strongly influence i (CSR s_ptr/s_col, j != i).
 * lambda_i starts as the number of points strongly influenced by i; the loop
 * picks the undecided point with maximal lambda (ties: lowest index), makes
 * it C, makes the undecided points it strongly influences F, and increments
 * lambda of the undecided points that strongly influence those new F points.
 * Output cf[i] = 1 (C) or 0 (F).  The max-selection uses a binary heap keyed
 * on (lambda desc, index asc); it selects exactly the point the algorithm
 * names.  Returns 0, or -1 on allocation failure.
 * ---------------------------------------------------------------------- */
static int heap_before(const int64_t *lam, int32_t a, int32_t b)
{
    return lam[a] > lam[b] || (lam[a] == lam[b] && a < b);
}

static void heap_up(int32_t *heap, int32_t *pos, const int64_t *lam, int32_t k)
{
    while (k > 0) {
        int32_t parent = (k - 1) / 2;
        if (!heap_before(lam, heap[k], heap[parent]))
            break;
        int32_t t = heap[k]; heap[k] = heap[parent]; heap[parent] = t;
        pos[heap[k]] = k; pos[heap[parent]] = parent;
        k = parent;
    }
}

static void heap_down(int32_t *heap, int32_t *pos, const int64_t *lam, int32_t size, int32_t k)
{
    for (;;) {
        int32_t l = 2 * k + 1, r = l + 1, best = k;
        if (l < size && heap_before(lam, heap[l], heap[best])) best = l;
        if (r < size && heap_before(lam, heap[r], heap[best])) best = r;
        if (best == k)
            break;
        int32_t t = heap[k]; heap[k] = heap[best]; heap[best] = t;
        pos[heap[k]] = k; pos[heap[best]] = best;
        k = best;
    }
}

static void heap_remove(int32_t *heap, int32_t *pos, const int64_t *lam, int32_t *size, int32_t pt)
{
    int32_t k = pos[pt];
    int32_t last = heap[*size - 1];
    (*size)--;
    pos[pt] = -1;
    if (k == *size)
        return;
    heap[k] = last;
    pos[last] = k;
    heap_up(heap, pos, lam, k);
    heap_down(heap, pos, lam, *size, pos[last]);
}

int oracle_rs_coarsen(int32_t n, const int64_t *s_ptr, const int32_t *s_col, int32_t *cf)
{
    int64_t nnz = s_ptr[n];
    int64_t *st_ptr = calloc((size_t)n + 1, sizeof(int64_t));
    int32_t *st_col = malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int32_t));
    int64_t *fill = malloc((size_t)n * sizeof(int64_t));
    int64_t *lam = malloc((size_t)n * sizeof(int64_t));
    int32_t *heap = malloc((size_t)n * sizeof(int32_t));
    int32_t *pos = malloc((size_t)n * sizeof(int32_t));
    int8_t *state = malloc((size_t)n); /* 0 undecided, 1 C, 2 F */
    if (!st_ptr || !st_col || !fill || !lam || !heap || !pos || !state) {
        free(st_ptr); free(st_col); free(fill); free(lam); free(heap); free(pos); free(state);
        return -1;
    }
    /* S^t_i = points strongly influenced by i */
    for (int64_t e = 0; e < nnz; ++e)
        st_ptr[s_col[e] + 1]++;
    for (int32_t i = 0; i < n; ++i)
        st_ptr[i + 1] += st_ptr[i];
    for (int32_t i = 0; i < n; ++i)
        fill[i] = st_ptr[i];
    for (int32_t i = 0; i < n; ++i)
        for (int64_t e = s_ptr[i]; e < s_ptr[i + 1]; ++e)
            st_col[fill[s_col[e]]++] = i;
    for (int32_t i = 0; i < n; ++i) {
        lam[i] = st_ptr[i + 1] - st_ptr[i];
        state[i] = 0;
        heap[i] = i;
        pos[i] = i;
    }
    int32_t size = n;
    for (int32_t k = n / 2; k >= 0; --k)
        heap_down(heap, pos, lam, size, k);
    while (size > 0) {
        int32_t i = heap[0];
        heap_remove(heap, pos, lam, &size, i);
        state[i] = 1;
        for (int64_t e = st_ptr[i]; e < st_ptr[i + 1]; ++e) {
            int32_t j = st_col[e];
            if (state[j] != 0)
                continue;
            state[j] = 2;
            heap_remove(heap, pos, lam, &size, j);
        }
        for (int64_t e = st_ptr[i]; e < st_ptr[i + 1]; ++e) {
            int32_t j = st_col[e];
            if (state[j] != 2)
                continue;
            /* only the F points made in this step: they have pos == -1 and
             * were undecided a moment ago; mark them handled with state 3 */
            state[j] = 3;
            for (int64_t f = s_ptr[j]; f < s_ptr[j + 1]; ++f) {
                int32_t k = s_col[f];
                if (state[k] != 0)
                    continue;
                lam[k]++;
                heap_up(heap, pos, lam, pos[k]);
            }
        }
    }
    for (int32_t i = 0; i < n; ++i)
        cf[i] = (state[i] == 1) ? 1 : 0;
    free(st_ptr); free(st_col); free(fill); free(lam); free(heap); free(pos); free(state);
    return 0;
}

/* ------------------------------------------------------------------------
 * Weighted least-squares interpolation weights (Sec. 3.8, Eq. LS).
 * For every F point i with interpolatory set C^i (ci_ptr/ci_col, fine
 * indices of C points), solve
 *     min_p  sum_k w_k ( yF[i,k] - sum_{j in C^i} p_j * yC[j,k] )^2
 * through the normal equations (G^t W G) p = G^t W y with G_kj = yC[j,k],
 * by Cholesky.  yF holds the (possibly Jacobi-relaxed) F-point values, yC
 * the injected C-point values; both n x nf row-major.  If a Cholesky pivot
 * is not positive, the last (weakest) member of C^i is dropped and the fit
 * is repeated; its weight is returned as 0.
 * Output p_val aligned with ci_col.  Returns the number of rows that had to
 * drop members.
 * ---------------------------------------------------------------------- */
int64_t oracle_ls_fit(int32_t n, int32_t nf, const int64_t *ci_ptr, const int32_t *ci_col,
                      const double *yF, const double *yC, const double *w, double *p_val)
{
    int64_t dropped = 0;
    int32_t cap = 0;
    for (int32_t i = 0; i < n; ++i) {
        int32_t len = (int32_t)(ci_ptr[i + 1] - ci_ptr[i]);
        if (len > cap) cap = len;
    }
    double *N = malloc((size_t)(cap * cap + 2 * cap + 1) * sizeof(double));
    double *rhs = N + (size_t)cap * cap;
    double *sol = rhs + cap;
    for (int32_t i = 0; i < n; ++i) {
        int64_t b = ci_ptr[i];
        int32_t len = (int32_t)(ci_ptr[i + 1] - b);
        for (int32_t t = 0; t < len; ++t)
            p_val[b + t] = 0.0;
        int did_drop = 0;
        while (len > 0) {
            /* normal equations */
            for (int32_t r = 0; r < len; ++r) {
                for (int32_t c = 0; c < len; ++c) {
                    double acc = 0.0;
                    for (int32_t k = 0; k < nf; ++k)
                        acc += w[k] * yC[(int64_t)ci_col[b + r] * nf + k] *
                               yC[(int64_t)ci_col[b + c] * nf + k];
                    N[r * cap + c] = acc;
                }
                double acc = 0.0;
                for (int32_t k = 0; k < nf; ++k)
                    acc += w[k] * yC[(int64_t)ci_col[b + r] * nf + k] * yF[(int64_t)i * nf + k];
                rhs[r] = acc;
            }
            /* Cholesky N = L L^t in place (lower triangle) */
            int ok = 1;
            for (int32_t c = 0; c < len && ok; ++c) {
                double d = N[c * cap + c];
                for (int32_t k = 0; k < c; ++k)
                    d -= N[c * cap + k] * N[c * cap + k];
                if (!(d > 0.0)) { ok = 0; break; }
                d = sqrt(d);
                N[c * cap + c] = d;
                for (int32_t r = c + 1; r < len; ++r) {
                    double v = N[r * cap + c];
                    for (int32_t k = 0; k < c; ++k)
                        v -= N[r * cap + k] * N[c * cap + k];
                    N[r * cap + c] = v / d;
                }
            }
            if (!ok) {
                len -= 1;
                did_drop = 1;
                continue;
            }
            /* forward then backward substitution */
            for (int32_t r = 0; r < len; ++r) {
                double v = rhs[r];
                for (int32_t k = 0; k < r; ++k)
                    v -= N[r * cap + k] * sol[k];
                sol[r] = v / N[r * cap + r];
            }
            for (int32_t r = len - 1; r >= 0; --r) {
                double v = sol[r];
                for (int32_t k = r + 1; k < len; ++k)
                    v -= N[k * cap + r] * sol[k];
                sol[r] = v / N[r * cap + r];
            }
            for (int32_t t = 0; t < len; ++t)
                p_val[b + t] = sol[t];
            break;
        }
        dropped += did_drop;
    }
    free(N);
    return dropped;
}

/* ------------------------------------------------------------------------
 * Greedy row colouring for the coloured-order Kaczmarz variant (not the
 * paper's order, which is the natural one, Sec. 5.3).  Rows are taken in
 * natural order; row i gets the smallest colour c such that no earlier row
 * sharing a column with row i has colour c.  Rows of one colour then share
 * no column, so their Kaczmarz projections commute.  used[] keeps, per
 * column, the colours of the earlier rows touching it (bit c of word
 * c / 64).  Returns the number of colours, or -1 if more than 128 are
 * needed or memory runs out.
 * ---------------------------------------------------------------------- */
int32_t oracle_row_colours(int64_t nrows, int32_t ncols, const int64_t *rp, const int32_t *ci,
                           int32_t *colour)
{
    uint64_t *used = (uint64_t *)calloc((size_t)ncols * 2 + 1, sizeof(uint64_t));
    if (!used)
        return -1;
    int32_t ncolour = 0;
    for (int64_t i = 0; i < nrows; ++i) {
        uint64_t forbid[2] = {0, 0};
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
            forbid[0] |= used[2 * (int64_t)ci[e]];
            forbid[1] |= used[2 * (int64_t)ci[e] + 1];
        }
        int32_t c = 0;
        while (c < 128 && ((forbid[c / 64] >> (c % 64)) & 1u))
            ++c;
        if (c == 128) {
            free(used);
            return -1;
        }
        colour[i] = c;
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e)
            used[2 * (int64_t)ci[e] + c / 64] |= (uint64_t)1 << (c % 64);
        if (c + 1 > ncolour)
            ncolour = c + 1;
    }
    free(used);
    return ncolour;
}
