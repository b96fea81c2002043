// coloured.cuh -- the coloured-order Kaczmarz variant of the solve phase's
// smoothing (not the paper's order, which is the natural one, Sec. 5.3).
//
// Each sweep of a smoothing phase visits its rows colour by colour: rows are
// coloured greedily in natural order (a row takes the smallest colour that no
// earlier row sharing an updated column has), so the rows of one colour
// share no updated column and their projections commute.  A colour class is
// then one fully parallel pass: each row reads its entries, forms its
// correction and writes its updated columns, with no ordering inside the
// class.  The classes run one kernel launch each, in order on the stream.
#pragma once

#include <vector>

#include "common.cuh"

namespace samg {

struct CSched {
    int rows = 0, cols = 0, mode = 0;  // mode 1: rows of A - s B; 2: fused relaxations
    int64_t nent = 0;
    std::vector<int> class_off;        // classes in program order: row ranges
    std::vector<int> class_lg;         // log2 lanes per row of each class
    int ncolour_max = 0;               // colours of the most coloured sweep
    int max_class_threads = 0;         // largest rows x lanes of one class
    DBuf<int> d_class_off, d_class_lg; // the classes on the device (one-CTA path)
    DBuf<int> rp, ci, rrow;            // permuted rows: entries, right-hand-side row
    DBuf<double> ad, bd, invd;         // coefficients (b: modes 1 and 2), 1/|a|^2
    DBuf<float> af, bf, invf;
};

// Greedy colouring of the rows of a CSR pattern in natural order (host):
// colour[i] = smallest c not used by an earlier row sharing a column with
// row i.  Returns the number of colours.
int greedy_row_colours(int rows, int cols, const std::vector<int64_t> &rp,
                       const std::vector<int> &ci, std::vector<int> &colour);

// The coloured program of count block Gauss-Seidel relaxations of the
// minimal SVD kind (mode 2, unknown [v; u], as the exact-order fused
// program) or of count stacked sweeps over the rows of A - s B (SPD kind,
// mode 1).  B, C: the level's mass matrices (identity on the finest level).
void build_cschedule_fused(const HCsr &A, const HCsr &At, const HCsr &B, const HCsr &C, int count,
                           CSched &cs, cudaStream_t s);
void build_cschedule_stacked(const HCsr &A, const HCsr &B, int count, CSched &cs, cudaStream_t s);

// Runs the program on x (cols x ld); rhs (program right-hand-side rows x ld);
// shift: ld device values.  A program whose every class fits COLOURED_CTA_ROWS
// row-lane slots runs as one launch of one CTA that steps through the
// classes with a CTA barrier between them; larger ones launch a grid per
// class.
template <typename T>
void launch_coloured(const CSched &cs, int ld, const T *rhs, T *x, const double *shift,
                     cudaStream_t s);

}  // namespace samg
