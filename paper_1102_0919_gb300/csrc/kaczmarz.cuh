// kaczmarz.cuh -- exact-order Kaczmarz sweeps (Sec. 5.3) on the GPU.
//
// A sweep projects x onto the hyperplanes r_i . x = b_i for i = 0 .. rows-1
// in natural row order.  Two rows commute exactly when they share no column,
// so the sweep is scheduled without changing its result:
//  * rows are cut into contiguous bands; inside a band every row gets a level
//    = 1 + the level of the latest earlier in-band row that shares a column,
//    and the rows of one level (disjoint columns) are updated in parallel;
//  * a band that touches a column last written by an earlier band waits until
//    that band has published the level of its last touch (bounded spin on a
//    progress word; a timeout sets an error flag and the kernel returns);
//  * values of columns touched more than once inside a band live in a
//    shared-memory window slot between their first and last touch; the first
//    touch loads from global memory, the last touch stores to it.
// Bands are handed out in increasing order by an atomic ticket, so a band only
// ever waits for bands that are already running or finished.
#pragma once

#include "common.cuh"

namespace samg {

struct KCtl {                 // device control block of one schedule
    unsigned long long epoch;  // launch counter (progress words carry it)
    unsigned int ticket;
    unsigned int done;
    int err;                   // 1 = a wait timed out
    int pad;
};

struct KSched {
    int rows = 0, cols = 0, nbands = 0, nlevels = 0, nchunks = 0;
    int max_slots = 0;
    int64_t nent = 0;
    bool shifted = false;      // rows of A - shift_j B (SPD kind)
    DBuf<int> band_chunk;      // nbands + 1: first staging chunk of each band
    DBuf<int4> chunk;          // 2 per chunk: {L0, L1, R0, R1}, {E0, E1, X0, X1}
    DBuf<int4> lvl;            // nlevels + 1: {first sched row, first req, publish, 0}
    DBuf<int2> rinfo;          // scheduled row -> {original row, first entry} (+ sentinel)
    DBuf<int2> ent;            // {column, 1 first | 2 last | 4 staged | slot << 3 | xs << 15}
    DBuf<int> xsc;             // per chunk: columns whose first values are staged
    DBuf<double> ea_d, eb_d;   // entry coefficients (a; b for the shifted form)
    DBuf<float> ea_f, eb_f;
    DBuf<double> inv_d;        // 1 / ||r_i||^2 per scheduled row (unshifted form)
    DBuf<float> inv_f;
    DBuf<int2> req;            // {band, level that band must have completed}
    DBuf<unsigned long long> progress;  // nbands
    DBuf<KCtl> ctl;
    mutable int grid_cache[256] = {};  // resident CTAs per kernel instance
    int *err = nullptr;        // error word shared by a context's schedules
                               // (null: the schedule's own ctl->err)
};

// Build the schedule of the rows of A (shift form when B != nullptr: rows of
// A - s B over the union pattern).  Host CSR inputs.
void build_kschedule(const HCsr &A, const HCsr *B, KSched &ks, cudaStream_t s);

// One sweep: x (cols x ld) updated in place; rhs (rows x ld) or null for 0;
// shift: ld device values (shifted form).  Returns after queuing the kernel.
template <typename T>
void launch_kaczmarz(const KSched &ks, int ld, const T *rhs, T *x, const double *shift,
                     cudaStream_t s);

// Reads the error flag (synchronizes the stream); throws SAMG_E_TIMEOUT if set.
void kaczmarz_check(const KSched &ks, cudaStream_t s);

}  // namespace samg
