// kaczmarz.cuh -- exact-order Kaczmarz sweeps (Sec. 5.3) on the GPU.
//
// A sweep projects x onto the hyperplanes r_i . x = b_i for i = 0 .. rows-1
// in natural row order.  Two rows commute exactly when they share no column,
// so the sweep is scheduled without changing its result:
//  * every row gets a global level = 1 + the level of the latest earlier row
//    that shares a column; rows are cut into contiguous bands, a row's band
//    level is the rank of its global level inside its band, and the rows of
//    one level (disjoint columns) are updated in parallel;
//  * a band that touches a column last written by an earlier band waits until
//    that band has published the level of its last touch (bounded spin on a
//    progress word; a timeout sets an error flag and the kernel returns);
//  * values of columns touched more than once inside a band live in a
//    shared-memory window slot between their first and last touch; the first
//    touch loads from global memory (staged ahead by the producer warp when no
//    earlier band writes the column), the last touch stores to it;
//  * a band's levels are packed into chunks whose schedules are copied to
//    shared memory by bulk copies a producer warp issues ahead of the compute
//    warps.
// Bands are handed out in increasing order by an atomic ticket, so a band only
// ever waits for bands that are already running or finished.
#pragma once

#include <vector>

#include "common.cuh"

namespace samg {

struct KCtl {                 // device control block of one schedule
    unsigned long long epoch;  // launch counter (progress words carry it)
    unsigned int ticket;
    unsigned int done;
    int err;                   // 1 = a wait timed out
    int mute;                  // band that never publishes its progress (testing the
                               // bounded waits); -1 = none
};

// One staging chunk: up to 32 levels of one band whose rows, entries and
// staged first values fit one shared-memory buffer.  Its schedule is a
// self-contained image (chunk-local row and entry numbers), one per
// coefficient precision, copied to shared memory in one bulk copy.
struct KChunk {
    int L0, nl;                // first (global) level, levels
    int nr, ne, nx;            // rows, entries, staged first values
    int bytes_f, bytes_d;      // image sizes (multiples of 16)
    int nq;                    // cross-band requirements carried in the image
    long long off_f, off_d;    // image byte offsets (multiples of 16)
};

struct KSched {
    int rows = 0, cols = 0, nbands = 0, nlevels = 0, nchunks = 0;
    int max_slots = 0;
    int64_t nent = 0;
    bool shifted = false;      // entries carry b coefficients (modes 1 and 2)
    int mode = 0;              // 0 rows of A; 1 rows of A - s_j B; 2 fused relaxations
    DBuf<int> band_chunk;      // nbands + 1: first staging chunk of each band
    DBuf<KChunk> chunk;
    DBuf<int4> lvl;            // per level: {first req, requirement count, publish, 0}
    DBuf<unsigned char> img_f, img_d;  // chunk images, float / double coefficients
    DBuf<int2> req;            // {band, level that band must have completed}
    DBuf<int> order;           // nbands: the band each ticket claims
    DBuf<unsigned long long> progress;  // nbands
    DBuf<KCtl> ctl;
    mutable int grid_cache[256] = {};  // resident CTAs per kernel instance
    int *err = nullptr;        // error word shared by a context's schedules
                               // (null: the schedule's own ctl->err)
};

// The host side of a schedule, before upload (same arrays as KSched).
struct HostSched {
    int rows = 0, cols = 0, nbands = 0, nlevels = 0, nchunks = 0, max_slots = 0;
    int64_t nent = 0;
    bool shifted = false;
    int mode = 0;
    std::vector<int> band_chunk;
    std::vector<KChunk> chunk;
    std::vector<int4> lvl;
    std::vector<unsigned char> img_f, img_d;
    std::vector<int2> req;
    std::vector<int> order;    // ticket -> band
};

// Host-only: the schedule, as the kernels receive it, of one sweep over the
// rows of A (fused_count 0, mode 0), of the fused program of fused_count
// minimal-SVD relaxations with the level's B and C (mode 2), or, with spd,
// of max(1, fused_count) stacked sweeps over the rows of A - s B (mode 1).
// B, C null: identity.  The same pattern builders as the solve's.
// resident_cap > 0 (at most 4095): a program that keeps at most that many
// columns live is built as one band with every column resident (a mode the
// solve does not use yet).  band_rows: rows per level a band grows to (0:
// 32).  slot_cap: live columns per band (0: 512).
void host_schedule(const HCsr &A, const HCsr *B, const HCsr *C, int fused_count, bool spd,
                   HostSched &h, int resident_cap = 0, int band_rows = 0, int slot_cap = 0);

// Build the schedule of the rows of A (shift form when B != nullptr: rows of
// A - s B over the union pattern).  Host CSR inputs.
void build_kschedule(const HCsr &A, const HCsr *B, KSched &ks, cudaStream_t s);

// count sweeps over the rows of A - s B in sequence (SPD kind): one program,
// so a sweep's rows start as soon as the rows they depend on are done.
void build_kschedule_stacked(const HCsr &A, const HCsr &B, int count, KSched &ks, cudaStream_t s,
                             int ld = 0, bool wide = true, int band_rows = 0);

// count block Gauss-Seidel relaxations of the minimal SVD kind as one
// program over the unknown [v; u] (n + m rows of ld values): per relaxation
// the rows of A (v updated, s_j B u read, right-hand side kappa_i) and then
// the rows of A^t (u updated, s_j C v read, right-hand side tau_j); the
// right-hand side block is [kappa; tau] (m + n rows).  The order of every
// row's updates is that of the sequential relaxations.
// Both builders band the program with kz_window_cap(ld, mode, wide) live
// columns and about band_rows rows per level (0: 32).  wide: the schedule
// serves float64 launches too; otherwise only float32 windows (float32 and
// bfloat16 storage), which hold more columns.
void build_kschedule_fused(const HCsr &A, const HCsr &At, const HCsr &B, const HCsr &C, int count,
                           KSched &ks, cudaStream_t s, int ld = 0, bool wide = true,
                           int band_rows = 0);

// The largest window (live columns per band) whose launch fits a CTA's
// shared memory at block width ld (at least 512): for float64 and float32
// windows (wide), or float32 windows only.
int kz_window_cap(int ld, int mode, bool wide = true);


// One sweep: x (cols x ld) updated in place; rhs (rows x ld) or null for 0;
// shift: ld device values (shifted form).  Returns after queuing the kernel.
template <typename T>
void launch_kaczmarz(const KSched &ks, int ld, const T *rhs, T *x, const double *shift,
                     cudaStream_t s);

// Host-only analysis of a sweep program (no device work): the global
// dependency level of every row and the number of bands.  fused_count = 0:
// one sweep over the rows of A; >= 1: the fused program of that many
// minimal-SVD relaxations with B = I, C = I (rows: per relaxation the m rows
// of A, then the n rows of A^t).
void plan_sweep(const HCsr &A, int fused_count, std::vector<int> &levels, int *nbands);

// Test hook: the given band (-1: none) never publishes its progress, so later
// bands that need it give up after their bounded wait.
void kaczmarz_mute_band(KSched &ks, int band, cudaStream_t s);

// Reads the error flag (synchronizes the stream); throws SAMG_E_TIMEOUT if set.
void kaczmarz_check(const KSched &ks, cudaStream_t s);

}  // namespace samg
