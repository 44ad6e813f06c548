// internal.h -- host-side interfaces between the translation units of libcmg.
#pragma once

#include "common.cuh"

namespace cmg {

// Lanes per CSR row for a level of average row length `avg` (1..32, power of 2).
int lanes_for_avg(double avg);

// ---------------------------------------------------------------- hec.cu
// Alg. 2 on one level: heaviest neighbours, visit ranks (Feistel keyed by
// seed/level unless `rank` is given), round-based resolution and labelling.
// agg_out: device int32[n].  *c_host receives the aggregate count.
cmg_status_t hec_level(int n, long long nnz, const int *rp, const int *col, const double *w,
                       uint64_t seed, int level, const uint32_t *rank, int *agg_out, int *c_host,
                       cudaStream_t s);
// The same without host synchronisation: c to *c_dev, barrier state to *gs.
cmg_status_t hec_level_async(int n, long long nnz, const int *rp, const int *col, const double *w,
                             uint64_t seed, int level, const uint32_t *rank, int *agg_out,
                             int *c_dev, GridSync *gs, cudaStream_t s);
// avg = average row length (chooses the lanes per row).
cmg_status_t launch_heaviest(int n, double avg, const int *rp, const int *col, const double *w,
                             int *m, cudaStream_t s);
cmg_status_t launch_ranks(int n, uint64_t seed, int level, uint32_t *r, cudaStream_t s);
// Ranks of a block-diagonal union of G graphs with vertex offsets voff (device).
cmg_status_t launch_ranks_batch(int n, int G, const int *voff, uint64_t seed, int level, uint32_t *r,
                                cudaStream_t s);

// ---------------------------------------------------------------- primitives.cu
// Exclusive scan of int32 in[0..n) into out[0..n]; out[n] = total (device).
cmg_status_t exclusive_scan(const int *in, int *out, int n, Scratch &scr, cudaStream_t s);
// Stable LSD radix sort of (key, val) by the low `bits` bits of key; the item
// count is read from device memory (count_dev) and is at most `cap`, the
// buffers' capacity.  On return *keys / *vals point at the sorted arrays
// (one of the two buffers).
cmg_status_t radix_sort_pairs(uint64_t **keys, uint32_t **vals, uint64_t *keys_alt,
                              uint32_t *vals_alt, int cap, const int *count_dev, int bits,
                              Scratch &scr, cudaStream_t s);

// ---------------------------------------------------------------- galerkin.cu
// Option checks shared by the single-graph and batched setup.
cmg_status_t check_options(const cmg_options_t &o);
// Level 0 of a hierarchy: copies the CSR (host or device, int64 row pointers)
// into new device arrays (int32 row pointers) and, with `validate`, checks
// the input contract of cmg_setup.  The arrays belong to the caller as soon
// as they are allocated, also when an error is returned.
cmg_status_t load_level0(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *w,
                         int32_t mem, int validate, int **rp_out, int **col_out, double **w_out,
                         long long *nnz_out, cudaStream_t s);
// w32[k] = (float)w[k].
cmg_status_t launch_to_float(long long m, const double *w, float *w32, cudaStream_t s);

// Sweep layout of a level, per graph (built at setup): rows renumbered by
// decreasing degree (stable); the rows with more than kHeavy entries come
// first and keep CSR form ("heavy" rows), the others form slices of 32 rows
// whose entries are interleaved -- entry k of the slice's row l sits at
// slice_offset + 32 k + l, shorter rows padded with weight 0 -- so a warp
// reads a slice with coalesced loads that do not depend on each other.
// Columns are renumbered local ids (16-bit when every graph of the level
// has at most 65536 vertices).  meta of a graph: the entry offsets (local to
// the graph) of its h heavy rows, then of its nsl slices, then the end.
#ifndef CMG_HEAVY_ROW
#define CMG_HEAVY_ROW 128
#endif
constexpr int kHeavy = CMG_HEAVY_ROW;

struct SweepLayout {
    uint32_t *perm = nullptr;   // new position -> original vertex (union numbering)
    int *inv = nullptr;         // original vertex -> new position
    int *heavy = nullptr;       // [G] heavy rows per graph
    int *eoff = nullptr;        // [G+1] first layout entry of each graph
    int *moff = nullptr;        // [G+1] first meta word of each graph
    int *meta = nullptr;        // per graph: offsets of h heavy rows, nsl slices, end
    void *bcol = nullptr;       // uint16 (col16) or int32 local columns
    void *bw = nullptr;         // weights in the sweep precision
    int col16 = 1;
    long long entries = 0;
    std::vector<int> hecnt, hmcnt, hheavy;   // per graph, host copies
    // single-graph layouts: heavy rows (stored padded to a multiple of 8
    // entries) cut into chunks of at most kHeavyChunk entries
    int *hchunk = nullptr;      // [h+1] first chunk of each heavy row
    int *crow = nullptr;        // [nchunks] heavy row of each chunk
    int *hcount = nullptr;      // [h] chunks finished (zeroed per launch)
    void *cpart = nullptr;      // [nchunks] chunk partial sums (sweep precision)
    int nchunks = 0;
    // single-graph layouts: iterate entries the slice kernel stages in shared
    // memory per sweep (0: none)
    int stage_n = 0;
};
constexpr int kHeavyChunk = 2048;
// Builds the layout of the N rows of a level holding G graphs at union
// offsets voff (device, G+1; host copy hvoff) from the level's CSR; fp32
// selects float weights.  Adds its device bytes to *bytes (nullable).
// perm_only: only the row order (perm, inv), for a level swept through its
// two-phase layout (no heavy rows, slices or entries).
cmg_status_t build_sweep_layout(int G, const int *voff, const std::vector<int> &hvoff, int N,
                                const int *rp, const int *col, const double *w, int fp32,
                                SweepLayout *L, size_t *bytes, cudaStream_t s, bool perm_only = false);
void free_sweep_layout(SweepLayout &L, cudaStream_t s);

// Two-phase sweep layout of a large single-graph level whose gathers have no
// locality.  Rows and columns are in the sweep layout's order (perm).  A sweep
// y = B_g x runs in T passes; pass t owns a contiguous range of rows (about
// nnz / T entries) and takes two phases:
//   phase 1: the columns are cut into source blocks of SB vertices; CTA b
//     copies the source blocks its share of the pass's stream needs into
//     shared memory and writes x_c of every entry into xbuf, at the entry's
//     position in list order -- the stream is ordered (source block, dest
//     block, row, CSR position), so its writes are runs ("cells": one source
//     block's entries of one dest block) that are contiguous in both orders;
//   phase 2 (after a grid barrier): the pass's rows are cut into a multiple
//     of P dest blocks (one or more per CTA); the CTA streams its block's
//     list -- (row offset, weight, x_c) at consecutive positions -- and adds
//     each term into a 64-bit fixed-point accumulator of its row in shared
//     memory (integer adds commute, so every order gives the same sums).
// Every global access is contiguous; the random accesses are to shared
// memory only; the sums are exact up to one rounding per term.
struct XLayout {
    int P = 0, T = 0, Q = 0, SB = 0, VMAX = 0;
    long long entries = 0;
    int ncells = 0;
    int nblocks = 0;              // dest blocks over all passes
    size_t smem = 0;              // dynamic shared memory of the sweep kernel
    long long xcap = 0;           // elements of each of the two xbufs
    uint16_t *src = nullptr;      // phase-1 stream, pass t from sal[t] on: column - block start
    uint16_t *dst = nullptr;      // [entries] list order: row - first row of its dest block
    void *w = nullptr;            // [entries] list order: weights in the sweep precision
    int *pass_s = nullptr;        // [T + 1] first entry of each pass (both orders)
    int *sal = nullptr;           // [T + 1] first element of each pass's stream in src (multiples of 8)
    int *qoff = nullptr;          // [T*(Q+1)] stream offset of each source block within its pass
    int *ndb = nullptr;           // [T + 1] first dest block of each pass
    int *dbr = nullptr;           // [nblocks + 1] first row of each dest block
    int *dbl = nullptr;           // [nblocks + 1] first list entry of each dest block
    int *cdel = nullptr;          // [ncells] list position - stream position of each cell's entries
    int *choff = nullptr;         // [T + 1] first chunk of each pass
    uint2 *chk = nullptr;         // [nchunks] per 32-entry stream chunk: its first entry's cell,
                                  // and bit l (1..31) set where entry l starts a cell
    int nchunks = 0;
    double *pmax = nullptr;       // [2][P] per-CTA max |x| of the sweeps' iterates
    void *xbuf[2] = {nullptr, nullptr};
};
// Knobs of the two-phase layout (0: default).
struct XParams {
    int sb = 0;                   // source block vertices
    long long xcap_bytes = 0;     // bytes of each xbuf (sets the pass count)
};
// Builds it from the level's CSR (original ids) and the sweep layout's row
// order; fp32 selects float weights.  P = the SM count.  Returns
// CMG_ERR_TOO_LARGE when the level does not fit the layout's limits (the
// caller then uses the slice layout).  Adds its device bytes to *bytes.
cmg_status_t build_xlayout(int n, long long nnz, const int *rp, const int *col, const double *w, int fp32,
                           const uint32_t *perm, const int *inv, const XParams &prm, XLayout *X,
                           size_t *bytes, cudaStream_t s);
void free_xlayout(XLayout &X, cudaStream_t s);
// Dynamic shared memory of the two-phase sweep kernel (FP32 or FP64 sweeps).
size_t xsweep_smem(int fp32);
// Adds to *out (zeroed first) the layout entries whose column is below S.
cmg_status_t layout_count_below(const SweepLayout &L, int S, unsigned long long *out, cudaStream_t s);
// Iterate entries the staged slice kernel can hold in shared memory (FP32 or
// FP64 sweeps).
int stage_capacity(int fp32);
// Staging pays when the staged prefix serves nearly all gathers of a sweep
// (`below` of the layout's `entries`; the large shared-memory carve-out
// leaves little L1 for the other gathers and for loads in flight) and a sweep
// holds enough gathers per SM to repay the copy.
inline bool stage_pays(unsigned long long below, long long entries, int sms) {
    return entries >= 16384ll * sms && below * 10ull >= (unsigned long long)entries * 9ull;
}
// FP32 sweeps of a level the rule above leaves unstaged: a short prefix of
// kPartialStage entries leaves most of L1 to the other gathers and pays when
// it serves at least 3 times its share of the rows (`below` of `entries`
// gathers for kPartialStage of n rows): the hub columns of a power-law
// level, not the even columns of a grid level.
constexpr int kPartialStage = 32768;
inline bool partial_stage_pays(unsigned long long below, long long entries, int n, int sms) {
    return entries >= 16384ll * sms && n > 2 * kPartialStage &&
           (double)below * (double)n >= 3.0 * (double)kPartialStage * (double)entries;
}

// Bits needed for the ids 0..c-1 (at least 1).
inline int bits_for(int c) {
    int b = 1;
    while ((1ll << b) < (long long)c) b++;
    return b;
}

// Device-side sizes of one coarsening step, read back once per level.
struct LevelCounts {
    int c;                      // aggregates (coarse vertices)
    int m;                      // emitted Galerkin records (2 x cross entries)
    int nseg;                   // coarse stored entries
    int pad;
    unsigned long long gbits;   // coarse Gershgorin shift (bits of a double)
    unsigned long long sell;    // SELL-32 size of the coarse level
    GridSync gs;                // barrier state of the coarsening kernel
};

// Galerkin product I L I^T of the level (rp, col, w) with aggregate map agg
// onto cnt->c aggregates (device), without host synchronisation.  Outputs
// go to caller buffers sized by upper bounds: rp_c int[n+1], col_c int[nnz],
// w_c double[nnz]; cnt->nseg and cnt->gbits receive the coarse nnz and g.
// key_bits: bits of an upper bound of c (keys pack two aggregate ids).
cmg_status_t galerkin_async(int n, long long nnz, const int *rp, const int *col, const double *w,
                            const int *agg, int key_bits, LevelCounts *cnt, int *rp_c, int *col_c,
                            double *w_c, cudaStream_t s);
// Gershgorin shift g = max_i 2 * sum_j w_ij into *g_dev (device double).
cmg_status_t launch_gershgorin(int n, const int *rp, const double *w, double *g_dev,
                               cudaStream_t s);

// ---------------------------------------------------------------- refine.cu
// Result record of one power-iteration run (device memory).
struct PiResult {
    double mu;       // mean of the raw result buffer
    double inv_s;    // 1 / ||raw - mu||
    double cos;      // cosine between the last two iterates
    double mu_prev;  // scalars of the previous iterate (used by the FP64 final sweep)
    double inv_s_prev;
    int buf;         // index (0..2) of the buffer that holds the raw result
    int buf_prev;    // index of the buffer that holds the previous iterate
    int sweeps;
    int capped;
    int zero;        // the last sweep annihilated the iterate (B_g v = 0)
    int pad;
};

struct PiLevel {
    int n;
    long long nnz;
    const int *rp;
    const int *col;
    const double *w;     // FP64 weights
    const float *w32;    // FP32 weights (FP32 sweep form) or nullptr
    double g;
    const int *agg;      // this level -> next coarser level (nullptr at the coarsest)
    const int *tile_row; // row tiles of the sweep kernel (nullptr: built on demand)
    int ntiles;
    long long sell_nnz;  // SELL-32 size for the shared-memory kernel (0: unknown)
    // sweep layout (one graph) for the slice kernel, or nullptr; with a layout
    // the level's iterates are stored in the layout's row order
    const SweepLayout *lay;
    // two-phase layout (same row order as lay), or nullptr
    const XLayout *xl;
    // FP64 sweeps in one thread-block cluster (cluster_plan): CTAs (0: not
    // planned), threads per CTA, dynamic shared memory per CTA, and the
    // largest SELL-32 entry count a CTA holds
    int cl_ctas, cl_threads, cl_emax;
    size_t cl_smem;
};

// Plans a level's FP64 sweeps in one thread-block cluster of 2..8 CTAs,
// each holding the whole iterate ring and the SELL-32 slices of its share
// of the rows, from the level's row pointers (host copy, n + 1).  Leaves
// lv->cl_ctas at 0 when the level is outside the plan's range or no cluster
// of that size can be resident.
void cluster_plan(PiLevel *lv, const int *rp_host);
// Whether a cluster CTA could hold an n-row level's iterate ring (3 x n
// values), g - d_i and slot order at all: the check before cluster_plan,
// which needs the level's row pointers on the host.
bool cluster_may_hold(int n);

// SELL-32 size of a CSR level (sum over 32-row slices of 32 x longest row);
// dev_counter: one device unsigned long long of scratch.  Synchronises s.
cmg_status_t sell_size(int n, const int *rp, unsigned long long *dev_counter, long long *out,
                       cudaStream_t s);
// The same for a level whose row count is in device memory (at most n_cap),
// without host synchronisation (the caller reads *dev_counter later).
cmg_status_t sell_size_async(const int *n_dev, int n_cap, const int *rp,
                             unsigned long long *dev_counter, cudaStream_t s);

// Row tiles of a level for the tiled sweep kernel (tile_count + 1 entries).
int tile_count(int n, long long nnz);
cmg_status_t build_tiles(int n, long long nnz, const int *rp, int *tile_row, cudaStream_t s);

// Power iteration (Alg. 3) on one level.  Start vector: x_init if given;
// else, if coarse_res is given, the prolongation (I_j^{j+1})^T of the coarse
// result held in coarse_bufs[coarse_res->buf]; else the Gaussian start of
// Alg. 1 Step 2 keyed by `seed`.
// bufs: three vectors of n elements (double, or float when fp32) and, for
// FP64, gd: n doubles of scratch for g - d_i.
// mode 0: stop on the cosine rule or after max_sweeps; mode 1: exactly k_fixed sweeps.
struct PiRun {
    const PiLevel *lv;
    int fp32;
    int mode;
    int k_fixed;
    int max_sweeps;
    double tol;
    uint64_t seed;
    const void *coarse_bufs[3];
    int coarse_fp64;                 // the coarse level's iterates are doubles
    const PiResult *coarse_res;
    const int *coarse_agg;           // agg of this level onto the coarse level
    const int *coarse_inv;           // the coarse level's layout order (nullptr: natural)
    const double *x_init;
    void *bufs[3];
    double *gd;
    PiResult *res;
};
// Caller-provided scratch for power_iteration / finalize (nullptr: the
// functions allocate their own).  Capacities are in elements.
struct PiWorkspace {
    int *tile_row;
    int tile_cap;
    double *partials;
    int partials_cap;
    double *fin_part;
    int fin_part_cap;
};
cmg_status_t power_iteration(const PiRun &run, GridSync *gs, cudaStream_t s,
                             const PiWorkspace *ws = nullptr);

// Level-0 finalisation in one cooperative launch:
//   - unless `fresh`: u = (y - mu) / s from the result buffer (FP64 form), or,
//     for the FP32 form, the last sweep recomputed in FP64 from the previous
//     iterate and normalised;
//   - if `sign`: scale u so that its largest-|u_i| entry (lowest index on
//     ties) is positive;
//   - out2[0] = u^T L u / u^T u, out2[1] = ||(L - out2[0] I) u|| / ||u||.
// True when the shared-memory kernel can hold the whole level.
bool small_level_fits(const PiLevel &lv, int fp32);

// Read-only view of a resident hierarchy's levels (FP64 CSR, shifts, maps),
// its device, its options' seed and its barrier state (api.cu).
struct HierarchyView {
    std::vector<PiLevel> lv;
    int device;
    uint64_t seed;
    cmg_options_t opts;
    GridSync *gs;
};
cmg_status_t hierarchy_view(cmg_hierarchy_t h, HierarchyView *out);

cmg_status_t finalize(const PiLevel &lv, int fp32, void *const bufs[3], const PiResult *res,
                      double *u, int sign, int fresh, double *out2, GridSync *gs, cudaStream_t s,
                      const PiWorkspace *ws = nullptr);

}  // namespace cmg
