// Internal interface between the host orchestration (api.cu) and the kernel
// translation units. Not part of the public ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ops {

constexpr int kMaxBins = 16;

// Learned sizing, load feedback: each class of rows (the numeric bin of a
// row's predicted size) has a factor 2^k on its predicted sizes,
// |k| <= kMaxFactorLog2. The one-phase kernels count, per class, the rows
// tried (group 0), those that ended more than 3/4 full (1), those that the
// next smaller table would hold at most 3/4 full (2) and the mispredicted
// ones (3), each spread over kLoadSlots counters (by block) against
// contention: counter (group * kMaxBins + class) * kLoadSlots + slot.
constexpr int kMaxFactorLog2 = 4;
constexpr int kLoadSlots = 8;
constexpr int kFbGroups = 4;
constexpr int kFbCounters = kFbGroups * kMaxBins * kLoadSlots;

struct SizeFactors {
    long long lim[kMaxBins];   // class j: sizes in (lim[j-1], lim[j]]; the last class takes the rest
    int k[kMaxBins];           // exponent of each class's factor
    int nb;
};

// Operands of one SpGEMM row window, as the kernels see them.
struct Operands {
    const void *arpt; int a64; const int32_t *acol; const double *aval;
    const void *brpt; int b64; const int32_t *bcol; const double *bval;
    int64_t row0;   // A row of window row 0
    int64_t mw;     // rows in the window
    int64_t ncols;  // columns of B (and C)
};

// What one bin kernel launch works on.
struct BinWork {
    const int32_t *bins;  // window row ids grouped by bin; nullptr = identity
    int64_t off, cnt;     // this bin's slice of `bins`
    int64_t *crpt;        // window C.rpt (int64, mw + 1)
    int32_t *ccol;        // numeric only
    double *cval;         // numeric only
    int lanes;            // threads per B row, 0 = per-row automatic
    int unroll;           // bitmap kernels: products in flight per lane (4 or 8; 0 = 4)
    int multi;            // plain hash kernels: read a slot before its compare-and-swap
    int distinct;         // every row of B has distinct columns (checked): warp-row numeric
                          // hash kernels may update values without atomics
    int *err;             // device error word
    // numeric bitmap kernel, pass 2 by column windows (B rows sorted)
    const int32_t *bs;    // run boundaries of B rows at the sub-ranges (G + 1 per row), or nullptr
    int G, gshift;        // sub-ranges of 2^gshift columns
    int wlists;           // rows with more A entries use the whole-row pass 2
    int wentries;         // C entries per window, about
    int head;             // shared bytes before the bitmap (set by launch_num)
    // one-phase (learned sizing) numeric kernels only
    int32_t *tcol;        // temporary rows: bin-local row r of this bin at
    double *tval;         //   tcol/tval + tbase + r * tcap
    long long tbase, tcap;
    long long tlimit;     // entries of tcol/tval (bounds check)
    long long *pred;      // predicted sizes; set to -1 for a row that overflowed
    int32_t *xlist;       // rows for the exact path (overflowed rows are appended)
    unsigned long long *xcount;
    long long xlimit;     // entries of xlist (bounds check)
    const uint8_t *lcls;  // class of each window row (the bin of its prediction)
    unsigned long long *fb;   // load feedback counters (kFbCounters), or nullptr
    long long tprev;      // slots of the next smaller table (0: none)
    // symbolic bitmap kernel: per-cell entry counts for the column-window
    // numeric kernel (nullptr: not wanted)
    uint16_t *cells;      // bin-local row r: cells[r * ncells + c] = entries in cell c
    int32_t *cslot;       // window row -> its bin-local index in this bin
    int cs, ncells;       // cells of 2^cs columns
    // numeric bitmap kernel over several column windows with rows of B
    // sorted: cell index of the long B rows, so each window walks only its runs
    const int32_t *bslot;
    const int32_t *bidx;
    // symbolic bitmap kernel: bit 0 set = some row of B is not sorted (the
    // runs are then not used); nullptr = B known sorted
    const unsigned long long *bflags;
    // numeric bitmap kernel (whole-row form): per-phase SM clock sums
    // (kPhaseClocks), or nullptr; a profiling aid
    unsigned long long *clk;
};

// Phases of the numeric bitmap kernel that spgemm_bitmap_phase_clocks reports.
constexpr int kPhaseClocks = 7;

struct Ranges {
    long long r[kMaxBins];
    int nb;
};

// Counters written by the binning passes (device memory, zeroed per call).
struct Counters {
    unsigned long long bin_cnt[kMaxBins];   // pass 1: rows per bin
    unsigned long long cursor[kMaxBins];    // pass 2: fill cursor per bin
    unsigned long long bin_sum[kMaxBins];   // pass 1: sum of the sizes per bin
    unsigned long long bin_nnza[kMaxBins];  // pass 1: A entries of the bin's rows
    unsigned long long max_size;
    unsigned long long total;
    unsigned long long flags;         // bit 0: some row of B has decreasing columns; bit 1: repeated ones
    unsigned long long windows;       // column windows of the large rows (win_count_kernel)
    unsigned long long wcol;          // those of them that accumulate by column
};

// Windowed pass 2 of the numeric bitmap kernel: at most kWinMaxLists A
// entries per row, at most kRunMaxSub column sub-ranges.
constexpr int kWinMaxLists = 1024;
constexpr int kRunMaxSub = 64;
constexpr int kRunDefaultEntries = 12288;

// Kernel table entry (host side).
struct KernelDesc {
    int tpr;          // threads per row (row group)
    int block;        // threads per block
    long long table;  // hash slots per row, or bitmap columns per pass
    long long max_size;  // largest row size the kernel accepts
    int bitmap;       // 1: shared-memory column bitmap kernel
    size_t smem;      // dynamic shared memory per block
};

// --- setup.cu ----------------------------------------------------------------
cudaError_t launch_nprod(const Operands &op, int64_t *nprod, int grid, cudaStream_t s);
cudaError_t launch_bin_pass1(const int64_t *sizes, int64_t n, const Ranges &rg,
                             const Operands &op, Counters *cnt, long long *tile_sums,
                             cudaStream_t s);
cudaError_t launch_bin_pass2(const int64_t *sizes, int64_t n, const Ranges &rg,
                             const long long *offsets, Counters *cnt, int32_t *bins,
                             cudaStream_t s);
// Sets bit 0 of cnt->flags when some row of B has a column smaller than the
// one before it.
cudaError_t launch_sorted_check(const Operands &op, int64_t brows, int64_t bnnz, Counters *cnt,
                                int grid, cudaStream_t s);
// In-place exclusive scan of crpt[0..n) using per-tile sums from pass 1;
// writes crpt[n] = total. tile_sums needs room for ntiles + 1 entries.
cudaError_t launch_scan(int64_t *crpt, int64_t n, long long *tile_sums, cudaStream_t s);
int64_t bin_tile_rows();
cudaError_t launch_iota(int32_t *out, int64_t n, cudaStream_t s);


// --- symbolic.cu / numeric.cu -------------------------------------------------
int sym_kernel_count();
int num_kernel_count();
const KernelDesc &sym_kernel(int id);
const KernelDesc &num_kernel(int id);
cudaError_t sym_prepare(int device_smem_optin);
cudaError_t num_prepare(int device_smem_optin);
// Default symbolic bin ranges and kernels (returns the bin count).
int default_sym_bins(long long *range, int32_t *kernel);
// Kernel attributes of every kernel on device `dev` (the current device),
// once per device; serialised by a lock, so handles and the
// allocation-free entry point may be set up from several host threads.
cudaError_t prepare_device(int dev, int smem_dyn_max);
cudaError_t launch_sym(int id, const Operands &op, const BinWork &w, size_t smem_bitmap,
                       cudaStream_t s);
cudaError_t launch_num(int id, const Operands &op, const BinWork &w, size_t smem_bitmap,
                       cudaStream_t s);
// one-phase numeric kernel `id` (a hash kernel of the numeric table)
cudaError_t launch_num_onephase(int id, const Operands &op, const BinWork &w, cudaStream_t s);

// --- runs.cu -------------------------------------------------------------------
// Run boundaries of B rows at column sub-ranges of 2^gshift columns
// (G + 1 int32 per row of B: offset of the first entry of each sub-range).
cudaError_t launch_bsplit(const Operands &op, int64_t brows, int64_t bnnz, int gshift, int G,
                          int32_t *bs, int grid, cudaStream_t s);
// numeric.cu: shared bytes before the bitmap of num_bitmap_kernel (walk
// scratch, or the run metadata of a windowed pass 2).
size_t num_bitmap_head_bytes(bool runs);

// --- window.cu -----------------------------------------------------------------
// Column-window numeric kernel for the rows of the last numeric bin (the
// large rows), used when every row of B is sorted. The column space is cut
// into cells of 2^cs columns (at most kWinMaxCells); the symbolic bitmap
// kernel counts each large row's entries per cell, and a planner cuts the
// row into windows of whole cells that fit one block's shared memory:
//   column window: a dense accumulator indexed by column (8 bytes per
//                  column) plus a presence bitmap; one pass over the products;
//   rank window:   a column bitmap with per-word ranks; one pass marks the
//                  columns, a second adds the values into C.val in L2.
// Rows with at most e1 entries take one rank window over all columns and need
// no cell counts.
constexpr int kWinMaxCells = 256;
constexpr int kWinMinCellLog2 = 12;
constexpr int kWinMaxColsLog2 = 22;
enum : int { kWinRank = 0, kWinCol = 1 };
constexpr long long kWinSingleMax = 16384;   // rows up to this size: one rank window

struct WinPlan {
    int cs = 0, ncells = 0;
    long long ncols = 0;
    long long budget = 0;   // shared bytes of a window's accumulator, bitmap and ranks
    int kc = 0;             // cells of a column window, at most (0: no column windows)
    long long e1 = -1;      // rows with at most e1 entries: one rank window
    long long cut = 0;      // rows of the last numeric bin have more than `cut` entries
};

struct Win {
    int32_t row;            // window row
    int32_t c0, c1;         // columns [c0, c1)
    int32_t mode;           // kWinRank / kWinCol
    uint32_t r0;            // rank of the window's first entry in its row
    uint32_t n;             // entries of the window
};

struct WinWork {
    const Win *win;
    long long nwin;
    unsigned long long *next;      // work counter of the persistent kernel (zeroed)
    const int32_t *bslot;          // B row -> slot of its cell index, or -1
    const int32_t *bidx;           // slot s: (ncells + 1) offsets of the first entry of each cell
    int cs, ncells;
    long long budget;
    // L2 spill of contended accumulations: block b owns spill[b * spill_stride ..),
    // one double per accumulator entry, zero between windows
    double *spill;
    long long spill_stride;
};

long long win_rank_bytes(long long width, long long n);
long long win_col_bytes(long long width);
size_t win_head_bytes();
cudaError_t win_prepare(int smem_optin);
// Window count of each row of the window with more than plan.cut entries
// (crpt holds n_nz), summed into *total.
cudaError_t launch_win_count(const WinPlan &plan, const int64_t *crpt, int64_t mw, const uint16_t *cells,
                             const int32_t *cslot, unsigned long long *total, unsigned long long *total_col,
                             int *err, cudaStream_t s);
// Cell index of the rows of B with at least `min_len` entries (slots up to cap).
cudaError_t launch_win_bindex(const Operands &op, int64_t brows, const WinPlan &plan, long long min_len,
                              int32_t *bslot, int32_t *bidx, long long cap, unsigned long long *nslot,
                              cudaStream_t s);
// Windows of the rows of bin w (crpt holds offsets), appended at *cursor.
cudaError_t launch_win_plan(const WinPlan &plan, const BinWork &w, const uint16_t *cells, const int32_t *cslot,
                            Win *list, long long cap, unsigned long long *cursor, cudaStream_t s);
cudaError_t launch_win_numeric(const Operands &op, const BinWork &w, const WinWork &ww, int grid, size_t smem,
                               cudaStream_t s);

// --- batch.cu ------------------------------------------------------------------
struct BatchProb {
    const void *arpt; int a64; const int32_t *acol; const double *aval;
    const void *brpt; int b64; const int32_t *bcol; const double *bval;
    int64_t M, N;
    int64_t *crpt; int32_t *ccol; double *cval; int64_t ccap;
    int32_t ntiles;
    int32_t dep;        // product whose C is this B, -1 when B is an input
    int32_t tiny;       // 1: every row has at most kBatchTiny products; 0: rows try one thread
                        // per row first (kBatchTiny distinct columns); -1: hash tables only
    int32_t pad;
    long long *tsum;    // per row tile: n_nz sum (symbolic tiles), then its exclusive prefix (scan)
};

constexpr int kBatchTiny = 8;
constexpr int kBatchMaxTile = 1024;   // rows per work item, at most

struct BatchItem {
    int32_t type;       // 0 symbolic tile, 1 scan, 2 numeric tile
    int32_t prob;
    int32_t tile;
    int32_t pad;
};

// Device state, zeroed before every run: queue head, error word and where,
// then per product: symbolic tiles done, scan done, numeric tiles done.
struct BatchState {
    unsigned long long head;
    int err;
    int where;
};

int batch_variant_count();
int batch_variant_table(int v);
int batch_variant_lanes(int v);
int batch_blocks_per_sm(int variant);
cudaError_t launch_batch(int variant, int grid, const BatchProb *probs, const BatchItem *items,
                         int nitems, BatchState *st, int *done_s, int *xflag, int *done_n,
                         int tile_rows, long long spin_limit, cudaStream_t s);

// --- learned.cu ----------------------------------------------------------------
int mlp_param_count();
cudaError_t launch_features(const Operands &op, int64_t mrows, long long *nprod, unsigned *maxlen,
                            unsigned *minlen, float *X, int grid, cudaStream_t s);
cudaError_t launch_mlp_forward(const float *theta, const float *X, int64_t n, float *y,
                               long long *sizes, float margin, long long cap, cudaStream_t s);
cudaError_t launch_mlp_train(const float *theta, const float *X, const float *t, int64_t n,
                             int64_t n_total, float *grad, float *loss, cudaStream_t s);
cudaError_t launch_adam(float *theta, const float *grad, float *m, float *v, int n, int step,
                        float lr, float b1, float b2, float eps, cudaStream_t s);
// sizes[i] = min(pred[i], n_prod[i]), or `huge` when n_prod[i] > exact_above
cudaError_t launch_learned_sizes(const int64_t *nprod, const long long *pred, int64_t n,
                                 long long exact_above, long long huge, int64_t *sizes,
                                 const SizeFactors &sf, uint8_t *cls, unsigned long long *fb,
                                 cudaStream_t s);
// copy one-phase rows from temporary memory into C (rows whose pred is -1 skipped)
cudaError_t launch_copy_rows(const BinWork &w, cudaStream_t s);

}  // namespace ops
