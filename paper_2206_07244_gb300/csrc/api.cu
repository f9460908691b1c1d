// Host orchestration and the C ABI (include/opsparse.h).
//
// One call of the plain path follows the paper's six steps (Sec. 5):
//   1 setup     C.rpt allocated; n_prod per row computed into it; scratch
//               reserved while that kernel runs (Sec. 5.4).
//   2 binning   Algorithm 1 on n_prod, one 16-word device->host read of the
//               bin sizes, Algorithm 2 (or the identity order of Algorithm 3
//               when one bin holds every row).
//   3 symbolic  one kernel per non-empty bin, largest rows first, each on its
//               own stream so small-row kernels fill SMs around the large
//               ones (Sec. 5.5); n_nz overwrites n_prod in C.rpt.
//   4 binning   Algorithm 1 on n_nz gives the total; one device->host read.
//   5 numeric   Algorithm 2 on n_nz, in-place exclusive scan of C.rpt,
//               C.col / C.val allocated after those kernels are queued
//               (Sec. 5.4), one numeric kernel per bin, largest first.
//   6 cleanup   scratch is kept in the handle for the next call; nothing is
//               freed between launches (Sec. 5.5).
#include <algorithm>
#include <climits>
#include <mutex>
#include <vector>
#include <cstdio>
#include <cstring>
#include <new>

#include "common.cuh"
#include "internal.h"
#include "opsparse.h"

using namespace ops;

namespace {

constexpr int kSide = 8;              // side streams for concurrent bin kernels
constexpr size_t kCountersBytes = 2048;  // 2 x Counters + the error word + the exact-list count
static_assert(2 * sizeof(ops::Counters) + 16 <= kCountersBytes, "counter block too small");

// Event-timing slots: 0..15 symbolic bins, 16..31 numeric bins, then the
// setup/binning/scan kernels.
enum Slot {
    kSlotSymBin = 0,
    kSlotNumBin = 16,
    kSlotNprod = 32,
    kSlotSymPass1 = 33,
    kSlotSymPass2 = 34,
    kSlotNumPass1 = 35,
    kSlotNumPass2 = 36,
    kSlotScan = 37,
    kSlotFeatures = 38,   // learned mode: row features
    kSlotMlp = 39,        // learned mode: MLP forward, sizes, binning by prediction
    kSlotCopy = 40,       // learned mode: one-phase rows copied into C
    kSlots = 41,
};

}  // namespace

// Pass 2 of the numeric bitmap kernel by column windows: rows with at most
// `lists` A entries (0: not used), G sub-ranges of 2^gshift columns, about
// `entries` C entries per window.
struct RunPlan {
    int lists = 0;
    int G = 0, gshift = 0;
    int entries = 0;
    const int32_t *bs = nullptr;     // run boundaries of B rows (set by the numeric phase)
};

struct spgemm_handle {
    int device = 0;
    int sm_count = 0;
    int smem_dyn_max = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t side[kSide] = {};
    cudaStream_t copyst[2] = {};   // device -> host copies of spgemm_multiply_host
    cudaEvent_t ev_fork = nullptr;
    cudaEvent_t ev_side[kSide] = {};
    spgemm_alloc_fn alloc = nullptr;
    spgemm_free_fn freefn = nullptr;
    void *ctx = nullptr;
    cudaMemPool_t pool = nullptr;
    spgemm_config cfg{};
    bool cfg_auto = false;   // default configuration: hash/bitmap cut derived per call from N
    // scratch arena: [Counters sym | Counters num | err] [bins] [tile sums]
    unsigned char *arena = nullptr;
    size_t arena_bytes = 0;
    Counters *h_cnt = nullptr;  // pinned, 2 entries
    // state between symbolic and numeric
    int state = 0;
    int64_t row0 = 0, mw = 0, ncols = 0, nnz = 0;
    int64_t *crpt = nullptr;
    long long num_size[kMaxBins] = {};
    RunPlan rplan;               // windowed pass 2 plan of the last symbolic call
    bool b_unsorted = false;     // some row of B has decreasing columns
    bool b_distinct = false;     // every row of B has strictly increasing columns
    // the last plain numeric call's rows stay in their bins (numeric order)
    // until the next symbolic call: spgemm_numeric_values runs them again
    bool reuse = false;
    int64_t reuse_arows = 0, reuse_annz = 0, reuse_brows = 0, reuse_bnnz = 0;
    int64_t stats[4 + 2 * SPGEMM_MAX_BINS] = {};
    int64_t bin_stats[2][3 * SPGEMM_MAX_BINS] = {};
    // learned sizing
    int mode = 0;                 // SPGEMM_MODE_PLAIN / SPGEMM_MODE_LEARNED
    float *theta = nullptr;       // predictor parameters (device)
    float margin = 0.25f;
    int lfk[kMaxBins] = {};       // per class: exponent of the factor on the predicted sizes,
                                  // adapted from call to call (load feedback)
    unsigned char *lscratch = nullptr;
    size_t lscratch_bytes = 0;
    int32_t *tcol = nullptr;      // temporary one-phase rows of the current call
    double *tval = nullptr;
    long long lsize[kMaxBins] = {}, loff[kMaxBins] = {}, ltbase[kMaxBins] = {}, ltcap[kMaxBins] = {};
    long long ltotal = 0;
    bool lid = false;
    int64_t xcount = 0;
    int64_t lstats[6 + kMaxBins] = {};  // one-phase rows, mispredicted rows, exact rows, temp
                                        // entries, rows > 3/4 full, rows that fit the next
                                        // smaller table, factor exponents used per class
    // column-window numeric path for the last numeric bin (window.cu)
    WinPlan wplan;                // plan of the last symbolic call
    bool wp_on = false;           // the symbolic call prepared cell counts and a window count
    uint16_t *wcells = nullptr;   // cell counts of the symbolic bitmap bin's rows
    size_t wcells_bytes = 0;
    int32_t *wcslot = nullptr;    // window row -> its index in the symbolic bitmap bin
    size_t wcslot_bytes = 0;
    long long nwin = 0;           // windows of the last symbolic call
    long long nwin_col = 0;       // those that accumulate by column
    // the last numeric call's windows and cell index of B, kept for
    // spgemm_numeric_values while the structure is kept
    Win *wlist = nullptr;
    int32_t *wbslot = nullptr;
    int32_t *wbidx = nullptr;
    unsigned long long *wctr = nullptr;   // cursor, work counter, index slots
    double *wspill = nullptr;     // L2 spill of the window kernel's blocks (kept zero)
    size_t wspill_bytes = 0;
    bool wkeep = false;
    bool win_used = false;        // the last numeric call ran the column windows
    // whole-row bitmap kernel walked by half-width column windows (sorted B)
    bool split_on = false;        // planned by the symbolic call
    bool split_idx = false;       // the symbolic call built the cell index of B
    bool split_keep = false;      // the last numeric call used it (index kept)
    int split_cs = 0, split_ncells = 0;
    // per-kernel CUDA-event timing (off unless requested)
    // pinned staging for spgemm_multiply_host
    unsigned char *stage = nullptr;
    size_t stage_bytes = 0;
    int64_t *stage_rpt = nullptr;
    size_t stage_rpt_n = 0;
    bool timing = false;
    bool serial = false;   // timing mode 2: every bin kernel on the main stream, one after another
    // phase clocks of the numeric bitmap kernel (profiling; off unless requested)
    bool phase_clk = false;
    unsigned long long *d_clk = nullptr;   // kPhaseClocks sums
    cudaEvent_t t0[kSlots] = {}, t1[kSlots] = {};
    bool pending[kSlots] = {};
    double ms[kSlots] = {};
    long long launches[kSlots] = {};
};

namespace {

void *dev_alloc(spgemm_handle *h, size_t bytes) {
    bytes = std::max<size_t>(bytes, 256);
    if (h->alloc) return h->alloc(bytes, h->stream, h->ctx);
    void *p = nullptr;
    if (cudaMallocFromPoolAsync(&p, bytes, h->pool, h->stream) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void dev_free(spgemm_handle *h, void *p) {
    if (!p) return;
    if (h->freefn) h->freefn(p, h->stream, h->ctx);
    else cudaFreeAsync(p, h->stream);
}

void flush_slot(spgemm_handle *h, int k) {
    if (!h->pending[k]) return;
    cudaEventSynchronize(h->t1[k]);
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->t0[k], h->t1[k]) == cudaSuccess) h->ms[k] += ms;
    cudaGetLastError();
    h->pending[k] = false;
}

void time_begin(spgemm_handle *h, int k, cudaStream_t s) {
    if (!h->timing) return;
    flush_slot(h, k);
    cudaEventRecord(h->t0[k], s);
}

void time_end(spgemm_handle *h, int k, cudaStream_t s) {
    if (!h->timing) return;
    cudaEventRecord(h->t1[k], s);
    h->pending[k] = true;
    h->launches[k] += 1;
}

Counters *d_counters(spgemm_handle *h, int phase) {
    return reinterpret_cast<Counters *>(h->arena) + phase;
}

int *d_err(spgemm_handle *h) {
    return reinterpret_cast<int *>(h->arena + 2 * sizeof(Counters));
}

size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

int ensure_arena(spgemm_handle *h, int64_t mw) {
    const int64_t ntiles = (mw + bin_tile_rows() - 1) / bin_tile_rows();
    const size_t need = kCountersBytes + align256(sizeof(int32_t) * (size_t)std::max<int64_t>(mw, 1)) +
                        align256(sizeof(long long) * (size_t)(ntiles + 2));
    if (h->arena && h->arena_bytes >= need) return SPGEMM_OK;
    int keep_err = 0;
    if (h->arena) {
        if (cudaStreamSynchronize(h->stream) != cudaSuccess) return SPGEMM_ERR_CUDA;
        cudaMemcpy(&keep_err, d_err(h), sizeof(int), cudaMemcpyDeviceToHost);
        dev_free(h, h->arena);
        h->arena = nullptr;
        h->arena_bytes = 0;
    }
    const size_t bytes = need + need / 4;
    h->arena = static_cast<unsigned char *>(dev_alloc(h, bytes));
    if (!h->arena) return SPGEMM_ERR_OOM;
    h->arena_bytes = bytes;
    if (cudaMemsetAsync(h->arena, 0, kCountersBytes, h->stream) != cudaSuccess) return SPGEMM_ERR_CUDA;
    if (keep_err &&
        cudaMemcpyAsync(d_err(h), &keep_err, sizeof(int), cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
        return SPGEMM_ERR_CUDA;
    return SPGEMM_OK;
}

int32_t *d_bins(spgemm_handle *h) {
    return reinterpret_cast<int32_t *>(h->arena + kCountersBytes);
}

long long *d_tiles(spgemm_handle *h) {
    return reinterpret_cast<long long *>(h->arena + kCountersBytes +
                                         align256(sizeof(int32_t) * (size_t)std::max<int64_t>(h->mw, 1)));
}

// Learned-sizing scratch per window row: features (6 floats), prediction,
// binning size, exact-path list, and the feature kernel's n_prod/max/min.
struct LScratch {
    float *X;
    long long *pred;
    int64_t *lsizes;
    int32_t *xlist;
    uint8_t *cls;         // class of each row (bin of its prediction)
    unsigned long long *fb;   // load feedback counters (kFbCounters)
    unsigned char *fws;   // n_prod (8 B) + max (4 B) + min (4 B) per row
};

LScratch lscratch_layout(spgemm_handle *h, int64_t mw) {
    const size_t m = (size_t)std::max<int64_t>(mw, 1);
    unsigned char *p = h->lscratch;
    LScratch L;
    L.X = reinterpret_cast<float *>(p);                 p += align256(sizeof(float) * 6 * m);
    L.pred = reinterpret_cast<long long *>(p);          p += align256(sizeof(long long) * m);
    L.lsizes = reinterpret_cast<int64_t *>(p);          p += align256(sizeof(int64_t) * m);
    L.xlist = reinterpret_cast<int32_t *>(p);           p += align256(sizeof(int32_t) * m);
    L.cls = reinterpret_cast<uint8_t *>(p);             p += align256(m);
    L.fb = reinterpret_cast<unsigned long long *>(p);   p += align256(sizeof(unsigned long long) * kFbCounters);
    L.fws = p;
    return L;
}

int ensure_lscratch(spgemm_handle *h, int64_t mw) {
    const size_t m = (size_t)std::max<int64_t>(mw, 1);
    const size_t need = align256(24 * m) + 2 * align256(8 * m) + align256(4 * m) + align256(m) +
                        align256(sizeof(unsigned long long) * kFbCounters) + align256(16 * m) + 256;
    if (h->lscratch && h->lscratch_bytes >= need) return SPGEMM_OK;
    if (h->lscratch) {
        if (cudaStreamSynchronize(h->stream) != cudaSuccess) return SPGEMM_ERR_CUDA;
        dev_free(h, h->lscratch);
    }
    h->lscratch = static_cast<unsigned char *>(dev_alloc(h, need));
    h->lscratch_bytes = h->lscratch ? need : 0;
    return h->lscratch ? SPGEMM_OK : SPGEMM_ERR_OOM;
}

unsigned long long *d_xcount(spgemm_handle *h) {
    return reinterpret_cast<unsigned long long *>(h->arena + 2 * sizeof(Counters) + 8);
}

bool is_pow2_lanes(int x) { return x == 0 || x == 1 || x == 2 || x == 4 || x == 8 || x == 16 || x == 32; }

int validate_config(const spgemm_config &c) {
    if (!is_pow2_lanes(c.lanes_per_brow) || !is_pow2_lanes(c.num_lanes_per_brow))
        return SPGEMM_ERR_INVALID;
    if (c.bitmap_unroll != 0 && c.bitmap_unroll != 4 && c.bitmap_unroll != 8) return SPGEMM_ERR_INVALID;
    if (c.window_lists < 0 || c.window_lists > kWinMaxLists || c.window_entries < 0) return SPGEMM_ERR_INVALID;
    if (c.hash_access != 0 && c.hash_access != 1) return SPGEMM_ERR_INVALID;
    if (c.bitmap_path < 0 || c.bitmap_path > 2) return SPGEMM_ERR_INVALID;
    if (c.window_budget < 0) return SPGEMM_ERR_INVALID;
    for (int phase = 0; phase < 2; ++phase) {
        const int nb = phase ? c.num_nbins : c.sym_nbins;
        const int32_t *k = phase ? c.num_kernel : c.sym_kernel;
        const int64_t *r = phase ? c.num_range : c.sym_range;
        const int nk = phase ? num_kernel_count() : sym_kernel_count();
        if (nb < 1 || nb > SPGEMM_MAX_BINS) return SPGEMM_ERR_INVALID;
        for (int j = 0; j < nb; ++j) {
            if (k[j] < 0 || k[j] >= nk) return SPGEMM_ERR_INVALID;
            const KernelDesc &d = phase ? num_kernel(k[j]) : sym_kernel(k[j]);
            const bool last = j == nb - 1;
            if (last != (r[j] < 0)) return SPGEMM_ERR_INVALID;      // only the last bin is unbounded
            if (last) {
                if (!d.bitmap) return SPGEMM_ERR_INVALID;          // it must take any row size
            } else {
                if (r[j] > d.max_size) return SPGEMM_ERR_INVALID;
                if (j > 0 && r[j] <= r[j - 1]) return SPGEMM_ERR_INVALID;
            }
        }
    }
    return SPGEMM_OK;
}

void default_config(spgemm_config &c) {
    std::memset(&c, 0, sizeof(c));
    // Symbolic: every table at least 1.2x the largest n_prod of its bin
    // (Sec. 5.7, the paper's choice "Sym_1.2x"); the bitmap takes the rest.
    long long sr[kMaxBins];
    c.sym_nbins = default_sym_bins(sr, c.sym_kernel);
    for (int j = 0; j < c.sym_nbins; ++j) c.sym_range[j] = sr[j];
    // Numeric: every table at least 2x the largest n_nz of its bin (Sec. 5.7,
    // "Num_2x").
    const int nn = num_kernel_count();
    c.num_nbins = nn;
    for (int j = 0; j < nn; ++j) {
        c.num_kernel[j] = j;
        const KernelDesc &d = num_kernel(j);
        c.num_range[j] = d.bitmap ? -1 : static_cast<int64_t>(d.table / 2);
    }
    c.lanes_per_brow = 0;
}

// The default configuration adapts where large rows leave the hash bins
// for the bitmap kernels to the number of columns N: a bitmap kernel clears
// and scans N bits per row (N/64 words with rank counts in the numeric
// phase), so its fixed cost per row grows with N while a hash bin's
// condense/sort cost grows with the row. Measured on GB300 (R-MAT n = 2^16,
// 2^18, 2^20), numeric rows above max(1024, N/512) entries and symbolic rows
// above max(6826, N/128) products run faster in the bitmap kernels.
void auto_cut(spgemm_config &c, int64_t ncols) {
    default_config(c);
    const int64_t num_lim = std::max<int64_t>(1024, ncols / 512);
    const int64_t sym_lim = std::max<int64_t>(6826, ncols / 128);
    for (int phase = 0; phase < 2; ++phase) {
        int32_t *k = phase ? c.num_kernel : c.sym_kernel;
        int64_t *r = phase ? c.num_range : c.sym_range;
        int32_t &nb = phase ? c.num_nbins : c.sym_nbins;
        const int64_t lim = phase ? num_lim : sym_lim;
        int keep = 0;
        while (keep < nb - 1 && r[keep] <= lim) ++keep;
        if (keep == 0) keep = 1;  // always keep the smallest hash bin
        k[keep] = k[nb - 1];      // the bitmap kernel takes everything larger
        r[keep] = -1;
        nb = keep + 1;
    }
}

RunPlan run_plan(const spgemm_config &c, int smem_dyn_max, int64_t ncols) {
    RunPlan p;
    if (c.window_lists <= 0 || ncols <= 0) return p;
    // the whole column range must fit one bitmap window next to the run metadata
    const int64_t words = (ncols + 63) / 64;
    if (words * 12 > smem_dyn_max - static_cast<int64_t>(num_bitmap_head_bytes(true))) return p;
    int gshift = 6;
    while (((ncols + (int64_t{1} << gshift) - 1) >> gshift) > kRunMaxSub) ++gshift;
    p.lists = c.window_lists;
    p.gshift = gshift;
    p.G = static_cast<int>((ncols + (int64_t{1} << gshift) - 1) >> gshift);
    p.entries = c.window_entries > 0 ? c.window_entries : kRunDefaultEntries;
    return p;
}

// Column-window plan for the last numeric bin (window.cu), for B with
// `ncols` columns. Cells of 2^cs columns, at most kWinMaxCells of them; a
// window's accumulator, bitmap and ranks get the shared memory left after
// the walk's head. Rows with more entries than a whole-width rank window
// holds (e1) need the cell counts of the symbolic bitmap kernel, so every
// such row must pass through it: the symbolic threshold must not exceed
// max(numeric threshold, e1). The default configuration lowers it where
// needed; an explicit configuration that breaks the rule keeps the
// whole-row bitmap kernel. Returns false when the path is not used.
bool win_setup(spgemm_handle *h, int64_t ncols) {
    spgemm_config &c = h->cfg;
    if (c.bitmap_path != 2 || ncols <= 0 || ncols > (int64_t{1} << kWinMaxColsLog2)) return false;
    if (!num_kernel(c.num_kernel[c.num_nbins - 1]).bitmap || !sym_kernel(c.sym_kernel[c.sym_nbins - 1]).bitmap)
        return false;
    int lg = 0;
    while ((int64_t{1} << lg) < ncols) ++lg;
    WinPlan p;
    p.cs = std::max(kWinMinCellLog2, lg - 8);
    const int64_t cw = int64_t{1} << p.cs;
    p.ncells = static_cast<int>((ncols + cw - 1) / cw);
    p.ncols = ncols;
    p.budget = ((static_cast<long long>(h->smem_dyn_max) - static_cast<long long>(win_head_bytes())) / 16) * 16;
    if (c.window_budget > 0) p.budget = std::min<long long>(p.budget, (c.window_budget / 16) * 16);
    if (p.ncells > kWinMaxCells || win_rank_bytes(cw, cw) > p.budget) return false;
    p.kc = 0;
    while (p.kc < p.ncells && win_col_bytes((p.kc + 1) * cw) <= p.budget) ++p.kc;
    // rows with at most e1 entries take one rank window over all columns
    // (when its bitmap fits): too sparse for column windows to pay
    p.e1 = win_rank_bytes(ncols, 0) <= p.budget ? kWinSingleMax : -1;
    p.cut = c.num_nbins >= 2 ? c.num_range[c.num_nbins - 2] : 0;
    const long long lim = std::max(p.cut, p.e1);
    if (c.sym_nbins >= 2 && c.sym_range[c.sym_nbins - 2] > lim) {
        if (!h->cfg_auto) return false;
        int keep = c.sym_nbins - 1;   // hash bins kept
        while (keep > 1 && c.sym_range[keep - 1] > lim) --keep;
        if (c.sym_range[keep - 1] > lim) return false;
        c.sym_kernel[keep] = c.sym_kernel[c.sym_nbins - 1];
        c.sym_range[keep] = -1;
        c.sym_nbins = keep + 1;
    }
    h->wplan = p;
    return true;
}

// Whole-row numeric bitmap kernel by column windows with rows of B sorted:
// each window walks only the runs of B rows inside it (cell index of the
// long B rows), instead of every product of the row once per window. Form 0
// uses it when one bitmap cannot hold every column; form 1 always, with
// windows of about half an SM's shared memory so two blocks run per SM (one
// block's bitmap and C.col phases overlap the other's float64 reductions).
// Needs at most kWinMaxCells cells of 2^cs >= 2^12 columns.
bool split_setup(spgemm_handle *h, int64_t ncols) {
    const spgemm_config &c = h->cfg;
    if (c.bitmap_path > 1 || ncols <= 0 || ncols > (int64_t{1} << kWinMaxColsLog2)) return false;
    // form 0 needs windows only when one bitmap cannot hold every column
    const int64_t full = (h->smem_dyn_max - static_cast<int64_t>(num_bitmap_head_bytes(false))) / 12 * 64;
    if (c.bitmap_path == 0 && ncols <= full) return false;
    if (c.window_lists > 0 || !num_kernel(c.num_kernel[c.num_nbins - 1]).bitmap) return false;
    int lg = 0;
    while ((int64_t{1} << lg) < ncols) ++lg;
    h->split_cs = std::max(kWinMinCellLog2, lg - 8);
    const int64_t cw = int64_t{1} << h->split_cs;
    h->split_ncells = static_cast<int>((ncols + cw - 1) / cw);
    return h->split_ncells <= kWinMaxCells;
}

// Grow-only device buffer of the handle.
template <typename T>
int ensure_buf(spgemm_handle *h, T **p, size_t *have, size_t need) {
    if (*p && *have >= need) return SPGEMM_OK;
    dev_free(h, *p);
    *p = static_cast<T *>(dev_alloc(h, need + need / 4));
    *have = *p ? need + need / 4 : 0;
    return *p ? SPGEMM_OK : SPGEMM_ERR_OOM;
}

// Drop the windows and B index kept for spgemm_numeric_values.
void win_release(spgemm_handle *h) {
    dev_free(h, h->wlist);
    dev_free(h, h->wbslot);
    dev_free(h, h->wbidx);
    dev_free(h, h->wctr);
    h->wlist = nullptr;
    h->wbslot = nullptr;
    h->wbidx = nullptr;
    h->wctr = nullptr;
    h->wkeep = false;
    h->split_idx = false;
}

// L2 spill slots of the window kernel: one accumulator's worth per block,
// zeroed when allocated; the kernel leaves every slot it uses zero.
int ensure_spill(spgemm_handle *h, long long stride) {
    const size_t need = sizeof(double) * static_cast<size_t>(stride) * static_cast<size_t>(h->sm_count);
    if (h->wspill && h->wspill_bytes >= need) return SPGEMM_OK;
    dev_free(h, h->wspill);
    h->wspill = static_cast<double *>(dev_alloc(h, need));
    h->wspill_bytes = h->wspill ? need : 0;
    if (!h->wspill) return SPGEMM_ERR_OOM;
    return cudaMemsetAsync(h->wspill, 0, need, h->stream) == cudaSuccess ? SPGEMM_OK : SPGEMM_ERR_CUDA;
}

// Cell index of B's long rows (launch_win_bindex), kept in the handle.
int build_bindex(spgemm_handle *h, const Operands &op, const spgemm_csr_in *B) {
    const long long min_len = std::max<long long>(32, (h->split_ncells + 1) / 2);
    const long long cap = B->nnz / min_len + 1;
    h->wctr = static_cast<unsigned long long *>(dev_alloc(h, 4 * sizeof(unsigned long long)));
    h->wbslot = static_cast<int32_t *>(dev_alloc(h, sizeof(int32_t) * (size_t)std::max<int64_t>(B->rows, 1)));
    h->wbidx = static_cast<int32_t *>(dev_alloc(h, sizeof(int32_t) * (size_t)cap * (size_t)(h->split_ncells + 1)));
    if (!h->wctr || !h->wbslot || !h->wbidx) {
        win_release(h);
        return SPGEMM_ERR_OOM;
    }
    WinPlan ip;
    ip.cs = h->split_cs;
    ip.ncells = h->split_ncells;
    if (cudaMemsetAsync(h->wctr, 0, 4 * sizeof(unsigned long long), h->stream) != cudaSuccess ||
        launch_win_bindex(op, B->rows, ip, min_len, h->wbslot, h->wbidx, cap, h->wctr + 2, h->stream) !=
            cudaSuccess) {
        win_release(h);
        return SPGEMM_ERR_CUDA;
    }
    h->split_idx = true;
    return SPGEMM_OK;
}

// What the numeric phase needs to run the last bin by column windows.
struct WinCall {
    bool on = false;
    bool plan = true;          // build the B index and the window list first
    WinWork ww{};
    Win *list = nullptr;
    long long cap = 0;
    unsigned long long *cursor = nullptr, *nslot = nullptr;
    int32_t *bslot = nullptr, *bidx = nullptr;
    long long bcap = 0, min_len = 0;
    int64_t brows = 0;
    // whole-row bitmap kernel by half-width column windows over sorted B
    bool split = false;
    int cs = 0, ncells = 0;
};

// Last CUDA runtime error the library turned into an error code on this
// thread (spgemm_last_cuda_error).
thread_local cudaError_t g_last_cuda = cudaSuccess;

cudaError_t note(cudaError_t e) {
    if (e != cudaSuccess) g_last_cuda = e;
    return e;
}

int cuda_rc(cudaError_t e) {
    note(e);
    if (e == cudaSuccess) return SPGEMM_OK;
    if (e == cudaErrorMemoryAllocation) return SPGEMM_ERR_OOM;
    return SPGEMM_ERR_CUDA;
}

#define CK(call)                                   \
    do {                                           \
        cudaError_t e_ = (call);                   \
        if (e_ != cudaSuccess) return cuda_rc(e_); \
    } while (0)

int check_csr_in(const spgemm_csr_in *m) {
    if (!m || m->rows < 0 || m->cols < 0 || m->nnz < 0 || !m->rpt) return SPGEMM_ERR_INVALID;
    if (m->nnz > 0 && !m->col) return SPGEMM_ERR_INVALID;
    if (m->cols > INT32_MAX || m->rows > INT32_MAX) return SPGEMM_ERR_INVALID;
    if (!m->rpt_is_i64 && m->nnz > INT32_MAX) return SPGEMM_ERR_INVALID;
    return SPGEMM_OK;
}

Operands make_operands(const spgemm_csr_in *A, const spgemm_csr_in *B, int64_t r0, int64_t mw) {
    Operands op;
    op.arpt = A->rpt; op.a64 = A->rpt_is_i64 ? 1 : 0; op.acol = A->col; op.aval = A->val;
    op.brpt = B->rpt; op.b64 = B->rpt_is_i64 ? 1 : 0; op.bcol = B->col; op.bval = B->val;
    op.row0 = r0; op.mw = mw; op.ncols = B->cols;
    return op;
}

// Launch the kernels of one phase, one per non-empty bin, largest rows first,
// spread over the side streams. runs: plan of a windowed pass 2 for the
// numeric bitmap kernel (nullptr or runs->lists == 0: whole-row pass 2).
int run_bins(spgemm_handle *h, int phase, const Operands &op, const long long *size,
             const long long *offset, bool identity, int64_t *crpt, int32_t *ccol, double *cval,
             const RunPlan *runs = nullptr, const WinCall *win = nullptr) {
    const int nb = phase ? h->cfg.num_nbins : h->cfg.sym_nbins;
    const int32_t *kid = phase ? h->cfg.num_kernel : h->cfg.sym_kernel;
    CK(cudaEventRecord(h->ev_fork, h->stream));
    int used = 0;
    for (int j = nb - 1; j >= 0; --j) {
        if (size[j] <= 0) continue;
        cudaStream_t s = h->serial ? h->stream : h->side[used % kSide];
        if (!h->serial && used < kSide) CK(cudaStreamWaitEvent(s, h->ev_fork, 0));
        BinWork w{};
        w.bins = identity ? nullptr : d_bins(h);
        w.off = identity ? 0 : offset[j];
        w.cnt = size[j];
        w.crpt = crpt; w.ccol = ccol; w.cval = cval;
        w.lanes = phase ? h->cfg.num_lanes_per_brow : h->cfg.lanes_per_brow;
        w.unroll = h->cfg.bitmap_unroll;
        w.multi = h->cfg.hash_access;
        w.distinct = phase == 1 && h->b_distinct;
        w.clk = phase == 1 && h->phase_clk ? h->d_clk : nullptr;
        w.err = d_err(h);
        const KernelDesc &d = phase ? num_kernel(kid[j]) : sym_kernel(kid[j]);
        size_t smem = 0;
        const int slot = (phase ? kSlotNumBin : kSlotSymBin) + j;
        if (d.bitmap && phase == 1 && win && win->on) {
            // column windows: index of B's long rows, the window list, then
            // the persistent window kernel, one block per SM
            time_begin(h, slot, s);
            if (win->plan) {
                CK(launch_win_bindex(op, win->brows, h->wplan, win->min_len, win->bslot, win->bidx, win->bcap,
                                     win->nslot, s));
                CK(launch_win_plan(h->wplan, w, h->wcells, h->wcslot, win->list, win->cap, win->cursor, s));
            }
            CK(launch_win_numeric(op, w, win->ww, h->sm_count, win_head_bytes() + static_cast<size_t>(win->ww.budget),
                                  s));
            time_end(h, slot, s);
            ++used;
            continue;
        }
        if (d.bitmap) {
            // bitmap bytes; the kernels add their head (walk scratch / run metadata)
            if (phase == 0) {
                const int64_t budget = h->smem_dyn_max - static_cast<int64_t>(sizeof(WalkScratch));
                int64_t words = std::min<int64_t>((op.ncols + 31) / 32, budget / 4);
                if (h->split_idx) {
                    // several passes over the columns: each walks only its runs
                    w.bslot = h->wbslot;
                    w.bidx = h->wbidx;
                    w.cs = h->split_cs;
                    w.ncells = h->split_ncells;
                    w.bflags = &d_counters(h, 1)->flags;
                    const int64_t cwords = int64_t{1} << (h->split_cs - 5);
                    if (words < (op.ncols + 31) / 32) words = std::max<int64_t>(cwords, (words / cwords) * cwords);
                }
                if (win && win->on && h->wcells) {
                    // per-cell counts: a pass covers whole cells
                    const int64_t cwords = int64_t{1} << (h->wplan.cs - 5);
                    if (words < (op.ncols + 31) / 32) words = (words / cwords) * cwords;
                    w.cells = h->wcells;
                    w.cslot = h->wcslot;
                    w.cs = h->wplan.cs;
                    w.ncells = h->wplan.ncells;
                }
                smem = static_cast<size_t>(std::max<int64_t>(words, 1)) * 4;
            } else {
                const bool r = runs && runs->lists > 0 && runs->bs;
                if (r) {
                    w.bs = runs->bs;
                    w.G = runs->G;
                    w.gshift = runs->gshift;
                    w.wlists = runs->lists;
                    w.wentries = runs->entries;
                }
                int64_t budget = h->smem_dyn_max - static_cast<int64_t>(num_bitmap_head_bytes(r));
                const bool split = !r && win && win->split;
                if (split) {
                    w.bslot = win->bslot;
                    w.bidx = win->bidx;
                    w.cs = win->cs;
                    w.ncells = win->ncells;
                }
                if (split && h->cfg.bitmap_path == 1) {
                    // half an SM's shared memory per block (two blocks per SM),
                    // windows of whole cells
                    budget = std::min<int64_t>(budget, (228 * 1024 - 2 * 1024) / 2 - 512 -
                                                           static_cast<int64_t>(num_bitmap_head_bytes(false)));
                }
                int64_t words = std::min<int64_t>((op.ncols + 63) / 64, budget / 12);
                if (split && words < (op.ncols + 63) / 64) {
                    const int64_t cwords = int64_t{1} << (win->cs - 6);
                    words = std::max<int64_t>(cwords, (words / cwords) * cwords);
                }
                smem = static_cast<size_t>(std::max<int64_t>(words, 1)) * 12;
            }
        }
        time_begin(h, slot, s);
        CK(phase ? launch_num(kid[j], op, w, smem, s) : launch_sym(kid[j], op, w, smem, s));
        time_end(h, slot, s);
        ++used;
    }
    for (int i = 0; !h->serial && i < std::min(used, kSide); ++i) {
        CK(cudaEventRecord(h->ev_side[i], h->side[i]));
        CK(cudaStreamWaitEvent(h->stream, h->ev_side[i], 0));
    }
    return SPGEMM_OK;
}

// Bin sizes -> (offsets, identity?) : identity when one bin holds every row
// (the generalisation of Algorithm 3: no scatter pass, rows in index order).
bool plan_bins(const Counters &c, int nb, long long *size, long long *offset) {
    long long acc = 0;
    int nonempty = 0;
    for (int j = 0; j < nb; ++j) {
        size[j] = static_cast<long long>(c.bin_cnt[j]);
        offset[j] = acc;
        acc += size[j];
        nonempty += size[j] > 0;
    }
    return nonempty <= 1;
}

int read_counters(spgemm_handle *h) {
    CK(cudaMemcpyAsync(h->h_cnt, h->arena, 2 * sizeof(Counters) + sizeof(int),
                       cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    const int err = *reinterpret_cast<const int *>(reinterpret_cast<const unsigned char *>(h->h_cnt) +
                                                   2 * sizeof(Counters));
    for (int phase = 0; phase < 2; ++phase)
        for (int j = 0; j < SPGEMM_MAX_BINS; ++j) {
            h->bin_stats[phase][j] = static_cast<int64_t>(h->h_cnt[phase].bin_cnt[j]);
            h->bin_stats[phase][SPGEMM_MAX_BINS + j] = static_cast<int64_t>(h->h_cnt[phase].bin_sum[j]);
            h->bin_stats[phase][2 * SPGEMM_MAX_BINS + j] = static_cast<int64_t>(h->h_cnt[phase].bin_nnza[j]);
        }
    return err ? SPGEMM_ERR_INTERNAL : SPGEMM_OK;
}

// --- learned sizing (one-phase rows with an exact fallback) -------------------
// Symbolic part: features -> MLP -> predicted sizes -> bins by prediction;
// rows predicted to fit a hash table are multiplied once (one-phase kernels,
// rows to temporary memory, n_nz to C.rpt); rows past the symbolic hash bins
// and mispredicted rows go to the exact bitmap kernels. Ends like the plain
// symbolic phase: C.rpt holds every row's n_nz and the total is known.
int symbolic_learned(spgemm_handle *h, const Operands &op, int64_t mrows, int64_t *crpt,
                     int64_t *nnz_out) {
    const int64_t mw = op.mw;
    int rc = ensure_lscratch(h, mw);
    if (rc) return rc;
    const LScratch L = lscratch_layout(h, mw);
    cudaStream_t s = h->stream;
    const int nb = h->cfg.num_nbins;
    const int last = nb - 1;   // the numeric bitmap bin: exact path
    const int64_t cap = nb >= 2 ? h->cfg.num_range[nb - 2] : 0;
    // the features kernel also leaves n_prod of every row in C.rpt (step 1)
    long long *fnp = reinterpret_cast<long long *>(crpt);
    unsigned *fmx = reinterpret_cast<unsigned *>(L.fws + sizeof(long long) * (size_t)mw);
    unsigned *fmn = fmx + mw;
    time_begin(h, kSlotFeatures, s);
    CK(launch_features(op, mrows, fnp, fmx, fmn, L.X, h->sm_count * 8, s));
    time_end(h, kSlotFeatures, s);
    time_begin(h, kSlotMlp, s);
    CK(launch_mlp_forward(h->theta, L.X, mw, nullptr, L.pred, h->margin, cap + 1, s));
    const int64_t exact_above = h->cfg.sym_nbins >= 2 ? h->cfg.sym_range[h->cfg.sym_nbins - 2] : -1;
    SizeFactors sf{};
    sf.nb = nb;
    for (int j = 0; j < nb; ++j) {
        sf.lim[j] = h->cfg.num_range[j];
        sf.k[j] = h->lfk[j];
    }
    CK(cudaMemsetAsync(L.fb, 0, sizeof(unsigned long long) * kFbCounters, s));
    CK(launch_learned_sizes(crpt, L.pred, mw, exact_above, LLONG_MAX / 4, L.lsizes, sf, L.cls, L.fb, s));
    Ranges rn{};
    rn.nb = nb;
    for (int j = 0; j < nb; ++j) rn.r[j] = h->cfg.num_range[j];
    CK(launch_bin_pass1(L.lsizes, mw, rn, op, d_counters(h, 0), nullptr, s));
    time_end(h, kSlotMlp, s);
    if ((rc = read_counters(h))) return rc;
    // B's column order (checked before this call): distinct columns let the
    // warp-row one-phase kernels update values without atomics
    h->b_distinct = (h->h_cnt[1].flags & 3ull) == 0;
    h->lid = plan_bins(h->h_cnt[0], nb, h->lsize, h->loff);
    if (!h->lid) CK(launch_bin_pass2(L.lsizes, mw, rn, h->loff, d_counters(h, 0), d_bins(h), s));
    // the exact list starts with the rows of the bitmap bin
    const long long cnt_last = h->lsize[last];
    if (cnt_last > 0) {
        if (h->lid) CK(launch_iota(L.xlist, mw, s));
        else CK(cudaMemcpyAsync(L.xlist, d_bins(h) + h->loff[last], sizeof(int32_t) * (size_t)cnt_last,
                                cudaMemcpyDeviceToDevice, s));
    }
    unsigned long long *h_x = reinterpret_cast<unsigned long long *>(
        reinterpret_cast<unsigned char *>(h->h_cnt) + 2 * sizeof(Counters) + 16);
    *h_x = static_cast<unsigned long long>(cnt_last);
    CK(cudaMemcpyAsync(d_xcount(h), h_x, sizeof(unsigned long long), cudaMemcpyHostToDevice, s));
    // temporary rows: bin j's row r at tbase_j + r * cap_j
    long long total_t = 0;
    for (int j = 0; j < last; ++j) {
        h->ltcap[j] = num_kernel(h->cfg.num_kernel[j]).max_size;
        h->ltbase[j] = total_t;
        total_t += h->lsize[j] * h->ltcap[j];
    }
    h->tcol = nullptr;
    h->tval = nullptr;
    h->ltotal = total_t;
    if (total_t > 0) {
        h->tcol = static_cast<int32_t *>(dev_alloc(h, sizeof(int32_t) * (size_t)total_t));
        h->tval = static_cast<double *>(dev_alloc(h, sizeof(double) * (size_t)total_t));
        if (!h->tcol || !h->tval) return SPGEMM_ERR_OOM;
    }
    // one-phase kernels, largest rows first on the side streams
    CK(cudaEventRecord(h->ev_fork, s));
    int used = 0;
    for (int j = last - 1; j >= 0; --j) {
        if (h->lsize[j] <= 0) continue;
        cudaStream_t ss = h->serial ? s : h->side[used % kSide];
        if (!h->serial && used < kSide) CK(cudaStreamWaitEvent(ss, h->ev_fork, 0));
        BinWork w{};
        w.bins = h->lid ? nullptr : d_bins(h);
        w.off = h->lid ? 0 : h->loff[j];
        w.cnt = h->lsize[j];
        w.crpt = crpt;
        w.lanes = h->cfg.num_lanes_per_brow;
        w.distinct = h->b_distinct;
        w.err = d_err(h);
        w.tcol = h->tcol; w.tval = h->tval;
        w.tbase = h->ltbase[j]; w.tcap = h->ltcap[j];
        w.tlimit = total_t;
        w.pred = L.pred; w.xlist = L.xlist; w.xcount = d_xcount(h);
        w.xlimit = mw;
        w.lcls = L.cls;
        w.fb = L.fb;
        w.tprev = j > 0 ? num_kernel(h->cfg.num_kernel[j - 1]).table : 0;
        const int slot = kSlotNumBin + j;
        time_begin(h, slot, ss);
        CK(launch_num_onephase(h->cfg.num_kernel[j], op, w, ss));
        time_end(h, slot, ss);
        ++used;
    }
    for (int i = 0; !h->serial && i < std::min(used, kSide); ++i) {
        CK(cudaEventRecord(h->ev_side[i], h->side[i]));
        CK(cudaStreamWaitEvent(s, h->ev_side[i], 0));
    }
    CK(cudaMemcpyAsync(h_x, d_xcount(h), sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    h->xcount = static_cast<int64_t>(*h_x);
    if (h->xcount > mw) return SPGEMM_ERR_INTERNAL;
    // exact symbolic for the bitmap-bin rows and the mispredicted rows
    if (h->xcount > 0) {
        BinWork w{};
        w.bins = L.xlist; w.off = 0; w.cnt = h->xcount;
        w.crpt = crpt;
        w.lanes = h->cfg.lanes_per_brow;
        w.unroll = h->cfg.bitmap_unroll;
        w.err = d_err(h);
        const int64_t budget = h->smem_dyn_max - static_cast<int64_t>(sizeof(WalkScratch));
        int64_t words = std::min<int64_t>((op.ncols + 31) / 32, budget / 4);
        if (h->split_idx) {   // several column passes: each walks only its runs
            w.bslot = h->wbslot;
            w.bidx = h->wbidx;
            w.cs = h->split_cs;
            w.ncells = h->split_ncells;
            w.bflags = &d_counters(h, 1)->flags;
            const int64_t cwords = int64_t{1} << (h->split_cs - 5);
            if (words < (op.ncols + 31) / 32) words = std::max<int64_t>(cwords, (words / cwords) * cwords);
        }
        time_begin(h, kSlotSymBin + 15, s);
        CK(launch_sym(sym_kernel_count() - 1, op, w, static_cast<size_t>(std::max<int64_t>(words, 1)) * 4, s));
        time_end(h, kSlotSymBin + 15, s);
    }
    // total n_nz and the scan's tile sums
    Ranges all{};
    all.nb = 1;
    all.r[0] = -1;
    time_begin(h, kSlotNumPass1, s);
    CK(launch_bin_pass1(crpt, mw, all, op, d_counters(h, 1), d_tiles(h), s));
    time_end(h, kSlotNumPass1, s);
    unsigned long long *h_fb = reinterpret_cast<unsigned long long *>(
        reinterpret_cast<unsigned char *>(h->h_cnt) + 2 * sizeof(Counters) + 64);
    CK(cudaMemcpyAsync(h_fb, L.fb, sizeof(unsigned long long) * kFbCounters, cudaMemcpyDeviceToHost, s));
    if ((rc = read_counters(h))) return rc;
    h->b_unsorted = (h->h_cnt[1].flags & 1ull) != 0;
    *nnz_out = static_cast<int64_t>(h->h_cnt[1].total);
    h->lstats[0] = 0;
    for (int j = 0; j < last; ++j) h->lstats[0] += h->lsize[j];
    h->lstats[1] = h->xcount - cnt_last;
    h->lstats[0] -= h->lstats[1];
    h->lstats[2] = cnt_last;
    h->lstats[3] = total_t;
    // Load feedback, per class of rows: the factor for the next call.
    // Doubling a class's factor moves its rows at most one table up, halving
    // it at most one table down. Double it when more than a quarter of the
    // class's rows tried in one phase overflowed or ended more than 3/4 full
    // (under-predicted: probes get long); halve it when at least 15/16 of
    // them would fill the next smaller table at most 3/4 (over-predicted:
    // set-up, condense and sort scan a table larger than needed).
    auto fbsum = [&](int grp, int b) {
        unsigned long long t = 0;
        for (int k = 0; k < kLoadSlots; ++k) t += h_fb[(grp * kMaxBins + b) * kLoadSlots + k];
        return static_cast<long long>(t);
    };
    h->lstats[4] = 0;
    h->lstats[5] = 0;
    for (int b = 0; b < kMaxBins; ++b) h->lstats[6 + b] = h->lfk[b];
    for (int b = 0; b + 1 < nb; ++b) {
        const long long tried = fbsum(0, b), hi = fbsum(1, b), lo = fbsum(2, b), mis = fbsum(3, b);
        h->lstats[4] += hi;
        h->lstats[5] += lo;
        if (tried <= 0) continue;
        if (4 * (hi + mis) > tried) h->lfk[b] = std::min(h->lfk[b] + 1, kMaxFactorLog2);
        else if (16 * lo >= 15 * tried) h->lfk[b] = std::max(h->lfk[b] - 1, -kMaxFactorLog2);
    }
    return SPGEMM_OK;
}

// Numeric part: scan, C allocation, copy of the one-phase rows, exact
// numeric kernel for the exact list.
int numeric_learned(spgemm_handle *h, const Operands &op, int64_t *crpt, int32_t **pcol,
                    double **pval, bool given) {
    cudaStream_t s = h->stream;
    const LScratch L = lscratch_layout(h, h->mw);
    time_begin(h, kSlotScan, s);
    CK(launch_scan(crpt, h->mw, d_tiles(h), s));
    time_end(h, kSlotScan, s);
    if (!given) {
        *pcol = static_cast<int32_t *>(dev_alloc(h, sizeof(int32_t) * (size_t)h->nnz));
        *pval = static_cast<double *>(dev_alloc(h, sizeof(double) * (size_t)h->nnz));
        if (!*pcol || !*pval) return SPGEMM_ERR_OOM;
    }
    const int last = h->cfg.num_nbins - 1;
    time_begin(h, kSlotCopy, s);
    for (int j = 0; j < last; ++j) {
        if (h->lsize[j] <= 0) continue;
        BinWork w{};
        w.bins = h->lid ? nullptr : d_bins(h);
        w.off = h->lid ? 0 : h->loff[j];
        w.cnt = h->lsize[j];
        w.crpt = crpt; w.ccol = *pcol; w.cval = *pval;
        w.tcol = h->tcol; w.tval = h->tval;
        w.tbase = h->ltbase[j]; w.tcap = h->ltcap[j];
        w.tlimit = h->ltotal;
        w.pred = L.pred;
        w.err = d_err(h);
        CK(launch_copy_rows(w, s));
    }
    time_end(h, kSlotCopy, s);
    if (h->xcount > 0) {
        BinWork w{};
        w.bins = L.xlist; w.off = 0; w.cnt = h->xcount;
        w.crpt = crpt; w.ccol = *pcol; w.cval = *pval;
        w.lanes = h->cfg.num_lanes_per_brow;
        w.unroll = h->cfg.bitmap_unroll;
        w.err = d_err(h);
        const int64_t budget = h->smem_dyn_max - static_cast<int64_t>(num_bitmap_head_bytes(false));
        int64_t words = std::min<int64_t>((op.ncols + 63) / 64, budget / 12);
        if (h->split_idx && !h->b_unsorted) {   // several column windows: each walks only its runs
            w.bslot = h->wbslot;
            w.bidx = h->wbidx;
            w.cs = h->split_cs;
            w.ncells = h->split_ncells;
            const int64_t cwords = int64_t{1} << (h->split_cs - 6);
            if (words < (op.ncols + 63) / 64) words = std::max<int64_t>(cwords, (words / cwords) * cwords);
        }
        time_begin(h, kSlotNumBin + 15, s);
        CK(launch_num(num_kernel_count() - 1, op, w, static_cast<size_t>(std::max<int64_t>(words, 1)) * 12, s));
        time_end(h, kSlotNumBin + 15, s);
    }
    dev_free(h, h->tcol);
    dev_free(h, h->tval);
    h->tcol = nullptr;
    h->tval = nullptr;
    return SPGEMM_OK;
}

}  // namespace

extern "C" {

const char *spgemm_last_cuda_error(void) {
    return g_last_cuda == cudaSuccess ? nullptr : cudaGetErrorName(g_last_cuda);
}

const char *spgemm_strerror(int code) {
    switch (code) {
        case SPGEMM_OK: return "ok";
        case SPGEMM_ERR_INVALID: return "invalid argument";
        case SPGEMM_ERR_SHAPE: return "shape mismatch (A.cols != B.rows)";
        case SPGEMM_ERR_OOM: return "out of device memory";
        case SPGEMM_ERR_STATE: return "call out of order";
        case SPGEMM_ERR_TIMEOUT: return "bounded device wait expired";
        case SPGEMM_ERR_CUDA: return "CUDA runtime error";
        case SPGEMM_ERR_INTERNAL: return "device-side check failed";
        case SPGEMM_ERR_ABORTED: return "the host sink stopped the transfer";
        default: return "unknown error";
    }
}

int spgemm_kernel_info(int phase, int id, int32_t *tpr, int32_t *block, int64_t *table,
                       int64_t *max_size) {
    const int n = phase ? num_kernel_count() : sym_kernel_count();
    if (phase < 0 || phase > 1 || id < 0 || id >= n) return SPGEMM_ERR_INVALID;
    const KernelDesc &d = phase ? num_kernel(id) : sym_kernel(id);
    if (tpr) *tpr = d.tpr;
    if (block) *block = d.block;
    if (table) *table = d.table;
    if (max_size) *max_size = d.bitmap ? -1 : d.max_size;
    return SPGEMM_OK;
}

int spgemm_create(spgemm_handle **out, const spgemm_config *cfg, spgemm_alloc_fn alloc,
                  spgemm_free_fn free_fn, void *ctx, void *stream) {
    if (!out) return SPGEMM_ERR_INVALID;
    *out = nullptr;
    if ((alloc == nullptr) != (free_fn == nullptr)) return SPGEMM_ERR_INVALID;
    spgemm_handle *h = new (std::nothrow) spgemm_handle();
    if (!h) return SPGEMM_ERR_OOM;
    int rc = SPGEMM_OK;
    do {
        if (cudaGetDevice(&h->device) != cudaSuccess) { rc = SPGEMM_ERR_CUDA; break; }
        int optin = 0;
        cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
        h->smem_dyn_max = optin - 1024;  // room for the kernels' static shared arrays
        if (prepare_device(h->device, h->smem_dyn_max) != cudaSuccess) {
            rc = SPGEMM_ERR_CUDA;
            break;
        }
        h->stream = static_cast<cudaStream_t>(stream);
        h->alloc = alloc;
        h->freefn = free_fn;
        h->ctx = ctx;
        for (int i = 0; i < kSide; ++i) {
            if (cudaStreamCreateWithFlags(&h->side[i], cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&h->ev_side[i], cudaEventDisableTiming) != cudaSuccess) {
                rc = SPGEMM_ERR_CUDA;
                break;
            }
        }
        if (rc) break;
        if (cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess) { rc = SPGEMM_ERR_CUDA; break; }
        if (cudaMallocHost(&h->h_cnt, 2 * sizeof(Counters) + 64 + sizeof(unsigned long long) * kFbCounters) !=
            cudaSuccess) { rc = SPGEMM_ERR_OOM; break; }
        if (!alloc) {
            cudaMemPoolProps props{};
            props.allocType = cudaMemAllocationTypePinned;
            props.handleTypes = cudaMemHandleTypeNone;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = h->device;
            if (cudaMemPoolCreate(&h->pool, &props) != cudaSuccess) { rc = SPGEMM_ERR_CUDA; break; }
            uint64_t thr = UINT64_MAX;
            cudaMemPoolSetAttribute(h->pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
        if (cfg) {
            if (validate_config(*cfg) != SPGEMM_OK) { rc = SPGEMM_ERR_INVALID; break; }
            h->cfg = *cfg;
        } else {
            default_config(h->cfg);
            h->cfg_auto = true;
        }
    } while (0);
    if (rc != SPGEMM_OK) {
        cudaGetLastError();
        spgemm_destroy(h);
        return rc;
    }
    *out = h;
    return SPGEMM_OK;
}

int spgemm_set_config(spgemm_handle *h, const spgemm_config *cfg) {
    if (!h) return SPGEMM_ERR_INVALID;
    h->reuse = false;   // the kept rows were binned for the old kernels
    if (!cfg) {
        default_config(h->cfg);
        h->cfg_auto = true;
        return SPGEMM_OK;
    }
    if (validate_config(*cfg) != SPGEMM_OK) return SPGEMM_ERR_INVALID;
    h->cfg = *cfg;
    h->cfg_auto = false;
    return SPGEMM_OK;
}

int spgemm_get_config(const spgemm_handle *h, spgemm_config *cfg) {
    if (!h || !cfg) return SPGEMM_ERR_INVALID;
    *cfg = h->cfg;
    return SPGEMM_OK;
}

int spgemm_symbolic(spgemm_handle *h, const spgemm_csr_in *A, const spgemm_csr_in *B,
                    int64_t row_begin, int64_t row_end, int64_t *nnzC) {
    if (!h || !nnzC) return SPGEMM_ERR_INVALID;
    int rc = check_csr_in(A);
    if (rc) return rc;
    if ((rc = check_csr_in(B))) return rc;
    if (A->cols != B->rows) return SPGEMM_ERR_SHAPE;
    if (row_begin < 0 || row_end < row_begin || row_end > A->rows) return SPGEMM_ERR_INVALID;
    h->reuse = false;   // the binning below overwrites the kept rows
    if (h->state == 1) {  // an earlier symbolic result was never consumed
        dev_free(h, h->crpt);
        dev_free(h, h->tcol);
        dev_free(h, h->tval);
        h->crpt = nullptr;
        h->tcol = nullptr;
        h->tval = nullptr;
        h->state = 0;
    }
    const int64_t mw = row_end - row_begin;
    h->mw = mw;
    if (h->cfg_auto) auto_cut(h->cfg, B->cols);
    win_release(h);
    h->wp_on = h->mode == SPGEMM_MODE_PLAIN && win_setup(h, B->cols);
    h->split_on = split_setup(h, B->cols);
    h->split_keep = false;
    h->split_idx = false;
    h->nwin = 0;
    h->nwin_col = 0;
    h->win_used = false;
    if ((rc = ensure_arena(h, mw))) return rc;
    int64_t *crpt = static_cast<int64_t *>(dev_alloc(h, sizeof(int64_t) * (size_t)(mw + 1)));
    if (!crpt) return SPGEMM_ERR_OOM;
    auto fail = [&](int code) {
        dev_free(h, crpt);
        return code;
    };
    // zero both phases' counters, keep the error word
    if (note(cudaMemsetAsync(h->arena, 0, 2 * sizeof(Counters), h->stream)) != cudaSuccess ||
        note(cudaMemsetAsync(crpt, 0, sizeof(int64_t) * (size_t)(mw + 1), h->stream)) != cudaSuccess)
        return fail(SPGEMM_ERR_CUDA);
    const Operands op = make_operands(A, B, row_begin, mw);
    // cell index of B's long rows for kernels that cover rows in several
    // column windows (built here, used by both phases; the symbolic kernel
    // checks on the device that B is sorted)
    if (h->split_on || h->mode == SPGEMM_MODE_LEARNED) {
        if (note(launch_sorted_check(op, B->rows, B->nnz, d_counters(h, 1), h->sm_count * 4, h->stream)) !=
            cudaSuccess)
            return fail(SPGEMM_ERR_CUDA);
        if (h->split_on && (rc = build_bindex(h, op, B))) return fail(rc);
    }
    if (h->mode == SPGEMM_MODE_LEARNED) {
        // the one-phase kernels multiply during this call: they read values
        if ((A->nnz > 0 && !A->val) || (B->nnz > 0 && !B->val)) return fail(SPGEMM_ERR_INVALID);
        int64_t nnz = 0;
        if ((rc = symbolic_learned(h, op, A->rows, crpt, &nnz))) {
            dev_free(h, h->tcol);
            dev_free(h, h->tval);
            h->tcol = nullptr;
            h->tval = nullptr;
            return fail(rc);
        }
        h->stats[0] = 0;
        h->stats[1] = 0;
        h->stats[2] = nnz;
        h->stats[3] = static_cast<int64_t>(h->h_cnt[1].max_size);
        h->crpt = crpt;
        h->row0 = row_begin;
        h->ncols = B->cols;
        h->nnz = nnz;
        h->state = 1;
        *nnzC = nnz;
        return SPGEMM_OK;
    }
    // rows of B must be sorted for the windowed pass 2 of the numeric bitmap kernel
    // step 1: n_prod per row into C.rpt
    time_begin(h, kSlotNprod, h->stream);
    if (note(launch_nprod(op, crpt, h->sm_count * 8, h->stream)) != cudaSuccess) return fail(SPGEMM_ERR_CUDA);
    time_end(h, kSlotNprod, h->stream);
    h->rplan = run_plan(h->cfg, h->smem_dyn_max, B->cols);
    // B's column order: the windowed kernels need sorted rows, the warp-row
    // numeric hash kernels skip value atomics when columns are distinct
    if (!h->split_on &&
        note(launch_sorted_check(op, B->rows, B->nnz, d_counters(h, 1), h->sm_count * 4, h->stream)) !=
            cudaSuccess)
        return fail(SPGEMM_ERR_CUDA);
    // step 2: symbolic binning by n_prod
    Ranges rs{};
    rs.nb = h->cfg.sym_nbins;
    for (int j = 0; j < rs.nb; ++j) rs.r[j] = h->cfg.sym_range[j];
    time_begin(h, kSlotSymPass1, h->stream);
    if (note(launch_bin_pass1(crpt, mw, rs, op, d_counters(h, 0), nullptr, h->stream)) != cudaSuccess)
        return fail(SPGEMM_ERR_CUDA);
    time_end(h, kSlotSymPass1, h->stream);
    if ((rc = read_counters(h))) return fail(rc);
    long long ssize[kMaxBins] = {}, soff[kMaxBins] = {};
    const bool sid = plan_bins(h->h_cnt[0], rs.nb, ssize, soff);
    h->stats[0] = static_cast<int64_t>(h->h_cnt[0].total);
    h->stats[1] = static_cast<int64_t>(h->h_cnt[0].max_size);
    for (int j = 0; j < SPGEMM_MAX_BINS; ++j) h->stats[4 + j] = j < rs.nb ? ssize[j] : 0;
    if (!sid) {
        time_begin(h, kSlotSymPass2, h->stream);
        if (note(launch_bin_pass2(crpt, mw, rs, soff, d_counters(h, 0), d_bins(h), h->stream)) != cudaSuccess)
            return fail(SPGEMM_ERR_CUDA);
        time_end(h, kSlotSymPass2, h->stream);
    }
    // cell counts of the symbolic bitmap bin's rows for the column windows
    WinCall wc0;
    if (h->wp_on) {
        const long long nbm = ssize[rs.nb - 1];
        if (nbm > 0 &&
            ((rc = ensure_buf(h, &h->wcells, &h->wcells_bytes,
                              sizeof(uint16_t) * (size_t)nbm * (size_t)h->wplan.ncells)) ||
             (rc = ensure_buf(h, &h->wcslot, &h->wcslot_bytes, sizeof(int32_t) * (size_t)std::max<int64_t>(mw, 1)))))
            return fail(rc);
        if (nbm > 0 && note(cudaMemsetAsync(h->wcslot, 0xff, sizeof(int32_t) * (size_t)mw, h->stream)) != cudaSuccess)
            return fail(SPGEMM_ERR_CUDA);
        wc0.on = nbm > 0;
    }
    // step 3: symbolic kernels, largest rows first
    if ((rc = run_bins(h, 0, op, ssize, soff, sid, crpt, nullptr, nullptr, nullptr, &wc0))) return fail(rc);
    // windows of the rows of the last numeric bin (their count sizes the list)
    if (h->wp_on &&
        note(launch_win_count(h->wplan, crpt, mw, wc0.on ? h->wcells : nullptr, wc0.on ? h->wcslot : nullptr,
                              &d_counters(h, 1)->windows, &d_counters(h, 1)->wcol, d_err(h), h->stream)) !=
            cudaSuccess)
        return fail(SPGEMM_ERR_CUDA);
    // step 4: numeric binning pass 1 -> total n_nz (and tile sums for the scan)
    Ranges rn{};
    rn.nb = h->cfg.num_nbins;
    for (int j = 0; j < rn.nb; ++j) rn.r[j] = h->cfg.num_range[j];
    time_begin(h, kSlotNumPass1, h->stream);
    if (note(launch_bin_pass1(crpt, mw, rn, op, d_counters(h, 1), d_tiles(h), h->stream)) != cudaSuccess)
        return fail(SPGEMM_ERR_CUDA);
    time_end(h, kSlotNumPass1, h->stream);
    if ((rc = read_counters(h))) return fail(rc);
    h->b_unsorted = (h->h_cnt[1].flags & 1ull) != 0;
    h->b_distinct = (h->h_cnt[1].flags & 3ull) == 0;
    h->nwin = static_cast<long long>(h->h_cnt[1].windows);
    h->nwin_col = static_cast<long long>(h->h_cnt[1].wcol);
    h->stats[2] = static_cast<int64_t>(h->h_cnt[1].total);
    h->stats[3] = static_cast<int64_t>(h->h_cnt[1].max_size);
    for (int j = 0; j < SPGEMM_MAX_BINS; ++j)
        h->stats[4 + SPGEMM_MAX_BINS + j] = j < rn.nb ? static_cast<int64_t>(h->h_cnt[1].bin_cnt[j]) : 0;
    for (int j = 0; j < kMaxBins; ++j) h->num_size[j] = j < rn.nb ? h->h_cnt[1].bin_cnt[j] : 0;
    h->crpt = crpt;
    h->row0 = row_begin;
    h->ncols = B->cols;
    h->nnz = static_cast<int64_t>(h->h_cnt[1].total);
    h->state = 1;
    *nnzC = h->nnz;
    return SPGEMM_OK;
}

int spgemm_numeric(spgemm_handle *h, const spgemm_csr_in *A, const spgemm_csr_in *B,
                   spgemm_csr_out *C) {
    if (!h || !C) return SPGEMM_ERR_INVALID;
    if (h->state != 1) return SPGEMM_ERR_STATE;
    int rc = check_csr_in(A);
    if (rc) return rc;
    if ((rc = check_csr_in(B))) return rc;
    if (A->cols != B->rows) return SPGEMM_ERR_SHAPE;
    if (h->row0 + h->mw > A->rows || B->cols != h->ncols) return SPGEMM_ERR_STATE;
    if ((A->nnz > 0 && !A->val) || (B->nnz > 0 && !B->val)) return SPGEMM_ERR_INVALID;
    const bool given = C->col != nullptr && C->val != nullptr;
    // from here on the symbolic result is consumed
    h->state = 0;
    h->reuse = false;
    int64_t *crpt = h->crpt;
    h->crpt = nullptr;
    const Operands op = make_operands(A, B, h->row0, h->mw);
    if (h->mode == SPGEMM_MODE_LEARNED) {
        int32_t *ccol = C->col;
        double *cval = C->val;
        rc = numeric_learned(h, op, crpt, &ccol, &cval, given);
        if (rc) {
            dev_free(h, crpt);
            if (!given) {
                dev_free(h, ccol);
                dev_free(h, cval);
            }
            dev_free(h, h->tcol);
            dev_free(h, h->tval);
            h->tcol = nullptr;
            h->tval = nullptr;
            return rc;
        }
        C->rows = h->mw; C->cols = h->ncols; C->nnz = h->nnz;
        C->rpt = crpt; C->col = ccol; C->val = cval;
        return SPGEMM_OK;
    }
    const int nb = h->cfg.num_nbins;
    long long off[kMaxBins] = {};
    long long acc = 0;
    int nonempty = 0;
    for (int j = 0; j < nb; ++j) {
        off[j] = acc;
        acc += h->num_size[j];
        nonempty += h->num_size[j] > 0;
    }
    // windowed pass 2 for the bitmap bin when every row of B is sorted
    RunPlan rp = h->rplan;
    if (h->b_unsorted || !num_kernel(h->cfg.num_kernel[nb - 1]).bitmap || h->num_size[nb - 1] <= 0)
        rp = RunPlan{};
    const bool nid = nonempty <= 1;
    Ranges rn{};
    rn.nb = nb;
    for (int j = 0; j < nb; ++j) rn.r[j] = h->cfg.num_range[j];
    int32_t *ccol = C->col;
    double *cval = C->val;
    auto fail = [&](int code) {
        dev_free(h, crpt);
        if (!given) {
            dev_free(h, ccol);
            dev_free(h, cval);
        }
        return code;
    };
    if (!nid) {
        time_begin(h, kSlotNumPass2, h->stream);
        if (note(launch_bin_pass2(crpt, h->mw, rn, off, d_counters(h, 1), d_bins(h), h->stream)) != cudaSuccess)
            return fail(SPGEMM_ERR_CUDA);
        time_end(h, kSlotNumPass2, h->stream);
    }
    time_begin(h, kSlotScan, h->stream);
    if (note(launch_scan(crpt, h->mw, d_tiles(h), h->stream)) != cudaSuccess) return fail(SPGEMM_ERR_CUDA);
    time_end(h, kSlotScan, h->stream);
    // C.col / C.val allocated while the binning and scan kernels run (Sec. 5.4)
    if (!given) {
        ccol = static_cast<int32_t *>(dev_alloc(h, sizeof(int32_t) * (size_t)h->nnz));
        cval = static_cast<double *>(dev_alloc(h, sizeof(double) * (size_t)h->nnz));
        if (!ccol || !cval) return fail(SPGEMM_ERR_OOM);
    }
    // column windows for the last bin
    WinCall wc;
    const int last = nb - 1;
    if (h->wp_on && !h->b_unsorted && h->num_size[last] > 0 && h->nwin > 0 &&
        num_kernel(h->cfg.num_kernel[last]).bitmap) {
        win_release(h);
        const WinPlan &p = h->wplan;
        wc.on = true;
        wc.min_len = std::max<long long>(32, (p.ncells + 1) / 2);
        wc.bcap = B->nnz / wc.min_len + 1;
        wc.brows = B->rows;
        wc.cap = h->nwin;
        h->wlist = static_cast<Win *>(dev_alloc(h, sizeof(Win) * (size_t)h->nwin));
        h->wctr = static_cast<unsigned long long *>(dev_alloc(h, 4 * sizeof(unsigned long long)));
        h->wbslot = static_cast<int32_t *>(dev_alloc(h, sizeof(int32_t) * (size_t)std::max<int64_t>(B->rows, 1)));
        h->wbidx = static_cast<int32_t *>(dev_alloc(h, sizeof(int32_t) * (size_t)wc.bcap * (size_t)(p.ncells + 1)));
        if (!h->wlist || !h->wctr || !h->wbslot || !h->wbidx) {
            win_release(h);
            return fail(SPGEMM_ERR_OOM);
        }
        if (note(cudaMemsetAsync(h->wctr, 0, 4 * sizeof(unsigned long long), h->stream)) != cudaSuccess) {
            win_release(h);
            return fail(SPGEMM_ERR_CUDA);
        }
        wc.list = h->wlist;
        wc.cursor = h->wctr;
        wc.nslot = h->wctr + 2;
        wc.bslot = h->wbslot;
        wc.bidx = h->wbidx;
        wc.ww.win = h->wlist;
        wc.ww.nwin = h->nwin;
        wc.ww.next = h->wctr + 1;
        wc.ww.bslot = h->wbslot;
        wc.ww.bidx = h->wbidx;
        wc.ww.cs = p.cs;
        wc.ww.ncells = p.ncells;
        wc.ww.budget = p.budget;
        wc.ww.spill_stride = p.budget / 8;
        if ((rc = ensure_spill(h, wc.ww.spill_stride))) {
            win_release(h);
            return fail(rc);
        }
        wc.ww.spill = h->wspill;
        rp = RunPlan{};
    }
    // whole-row bitmap kernel by column windows over the cell index that the
    // symbolic call built
    if (!wc.on && h->split_idx && !h->b_unsorted && h->num_size[last] > 0 && rp.lists == 0 &&
        num_kernel(h->cfg.num_kernel[last]).bitmap) {
        wc.split = true;
        wc.cs = h->split_cs;
        wc.ncells = h->split_ncells;
        wc.bslot = h->wbslot;
        wc.bidx = h->wbidx;
    }
    // run boundaries of B's rows at the column sub-ranges, for the windowed pass 2
    int32_t *bs = nullptr;
    if (rp.lists > 0) {
        bs = static_cast<int32_t *>(dev_alloc(h, sizeof(int32_t) * (size_t)B->rows * (size_t)(rp.G + 1)));
        if (!bs) return fail(SPGEMM_ERR_OOM);
        if (note(launch_bsplit(op, B->rows, B->nnz, rp.gshift, rp.G, bs, h->sm_count * 4, h->stream)) !=
            cudaSuccess) {
            dev_free(h, bs);
            return fail(SPGEMM_ERR_CUDA);
        }
        rp.bs = bs;
    }
    rc = run_bins(h, 1, op, h->num_size, off, nid, crpt, ccol, cval, &rp, &wc);
    dev_free(h, bs);
    if (rc) {
        win_release(h);
        return fail(rc);
    }
    h->wkeep = wc.on;
    h->win_used = wc.on;
    h->split_keep = wc.split;
    h->reuse = true;
    h->reuse_arows = A->rows;
    h->reuse_annz = A->nnz;
    h->reuse_brows = B->rows;
    h->reuse_bnnz = B->nnz;
    C->rows = h->mw;
    C->cols = h->ncols;
    C->nnz = h->nnz;
    C->rpt = crpt;
    C->col = ccol;
    C->val = cval;
    return SPGEMM_OK;
}

// Numeric kernels again over the kept bins and C.rpt (same structure, new
// values): no n_prod, binning, symbolic, scan or allocation. The bitmap bin
// takes the whole-row pass 2 (its windowed form needs a scratch buffer).
int spgemm_numeric_values(spgemm_handle *h, const spgemm_csr_in *A, const spgemm_csr_in *B,
                          const spgemm_csr_out *C) {
    if (!h || !C) return SPGEMM_ERR_INVALID;
    int rc = check_csr_in(A);
    if (rc) return rc;
    if ((rc = check_csr_in(B))) return rc;
    if (A->cols != B->rows) return SPGEMM_ERR_SHAPE;
    if (!h->reuse) return SPGEMM_ERR_STATE;
    if (A->rows != h->reuse_arows || A->nnz != h->reuse_annz || B->rows != h->reuse_brows ||
        B->nnz != h->reuse_bnnz || B->cols != h->ncols)
        return SPGEMM_ERR_STATE;
    if ((A->nnz > 0 && !A->val) || (B->nnz > 0 && !B->val)) return SPGEMM_ERR_INVALID;
    if (C->rows != h->mw || C->cols != h->ncols || C->nnz != h->nnz || !C->rpt ||
        (C->nnz > 0 && (!C->col || !C->val)))
        return SPGEMM_ERR_INVALID;
    const int nb = h->cfg.num_nbins;
    long long off[kMaxBins] = {};
    long long acc = 0;
    int nonempty = 0;
    for (int j = 0; j < nb; ++j) {
        off[j] = acc;
        acc += h->num_size[j];
        nonempty += h->num_size[j] > 0;
    }
    const Operands op = make_operands(A, B, h->row0, h->mw);
    // the last bin reuses the windows and B index of the numeric call
    WinCall wc;
    if (h->wkeep) {
        wc.on = true;
        wc.plan = false;
        wc.ww.win = h->wlist;
        wc.ww.nwin = h->nwin;
        wc.ww.next = h->wctr + 1;
        wc.ww.bslot = h->wbslot;
        wc.ww.bidx = h->wbidx;
        wc.ww.cs = h->wplan.cs;
        wc.ww.ncells = h->wplan.ncells;
        wc.ww.budget = h->wplan.budget;
        wc.ww.spill_stride = h->wplan.budget / 8;
        wc.ww.spill = h->wspill;
        CK(cudaMemsetAsync(h->wctr + 1, 0, sizeof(unsigned long long), h->stream));
    } else if (h->split_keep) {
        wc.split = true;
        wc.cs = h->split_cs;
        wc.ncells = h->split_ncells;
        wc.bslot = h->wbslot;
        wc.bidx = h->wbidx;
    }
    return run_bins(h, 1, op, h->num_size, off, nonempty <= 1, static_cast<int64_t *>(C->rpt), C->col,
                    C->val, nullptr, &wc);
}

int spgemm_multiply(spgemm_handle *h, const spgemm_csr_in *A, const spgemm_csr_in *B,
                    spgemm_csr_out *C) {
    if (!h || !A || !C) return SPGEMM_ERR_INVALID;
    int64_t nnz = 0;
    int rc = spgemm_symbolic(h, A, B, 0, A->rows, &nnz);
    if (rc) return rc;
    return spgemm_numeric(h, A, B, C);
}

int spgemm_status(spgemm_handle *h) {
    if (!h) return SPGEMM_ERR_INVALID;
    CK(cudaStreamSynchronize(h->stream));
    if (!h->arena) return SPGEMM_OK;
    int err = 0;
    CK(cudaMemcpy(&err, d_err(h), sizeof(int), cudaMemcpyDeviceToHost));
    if (err) {
        CK(cudaMemset(d_err(h), 0, sizeof(int)));
        return SPGEMM_ERR_INTERNAL;
    }
    return SPGEMM_OK;
}

int spgemm_free(spgemm_handle *h, void *ptr) {
    if (!h) return SPGEMM_ERR_INVALID;
    dev_free(h, ptr);
    return SPGEMM_OK;
}

int spgemm_last_stats(const spgemm_handle *h, int64_t *out, int n) {
    if (!h || !out || n < 0) return SPGEMM_ERR_INVALID;
    const int m = std::min<int>(n, 4 + 2 * SPGEMM_MAX_BINS);
    std::memcpy(out, h->stats, sizeof(int64_t) * (size_t)m);
    return SPGEMM_OK;
}

static int multiply_host(spgemm_handle *h, const spgemm_csr_in *A, const spgemm_csr_in *B,
                         int64_t chunk_bytes, spgemm_host_sink_fn sink, void *ctx,
                         int64_t *nnzC) {
    if (!h || !A || !B || !sink) return SPGEMM_ERR_INVALID;
    int rc = check_csr_in(A);
    if (rc) return rc;
    if ((rc = check_csr_in(B))) return rc;
    if (A->cols != B->rows) return SPGEMM_ERR_SHAPE;
    if ((A->nnz > 0 && !A->val) || (B->nnz > 0 && !B->val)) return SPGEMM_ERR_INVALID;
    if (chunk_bytes < (1 << 20)) chunk_bytes = 1 << 20;
    for (auto &cs : h->copyst)
        if (!cs && cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return SPGEMM_ERR_CUDA;
    const bool same = A->rpt == B->rpt && A->col == B->col && A->val == B->val &&
                      A->rows == B->rows && A->rpt_is_i64 == B->rpt_is_i64;
    // host -> device copies of the operands
    void *dev[7] = {};
    auto release = [&]() {
        for (void *p : dev) dev_free(h, p);
    };
    auto upload = [&](const spgemm_csr_in *m, void **slot, spgemm_csr_in *d) -> int {
        const size_t rb = (size_t)(m->rows + 1) * (m->rpt_is_i64 ? 8 : 4);
        slot[0] = dev_alloc(h, rb);
        slot[1] = dev_alloc(h, sizeof(int32_t) * (size_t)m->nnz);
        slot[2] = dev_alloc(h, sizeof(double) * (size_t)m->nnz);
        if (!slot[0] || !slot[1] || !slot[2]) return SPGEMM_ERR_OOM;
        CK(cudaMemcpyAsync(slot[0], m->rpt, rb, cudaMemcpyHostToDevice, h->stream));
        if (m->nnz) {
            CK(cudaMemcpyAsync(slot[1], m->col, sizeof(int32_t) * (size_t)m->nnz,
                               cudaMemcpyHostToDevice, h->stream));
            CK(cudaMemcpyAsync(slot[2], m->val, sizeof(double) * (size_t)m->nnz,
                               cudaMemcpyHostToDevice, h->stream));
        }
        *d = *m;
        d->rpt = slot[0];
        d->col = static_cast<const int32_t *>(slot[1]);
        d->val = static_cast<const double *>(slot[2]);
        return SPGEMM_OK;
    };
    spgemm_csr_in dA{}, dB{};
    if ((rc = upload(A, dev, &dA))) { release(); return rc; }
    if (same) dB = dA;
    else if ((rc = upload(B, dev + 3, &dB))) { release(); return rc; }
    const int64_t M = A->rows;

    // Slabs of rows with about equal n_prod: slab s + 1 is computed while
    // slab s is copied to the host, so the copies (bound by the host link)
    // hide the arithmetic.
    std::vector<int64_t> cut{0, M};
    if (M > 1) {
        int64_t *d_np = static_cast<int64_t *>(dev_alloc(h, sizeof(int64_t) * (size_t)M));
        dev[6] = d_np;
        if (!d_np) { release(); return SPGEMM_ERR_OOM; }
        const Operands op = make_operands(&dA, &dB, 0, M);
        std::vector<int64_t> np((size_t)M);
        if (cudaMemsetAsync(d_np, 0, sizeof(int64_t) * (size_t)M, h->stream) != cudaSuccess ||
            note(launch_nprod(op, d_np, h->sm_count * 8, h->stream)) != cudaSuccess ||
            cudaMemcpyAsync(np.data(), d_np, sizeof(int64_t) * (size_t)M, cudaMemcpyDeviceToHost,
                            h->stream) != cudaSuccess ||
            cudaStreamSynchronize(h->stream) != cudaSuccess) {
            release();
            return SPGEMM_ERR_CUDA;
        }
        // integer sums and double ratios: long double is a software type on
        // some hosts (128-bit on aarch64), far too slow for a loop over rows
        int64_t total = 0;
        for (int64_t v : np) total += v;
        // about 1.5e9 products per slab, and at least one slab per 8 chunks
        // of C at the n_prod upper bound (12 bytes per entry)
        const double by_work = static_cast<double>(total) / 1.5e9;
        const double by_copy = 12.0 * static_cast<double>(total) / (8.0 * static_cast<double>(chunk_bytes));
        const int S = static_cast<int>(std::min(64.0, std::max(1.0, std::max(by_work, by_copy))));
        cut.assign(1, 0);
        // cut c (1 <= c < S) at the first row where the prefix reaches c / S of the total
        int64_t acc = 0;
        double next = static_cast<double>(total) / S;
        for (int64_t r = 0; r < M; ++r) {
            acc += np[(size_t)r];
            if ((int)cut.size() < S && static_cast<double>(acc) >= next) {
                cut.push_back(r + 1);
                next = static_cast<double>(total) * static_cast<double>(cut.size()) / S;
            }
        }
        if (cut.back() != M) cut.push_back(M);
        dev_free(h, d_np);
        dev[6] = nullptr;
    }
    const int S = static_cast<int>(cut.size()) - 1;

    // pinned staging: row pointers of one slab plus two chunk buffers
    int64_t max_rows = 0;
    for (int k = 0; k < S; ++k) max_rows = std::max(max_rows, cut[k + 1] - cut[k]);
    const size_t nr = (size_t)max_rows + 1;
    if (h->stage_rpt_n < nr) {
        if (h->stage_rpt) cudaFreeHost(h->stage_rpt);
        h->stage_rpt = nullptr;
        h->stage_rpt_n = 0;
        if (cudaMallocHost(&h->stage_rpt, sizeof(int64_t) * nr) != cudaSuccess) {
            release();
            return SPGEMM_ERR_OOM;
        }
        h->stage_rpt_n = nr;
    }
    if (h->stage_bytes < 2 * (size_t)chunk_bytes) {
        if (h->stage) cudaFreeHost(h->stage);
        h->stage = nullptr;
        h->stage_bytes = 0;
        if (cudaMallocHost(&h->stage, 2 * (size_t)chunk_bytes) != cudaSuccess) {
            release();
            return SPGEMM_ERR_OOM;
        }
        h->stage_bytes = 2 * (size_t)chunk_bytes;
    }
    cudaEvent_t ev_c[2] = {}, part_done[2][2] = {};
    auto destroy_events = [&]() {
        for (auto &e : ev_c)
            if (e) cudaEventDestroy(e);
        for (auto &row : part_done)
            for (auto &e : row)
                if (e) cudaEventDestroy(e);
    };
    bool ev_ok = true;
    for (auto &e : ev_c) ev_ok &= cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    for (auto &row : part_done)
        for (auto &e : row) ev_ok &= cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    if (!ev_ok) {
        destroy_events();
        release();
        return SPGEMM_ERR_CUDA;
    }

    spgemm_csr_out C[2] = {};
    int64_t nnz_s[2] = {0, 0};
    auto free_c = [&](int b) {
        dev_free(h, C[b].rpt);
        dev_free(h, C[b].col);
        dev_free(h, C[b].val);
        C[b] = spgemm_csr_out{};
    };
    auto compute = [&](int k) -> int {
        const int b = k & 1;
        int r = spgemm_symbolic(h, &dA, &dB, cut[k], cut[k + 1], &nnz_s[b]);
        if (r) return r;
        if ((r = spgemm_numeric(h, &dA, &dB, &C[b]))) return r;
        CK(cudaEventRecord(ev_c[b], h->stream));
        return SPGEMM_OK;
    };
    // chunk copies: (col, val) of rows [r0, r1) of the slab in buffer `buf`,
    // split over the two copy streams
    int64_t *rpt = h->stage_rpt;
    // a chunk of n entries holds n columns, padding to 256 bytes, n values
    auto fits = [&](int64_t n) { return ((4 * n + 255) & ~int64_t{255}) + 8 * n <= chunk_bytes; };
    auto next_rows = [&](int64_t r0, int64_t rows) {
        int64_t r1 = r0 + 1, lo = r0 + 1, hi = rows;
        while (lo <= hi) {   // largest r1 whose entries fit one chunk
            const int64_t mid = lo + (hi - lo) / 2;
            if (fits(rpt[mid] - rpt[r0])) { r1 = mid; lo = mid + 1; }
            else hi = mid - 1;
        }
        return r1;
    };
    auto enqueue = [&](const spgemm_csr_out &c, int64_t r0, int64_t r1, int buf) -> bool {
        const int64_t n = rpt[r1] - rpt[r0];
        if (!fits(n)) return false;   // one row larger than a chunk
        unsigned char *base = h->stage + (size_t)buf * (size_t)chunk_bytes;
        int32_t *hcol = reinterpret_cast<int32_t *>(base);
        double *hval = reinterpret_cast<double *>(base + ((sizeof(int32_t) * (size_t)n + 255) & ~size_t(255)));
        const int64_t off = rpt[r0] - rpt[0];
        for (int k = 0; k < 2; ++k) {
            const int64_t lo = n * k / 2, hi = n * (k + 1) / 2;
            cudaStream_t cs = h->copyst[k];
            if (hi > lo &&
                (cudaMemcpyAsync(hcol + lo, c.col + off + lo, sizeof(int32_t) * (size_t)(hi - lo),
                                 cudaMemcpyDeviceToHost, cs) != cudaSuccess ||
                 cudaMemcpyAsync(hval + lo, c.val + off + lo, sizeof(double) * (size_t)(hi - lo),
                                 cudaMemcpyDeviceToHost, cs) != cudaSuccess))
                return false;
            if (cudaEventRecord(part_done[buf][k], cs) != cudaSuccess) return false;
        }
        return true;
    };
    auto wait_buf = [&](int buf) -> bool {
        for (int k = 0; k < 2; ++k)
            if (cudaEventSynchronize(part_done[buf][k]) != cudaSuccess) return false;
        return true;
    };

    rc = S > 0 ? compute(0) : SPGEMM_OK;
    int64_t nnz_total = 0, nnz_before = 0;
    for (int k = 0; k < S && rc == SPGEMM_OK; ++k) {
        const int b = k & 1;
        const int64_t rows = cut[k + 1] - cut[k];
        // slab k's row pointers (the copy streams wait for its kernels)
        bool ok = true;
        for (auto &cs : h->copyst) ok &= cudaStreamWaitEvent(cs, ev_c[b], 0) == cudaSuccess;
        ok = ok && cudaMemcpyAsync(rpt, C[b].rpt, sizeof(int64_t) * (size_t)(rows + 1), cudaMemcpyDeviceToHost,
                                   h->copyst[0]) == cudaSuccess &&
             cudaStreamSynchronize(h->copyst[0]) == cudaSuccess;
        if (!ok) { rc = SPGEMM_ERR_CUDA; break; }
        if (rows > 0 && rpt[rows] - rpt[0] != nnz_s[b]) { rc = SPGEMM_ERR_INTERNAL; break; }
        int64_t r0 = 0, r1 = rows > 0 ? next_rows(0, rows) : 0;
        int buf = 0;
        if (rows > 0 && !enqueue(C[b], r0, r1, buf)) { rc = SPGEMM_ERR_INVALID; break; }
        // the next slab's kernels run while this slab's copies are in flight
        if (k + 1 < S && (rc = compute(k + 1))) break;
        while (rows > 0) {
            const bool more = r1 < rows;
            int64_t n0 = r1, n1 = r1;
            if (more) {
                n1 = next_rows(n0, rows);
                if (!enqueue(C[b], n0, n1, buf ^ 1)) { rc = SPGEMM_ERR_INVALID; break; }
            }
            if (!wait_buf(buf)) { rc = SPGEMM_ERR_CUDA; break; }
            const int64_t n = rpt[r1] - rpt[r0];
            unsigned char *base = h->stage + (size_t)buf * (size_t)chunk_bytes;
            const int32_t *hc = reinterpret_cast<const int32_t *>(base);
            const double *hv = reinterpret_cast<const double *>(
                base + ((sizeof(int32_t) * (size_t)n + 255) & ~size_t(255)));
            // row pointers handed over are absolute in the whole C
            const int64_t shift = nnz_before - rpt[0];
            for (int64_t i = r0; i <= r1; ++i) rpt[i] += shift;
            const int sr = sink(ctx, cut[k] + r0, r1 - r0, rpt + r0, hc, hv, n);
            for (int64_t i = r0; i <= r1; ++i) rpt[i] -= shift;
            if (sr != 0) { rc = SPGEMM_ERR_ABORTED; break; }
            if (!more) break;
            r0 = n0;
            r1 = n1;
            buf ^= 1;
        }
        if (rc != SPGEMM_OK) break;
        nnz_before += nnz_s[b];
        nnz_total += nnz_s[b];
        free_c(b);
    }
    for (auto &cs : h->copyst) cudaStreamSynchronize(cs);
    cudaStreamSynchronize(h->stream);
    free_c(0);
    free_c(1);
    destroy_events();
    release();
    if (rc == SPGEMM_OK && nnzC) *nnzC = nnz_total;
    return rc;
}

int spgemm_multiply_host(spgemm_handle *h, const spgemm_csr_in *A, const spgemm_csr_in *B,
                         int64_t chunk_bytes, spgemm_host_sink_fn sink, void *ctx,
                         int64_t *nnzC) {
    const int rc = multiply_host(h, A, B, chunk_bytes, sink, ctx, nnzC);
    if (h) h->reuse = false;   // its device copies of A, B and C are gone
    return rc;
}

int spgemm_bin_stats(const spgemm_handle *h, int phase, int64_t *out, int n) {
    if (!h || !out || phase < 0 || phase > 1 || n < 0) return SPGEMM_ERR_INVALID;
    const int m = std::min<int>(n, 3 * SPGEMM_MAX_BINS);
    std::memcpy(out, h->bin_stats[phase], sizeof(int64_t) * (size_t)m);
    return SPGEMM_OK;
}

int spgemm_window_stats(const spgemm_handle *h, int64_t *out, int n) {
    if (!h || !out || n < 0) return SPGEMM_ERR_INVALID;
    const int64_t v[9] = {h->wp_on ? 1 : 0, h->win_used ? 1 : 0, h->nwin, h->nwin_col,
                          h->wp_on ? h->wplan.cs : 0, h->wp_on ? h->wplan.ncells : 0,
                          h->wp_on ? h->wplan.budget : 0, h->wp_on ? h->wplan.e1 : 0,
                          h->split_keep ? 1 : 0};
    for (int i = 0; i < std::min(n, 9); ++i) out[i] = v[i];
    return SPGEMM_OK;
}

int spgemm_set_timing(spgemm_handle *h, int enable) {
    if (!h) return SPGEMM_ERR_INVALID;
    if (enable && !h->t0[0]) {
        for (int k = 0; k < kSlots; ++k) {
            if (cudaEventCreate(&h->t0[k]) != cudaSuccess || cudaEventCreate(&h->t1[k]) != cudaSuccess)
                return SPGEMM_ERR_CUDA;
        }
    }
    h->timing = enable != 0;
    h->serial = enable == 2;
    return SPGEMM_OK;
}

int spgemm_set_phase_clocks(spgemm_handle *h, int enable) {
    if (!h) return SPGEMM_ERR_INVALID;
    if (enable && !h->d_clk) {
        h->d_clk = static_cast<unsigned long long *>(dev_alloc(h, sizeof(unsigned long long) * kPhaseClocks));
        if (!h->d_clk) return SPGEMM_ERR_OOM;
        if (cudaMemsetAsync(h->d_clk, 0, sizeof(unsigned long long) * kPhaseClocks, h->stream) != cudaSuccess)
            return SPGEMM_ERR_CUDA;
    }
    h->phase_clk = enable != 0;
    return SPGEMM_OK;
}

int spgemm_bitmap_phase_clocks(spgemm_handle *h, int64_t *out, int n, int reset) {
    if (!h || n < 0 || (n > 0 && !out)) return SPGEMM_ERR_INVALID;
    unsigned long long v[kPhaseClocks] = {};
    if (h->d_clk) {
        if (cudaMemcpyAsync(v, h->d_clk, sizeof(v), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
            (reset && cudaMemsetAsync(h->d_clk, 0, sizeof(v), h->stream) != cudaSuccess) ||
            cudaStreamSynchronize(h->stream) != cudaSuccess)
            return SPGEMM_ERR_CUDA;
    }
    for (int k = 0; k < n && k < kPhaseClocks; ++k) out[k] = static_cast<int64_t>(v[k]);
    return SPGEMM_OK;
}

int spgemm_kernel_times(spgemm_handle *h, double *ms, int64_t *launches, int n, int reset) {
    if (!h || n < 0) return SPGEMM_ERR_INVALID;
    CK(cudaStreamSynchronize(h->stream));
    for (int k = 0; k < kSlots; ++k) {
        if (h->t1[k]) flush_slot(h, k);
    }
    const int m = std::min<int>(n, kSlots);
    for (int k = 0; k < m; ++k) {
        if (ms) ms[k] = h->ms[k];
        if (launches) launches[k] = h->launches[k];
    }
    if (reset) {
        for (int k = 0; k < kSlots; ++k) {
            h->ms[k] = 0.0;
            h->launches[k] = 0;
        }
    }
    return SPGEMM_OK;
}

int spgemm_set_predictor(spgemm_handle *h, const float *theta, float margin) {
    if (!h || !theta || !(margin >= 0.f)) return SPGEMM_ERR_INVALID;
    if (!h->theta) {
        h->theta = static_cast<float *>(dev_alloc(h, sizeof(float) * (size_t)mlp_param_count()));
        if (!h->theta) return SPGEMM_ERR_OOM;
    }
    CK(cudaMemcpyAsync(h->theta, theta, sizeof(float) * (size_t)mlp_param_count(), cudaMemcpyDefault,
                       h->stream));
    h->margin = margin;
    for (int &k : h->lfk) k = 0;
    return SPGEMM_OK;
}

int spgemm_set_mode(spgemm_handle *h, int mode) {
    if (!h || (mode != SPGEMM_MODE_PLAIN && mode != SPGEMM_MODE_LEARNED)) return SPGEMM_ERR_INVALID;
    if (mode == SPGEMM_MODE_LEARNED && !h->theta) return SPGEMM_ERR_STATE;
    if (h->state == 1) return SPGEMM_ERR_STATE;
    h->mode = mode;
    return SPGEMM_OK;
}

int spgemm_learned_stats(const spgemm_handle *h, int64_t *out, int n) {
    if (!h || !out || n < 0) return SPGEMM_ERR_INVALID;
    for (int i = 0; i < std::min(n, 6 + kMaxBins); ++i) out[i] = h->lstats[i];
    return SPGEMM_OK;
}

int spgemm_destroy(spgemm_handle *h) {
    if (!h) return SPGEMM_OK;
    if (h->side[0]) cudaStreamSynchronize(h->stream);
    if (h->state == 1) dev_free(h, h->crpt);
    dev_free(h, h->tcol);
    dev_free(h, h->tval);
    dev_free(h, h->theta);
    dev_free(h, h->lscratch);
    dev_free(h, h->arena);
    win_release(h);
    dev_free(h, h->wcells);
    dev_free(h, h->wcslot);
    dev_free(h, h->wspill);
    dev_free(h, h->d_clk);
    if (h->side[0]) cudaStreamSynchronize(h->stream);
    for (int i = 0; i < kSide; ++i) {
        if (h->side[i]) cudaStreamDestroy(h->side[i]);
        if (h->ev_side[i]) cudaEventDestroy(h->ev_side[i]);
    }
    for (auto &cs : h->copyst)
        if (cs) cudaStreamDestroy(cs);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    for (int k = 0; k < kSlots; ++k) {
        if (h->t0[k]) cudaEventDestroy(h->t0[k]);
        if (h->t1[k]) cudaEventDestroy(h->t1[k]);
    }
    if (h->h_cnt) cudaFreeHost(h->h_cnt);
    if (h->stage) cudaFreeHost(h->stage);
    if (h->stage_rpt) cudaFreeHost(h->stage_rpt);
    if (h->pool) cudaMemPoolDestroy(h->pool);
    delete h;
    return SPGEMM_OK;
}

}  // extern "C"

// --- batched products (one persistent launch under a CUDA graph) ---------------
struct spgemm_batch {
    spgemm_handle *h = nullptr;
    int n = 0;
    std::vector<BatchProb> probs;
    std::vector<int64_t> M, N;
    BatchProb *d_probs = nullptr;
    BatchItem *d_items = nullptr;
    int nitems = 0;
    unsigned char *d_state = nullptr;   // BatchState, then done_s, xflag, done_n
    size_t state_bytes = 0;
    unsigned char *arena = nullptr;
    size_t arena_bytes = 0;
    int variant = 0, tile_rows = 0, grid = 0;
    long long spin_limit = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t *d_totals = nullptr;        // gathered C.rpt[M] of every product
    std::vector<int64_t> nnz;
    int last_rc = SPGEMM_OK;
};

namespace {

__global__ void gather_totals_kernel(const BatchProb *probs, int n, int64_t *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = probs[i].crpt[probs[i].M];
}

void batch_release(spgemm_batch *b) {
    spgemm_handle *h = b->h;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    dev_free(h, b->d_probs);
    dev_free(h, b->d_items);
    dev_free(h, b->d_state);
    dev_free(h, b->arena);
    dev_free(h, b->d_totals);
}

}  // namespace

extern "C" {

int spgemm_batch_create(spgemm_batch **out, spgemm_handle *h, int n, const spgemm_csr_in *A,
                        const spgemm_csr_in *B, const int32_t *b_from,
                        const spgemm_batch_options *opt) {
    if (!out || !h || n < 0 || (n > 0 && (!A || !B))) return SPGEMM_ERR_INVALID;
    *out = nullptr;
    spgemm_batch *b = new (std::nothrow) spgemm_batch();
    if (!b) return SPGEMM_ERR_OOM;
    b->h = h;
    b->n = n;
    b->probs.resize(n);
    b->M.resize(n);
    b->N.resize(n);
    b->nnz.assign(n, 0);
    int rc = SPGEMM_OK;
    auto fail = [&](int code) {
        cudaStreamSynchronize(h->stream);
        batch_release(b);
        delete b;
        return code;
    };
    // shapes and dependencies
    std::vector<int> level(n, 0);
    for (int i = 0; i < n; ++i) {
        const int dep = b_from ? b_from[i] : -1;
        if ((rc = check_csr_in(&A[i]))) return fail(rc);
        if (dep >= i) return fail(SPGEMM_ERR_INVALID);
        if (dep < 0) {
            if ((rc = check_csr_in(&B[i]))) return fail(rc);
            if (A[i].cols != B[i].rows) return fail(SPGEMM_ERR_SHAPE);
            if ((A[i].nnz > 0 && !A[i].val) || (B[i].nnz > 0 && !B[i].val)) return fail(SPGEMM_ERR_INVALID);
            b->N[i] = B[i].cols;
        } else {
            if (A[i].cols != b->M[dep]) return fail(SPGEMM_ERR_SHAPE);
            if (A[i].nnz > 0 && !A[i].val) return fail(SPGEMM_ERR_INVALID);
            b->N[i] = b->N[dep];
            level[i] = level[dep] + 1;
        }
        b->M[i] = A[i].rows;
    }
    // row bounds: exact n_prod for products of input matrices; for a product
    // whose B is an earlier C, the n_prod of that C's rows bounds their size,
    // so a pseudo row pointer built from those bounds gives a bound here
    std::vector<std::vector<int64_t>> bound(n);
    std::vector<int64_t> cap(n, 0), pmax(n, 0);
    int64_t maxrow = 0;
    int64_t *d_b = nullptr, *d_rp = nullptr;
    size_t d_b_n = 0, d_rp_n = 0;
    for (int i = 0; i < n; ++i) {
        const int dep = b_from ? b_from[i] : -1;
        const int64_t M = b->M[i];
        if ((size_t)(M + 1) > d_b_n) {
            dev_free(h, d_b);
            d_b_n = (size_t)(M + 1);
            d_b = static_cast<int64_t *>(dev_alloc(h, sizeof(int64_t) * d_b_n));
            if (!d_b) return fail(SPGEMM_ERR_OOM);
        }
        Operands op{};
        op.arpt = A[i].rpt; op.a64 = A[i].rpt_is_i64 ? 1 : 0; op.acol = A[i].col;
        op.row0 = 0; op.mw = M; op.ncols = b->N[i];
        if (dep < 0) {
            op.brpt = B[i].rpt; op.b64 = B[i].rpt_is_i64 ? 1 : 0;
        } else {
            const std::vector<int64_t> &bd = bound[dep];
            std::vector<int64_t> rp(bd.size() + 1, 0);
            for (size_t k = 0; k < bd.size(); ++k) rp[k + 1] = rp[k] + bd[k];
            if (rp.size() > d_rp_n) {
                dev_free(h, d_rp);
                d_rp_n = rp.size();
                d_rp = static_cast<int64_t *>(dev_alloc(h, sizeof(int64_t) * d_rp_n));
                if (!d_rp) return fail(SPGEMM_ERR_OOM);
            }
            CK(cudaMemcpyAsync(d_rp, rp.data(), sizeof(int64_t) * rp.size(), cudaMemcpyHostToDevice, h->stream));
            op.brpt = d_rp; op.b64 = 1;
        }
        CK(cudaMemsetAsync(d_b, 0, sizeof(int64_t) * (size_t)(M + 1), h->stream));
        CK(launch_nprod(op, d_b, h->sm_count * 4, h->stream));
        bound[i].resize((size_t)M);
        if (M > 0)
            CK(cudaMemcpyAsync(bound[i].data(), d_b, sizeof(int64_t) * (size_t)M, cudaMemcpyDeviceToHost,
                               h->stream));
        CK(cudaStreamSynchronize(h->stream));
        for (int64_t v : bound[i]) {
            cap[i] += v;
            pmax[i] = std::max(pmax[i], v);
            maxrow = std::max(maxrow, v);
        }
    }
    dev_free(h, d_b);
    dev_free(h, d_rp);
    // kernel variant: the smallest table whose sort holds the largest row
    int64_t need = 1;
    while (need < maxrow) need <<= 1;
    b->variant = -1;
    for (int v = 0; v < batch_variant_count(); ++v)
        if (batch_variant_table(v) >= need) { b->variant = v; break; }
    if (opt && opt->variant >= 0) {
        if (opt->variant >= batch_variant_count() || batch_variant_table(opt->variant) < need)
            return fail(SPGEMM_ERR_INVALID);
        b->variant = opt->variant;
    }
    if (b->variant < 0) return fail(SPGEMM_ERR_INVALID);   // rows too large to batch
    const int rg = 256 / batch_variant_lanes(b->variant);
    b->tile_rows = (opt && opt->tile_rows > 0) ? opt->tile_rows : rg * 32;
    if (b->tile_rows % rg) b->tile_rows += rg - b->tile_rows % rg;
    if (b->tile_rows > kBatchMaxTile) return fail(SPGEMM_ERR_INVALID);
    b->spin_limit = (opt && opt->spin_limit > 0) ? opt->spin_limit : (1LL << 22);
    // arena: per product C.rpt (M+1 int64), C.col and C.val with room for the bound
    std::vector<size_t> off_rpt(n), off_col(n), off_val(n), off_tsum(n);
    size_t total = 0;
    for (int i = 0; i < n; ++i) {
        const int64_t nt = (b->M[i] + b->tile_rows - 1) / b->tile_rows;
        off_tsum[i] = total; total += align256(sizeof(long long) * (size_t)(nt + 1));
        off_rpt[i] = total; total += align256(sizeof(int64_t) * (size_t)(b->M[i] + 1));
        off_col[i] = total; total += align256(sizeof(int32_t) * (size_t)std::max<int64_t>(cap[i], 1));
        off_val[i] = total; total += align256(sizeof(double) * (size_t)std::max<int64_t>(cap[i], 1));
    }
    b->arena = static_cast<unsigned char *>(dev_alloc(h, std::max<size_t>(total, 256)));
    if (!b->arena) return fail(SPGEMM_ERR_OOM);
    b->arena_bytes = total;
    // problems and work items in dependency order
    std::vector<BatchItem> items;
    int maxlevel = 0;
    for (int i = 0; i < n; ++i) maxlevel = std::max(maxlevel, level[i]);
    for (int i = 0; i < n; ++i) {
        BatchProb &P = b->probs[i];
        const int dep = b_from ? b_from[i] : -1;
        P.arpt = A[i].rpt; P.a64 = A[i].rpt_is_i64 ? 1 : 0; P.acol = A[i].col; P.aval = A[i].val;
        P.M = b->M[i];
        P.N = b->N[i];
        P.crpt = reinterpret_cast<int64_t *>(b->arena + off_rpt[i]);
        P.ccol = reinterpret_cast<int32_t *>(b->arena + off_col[i]);
        P.cval = reinterpret_cast<double *>(b->arena + off_val[i]);
        P.ccap = cap[i];
        P.tsum = reinterpret_cast<long long *>(b->arena + off_tsum[i]);
        P.ntiles = static_cast<int32_t>((P.M + b->tile_rows - 1) / b->tile_rows);
        P.dep = dep;
        // 1: every row fits the one-thread path; 0: rows try it first; -1: never
        P.tiny = (opt && opt->no_tiny) ? -1 : (pmax[i] <= kBatchTiny ? 1 : 0);
        P.pad = 0;
        if (dep < 0) {
            P.brpt = B[i].rpt; P.b64 = B[i].rpt_is_i64 ? 1 : 0; P.bcol = B[i].col; P.bval = B[i].val;
        } else {
            P.brpt = b->probs[dep].crpt; P.b64 = 1; P.bcol = b->probs[dep].ccol; P.bval = b->probs[dep].cval;
        }
    }
    for (int L = 0; L <= maxlevel; ++L)
        for (int type = 0; type < 3; ++type)
            for (int i = 0; i < n; ++i) {
                if (level[i] != L) continue;
                if (type == 1) items.push_back({1, i, 0, 0});
                else
                    for (int t = 0; t < b->probs[i].ntiles; ++t) items.push_back({type, i, t, 0});
            }
    b->nitems = static_cast<int>(items.size());
    b->d_probs = static_cast<BatchProb *>(dev_alloc(h, sizeof(BatchProb) * (size_t)std::max(n, 1)));
    b->d_items = static_cast<BatchItem *>(dev_alloc(h, sizeof(BatchItem) * std::max<size_t>(items.size(), 1)));
    b->state_bytes = sizeof(BatchState) + 3 * sizeof(int) * (size_t)std::max(n, 1);
    b->d_state = static_cast<unsigned char *>(dev_alloc(h, b->state_bytes));
    b->d_totals = static_cast<int64_t *>(dev_alloc(h, sizeof(int64_t) * (size_t)std::max(n, 1)));
    if (!b->d_probs || !b->d_items || !b->d_state || !b->d_totals) return fail(SPGEMM_ERR_OOM);
    if (n) CK(cudaMemcpyAsync(b->d_probs, b->probs.data(), sizeof(BatchProb) * (size_t)n,
                              cudaMemcpyHostToDevice, h->stream));
    if (!items.empty())
        CK(cudaMemcpyAsync(b->d_items, items.data(), sizeof(BatchItem) * items.size(),
                           cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    b->grid = std::max(1, h->sm_count * std::max(1, batch_blocks_per_sm(b->variant)));
    // capture: reset the queue state, then the persistent kernel
    cudaStream_t cs = h->side[0];
    BatchState *st = reinterpret_cast<BatchState *>(b->d_state);
    int *done_s = reinterpret_cast<int *>(b->d_state + sizeof(BatchState));
    int *xflag = done_s + std::max(n, 1);
    int *done_n = xflag + std::max(n, 1);
    CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    cudaError_t e1 = cudaMemsetAsync(b->d_state, 0, b->state_bytes, cs);
    cudaError_t e2 = launch_batch(b->variant, b->grid, b->d_probs, b->d_items, b->nitems, st, done_s,
                                  xflag, done_n, b->tile_rows, b->spin_limit, cs);
    cudaError_t e3 = cudaStreamEndCapture(cs, &b->graph);
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) return fail(SPGEMM_ERR_CUDA);
    CK(cudaGraphInstantiate(&b->exec, b->graph, 0));
    *out = b;
    return SPGEMM_OK;
}

int spgemm_batch_run(spgemm_batch *b) {
    if (!b) return SPGEMM_ERR_INVALID;
    CK(cudaGraphLaunch(b->exec, b->h->stream));
    return SPGEMM_OK;
}

int spgemm_batch_sync(spgemm_batch *b) {
    if (!b) return SPGEMM_ERR_INVALID;
    spgemm_handle *h = b->h;
    BatchState host{};
    if (b->n > 0) {
        gather_totals_kernel<<<(b->n + 255) / 256, 256, 0, h->stream>>>(b->d_probs, b->n, b->d_totals);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(b->nnz.data(), b->d_totals, sizeof(int64_t) * (size_t)b->n,
                           cudaMemcpyDeviceToHost, h->stream));
    }
    CK(cudaMemcpyAsync(&host, b->d_state, sizeof(BatchState), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    b->last_rc = host.err;
    return host.err;
}

int spgemm_batch_result(const spgemm_batch *b, int i, spgemm_csr_out *C) {
    if (!b || !C || i < 0 || i >= b->n) return SPGEMM_ERR_INVALID;
    const BatchProb &P = b->probs[i];
    C->rows = P.M;
    C->cols = P.N;
    C->nnz = b->nnz[i];
    C->rpt = P.crpt;
    C->col = P.ccol;
    C->val = P.cval;
    return SPGEMM_OK;
}

int spgemm_batch_info(const spgemm_batch *b, int64_t *out, int nvals) {
    if (!b || !out || nvals < 0) return SPGEMM_ERR_INVALID;
    const int64_t v[6] = {b->n, b->nitems, b->grid, batch_variant_lanes(b->variant),
                          batch_variant_table(b->variant), b->tile_rows};
    for (int k = 0; k < std::min(nvals, 6); ++k) out[k] = v[k];
    return SPGEMM_OK;
}

int spgemm_batch_destroy(spgemm_batch *b) {
    if (!b) return SPGEMM_OK;
    cudaStreamSynchronize(b->h->stream);
    batch_release(b);
    delete b;
    return SPGEMM_OK;
}

}  // extern "C"

namespace ops {

cudaError_t prepare_device(int dev, int smem_dyn_max) {
    constexpr int kMaxDev = 64;
    static std::mutex mu;
    static bool done[kMaxDev] = {};
    if (dev < 0 || dev >= kMaxDev) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (done[dev]) return cudaSuccess;
    cudaError_t e = sym_prepare(smem_dyn_max);
    if (e == cudaSuccess) e = num_prepare(smem_dyn_max);
    if (e == cudaSuccess) e = win_prepare(smem_dyn_max);
    if (e == cudaSuccess) done[dev] = true;
    return e;
}

}  // namespace ops
