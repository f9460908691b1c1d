/*
 * opsparse.h - C ABI of the GB300 (sm_103a) row-wise SpGEMM library.
 *
 * The library computes C = A * B for sparse A (M x K) and B (K x N) in CSR
 * form, row by row (Gustavson's row-wise dataflow, Eq. 2, Sec. 2.1), as a
 * two-phase method (Sec. 2.2): a symbolic phase counts the non-zeros of each
 * output row, C is allocated from the total, and a numeric phase writes each
 * row's sorted column indices and values.
 *
 * Conventions for every entry point:
 *   - Pointers inside spgemm_csr_in / spgemm_csr_out are DEVICE pointers on
 *     the handle's device unless a function says otherwise.
 *   - Integers: column indices int32; input row pointers int32 or int64
 *     (rpt_is_i64); the output row pointer is always int64 (an output row
 *     window may hold more than 2^31 - 1 entries).
 *   - Values are IEEE float64 (the paper evaluates in double precision,
 *     Sec. 6).
 *   - Every call is ordered on the handle's CUDA stream. Calls that must
 *     return a count to the host (spgemm_symbolic) synchronise that stream;
 *     the others only enqueue work.
 *   - A handle is not thread-safe; use one handle per host thread.
 *   - Return value: SPGEMM_OK (0) or one of the negative codes below;
 *     spgemm_strerror() names them. On error no output is handed over and
 *     the handle stays usable unless the code is SPGEMM_ERR_CUDA.
 */
#ifndef OPSPARSE_H
#define OPSPARSE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SPGEMM_OK                  0
#define SPGEMM_ERR_INVALID        -1  /* bad argument or malformed CSR      */
#define SPGEMM_ERR_SHAPE          -2  /* A.cols != B.rows                   */
#define SPGEMM_ERR_OOM            -3  /* an allocation failed               */
#define SPGEMM_ERR_STATE          -4  /* call out of order (numeric before symbolic) */
#define SPGEMM_ERR_TIMEOUT        -5  /* a bounded device wait ran out      */
#define SPGEMM_ERR_CUDA           -6  /* a CUDA runtime call failed         */
#define SPGEMM_ERR_INTERNAL       -7  /* a device-side check failed (table overflow) */
#define SPGEMM_ERR_ABORTED        -8  /* a host sink callback asked to stop  */

#define SPGEMM_MAX_BINS 16

/* Read-only CSR input (Sec. 2.1.1): rpt has rows+1 entries, col/val have
 * nnz = rpt[rows] entries. Columns inside a row need not be sorted and may
 * repeat; repeated (row, col) pairs are summed. Caller-owned device memory. */
typedef struct {
    int64_t rows, cols, nnz;
    const void *rpt;
    int32_t rpt_is_i64;          /* 0: int32 row pointers, 1: int64 */
    const int32_t *col;
    const double *val;           /* may be NULL for spgemm_symbolic */
} spgemm_csr_in;

/* CSR output written by the library: rows = row window length, cols = B.cols,
 * nnz = number of stored entries; rpt (int64, rows+1) starts at 0 for the
 * first row of the window; columns ascending and unique in every row.
 * Ownership of rpt/col/val passes to the caller (see spgemm_alloc_fn). */
typedef struct {
    int64_t rows, cols, nnz;
    int64_t *rpt;
    int32_t *col;
    double *val;
} spgemm_csr_out;

/* Device-memory allocator hooks. alloc returns a device pointer aligned to at
 * least 256 bytes or NULL; free releases it. `stream` is the cudaStream_t of
 * the handle, passed as void*. With both NULL the library uses a private
 * stream-ordered pool (cudaMallocAsync); output arrays then belong to the
 * caller, who releases them with spgemm_free(). */
typedef void *(*spgemm_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*spgemm_free_fn)(void *ptr, void *stream, void *ctx);

/* Bin configuration (Sec. 5.1, Sec. 5.6, Sec. 5.7). Bin j of a phase takes
 * the rows whose size (n_prod for the symbolic phase, n_nz for the numeric
 * phase) is <= range[j] and > range[j-1] (Algorithm 1: first j with
 * size <= r_range[j]); the last used bin must have range -1 (no bound).
 * kernel[j] picks the kernel that computes bin j from the table printed by
 * spgemm_kernel_info(); its capacity must hold range[j]. A handle created
 * with cfg NULL (or reset with spgemm_set_config(h, NULL)) uses the default
 * bins, every hash kernel with tables 1.2x (symbolic) and 2x (numeric) the
 * largest row of the bin (Sec. 5.7), and moves the switch to the bitmap
 * kernels with the number of columns of B at each spgemm_symbolic; the
 * configuration then in use is what spgemm_get_config returns.
 * lanes_per_brow / num_lanes_per_brow: threads that walk one row of B
 * together in the symbolic / numeric phase (1..32, a power of two), or 0 to
 * pick it per output row from the mean referenced B-row length.
 * bitmap_unroll: products each thread of a bitmap kernel loads before using
 * them (4 or 8; 0 = 4).
 * window_lists (0..1024, 0 = off, the default): when every row of B is
 * sorted by column and B's columns fit one bitmap, rows of the numeric
 * bitmap kernel with at most this many A entries (and at most as many as
 * the kernel's block has threads) sum their values window by window over
 * the column space, so that the C.val lines being summed into stay in L2.
 * This halves that kernel's DRAM traffic on power-law inputs but executes
 * more instructions per product. window_entries: C entries per such window,
 * about (0 = 12288).
 * hash_access: how a hash probe of the symbolic and numeric hash kernels
 * reaches its slot. 0 (the default): one atomicCAS per probe, whose result
 * is the slot's key (Sec. 5.6, Algorithms 4-5). 1: a plain read of the slot
 * first and an atomicCAS only when the slot is empty, the access pattern of
 * the libraries the paper compares its hashing against (Sec. 6). Results do
 * not depend on it; it exists for that comparison.
 * bitmap_path: how the last numeric bin (the rows past the hash tables) is
 * computed. All forms give the same C.
 *   0 (the default): one block per row with a column bitmap and its ranks
 *     in shared memory, one window over the whole column space when it fits;
 *     the values are summed in C.val by float64 L2 reductions. When B has
 *     more columns than one bitmap holds, the row is covered in several
 *     windows; with every row of B sorted by column (and at most 2^22
 *     columns) each window then walks only the runs of B rows inside it.
 *   1: the same, but when every row of B is sorted by column and B has at
 *     most 2^22 columns a row is covered in column windows of about half an
 *     SM's shared memory (two blocks per SM), each window walking only the
 *     runs of B rows inside it, found in a cell index of B's long rows.
 *     Unsorted B takes form 0.
 *   2: rows cut into column windows planned from per-cell entry counts that
 *     the symbolic bitmap kernel records, summed in shared memory (by column
 *     where a window is dense, by rank elsewhere); needs sorted B and at most
 *     2^22 columns, and lowers the symbolic bitmap kernel's threshold in the
 *     default configuration so every row with more entries than one
 *     whole-width window passes through it.
 * On GB300 form 0 is the fastest on power-law inputs: the kernels are bound
 * by the SM's rate of scattered L2 requests and float64 accumulation, which
 * splitting rows does not raise (measured in the design notes).
 * window_budget: shared-memory bytes a column window may use for its
 * accumulator, bitmap and ranks (0 = all that one block can have, the
 * default). Smaller budgets cut rows into more, smaller windows; a budget
 * too small for one fully dense cell turns the column windows off. */
typedef struct {
    int32_t sym_nbins;
    int32_t sym_kernel[SPGEMM_MAX_BINS];
    int64_t sym_range[SPGEMM_MAX_BINS];
    int32_t num_nbins;
    int32_t num_kernel[SPGEMM_MAX_BINS];
    int64_t num_range[SPGEMM_MAX_BINS];
    int32_t lanes_per_brow;
    int32_t num_lanes_per_brow;
    int32_t bitmap_unroll;
    int32_t window_lists;
    int32_t window_entries;
    int32_t hash_access;
    int32_t bitmap_path;
    int32_t window_budget;
} spgemm_config;

typedef struct spgemm_handle spgemm_handle;

/* Create a handle on the current CUDA device. cfg NULL = defaults; stream is
 * a cudaStream_t (NULL = legacy default stream). Creates the handle's side
 * streams (Sec. 5: bins of one phase run concurrently) and a small pinned
 * host buffer. */
int spgemm_create(spgemm_handle **h, const spgemm_config *cfg,
                  spgemm_alloc_fn alloc, spgemm_free_fn free_fn, void *ctx,
                  void *stream);

/* Replace the bin configuration (validated; SPGEMM_ERR_INVALID if a range
 * exceeds its kernel's capacity or the last range is bounded). */
int spgemm_set_config(spgemm_handle *h, const spgemm_config *cfg);
int spgemm_get_config(const spgemm_handle *h, spgemm_config *cfg);

/* Symbolic phase for output rows [row_begin, row_end) of C = A * B
 * (Sec. 5 steps 1-4): per-row intermediate-product count n_prod (Sec. 2.1.2)
 * written into C.rpt, symbolic binning (Algorithms 1-3), per-bin symbolic
 * kernels (Algorithm 4; large rows use a shared-memory column bitmap), and
 * the first numeric binning pass, which yields the total. Allocates the
 * output row pointer (row_end - row_begin + 1 int64) and keeps it in the
 * handle until spgemm_numeric. *nnzC receives the number of entries of the
 * window. In SPGEMM_MODE_PLAIN A.val/B.val are not read (they may be NULL);
 * in SPGEMM_MODE_LEARNED rows are multiplied during this call and NULL
 * values give SPGEMM_ERR_INVALID. Synchronises the handle's stream. */
int spgemm_symbolic(spgemm_handle *h, const spgemm_csr_in *A,
                    const spgemm_csr_in *B, int64_t row_begin, int64_t row_end,
                    int64_t *nnzC);

/* Numeric phase for the window of the last spgemm_symbolic (Sec. 5 steps
 * 4-6): second numeric binning pass, in-place exclusive scan of C.rpt
 * (Sec. 5.3), allocation of C.col/C.val overlapped with those kernels
 * (Sec. 5.4), then per-bin numeric kernels (Algorithm 5 hash, condense,
 * sort; large rows use the bitmap-rank kernel). If C->col and C->val are
 * non-NULL on entry they are used as the output buffers (each must hold
 * *nnzC entries); otherwise they are allocated. On return C describes the
 * window and owns rpt/col/val. Does not synchronise. */
int spgemm_numeric(spgemm_handle *h, const spgemm_csr_in *A,
                   const spgemm_csr_in *B, spgemm_csr_out *C);

/* spgemm_symbolic over all rows followed by spgemm_numeric. */
int spgemm_multiply(spgemm_handle *h, const spgemm_csr_in *A,
                    const spgemm_csr_in *B, spgemm_csr_out *C);

/* Numeric phase again over the structure of this handle's last
 * spgemm_numeric, for new values of A and B with the same structure (the
 * same rpt and col contents): the repeated products of an iterative setup
 * where only the values change. It rests on the two-phase split of Sec. 2.2
 * (structure first, values second); the paper itself always runs both.
 * Skips n_prod, both binning steps, the symbolic kernels, the scan and the
 * allocation: the rows keep the bins, kernels and C.rpt of the last call,
 * and only the per-bin numeric kernels run (Algorithm 5; large rows the
 * bitmap-rank kernel, with its whole-row pass 2).
 *   A, B  device CSR, caller-owned; rows, cols and nnz must equal those of
 *         the last numeric call and A.val/B.val must be non-NULL.
 *   C     the output of that call (or arrays with the same contents):
 *         C->rpt (int64, rows+1) is read, C->col is rewritten with the same
 *         columns and C->val (nnz float64) receives the new values. Nothing
 *         is allocated and ownership does not change.
 * Returns SPGEMM_ERR_STATE when the handle holds no plain-mode structure
 * (no numeric call yet, a spgemm_symbolic, spgemm_multiply_host or
 * spgemm_set_config since, or the last call was in SPGEMM_MODE_LEARNED) or
 * the shapes differ; SPGEMM_ERR_INVALID for a C that does not describe that
 * result. A or B with another structure but the same sizes is not detected
 * here: spgemm_status then reports SPGEMM_ERR_INTERNAL where a row's size no
 * longer matches, and C is undefined. Does not synchronise. */
int spgemm_numeric_values(spgemm_handle *h, const spgemm_csr_in *A,
                          const spgemm_csr_in *B, const spgemm_csr_out *C);

/* Wait for the handle's stream and report device-side checks raised by any
 * earlier call (a full hash table, a row whose numeric size differs from its
 * symbolic count): SPGEMM_OK or SPGEMM_ERR_INTERNAL (the check is then
 * cleared). */
int spgemm_status(spgemm_handle *h);

/* Release memory that the library allocated for an output when no allocator
 * hooks were given (stream-ordered on the handle's stream). */
int spgemm_free(spgemm_handle *h, void *ptr);

/* Free the handle's scratch memory, streams and host buffers. Never frees
 * an output handed to the caller. */
int spgemm_destroy(spgemm_handle *h);

/* Receives one chunk of C rows copied back to host memory:
 * rows [row_begin, row_begin + rows), rpt points at rows+1 int64 offsets
 * (absolute: rpt[k] - rpt[0] indexes col/val), col/val hold nnz entries.
 * All pointers are host memory owned by the library and valid only during
 * the call. Return 0 to continue, nonzero to stop (SPGEMM_ERR_ABORTED). */
typedef int (*spgemm_host_sink_fn)(void *ctx, int64_t row_begin, int64_t rows,
                                   const int64_t *rpt, const int32_t *col,
                                   const double *val, int64_t nnz);

/* C = A * B for operands in HOST memory (pinned memory gives full copy
 * speed): copies A and B to the device (once if A and B are the same
 * arrays), then computes C in slabs of rows with about equal n_prod (about
 * 1.5e9 products each, and at least one slab per 8 chunks of C at the
 * n_prod bound, at most 64) and streams each slab back in chunks of at most
 * chunk_bytes of (col, val) through two pinned staging buffers, on streams
 * of their own, while the next slab is computed. sink is called for each
 * chunk in row order while the next chunk is in flight. Neither C nor more
 * than two slabs of it have to fit in host or device memory. *nnzC (may be
 * NULL) receives the total. Device copies and C are released before
 * returning. */
int spgemm_multiply_host(spgemm_handle *h, const spgemm_csr_in *A,
                         const spgemm_csr_in *B, int64_t chunk_bytes,
                         spgemm_host_sink_fn sink, void *ctx, int64_t *nnzC);

/* Per-bin statistics of the last symbolic call for phase 0 (symbolic bins)
 * or 1 (numeric bins): 3 * SPGEMM_MAX_BINS int64: rows per bin, sum of the
 * row sizes per bin (n_prod or n_nz), A entries of the bin's rows. */
int spgemm_bin_stats(const spgemm_handle *h, int phase, int64_t *out, int n);

/* Column windows of the last symbolic/numeric pair (see bitmap_path), up to
 * 9 int64. For bitmap_path 2: 1 if the symbolic call prepared them, 1 if the
 * numeric call ran them, windows, windows that accumulate by column, log2 of
 * the cell width, cells per row, shared bytes per window, and the largest
 * row size that takes one window over all columns. Then 1 if the numeric
 * call ran the default form's run-restricted windows (bitmap_path 0). */
int spgemm_window_stats(const spgemm_handle *h, int64_t *out, int n);

/* Per-kernel timing with CUDA events recorded on the stream each kernel is
 * launched on. spgemm_kernel_times synchronises the handle's stream and
 * returns accumulated milliseconds and launch counts per slot: slots 0-15
 * the symbolic bins, 16-31 the numeric bins, 32 n_prod, 33/34 symbolic
 * binning passes 1/2, 35/36 numeric binning passes 1/2, 37 the scan; in
 * learned mode also 38 the row features, 39 the MLP forward with the sizes
 * and binning by prediction, 40 the copy of one-phase rows into C (41
 * slots). reset != 0 clears the totals. */
int spgemm_set_timing(spgemm_handle *h, int enable);
int spgemm_kernel_times(spgemm_handle *h, double *ms, int64_t *launches, int n,
                        int reset);

/* Phase clocks of the numeric bitmap kernel: a profiling aid with no
 * counterpart in the paper. With enable != 0, numeric calls from then on run
 * the 1024-thread, whole-row form of that kernel with a block barrier at the
 * end of each phase, and thread 0 of every block adds the SM clock cycles
 * its block spent in the phase to counters kept by the handle (a 56-byte
 * device buffer allocated at the first enable, freed by spgemm_destroy);
 * enable = 0 turns the barriers and counters off. C does not depend on it.
 * spgemm_bitmap_phase_clocks synchronises the handle's stream and writes
 * min(n, 7) int64 sums over blocks, one per phase in order: bitmap clear,
 * pass 1 (column bits), per-word prefix counts, C.col write, C.val clear,
 * pass 2 (float64 reductions into C.val), L2 priority reset of the row's
 * C.val lines; all 0 before the first enable. reset != 0 clears them. Cycles
 * of one SM's clock: divide the sum by the SM count and the clock rate for
 * the time each phase takes when all SMs run the kernel. Errors:
 * SPGEMM_ERR_INVALID (null handle, n < 0, null out with n > 0),
 * SPGEMM_ERR_OOM, SPGEMM_ERR_CUDA. */
int spgemm_set_phase_clocks(spgemm_handle *h, int enable);
int spgemm_bitmap_phase_clocks(spgemm_handle *h, int64_t *out, int n, int reset);

/* Per-phase statistics of the last symbolic/numeric call: 4 + 2 * NB
 * int64 values: total n_prod, max row n_prod, total n_nz, max row n_nz,
 * then the symbolic and numeric bin sizes (SPGEMM_MAX_BINS each). */
int spgemm_last_stats(const spgemm_handle *h, int64_t *out, int n);

/* Describe kernel `id` of a phase (0 symbolic, 1 numeric): its threads per
 * row, threads per block, table capacity (entries; for the bitmap kernel
 * the number of columns one pass covers) and the largest row size it
 * accepts. Returns SPGEMM_ERR_INVALID past the last kernel. */
int spgemm_kernel_info(int phase, int id, int32_t *threads_per_row,
                       int32_t *block, int64_t *table, int64_t *max_size);

/* ---- Learned row sizing ---------------------------------------------------
 * The paper sizes every output row with the exact symbolic phase (Sec. 2.2).
 * In SPGEMM_MODE_LEARNED a small perceptron predicts each row's n_nz from six
 * row features; a row predicted to fit a shared-memory hash table is
 * multiplied once into a table sized from the prediction (the one-phase
 * method of Sec. 2.2: the row goes to temporary memory and is copied into C
 * after the scan). A row whose keys do not fit is detected in the kernel
 * and recomputed by the exact symbolic and numeric kernels, as are rows
 * past the symbolic hash bins, so C is identical to SPGEMM_MODE_PLAIN.
 *
 * Predictor: 6 -> 64 -> 64 -> 1, ReLU, float32, parameters in one flat
 * vector W1 (6x64 row-major), b1 (64), W2 (64x64 row-major), b2 (64),
 * w3 (64), b3 (1) (spgemm_mlp_param_count() = 4673 floats). Features of
 * output row i (of M = A.rows): log1p(nnz of A row i), log1p(n_prod_i),
 * log1p of the max / mean / min length of the referenced B rows (0 for an
 * empty A row) and log((i + 1) / M). The output approximates log1p(n_nz);
 * the predicted size is p = max(1, ceil(expm1(y) * (1 + margin))). Rows are
 * put in classes by p (class j: the numeric bin that p falls in) and the
 * size used is ceil(p * 2^k_j), at least 1 and at most the row's n_prod.
 * The exponents k_j (|k_j| <= 4; 0 after spgemm_set_predictor) are the
 * handle's load feedback, updated by each learned-mode spgemm_symbolic for
 * the next one: k_j + 1 when more than a quarter of class j's rows tried in
 * one phase overflowed their table or filled it more than 3/4, k_j - 1 when
 * at least 15/16 of them would fill the next smaller table at most 3/4
 * (a factor of 2 moves a row at most one table). Results never depend on
 * the k_j; only the tables the rows use do. */
#define SPGEMM_MODE_PLAIN   0
#define SPGEMM_MODE_LEARNED 1

int spgemm_mlp_param_count(void);

/* Copy the predictor's parameters (host or device pointer, 4673 floats)
 * into the handle, with the safety margin of the predicted sizes. */
int spgemm_set_predictor(spgemm_handle *h, const float *theta, float margin);

/* SPGEMM_MODE_PLAIN or SPGEMM_MODE_LEARNED (needs a predictor; not between
 * spgemm_symbolic and spgemm_numeric: SPGEMM_ERR_STATE). */
int spgemm_set_mode(spgemm_handle *h, int mode);

/* After a learned-mode spgemm_symbolic (up to 6 + SPGEMM_MAX_BINS values):
 * rows multiplied in one phase, rows mispredicted (recomputed exactly), rows
 * past the hash bins (exact), entries of temporary memory used, one-phase
 * rows that filled their table more than 3/4, those that the next smaller
 * table would hold at most 3/4 full, then the factor exponent k_j that the
 * call used for each class j. */
int spgemm_learned_stats(const spgemm_handle *h, int64_t *out, int n);

/* Features of rows [row_begin, row_end) of C = A * B into X (device,
 * (row_end - row_begin) x 6 floats, row-major). workspace: device memory of
 * 16 bytes per row. Ordered on `stream`. */
int spgemm_features(const spgemm_csr_in *A, const spgemm_csr_in *B, int64_t row_begin,
                    int64_t row_end, float *X, void *workspace, void *stream);

/* y[i] = predictor(X[i]) for n rows (device pointers). */
int spgemm_mlp_forward(const float *theta, const float *X, int64_t n, float *y, void *stream);

/* Adds to grad (4673 floats, device) the gradient of
 * sum over these n samples of (y_i - t_i)^2 / n_total, and that sum to
 * *loss (device float): call once per part of a mini-batch of n_total
 * samples after zeroing grad and loss. */
int spgemm_mlp_train_step(const float *theta, const float *X, const float *t, int64_t n,
                          int64_t n_total, float *grad, float *loss, void *stream);

/* One Adam step (Kingma & Ba, with bias correction; step counts from 1) on
 * the 4673 parameters; m and v are the moment buffers (device). */
int spgemm_mlp_adam(float *theta, const float *grad, float *m, float *v, int step, float lr,
                    float beta1, float beta2, float eps, void *stream);

/* ---- Batched products ------------------------------------------------------
 * Many products C_i = A_i * B_i with small rows (for example the Galerkin
 * products P^T (A P) of an algebraic-multigrid setup) run in one persistent
 * kernel, captured once in a CUDA graph. B_i may be the C of an earlier
 * product j < i (b_from[i] = j; -1 or b_from NULL: B[i] is an input, and
 * B[i] is then ignored when b_from[i] >= 0). Each product follows the
 * two-phase method (symbolic row tiles, scan, numeric row tiles); blocks
 * take work items from a device queue and wait, with a bound, for the items
 * they depend on. Inputs are device CSR that must stay valid while the
 * batch exists. The plan (spgemm_batch_create) bounds every row's size by
 * its number of intermediate products and places every C in one arena; a
 * batch whose largest row bound exceeds the largest table (256) is
 * rejected with SPGEMM_ERR_INVALID. */
typedef struct spgemm_batch spgemm_batch;
typedef struct {
    int32_t variant;     /* -1: smallest table that holds the largest row;
                            0, 1, 2: 8 lanes / 64 slots, 16 / 128, 32 / 256 */
    int32_t tile_rows;   /* rows per work item, at most 1024 (0: 32 per row group) */
    int64_t spin_limit;  /* polls of a bounded wait, 200 ns apart (0: 2^22) */
    int32_t no_tiny;     /* 1: products whose rows have at most 8 products
                            also use the hash tables (0: one thread per row) */
    int32_t reserved;
} spgemm_batch_options;

int spgemm_batch_create(spgemm_batch **b, spgemm_handle *h, int n, const spgemm_csr_in *A,
                        const spgemm_csr_in *B, const int32_t *b_from,
                        const spgemm_batch_options *opt);
/* Enqueue one run (one graph launch) on the handle's stream. */
int spgemm_batch_run(spgemm_batch *b);
/* Wait for the last run: SPGEMM_OK, SPGEMM_ERR_TIMEOUT (a bounded wait ran
 * out) or SPGEMM_ERR_INTERNAL (a row outgrew its bound); reads the sizes. */
int spgemm_batch_sync(spgemm_batch *b);
/* Product i of the last synchronised run: device pointers into the batch's
 * arena (valid until the next run or destroy), C.rpt int64 (rows + 1). */
int spgemm_batch_result(const spgemm_batch *b, int i, spgemm_csr_out *C);
/* products, work items, blocks, lanes per row, table slots, rows per item */
int spgemm_batch_info(const spgemm_batch *b, int64_t *out, int n);
int spgemm_batch_destroy(spgemm_batch *b);

/* ---- Operation-rate probes --------------------------------------------------
 * Diagnostic, with no counterpart in the paper: the rates of the operations
 * the numeric kernels are built from, which bound them beside the memory
 * roofline. Every intermediate product costs one float64 multiply-add and
 * one accumulation into its output entry. One 1024-thread block per SM runs
 * `iters` operations per thread (after one untimed run); *gops receives
 * operations per second / 1e9 (op 0: fused multiply-adds, two flops each).
 *   op 0  float64 fma, 8 independent chains per thread
 *   op 1  shared float64 accumulation by compare-and-swap of fma (the
 *         kernels' update), over 16384 doubles
 *   op 2  shared float64 atomicAdd over 16384 doubles
 *   op 3  shared 32-bit atomicOr over 2^19 bits
 *   op 4  shared 32-bit atomicCAS over 2^15 slots (a hash probe)
 *   op 5  global float64 reduction (red.add) over at most 32 MB of buf
 *         (L2-resident)
 *   op 6  global float64 reduction over all of buf (mostly DRAM)
 *   op 7  as op 5, but the 32 lanes of a warp reduce into 32 consecutive
 *         doubles
 * hot = 0 spreads the addresses uniformly; hot = h > 0 sends every
 * operation to one of h addresses (contention). buf: device memory of
 * buf_bytes (at least 1 MB) for ops 5 to 7, zeroed by the call; may be NULL
 * otherwise. Synchronises `stream`. */
int spgemm_probe(int op, int hot, int64_t iters, void *buf, int64_t buf_bytes, double *gops, void *stream);

const char *spgemm_strerror(int code);
/* Name of the last CUDA runtime error that the library, on the calling
 * thread, turned into SPGEMM_ERR_CUDA or SPGEMM_ERR_OOM (e.g.
 * "cudaErrorInvalidValue"), or NULL if there was none. Diagnostic only; a
 * static string. */
const char *spgemm_last_cuda_error(void);

/* ---- Sizing C without allocating device memory --------------------------
 * The paper has no counterpart to this function; it serves callers that
 * cannot call cudaMalloc at run time, such as a serving loop whose device
 * memory is all owned by another framework's allocator, a runtime with a
 * memory budget fixed at start-up, or code that is itself an allocator.
 *
 * spgemm_rowptr_noalloc runs the symbolic phase of C = A * B over all rows
 * of A (n_prod, symbolic binning, the symbolic kernels, the exclusive scan)
 * and writes C's int64 row pointer into crpt (device memory, A->rows + 1
 * entries, caller-owned): crpt[i] is the offset of row i, crpt[A->rows] =
 * *nnzC (nnzC may be NULL). A->val and B->val are not read. The result is
 * the same row pointer that spgemm_symbolic followed by spgemm_numeric
 * produce with the default configuration.
 *
 * It allocates nothing and creates no handle, stream or event: its scratch
 * memory is one fixed array inside the library (about 4 MB, held by every
 * GPU that loads the library until the process exits), sized for at most
 * SPGEMM_NOALLOC_MAX_ROWS rows of A; larger A is rejected with
 * SPGEMM_ERR_INVALID. All work is ordered on `stream` (a cudaStream_t; NULL
 * = legacy default stream) and the call waits for it twice (to read the
 * bin sizes and the total).
 *
 * The first call on a device looks up the array's device address and
 * prepares the kernels on that device, with that device current; make that
 * first call before any stream capture. Every call uses the same array and
 * it keeps the previous call's contents (the call clears what must start at
 * zero), so calls that overlap on the GPU, from several host threads or on
 * several streams, race with each other and must be serialised by the
 * caller. */
#define SPGEMM_NOALLOC_MAX_ROWS (1 << 20)
int spgemm_rowptr_noalloc(const spgemm_csr_in *A, const spgemm_csr_in *B,
                          int64_t *crpt, void *stream, int64_t *nnzC);

#ifdef __cplusplus
}
#endif

#endif /* OPSPARSE_H */
