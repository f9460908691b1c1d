// Column-window numeric kernel for the large rows (the numeric phase of Sec.
// 2.2 and Sec. 5.2: Algorithm 5's accumulation followed by the condense, sort
// and store of Sec. 5.6.2), used when every row of B is sorted by column.
//
// A large output row is the union of many long, sorted B rows. Instead of
// one block per row that sums into C.val with global float64 reductions,
// the row is cut into windows of whole cells (2^cs columns each). The
// symbolic bitmap kernel counts each large row's entries per cell; a planner
// turns those counts into windows that fit one block's shared memory, and
// every window is summed in shared memory and written to C once, in column
// order:
//
//   column window  accumulator indexed by column (8 bytes per column) plus a
//                  presence bitmap; one pass over the window's products;
//                  used where at least one column in 8 holds an entry;
//   rank window    column bitmap, per-word ranks (16 bits) and an
//                  accumulator indexed by rank (8 bytes per entry); one pass
//                  marks the columns, a second adds the values at their ranks.
//
// With B sorted, the products of a window are, for every A entry of the row,
// one contiguous run of its B row; the run bounds come from a cell index of
// the long B rows (two loads) or a binary search of a short one. A persistent
// kernel (one block per SM) takes windows from a counter. Each window leaves
// the shared accumulator and bitmaps zero for the next one, so only the
// entries a window touched are cleared.
//
// This replaces the paper's global-memory hash kernel for its largest rows
// (its numeric kernel 7) and the in-row sort: the bitmap and its ranks give
// the sorted order directly.
#include <climits>

#include "common.cuh"
#include "internal.h"

namespace ops {

constexpr int kWinBlock = 1024;
constexpr int kWinIters = 4;    // products one lane loads before using them
constexpr int kWinBatch = 4;    // pieces a sub-group takes per grab of the piece counter

// Shared bytes of a window's body. A column window holds an accumulator
// per column, presence bits, their ranks and spill bits; a rank window only a
// bitmap of its columns and a 32-bit rank per 64-bit word (its values are
// summed in C.val itself).
__host__ __device__ inline long long rank_bytes(long long width, long long) {
    const long long nw = (width + 63) >> 6;
    return 12 * nw;
}
__host__ __device__ inline long long col_bytes(long long width) {
    const long long nw = (width + 31) >> 5;
    return 8 * width + 12 * nw;   // accumulator, presence bits, ranks, spill bits
}
long long win_rank_bytes(long long width, long long n) { return rank_bytes(width, n); }
long long win_col_bytes(long long width) { return col_bytes(width); }

struct WinHead {
    long long q[kWinBlock];          // first B entry of each run of the chunk
    int len[kWinBlock];              // run length
    int pstart[kWinBlock + 1];       // exclusive piece offsets
    long long red[34];
    Win win;                         // the window being computed
    long long widx;
    unsigned ctr;                    // piece counter of the chunk
    int S;                           // threads per run of the current chunk
    int bad;
};

constexpr size_t kWinHeadBytes = (sizeof(WinHead) + 15) & ~static_cast<size_t>(15);
size_t win_head_bytes() { return kWinHeadBytes; }

// acc[idx[u]] += a * b[u] for the entries with idx[u] >= 0, in shared
// memory, each with one compare-and-swap of the fused multiply-add. The
// loads, multiply-adds and compare-and-swaps of the N entries are issued
// together (no entry waits for another's round trip). A lost race (another
// thread updated the entry in between, or the same entry twice in the
// batch) does not retry: the product goes to the block's L2 spill slot
// g[idx] with a float64 reduction, and the entry's spill bit is set. On a hot
// entry (a column that many B rows share) shared-memory compare-and-swap
// serialises on its round trip, while the L2 adds same-address reductions
// in its own pipeline.
template <int N>
__device__ __forceinline__ void acc_add(double *acc, const int (&idx)[N], double a, const double (&b)[N], double *g,
                                        unsigned *spill) {
    unsigned long long *q = reinterpret_cast<unsigned long long *>(acc);
    unsigned long long old[N], got[N];
#pragma unroll
    for (int u = 0; u < N; ++u) old[u] = idx[u] >= 0 ? q[idx[u]] : 0ull;
#pragma unroll
    for (int u = 0; u < N; ++u) {
        got[u] = old[u];
        if (idx[u] >= 0) {
            const unsigned long long want = static_cast<unsigned long long>(
                __double_as_longlong(fma(a, b[u], __longlong_as_double(static_cast<long long>(old[u])))));
            got[u] = atomicCAS(q + idx[u], old[u], want);
        }
    }
#pragma unroll
    for (int u = 0; u < N; ++u) {
        if (idx[u] >= 0 && got[u] != old[u]) {
            asm volatile("red.global.add.f64 [%0], %1;" ::"l"(g + idx[u]), "d"(a * b[u]) : "memory");
            atomicOr(spill + (idx[u] >> 5), 1u << (idx[u] & 31));
        }
    }
}

// Value of accumulator entry i at the store: the shared sum plus, when its
// spill bit is set, the L2 part, whose slot is cleared for the next window.
__device__ __forceinline__ double acc_take(const double *acc, const unsigned *spill, double *g, unsigned i) {
    double v = acc[i];
    if ((spill[i >> 5] >> (i & 31)) & 1u) {
        v += __ldcg(g + i);
        __stcg(g + i, 0.0);
    }
    return v;
}

// --- planner -------------------------------------------------------------------
// Cuts one row into windows; emit(c0, c1, r0, n, mode) for each. Returns
// the number of windows, or -1 when the cells do not add up to n_nz (or a
// single cell does not fit). Rows with at most e1 entries (or no cells) take
// one rank window over all columns.
template <typename Emit>
__device__ int plan_row(const uint16_t *cells, long long n_nz, const WinPlan &pa, Emit &&emit) {
    if (n_nz <= 0) return 0;
    if (n_nz <= pa.e1) {
        emit(0LL, pa.ncols, 0LL, n_nz, static_cast<int>(kWinRank));
        return 1;
    }
    if (!cells) return -1;
    const long long cw = 1LL << pa.cs;
    int s = 0, cnt = 0;
    long long r = 0;
    while (s < pa.ncells) {
        if (cells[s] == 0) {
            ++s;
            continue;
        }
        int tc = s;
        long long ec = 0;
        while (tc < pa.ncells && tc - s < pa.kc) ec += cells[tc++];
        while (tc > s + 1 && cells[tc - 1] == 0) --tc;
        int tr = s;
        long long er = 0;
        while (tr < pa.ncells) {
            const long long c1 = min((tr + 1) * cw, pa.ncols);
            if (rank_bytes(c1 - s * cw, er + cells[tr]) > pa.budget) break;
            er += cells[tr++];
        }
        if (tr == s) return -1;
        while (tr > s + 1 && cells[tr - 1] == 0) --tr;
        const long long wc = min(tc * cw, pa.ncols) - s * cw;
        // by column where at least one column in 8 holds an entry: one pass
        // over the products instead of two outweighs the narrower window
        const bool col = pa.kc > 0 && 8 * ec >= wc;
        const int t = col ? tc : tr;
        const long long e = col ? ec : er;
        emit(s * cw, min(t * cw, pa.ncols), r, e, col ? static_cast<int>(kWinCol) : static_cast<int>(kWinRank));
        r += e;
        s = t;
        ++cnt;
    }
    return r == n_nz ? cnt : -1;
}

__global__ void __launch_bounds__(256)
win_count_kernel(WinPlan pa, const int64_t *crpt, int64_t mw, const uint16_t *cells, const int32_t *cslot,
                 unsigned long long *total, unsigned long long *total_col, int *err) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    unsigned long long c = 0, cc = 0;
    if (i < mw) {
        const long long n = crpt[i];
        if (n > pa.cut) {
            const uint16_t *cl = nullptr;
            if (n > pa.e1) {
                const int32_t slot = cslot ? cslot[i] : -1;
                if (slot >= 0) cl = cells + static_cast<int64_t>(slot) * pa.ncells;
            }
            const int k = plan_row(cl, n, pa, [&](long long, long long, long long, long long, int mode) {
                cc += mode == kWinCol;
            });
            if (k < 0) {
                set_error(err, DERR_WINDOW);
                cc = 0;
            } else {
                c = static_cast<unsigned long long>(k);
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        c += __shfl_xor_sync(0xffffffffu, c, o);
        cc += __shfl_xor_sync(0xffffffffu, cc, o);
    }
    if ((threadIdx.x & 31) == 0 && c) {
        atomicAdd(total, c);
        if (cc) atomicAdd(total_col, cc);
    }
}

cudaError_t launch_win_count(const WinPlan &plan, const int64_t *crpt, int64_t mw, const uint16_t *cells,
                             const int32_t *cslot, unsigned long long *total, unsigned long long *total_col,
                             int *err, cudaStream_t s) {
    if (mw <= 0) return cudaSuccess;
    win_count_kernel<<<static_cast<unsigned>((mw + 255) / 256), 256, 0, s>>>(plan, crpt, mw, cells, cslot,
                                                                             total, total_col, err);
    return cudaGetLastError();
}

// One thread per row of the bin: the same cut as win_count_kernel, written
// to the list at a range reserved with one atomic add.
__global__ void __launch_bounds__(256)
win_plan_kernel(WinPlan pa, BinWork w, const uint16_t *cells, const int32_t *cslot, Win *list, long long cap,
                unsigned long long *cursor) {
    const int64_t r = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (r >= w.cnt) return;
    const int64_t row = w.bins ? static_cast<int64_t>(w.bins[w.off + r]) : w.off + r;
    const long long n = w.crpt[row + 1] - w.crpt[row];
    const uint16_t *cl = nullptr;
    if (n > pa.e1) {
        const int32_t slot = cslot ? cslot[row] : -1;
        if (slot >= 0) cl = cells + static_cast<int64_t>(slot) * pa.ncells;
    }
    const int k = plan_row(cl, n, pa, [](long long, long long, long long, long long, int) {});
    if (k <= 0) {
        if (k < 0) set_error(w.err, DERR_WINDOW);
        return;
    }
    const unsigned long long at = atomicAdd(cursor, static_cast<unsigned long long>(k));
    if (at + k > static_cast<unsigned long long>(cap)) {
        set_error(w.err, DERR_WINDOW);
        return;
    }
    Win *out = list + at;
    plan_row(cl, n, pa, [&](long long c0, long long c1, long long r0, long long e, int mode) {
        Win v;
        v.row = static_cast<int32_t>(row);
        v.c0 = static_cast<int32_t>(c0);
        v.c1 = static_cast<int32_t>(c1);
        v.mode = mode;
        v.r0 = static_cast<uint32_t>(r0);
        v.n = static_cast<uint32_t>(e);
        *out++ = v;
    });
}

cudaError_t launch_win_plan(const WinPlan &plan, const BinWork &w, const uint16_t *cells, const int32_t *cslot,
                            Win *list, long long cap, unsigned long long *cursor, cudaStream_t s) {
    if (w.cnt <= 0) return cudaSuccess;
    win_plan_kernel<<<static_cast<unsigned>((w.cnt + 255) / 256), 256, 0, s>>>(plan, w, cells, cslot, list, cap,
                                                                               cursor);
    return cudaGetLastError();
}

// --- cell index of the long rows of B ------------------------------------------
// One warp per row of B. A row with at least min_len entries takes a slot s
// (up to cap) and gets bidx[s * (ncells + 1) + c] = offset in the row of its
// first entry with column >= c * 2^cs (c = 0..ncells): entry e writes the
// cells after the previous entry's cell up to its own; the last entry writes
// the rest. Shorter rows (and rows past the cap) get slot -1 and are
// searched.
__global__ void __launch_bounds__(256)
win_bindex_kernel(Operands op, int64_t brows, int cs, int ncells, long long min_len, int32_t *bslot,
                  int32_t *bidx, long long cap, unsigned long long *nslot) {
    const int64_t k = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (k >= brows) return;
    const int64_t q0 = ld_rpt(op.brpt, op.b64, k);
    const int64_t len = ld_rpt(op.brpt, op.b64, k + 1) - q0;
    long long slot = -1;
    if (len >= min_len && lane == 0) {
        slot = static_cast<long long>(atomicAdd(nslot, 1ull));
        if (slot >= cap) slot = -1;
    }
    slot = __shfl_sync(0xffffffffu, slot, 0);
    if (lane == 0) bslot[k] = static_cast<int32_t>(slot);
    if (slot < 0) return;
    int32_t *x = bidx + slot * (ncells + 1);
    for (int64_t e = lane; e < len; e += 32) {
        const int cc = min(__ldg(op.bcol + q0 + e) >> cs, ncells);
        const int pc = e == 0 ? -1 : min(__ldg(op.bcol + q0 + e - 1) >> cs, ncells);
        for (int c = pc + 1; c <= cc; ++c) x[c] = static_cast<int32_t>(e);
        if (e + 1 == len)
            for (int c = cc + 1; c <= ncells; ++c) x[c] = static_cast<int32_t>(len);
    }
}

cudaError_t launch_win_bindex(const Operands &op, int64_t brows, const WinPlan &plan, long long min_len,
                              int32_t *bslot, int32_t *bidx, long long cap, unsigned long long *nslot,
                              cudaStream_t s) {
    if (brows <= 0) return cudaSuccess;
    const int64_t threads = brows * 32;
    win_bindex_kernel<<<static_cast<unsigned>((threads + 255) / 256), 256, 0, s>>>(
        op, brows, plan.cs, plan.ncells, min_len, bslot, bidx, cap, nslot);
    return cudaGetLastError();
}

// --- the window kernel -----------------------------------------------------------
// First index in [lo, hi) of B.col with column >= c (B row sorted).
__device__ __forceinline__ long long lower_col(const int32_t *bcol, long long lo, long long hi, int c) {
    while (lo < hi) {
        const long long mid = lo + ((hi - lo) >> 1);
        if (__ldg(bcol + mid) < c) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Sum of one long long per thread over the block; every thread gets it.
__device__ __forceinline__ long long block_sum_ll(long long x, long long *sw) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = x;
    __syncthreads();
    long long t = (threadIdx.x & 31) < (blockDim.x >> 5) ? sw[threadIdx.x & 31] : 0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    return t;
}

// Visits every product of the current window:
// for each A entry of the row [p0, p1), the run of its B row inside columns
// [c0, c1). Runs are set up BLOCK at a time (one per thread); every run is
// cut into pieces of at most S * ITERS products, S the threads that read a
// run together (from the chunk's mean run length, so short runs do not
// leave lanes idle), and warps take pieces from a shared counter, a batch at
// a time, so a warp that drew long runs does not hold the others at the
// barrier. A lane loads its ITERS products, then hands them to
// f(key[ITERS], a_value, b_value[ITERS]) together (key -1: no product).
// keep: the row fits one chunk and the previous walk of this window left its
// runs in place.
template <int BLOCK, int ITERS, bool VAL, typename F>
__device__ __forceinline__ void win_walk(const Operands &op, const WinWork &ww, int64_t p0, int64_t p1, int c0,
                                         int c1, WinHead *hd, bool keep, F &&f) {
    const bool whole = c0 == 0 && c1 >= op.ncols;
    const int lane = threadIdx.x & 31;
    for (int64_t c = p0; c < p1; c += BLOCK) {
        const int cnt = static_cast<int>(p1 - c < BLOCK ? p1 - c : BLOCK);
        if (keep && p1 - p0 <= BLOCK) {
            if (threadIdx.x == 0) hd->ctr = 0;
            __syncthreads();
        } else {
            long long len = 0;
            if (threadIdx.x < cnt) {
                const int t = threadIdx.x;
                const int k = __ldg(op.acol + c + t);
                const long long q0 = ld_rpt(op.brpt, op.b64, k);
                const long long q1 = ld_rpt(op.brpt, op.b64, k + 1);
                long long s = q0, e = q1;
                if (!whole) {
                    const int32_t slot = ww.bslot ? __ldg(ww.bslot + k) : -1;
                    if (slot >= 0) {
                        const int32_t *x = ww.bidx + static_cast<long long>(slot) * (ww.ncells + 1);
                        if (c0 > 0) s = q0 + __ldg(x + (c0 >> ww.cs));
                        if (c1 < op.ncols) e = q0 + __ldg(x + (c1 >> ww.cs));
                    } else {
                        if (c0 > 0) s = lower_col(op.bcol, q0, q1, c0);
                        if (c1 < op.ncols) e = lower_col(op.bcol, s, q1, c1);
                    }
                }
                if (e < s) e = s;
                hd->q[t] = s;
                hd->len[t] = static_cast<int>(e - s);
                len = e - s;
            }
            // mean length of the non-empty runs -> S (sum and count in one reduction)
            const long long packed = block_sum_ll((len << 11) + (len > 0 ? 1 : 0), hd->red);
            const long long ne = packed & 2047, sum = packed >> 11;
            const long long mean = ne ? (sum + ne - 1) / ne : 1;
            int S = 1;
            while (S < 32 && static_cast<long long>(S) * ITERS < mean) S <<= 1;
            const long long W = static_cast<long long>(S) * ITERS;
            long long total;
            const long long ex = block_excl_scan_ll<BLOCK>((len + W - 1) / W, total, hd->red);
            hd->pstart[threadIdx.x] = static_cast<int>(ex);   // entries >= cnt hold `total`
            if (threadIdx.x == 0) {
                hd->pstart[BLOCK] = static_cast<int>(total);
                hd->S = S;
                hd->ctr = 0;
            }
            __syncthreads();
        }
        const int S = hd->S;
        const int total = hd->pstart[BLOCK];
        const int W = S * ITERS;
        const int spw = 32 / S, wsub = lane / S, ls = lane % S;
        const int a_off = static_cast<int>(c - p0);
        int lo = 0;
        for (;;) {
            unsigned base = 0;
            if (lane == 0) base = atomicAdd(&hd->ctr, static_cast<unsigned>(spw * kWinBatch));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (base >= static_cast<unsigned>(total)) break;
            const int it0 = static_cast<int>(base) + wsub * kWinBatch;
            const int it1 = it0 + kWinBatch < total ? it0 + kWinBatch : total;
            if (it0 >= it1) continue;
            {   // last e with pstart[e] <= it0, at or after the previous one
                int hi = cnt;
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (hd->pstart[mid] <= it0) lo = mid; else hi = mid;
                }
            }
            int next = hd->pstart[lo + 1];
            for (int it = it0; it < it1; ++it) {
                while (it >= next) {
                    ++lo;
                    next = hd->pstart[lo + 1];
                }
                const long long qb = hd->q[lo] + static_cast<long long>(it - hd->pstart[lo]) * W + ls;
                const long long qe = hd->q[lo] + hd->len[lo];
                const double a = VAL ? __ldg(op.aval + p0 + a_off + lo) : 0.0;
                int key[ITERS];
                double bv[ITERS];
#pragma unroll
                for (int u = 0; u < ITERS; ++u) {
                    const long long q = qb + static_cast<long long>(u) * S;
                    key[u] = q < qe ? __ldg(op.bcol + q) : -1;
                    bv[u] = (VAL && q < qe) ? __ldg(op.bval + q) : 0.0;
                }
                f(key, a, bv);
            }
        }
        __syncthreads();
    }
}

// Per-word ranks of a bitmap of nw 64-bit words: pre[i] = set bits in
// words [0, i); returns the total. Warps own contiguous ranges of words,
// lanes read consecutive words (no bank conflicts).
template <int BLOCK>
__device__ __forceinline__ unsigned ranks32(const unsigned long long *bm, unsigned *pre, int nw, long long *sw) {
    constexpr int kWarps = BLOCK / 32;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int per = (((nw + kWarps - 1) / kWarps) + 31) & ~31;
    const int w0 = wp * per;
    const int w1 = w0 + per < nw ? w0 + per : nw;
    unsigned cnt = 0;
    for (int i = w0 + lane; i < w1; i += 32) cnt += static_cast<unsigned>(__popcll(bm[i]));
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    long long total;
    const long long base0 = block_excl_scan_ll<BLOCK>(lane == 0 ? cnt : 0, total, sw);
    unsigned base = static_cast<unsigned>(__shfl_sync(0xffffffffu, base0, 0));
    for (int i0 = w0; i0 < w1; i0 += 32) {
        const int i = i0 + lane;
        const unsigned c = i < w1 ? static_cast<unsigned>(__popcll(bm[i])) : 0u;
        unsigned inc = c;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (i < w1) pre[i] = base + inc - c;
        base += __shfl_sync(0xffffffffu, inc, 31);
    }
    __syncthreads();
    return static_cast<unsigned>(total);
}

template <int BLOCK, int ITERS>
__global__ void __launch_bounds__(BLOCK, 1)
win_numeric_kernel(Operands op, BinWork w, WinWork ww) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    WinHead *hd = reinterpret_cast<WinHead *>(smem_raw);
    unsigned char *body = smem_raw + kWinHeadBytes;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int kWarps = BLOCK / 32;
    double *gsp = ww.spill + static_cast<long long>(blockIdx.x) * ww.spill_stride;
    // the body starts zero; every window leaves it zero
    {
        uint4 *b4 = reinterpret_cast<uint4 *>(body);
        const long long n16 = ww.budget >> 4;
        for (long long i = threadIdx.x; i < n16; i += BLOCK) b4[i] = make_uint4(0u, 0u, 0u, 0u);
    }
    __syncthreads();
    for (;;) {
        if (threadIdx.x == 0) {
            const long long i = static_cast<long long>(atomicAdd(ww.next, 1ull));
            hd->widx = i;
            if (i < ww.nwin) hd->win = ww.win[i];
            hd->bad = 0;
        }
        __syncthreads();
        if (hd->widx >= ww.nwin) break;
        const Win win = hd->win;
        const int64_t row = win.row;
        const int c0 = win.c0, c1 = win.c1;
        const long long width = static_cast<long long>(c1) - c0;
        const long long n = win.n;
        const int64_t out = w.crpt[row] + win.r0;
        const int64_t ar = op.row0 + row;
        const int64_t p0 = ld_rpt(op.arpt, op.a64, ar);
        const int64_t p1 = ld_rpt(op.arpt, op.a64, ar + 1);
        const unsigned uw = static_cast<unsigned>(width);
        bool bad = false;
        if (win.mode == kWinCol) {
            // accumulator by column, presence bits, their ranks, spill bits
            const int nw = static_cast<int>((width + 31) >> 5);
            double *acc = reinterpret_cast<double *>(body);
            unsigned *bits = reinterpret_cast<unsigned *>(body + 8 * width);
            unsigned *pre = bits + nw;
            unsigned *spl = pre + nw;
            if (width <= 0 || width > ww.spill_stride || col_bytes(width) > ww.budget) {
                if (threadIdx.x == 0) set_error(w.err, DERR_WINDOW);
                __syncthreads();
                continue;
            }
            win_walk<BLOCK, ITERS, true>(op, ww, p0, p1, c0, c1, hd, false,
                                         [&](const int (&key)[ITERS], double a, const double (&b)[ITERS]) {
                int idx[ITERS];
#pragma unroll
                for (int u = 0; u < ITERS; ++u) {
                    const unsigned rel = static_cast<unsigned>(key[u] - c0);
                    idx[u] = -1;
                    if (key[u] >= 0) {
                        if (rel < uw) {
                            atomicOr(bits + (rel >> 5), 1u << (rel & 31));
                            idx[u] = static_cast<int>(rel);
                        } else {
                            bad = true;
                        }
                    }
                }
                acc_add<ITERS>(acc, idx, a, b, gsp, spl);
            });
            // ranks of the presence words: one word per thread, block scan
            long long tot = 0;
            for (int base = 0; base < nw; base += BLOCK) {
                const int i = base + threadIdx.x;
                const long long cb = i < nw ? __popc(bits[i]) : 0;
                long long t;
                const long long ex = block_excl_scan_ll<BLOCK>(cb, t, hd->red);
                if (i < nw) pre[i] = static_cast<unsigned>(tot + ex);
                tot += t;
            }
            __syncthreads();
            const bool ok = tot == n;
            if (!ok && threadIdx.x == 0) set_error(w.err, DERR_COUNT_MISMATCH);
            // store: one word per warp iteration, lane = bit; present entries
            // of a word have consecutive ranks, so each store is one run
            const unsigned lt = (1u << lane) - 1u;
            for (int i = warp; i < nw; i += kWarps) {
                const unsigned x = bits[i];
                if (!x) continue;
                if ((x >> lane) & 1u) {
                    const unsigned rel = static_cast<unsigned>(i * 32 + lane);
                    const double v = acc_take(acc, spl, gsp, rel);
                    if (ok) {
                        const int64_t rk = out + pre[i] + __popc(x & lt);
                        w.ccol[rk] = c0 + static_cast<int>(rel);
                        w.cval[rk] = v;
                    }
                    acc[rel] = 0.0;
                }
            }
            __syncthreads();
            for (int i = threadIdx.x; i < nw; i += BLOCK) {
                bits[i] = 0u;
                pre[i] = 0u;
                spl[i] = 0u;
            }
        } else {
            // rank window: bitmap and 32-bit ranks per word; the values are
            // summed into C.val itself with float64 L2 reductions (the
            // entries of a sparse window rarely meet, so the L2 adds them
            // without the round trips of shared-memory compare-and-swap)
            const int nw = static_cast<int>((width + 63) >> 6);
            unsigned long long *bm = reinterpret_cast<unsigned long long *>(body);
            unsigned *bm32 = reinterpret_cast<unsigned *>(bm);
            unsigned *pre = reinterpret_cast<unsigned *>(bm + nw);
            if (width <= 0 || rank_bytes(width, n) > ww.budget) {
                if (threadIdx.x == 0) set_error(w.err, DERR_WINDOW);
                __syncthreads();
                continue;
            }
            win_walk<BLOCK, ITERS, false>(op, ww, p0, p1, c0, c1, hd, false,
                                          [&](const int (&key)[ITERS], double, const double (&)[ITERS]) {
#pragma unroll
                for (int u = 0; u < ITERS; ++u) {
                    const unsigned rel = static_cast<unsigned>(key[u] - c0);
                    if (key[u] < 0) continue;
                    if (rel < uw) atomicOr(bm32 + (rel >> 5), 1u << (rel & 31));
                    else bad = true;
                }
            });
            const unsigned tot = ranks32<BLOCK>(bm, pre, nw, hd->red);
            const bool ok = tot == n;
            if (!ok && threadIdx.x == 0) set_error(w.err, DERR_COUNT_MISMATCH);
            if (ok) {
                int32_t *ccol = w.ccol + out;
                double *cval = w.cval + out;
                const unsigned long long pol = l2_evict_last_policy();
                // C.col in column order: each warp takes a contiguous range of
                // words of about equal cost (entries + 2 per word); a lane
                // writes its own word, words with many entries are written by
                // the whole warp (lane = bit), so one store covers a run
                constexpr int kDense = 24;
                constexpr unsigned long long kWordCost = 2;
                const unsigned lt = (1u << lane) - 1u;
                const unsigned long long vtot = static_cast<unsigned long long>(n) + kWordCost * nw;
                auto first_word = [&](unsigned long long cost) {
                    int lo = 0, hi = nw;
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (pre[mid] + kWordCost * static_cast<unsigned long long>(mid) >= cost) hi = mid;
                        else lo = mid + 1;
                    }
                    return lo;
                };
                const unsigned long long wq = static_cast<unsigned long long>(warp);
                const int i_beg = first_word(vtot * wq / kWarps);
                const int i_end = first_word(vtot * (wq + 1) / kWarps);
                for (int ib = i_beg; ib < i_end; ib += 32) {
                    const int i = ib + lane;
                    const unsigned long long x = i < i_end ? bm[i] : 0ull;
                    const unsigned pos0 = i < i_end ? pre[i] : 0u;
                    const bool dense = __popcll(x) >= kDense;
                    unsigned dm = __ballot_sync(0xffffffffu, dense);
                    if (!dense) {
                        unsigned pos = pos0;
                        const int cb = c0 + i * 64;
                        unsigned lo = static_cast<unsigned>(x), hi = static_cast<unsigned>(x >> 32);
                        while (lo) {
                            const int b = __ffs(lo) - 1;
                            lo &= lo - 1;
                            ccol[pos++] = cb + b;
                        }
                        while (hi) {
                            const int b = __ffs(hi) - 1;
                            hi &= hi - 1;
                            ccol[pos++] = cb + 32 + b;
                        }
                    }
                    while (dm) {
                        const int src = __ffs(dm) - 1;
                        dm &= dm - 1;
                        const unsigned long long xw = __shfl_sync(0xffffffffu, x, src);
                        const unsigned pw = __shfl_sync(0xffffffffu, pos0, src);
                        const int cb = c0 + (ib + src) * 64;
                        const unsigned lo = static_cast<unsigned>(xw), hi = static_cast<unsigned>(xw >> 32);
                        if ((lo >> lane) & 1u) ccol[pw + __popc(lo & lt)] = cb + lane;
                        if ((hi >> lane) & 1u) ccol[pw + __popc(lo) + __popc(hi & lt)] = cb + 32 + lane;
                    }
                }
                // C.val starts at zero; its lines stay in L2 (evict-last) while summed
                for (long long t = threadIdx.x; t < n; t += BLOCK) st_keep(cval + t, 0.0, pol);
                __syncthreads();
                win_walk<BLOCK, ITERS, true>(op, ww, p0, p1, c0, c1, hd, true,
                                             [&](const int (&key)[ITERS], double a, const double (&b)[ITERS]) {
#pragma unroll
                    for (int u = 0; u < ITERS; ++u) {
                        const unsigned rel = static_cast<unsigned>(key[u] - c0);
                        if (key[u] >= 0 && rel < uw) {
                            const unsigned wi = rel >> 6, bi = rel & 63u;
                            const unsigned rk = pre[wi] + static_cast<unsigned>(__popcll(bm[wi] << (63u - bi))) - 1u;
                            if (rk < static_cast<unsigned>(n)) red_add_keep(cval + rk, a * b[u], pol);
                        }
                    }
                });
                // back to normal priority: every 128-byte line of the segment
                const uintptr_t l0 = reinterpret_cast<uintptr_t>(cval) & ~static_cast<uintptr_t>(127);
                const uintptr_t l1 = reinterpret_cast<uintptr_t>(cval + n);
                for (uintptr_t l = l0 + 128 * static_cast<uintptr_t>(threadIdx.x); l < l1;
                     l += 128 * static_cast<uintptr_t>(BLOCK))
                    l2_priority_normal(reinterpret_cast<const void *>(l));
            }
            __syncthreads();
            // leave the body zero: bitmap and ranks
            for (int i = threadIdx.x; i < nw; i += BLOCK) {
                bm[i] = 0ull;
                pre[i] = 0u;
            }
        }
        if (bad) hd->bad = 1;   // benign race: any writer sets 1
        __syncthreads();
        if (threadIdx.x == 0 && hd->bad) set_error(w.err, DERR_WINDOW);
    }
}

using WinFn = void (*)(Operands, BinWork, WinWork);
static const WinFn g_win_fn = &win_numeric_kernel<kWinBlock, kWinIters>;

cudaError_t win_prepare(int smem_optin) {
    return cudaFuncSetAttribute(reinterpret_cast<const void *>(g_win_fn),
                                cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin);
}

cudaError_t launch_win_numeric(const Operands &op, const BinWork &w, const WinWork &ww, int grid, size_t smem,
                               cudaStream_t s) {
    if (ww.nwin <= 0) return cudaSuccess;
    g_win_fn<<<grid, kWinBlock, smem, s>>>(op, w, ww);
    return cudaGetLastError();
}

}  // namespace ops
