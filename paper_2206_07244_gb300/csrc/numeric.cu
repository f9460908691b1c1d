// Numeric phase (Sec. 2.2, Sec. 5.2, Algorithm 5, Sec. 5.6.2): the sorted
// column indices and summed values of each output row, written at the row
// offsets that the scan left in C.rpt.
//
// Bins 0..8: a row group of TPR threads owns a shared-memory table of T
// (int32 key, float64 value) slots, 12 bytes each, keys -1 = empty. Each
// product probes with one atomicCAS; on an empty slot or the same key the
// value is added with a shared-memory float64 atomicAdd (Algorithm 5). Then
// the three phases of Sec. 5.6.2 follow: condense the occupied slots to the
// front of the table (ballot/popc prefix per chunk of TPR slots, in place),
// sort them by column (bitonic network in shared memory over the next power
// of two), and store them with coalesced writes. The row size is known from
// the symbolic phase and checked.
//
// Rows past the largest table go to num_bitmap_kernel (one 1024-thread block
// per row). Pass 1 marks the row's columns in a shared-memory bitmap (set
// with 32-bit atomicOr, read as 64-bit words) and forms per-word prefix counts, which give every column its rank
// in the sorted row: C.col is written straight from the bitmap in column
// order, no sort needed. Pass 2 adds each product into C.val[rank] with a
// float64 atomicAdd in global memory (L2). 227 KB cover 1.2M columns per
// pass; wider matrices take several column windows. This replaces the
// paper's global-memory hash kernel (its kernel 7) and its condense/sort.
#include <climits>

#include "common.cuh"
#include "internal.h"

namespace ops {

// Returns false when every slot holds another key (the table is full).
// MULTI: the access pattern the paper measures against (Sec. 6, the hashing
// comparison), a plain read of the slot first and the compare-and-swap only
// on an empty one; otherwise one access per probe (Algorithm 5).
template <int T, bool MULTI = false>
__device__ __forceinline__ bool num_insert(int *tk, double *tv, int key, double a, double b) {
    uint32_t h = hash_slot<T>(key);
    for (int it = 0; it < T; ++it) {
        if (MULTI) {
            const int cur = *static_cast<volatile int *>(tk + h);
            bool hit = cur == key;
            if (!hit && cur == -1) {
                const int old = atomicCAS(tk + h, -1, key);
                hit = old == -1 || old == key;
            }
            if (hit) {
                smem_fma_add(tv + h, a, b);
                return true;
            }
        } else {
            const int old = atomicCAS(tk + h, -1, key);
            if (old == -1 || old == key) {
                smem_fma_add(tv + h, a, b);
                return true;
            }
        }
        h = next_slot<T>(h);
    }
    return false;
}

// The same probe with the value updated by a plain read, fused
// multiply-add and write: for row groups whose steps touch distinct entries
// only (group_row_walk with SYNC), where no other thread can update the
// entry in between. The key still takes a compare-and-swap: distinct keys of
// one step may probe the same slot.
template <int T>
__device__ __forceinline__ bool num_insert_owned(int *tk, double *tv, int key, double a, double b) {
    uint32_t h = hash_slot<T>(key);
    for (int it = 0; it < T; ++it) {
        const int old = atomicCAS(tk + h, -1, key);
        if (old == -1 || old == key) {
            tv[h] = fma(a, b, tv[h]);
            return true;
        }
        h = next_slot<T>(h);
    }
    return false;
}

// Mean referenced B-row length decides how many threads walk one B row; the
// symbolic phase's n_prod is gone by now (C.rpt holds offsets), so the row
// group recomputes it from B.rpt (those lines are needed right after).
template <int TPR>
__device__ __forceinline__ int numeric_lanes(const Operands &op, int fixed, int64_t p0,
                                             int64_t p1, int lg, long long *red) {
    if (fixed > 0) return pick_lanes_distinct(fixed, 0, 1, TPR);
    long long sum = 0;
    for (int64_t p = p0 + lg; p < p1; p += TPR) {
        const int k = __ldg(op.acol + p);
        sum += ld_rpt(op.brpt, op.b64, k + 1) - ld_rpt(op.brpt, op.b64, k);
    }
    sum = group_sum<TPR>(sum, red);
    return pick_lanes_distinct(0, sum, p1 - p0, TPR);
}

// Ascending bitonic sort of the NR * 32 values one warp holds in registers,
// element e = r * 32 + lane in x[r] (striped, so the sorted result stores
// coalesced). Every loop has a compile-time trip count and unrolls fully, so
// register indices are constants: strides below 32 exchange through
// shuffles, larger ones between a lane's own registers.
template <int NR>
__device__ __forceinline__ void warp_bitonic(unsigned (&x)[NR]) {
    constexpr int P = NR * 32;
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 2; k <= P; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= 32) {
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    const int r2 = r ^ (j >> 5);
                    if (r2 > r) {
                        const bool up = ((r * 32 + lane) & k) == 0;
                        const unsigned a = x[r], b = x[r2];
                        const unsigned mn = a < b ? a : b, mx = a < b ? b : a;
                        x[r] = up ? mn : mx;
                        x[r2] = up ? mx : mn;
                    }
                }
            } else {
                const bool lower = (lane & j) == 0;
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    const unsigned o = __shfl_xor_sync(0xffffffffu, x[r], j);
                    const bool up = ((r * 32 + lane) & k) == 0;
                    const unsigned mn = x[r] < o ? x[r] : o, mx = x[r] < o ? o : x[r];
                    x[r] = lower == up ? mn : mx;
                }
            }
        }
    }
}

// One warp: sort the n condensed entries (tk[e], tv[e]), e < n <= NR * 32,
// by column and store the first m to ocol/oval. Keys are (column << 8 | e):
// columns below 2^24, n <= 256.
template <int NR>
__device__ __forceinline__ void warp_sort_store(const int *tk, const double *tv, int n, int64_t m,
                                                int32_t *ocol, double *oval, bool store) {
    const int lane = threadIdx.x & 31;
    unsigned x[NR];
#pragma unroll
    for (int q = 0; q < NR; ++q) {
        const int e = q * 32 + lane;
        x[q] = e < n ? (static_cast<unsigned>(tk[e]) << 8) | static_cast<unsigned>(e) : 0xffffffffu;
    }
    warp_bitonic<NR>(x);
    if (!store) return;
#pragma unroll
    for (int q = 0; q < NR; ++q) {
        const int e = q * 32 + lane;
        if (e < m) {
            ocol[e] = static_cast<int32_t>(x[q] >> 8);
            oval[e] = tv[x[q] & 255u];
        }
    }
}

// Minimum resident blocks: enough for 2048 threads per SM (<= 32 registers
// per thread, Sec. 5.6) for sub-warp row groups, unless the table is so
// large that one block fills the SM's shared memory anyway. Kernels whose
// walks and sorts spill at 32 registers get fewer threads and more
// registers: warp-per-row kernels that sort in registers 1280 threads (48
// registers; 27-point stencil 128^3: 10.64 -> 9.72 ms against 1536 threads),
// block-per-row kernels 1536 (40 registers; block-diagonal n = 2^20:
// 12.43 -> 10.44 ms against 2048).
// ONE_PHASE (learned sizing): the row's size is not known; the table was
// chosen from a prediction. A probe that finds no free slot, or more keys
// than the table can sort in place, marks the row as mispredicted: it is
// queued for the exact path and nothing is written. Otherwise the row's
// size goes to C.rpt and its sorted entries to its temporary slot.
template <int TPR, int BLOCK, int T, bool ONE_PHASE = false, bool MULTI = false>
__global__ void __launch_bounds__(BLOCK, (T * 12 * (BLOCK / TPR) > 110 * 1024) ? 1
                                         : ((TPR == 32 && T <= 256) ? 1280 : (TPR > 32 ? 1536 : 2048)) / BLOCK)
num_hash_kernel(Operands op, BinWork w) {
    constexpr int RPB = BLOCK / TPR;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *vals_all = reinterpret_cast<double *>(smem_raw);
    int *keys_all = reinterpret_cast<int *>(vals_all + RPB * T);
    __shared__ long long red64[32];
    __shared__ int red32[33];
    __shared__ int full[RPB];   // one-phase: a probe found no free slot in this row's table
    const int g = threadIdx.x / TPR, lg = threadIdx.x % TPR;
    int *tk = keys_all + g * T;
    double *tv = vals_all + g * T;
    bool failed = false;
    if (lg == 0) full[g] = 0;
    const int64_t r = static_cast<int64_t>(blockIdx.x) * RPB + g;
    const bool valid = r < w.cnt;
    const int64_t row = valid ? (w.bins ? static_cast<int64_t>(w.bins[w.off + r]) : w.off + r) : 0;
    for (int s = lg; s < T; s += TPR) {
        tk[s] = -1;
        tv[s] = 0.0;
    }
    int64_t cbase = 0, n_expect = 0, p0 = 0, p1 = 0;
    if (valid) {
        if (!ONE_PHASE) {
            cbase = w.crpt[row];
            n_expect = w.crpt[row + 1] - cbase;
        }
        const int64_t ar = op.row0 + row;
        p0 = ld_rpt(op.arpt, op.a64, ar);
        p1 = ld_rpt(op.arpt, op.a64, ar + 1);
    }
    const int S = numeric_lanes<TPR>(op, w.lanes, p0, p1, lg, red64);
    group_sync<TPR>();
    if constexpr (TPR > 32) {
        // one row per block: flattened walk over B-row pieces
        WalkScratch *sc = reinterpret_cast<WalkScratch *>(
            smem_raw + (sizeof(int) + sizeof(double)) * (size_t)RPB * T);
        block_row_walk<BLOCK, true>(op, p0, p1, S, sc, [&](int key, double a, double b) {
            if (!num_insert<T, MULTI>(tk, tv, key, a, b)) failed = true;
        });
    } else if (!MULTI && w.distinct && S == TPR) {
        // one B row per step, its columns distinct: values without atomics,
        // B's entries staged in shared memory by cp.async (after the tables:
        // kStage * TPR values, then as many columns, per row group)
        double *sv = reinterpret_cast<double *>(smem_raw + (sizeof(int) + sizeof(double)) * (size_t)RPB * T) +
                     static_cast<size_t>(g) * kStage * TPR;
        int *sc = reinterpret_cast<int *>(reinterpret_cast<double *>(smem_raw +
                                                                      (sizeof(int) + sizeof(double)) * (size_t)RPB * T) +
                                          static_cast<size_t>(RPB) * kStage * TPR) +
                  static_cast<size_t>(g) * kStage * TPR;
        group_row_walk_staged<TPR>(op, p0, p1, sc, sv, [&](int key, double a, double b) {
            if (!num_insert_owned<T>(tk, tv, key, a, b)) failed = true;
        });
    } else {
        group_row_walk<TPR, true>(op, p0, p1, S, [&](int key, double a, double b) {
            if (!num_insert<T, MULTI>(tk, tv, key, a, b)) failed = true;
        });
    }
    if (failed) {
        if (ONE_PHASE) full[g] = 1;
        else set_error(w.err, DERR_TABLE_FULL);
    }
    group_sync<TPR>();
    // condense: occupied slots move to the front, chunk by chunk; a write
    // never lands past the chunk that was just read.
    int n = 0;
    int kmin = INT_MAX, kmax = -1;   // this thread's smallest and largest key
    for (int c = 0; c < T; c += TPR) {
        const int s = c + lg;
        int k = -1;
        double v = 0.0;
        if (s < T) {
            k = tk[s];
            v = tv[s];
        }
        if (k >= 0) {
            kmin = min(kmin, k);
            kmax = max(kmax, k);
        }
        int pre, tot;
        group_excl_count<TPR>(k >= 0, pre, tot, red32);
        group_sync<TPR>();
        if (k >= 0) {
            tk[n + pre] = k;
            tv[n + pre] = v;
        }
        n += tot;
        group_sync<TPR>();
    }
    int P = 1;
    while (P < n) P <<= 1;
    if constexpr (ONE_PHASE) {
        // mispredicted: queue the row for the exact path, write nothing else
        if (full[g] || P > T) {
            if (valid && lg == 0) {   // C.rpt keeps n_prod for the exact symbolic kernel
                w.pred[row] = -1;
                if (w.fb)
                    atomicAdd(w.fb + (3 * kMaxBins + w.lcls[row]) * kLoadSlots + blockIdx.x % kLoadSlots, 1ull);
                const unsigned long long at = atomicAdd(w.xcount, 1ull);
                if (at < static_cast<unsigned long long>(w.xlimit)) w.xlist[at] = static_cast<int32_t>(row);
                else set_error(w.err, DERR_BOUNDS);
            }
            return;   // uniform over the row group
        }
        n_expect = n;
        if (valid && lg == 0) {
            w.crpt[row] = n;
            // load feedback: more than 3/4 full, or at most 3/4 of the next smaller table
            const int grp = 4 * n > 3 * T ? 1 : (w.tprev > 0 && 4ll * n <= 3 * w.tprev ? 2 : 0);
            if (w.fb && grp)
                atomicAdd(w.fb + (grp * kMaxBins + w.lcls[row]) * kLoadSlots + blockIdx.x % kLoadSlots, 1ull);
        }
    } else {
        if (valid && n != n_expect) set_error(w.err, DERR_COUNT_MISMATCH);
        if (P > T) {  // cannot happen within the kernel's capacity; never index past the table
            set_error(w.err, DERR_TABLE_FULL);
            P = 1;
        }
    }
    if constexpr (TPR == 32 && T <= 256) {
        if (op.ncols <= (int64_t{1} << 24)) {   // uniform
            // one warp per row: sort (column << 8 | slot) in registers, then
            // store columns and the values of their slots in order
            const int64_t m = n < n_expect ? n : n_expect;
            int32_t *ocol = w.ccol + cbase;
            double *oval = w.cval + cbase;
            bool in_bounds = true;
            if (ONE_PHASE) {
                ocol = w.tcol + w.tbase + r * w.tcap;
                oval = w.tval + w.tbase + r * w.tcap;
                in_bounds = m <= w.tcap && w.tbase + r * w.tcap + m <= w.tlimit;
                if (valid && !in_bounds && lg == 0) set_error(w.err, DERR_BOUNDS);
            }
            const bool store = valid && in_bounds;
            if (n <= 32) warp_sort_store<1>(tk, tv, n, m, ocol, oval, store);
            else if (n <= 64) warp_sort_store<2>(tk, tv, n, m, ocol, oval, store);
            else if (n <= 128 || T <= 128) warp_sort_store<(T < 128 ? T / 32 : 4)>(tk, tv, n, m, ocol, oval, store);
            else warp_sort_store<T / 32>(tk, tv, n, m, ocol, oval, store);
            return;   // uniform over the warp; no block barrier follows
        }
    }
    if constexpr (TPR > 32) {
        // One row per block. When the row's columns span few enough words,
        // each entry goes straight to its place in the sorted row: bit
        // (column - min) of a span bitmap is set for every entry, and the
        // set bits below it give its rank. The bitmap (nw words) and its
        // per-word prefix counts (nw words) take the top 2 nw words of the
        // key table, above the n condensed keys.
        if (n > 0) {   // uniform: n is the block's count
            kmin = block_min<TPR>(kmin, red32);
            kmax = -block_min<TPR>(-kmax, red32);
            const long long span = static_cast<long long>(kmax) - kmin + 1;
            const long long nwl = (span + 31) >> 5;
            if (n + 2 * nwl <= T) {   // uniform
                const int nw = static_cast<int>(nwl);
                unsigned *bits = reinterpret_cast<unsigned *>(tk + T - 2 * nw);
                unsigned *pre = bits + nw;
                for (int i = lg; i < nw; i += TPR) bits[i] = 0u;
                __syncthreads();
                for (int s = lg; s < n; s += TPR) {
                    const unsigned rel = static_cast<unsigned>(tk[s] - kmin);
                    atomicOr(bits + (rel >> 5), 1u << (rel & 31));
                }
                __syncthreads();
                // rank of each word's first column: thread lg owns words
                // [lg * per, (lg + 1) * per)
                const int per = (nw + TPR - 1) / TPR;
                const int w0 = lg * per, w1 = min(w0 + per, nw);
                unsigned mine = 0;
                for (int i = w0; i < w1; ++i) mine += __popc(bits[i]);
                unsigned total;
                unsigned run = block_excl_scan<TPR>(mine, total, reinterpret_cast<unsigned *>(red32));
                for (int i = w0; i < w1; ++i) {
                    pre[i] = run;
                    run += __popc(bits[i]);
                }
                __syncthreads();
                if (valid) {
                    const int64_t m = n < n_expect ? n : n_expect;
                    int32_t *ocol = w.ccol + cbase;
                    double *oval = w.cval + cbase;
                    bool in_bounds = true;
                    if (ONE_PHASE) {
                        ocol = w.tcol + w.tbase + r * w.tcap;
                        oval = w.tval + w.tbase + r * w.tcap;
                        in_bounds = m <= w.tcap && w.tbase + r * w.tcap + m <= w.tlimit;
                        if (!in_bounds && lg == 0) set_error(w.err, DERR_BOUNDS);
                    }
                    for (int s = lg; in_bounds && s < n; s += TPR) {
                        const int key = tk[s];
                        const unsigned rel = static_cast<unsigned>(key - kmin);
                        const unsigned wd = rel >> 5;
                        const int64_t rank = pre[wd] + __popc(bits[wd] & ((1u << (rel & 31)) - 1u));
                        if (rank < m) {
                            ocol[rank] = key;
                            oval[rank] = tv[s];
                        }
                    }
                }
                return;   // uniform over the block
            }
        }
    }
    for (int s = n + lg; s < P; s += TPR) tk[s] = INT_MAX;
    group_sync<TPR>();
    // bitonic sort of (key, value) pairs over P entries, ascending
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = lg; i < P; i += TPR) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const int ka = tk[i], kb = tk[ixj];
                    const bool up = (i & k) == 0;
                    if ((ka > kb) == up) {
                        tk[i] = kb;
                        tk[ixj] = ka;
                        const double va = tv[i];
                        tv[i] = tv[ixj];
                        tv[ixj] = va;
                    }
                }
            }
            group_sync<TPR>();
        }
    }
    if (valid) {
        const int64_t m = n < n_expect ? n : n_expect;
        int32_t *ocol = w.ccol + cbase;
        double *oval = w.cval + cbase;
        bool in_bounds = true;
        if (ONE_PHASE) {
            ocol = w.tcol + w.tbase + r * w.tcap;
            oval = w.tval + w.tbase + r * w.tcap;
            in_bounds = m <= w.tcap && w.tbase + r * w.tcap + m <= w.tlimit;
            if (!in_bounds && lg == 0) set_error(w.err, DERR_BOUNDS);
        }
        for (int64_t t = lg; in_bounds && t < m; t += TPR) {
            ocol[t] = tk[t];
            oval[t] = tv[t];
        }
    }
}

// Rank of every bitmap word's first column: pre[i] = set bits in words
// [0, i). Warp w owns words [w * per, (w + 1) * per) (per a multiple of 32)
// and its lanes read consecutive words, so no two lanes of a warp hit one
// bank. Returns the total. Synchronises the block; pre is complete on return.
template <int BLOCK>
__device__ __forceinline__ unsigned bitmap_ranks(const unsigned long long *bm, unsigned *pre, int nw,
                                                 unsigned *sw) {
    constexpr int kWarps = BLOCK / 32;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int per = (((nw + kWarps - 1) / kWarps) + 31) & ~31;
    const int w0 = wp * per;
    const int w1 = w0 + per < nw ? w0 + per : nw;
    unsigned cnt = 0;
    for (int i = w0 + lane; i < w1; i += 32) cnt += static_cast<unsigned>(__popcll(bm[i]));
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    __syncthreads();   // earlier readers of sw are done
    if (lane == 0) sw[wp] = cnt;
    __syncthreads();
    if (wp == 0) {
        const unsigned t = lane < kWarps ? sw[lane] : 0u;
        unsigned inc = t;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane < kWarps) sw[lane] = inc - t;
        if (lane == 31) sw[32] = inc;
    }
    __syncthreads();
    unsigned base = sw[wp];
    const unsigned total = sw[32];
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
    return total;
}

// Pass 2 by column windows (B rows sorted, run boundaries from bsplit): the
// row's products whose columns fall in sub-ranges [g, g2) of the column
// space are, per A entry, one run of its B row; the runs of a window are
// concatenated into one flat index space that the block's warps split into
// equal contiguous ranges. Windows hold about w.wentries entries of C, so
// the C.val lines that the float64 reductions of a window hit stay in L2.
struct RunMeta {
    long long q0[kWinMaxLists];      // first B entry of each A entry's B row
    double aval[kWinMaxLists];       // A values of the row
    int32_t ks[kWinMaxLists];        // B row of each A entry
    int32_t rs[kWinMaxLists];        // run start (offset in the B row) of the current window
    long long lp[kWinMaxLists + 1];  // exclusive prefix of the run lengths
    long long red[33];               // block scan scratch
    int g2;                          // end sub-range of the current window
};


size_t num_bitmap_head_bytes(bool runs) {
    const size_t a = sizeof(WalkScratch), b = sizeof(RunMeta);
    const size_t h = runs && b > a ? b : a;
    return (h + 15) & ~static_cast<size_t>(15);
}

// Calls f(col, a_value, b_value) for every product of the current window's
// runs (rm->lp holds their exclusive prefix, `total` the sum). A lane loads
// UNROLL products before using any.
template <int BLOCK, int UNROLL, typename F>
__device__ __forceinline__ void run_walk(const Operands &op, const RunMeta *rm, int nl, long long total,
                                         F &&f) {
    constexpr int kWarps = BLOCK / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long per = (total + kWarps - 1) / kWarps;
    const long long f0 = per * warp;
    const long long f1 = f0 + per < total ? f0 + per : total;
    if (f0 >= f1) return;
    int t = 0;
    {   // run of the lane's first index: last t with lp[t] <= f0 + lane
        const long long first = f0 + lane;
        int lo = 0, hi = nl;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (rm->lp[mid] <= first) lo = mid; else hi = mid;
        }
        t = lo;
    }
    for (long long base = f0; base < f1; base += 32 * UNROLL) {
        int c[UNROLL], tt[UNROLL];
        double b[UNROLL];
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
            const long long idx = base + u * 32 + lane;
            c[u] = -1;
            tt[u] = t;
            b[u] = 0.0;
            if (idx < f1) {
                while (rm->lp[t + 1] <= idx) ++t;   // runs are visited in order
                tt[u] = t;
                const long long q = rm->q0[t] + rm->rs[t] + (idx - rm->lp[t]);
                c[u] = __ldg(op.bcol + q);
                b[u] = __ldg(op.bval + q);
            }
        }
#pragma unroll
        for (int u = 0; u < UNROLL; ++u)
            if (c[u] >= 0) f(c[u], rm->aval[tt[u]], b[u]);
    }
}

// RUNS: the row is covered in several column windows and B's rows are
// sorted; each window's passes walk only the runs of B rows inside it
// (w.bslot / w.bidx), so a window costs its own products, not the row's.
template <int BLOCK, int ITERS, bool RUNS = false>
__global__ void __launch_bounds__(BLOCK, BLOCK == 1024 ? 1 : (RUNS ? 1024 : 1536) / BLOCK)
num_bitmap_kernel(Operands op, BinWork w, int words) {
    constexpr int kBmBlock = BLOCK;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // the head holds the walk scratch of pass 1, then the run metadata of a
    // windowed pass 2
    WalkScratch *sc = reinterpret_cast<WalkScratch *>(smem_raw);
    RunMeta *rm = reinterpret_cast<RunMeta *>(smem_raw);
    unsigned long long *bm = reinterpret_cast<unsigned long long *>(smem_raw + w.head);
    unsigned *bm32 = reinterpret_cast<unsigned *>(bm);   // same words, 32-bit halves
    unsigned *pre = reinterpret_cast<unsigned *>(bm + words);
    __shared__ unsigned sw[33];
    // phase clocks (profiling, w.clk set; 1024-thread blocks, whose
    // registers have room): a block barrier ends each phase, then thread 0
    // adds the SM clock cycles since the previous mark
    constexpr bool kClk = BLOCK == 1024;
    long long tmark = 0;
    if (kClk && w.clk && threadIdx.x == 0) tmark = clock64();
    auto phase_end = [&](int k) {
        if (!kClk || !w.clk) return;   // uniform: a kernel argument
        __syncthreads();
        if (threadIdx.x == 0) {
            const long long t = clock64();
            atomicAdd(w.clk + k, static_cast<unsigned long long>(t - tmark));
            tmark = t;
        }
    };
    // Block b takes the bin's row (b * P) mod cnt, P a prime that does not
    // divide cnt (a permutation): the binning leaves the bin's rows in row
    // order, and on power-law inputs the heaviest rows come first, so blocks
    // in launch order would sum dozens of multi-MB C.val segments at once and
    // push them out of L2 before their rows are done. Spread over the launch,
    // the rows summed together are a sample of the whole bin (R-MAT n = 2^20:
    // 192 -> 178 ms; groups of 256 consecutive rows spread the same way:
    // 183 ms).
    const long long kSpread = (w.cnt % 1000003ll == 0) ? 999983ll : 1000003ll;
    const int64_t pos = static_cast<int64_t>((static_cast<long long>(blockIdx.x) * kSpread) % w.cnt);
    const int64_t row = w.bins ? static_cast<int64_t>(w.bins[w.off + pos]) : w.off + pos;
    const int64_t cbase = w.crpt[row];
    const int64_t n_expect = w.crpt[row + 1] - cbase;
    const int64_t ar = op.row0 + row;
    const int64_t p0 = ld_rpt(op.arpt, op.a64, ar);
    const int64_t p1 = ld_rpt(op.arpt, op.a64, ar + 1);
    // threads per B row from the row's size instead of its n_prod (C.rpt
    // holds offsets by now): n_nz <= n_prod, so the choice is at most one
    // step narrower, and the A row is first read by pass 1 itself
    const int S = pick_lanes_distinct(w.lanes, n_expect, p1 - p0, 32);
    const int64_t span = static_cast<int64_t>(words) * 64;
    int64_t done = 0;
    bool ok = true;
    for (int64_t c0 = 0; c0 < op.ncols; c0 += span) {
        const int nw = static_cast<int>(((op.ncols - c0 < span ? op.ncols - c0 : span) + 63) / 64);
        for (int i = threadIdx.x; i < nw; i += kBmBlock) bm[i] = 0ull;
        __syncthreads();
        phase_end(0);
        // pass 1: the row's columns inside this window. 32-bit atomics on the
        // two halves of a 64-bit word: shared 64-bit atomics run several
        // times slower on this GPU
        const int c0i = static_cast<int>(c0);
        const unsigned span32 = static_cast<unsigned>(span);
        RunSel rsel{w.bslot, w.bidx, w.cs, w.ncells, c0i,
                    static_cast<int>(c0 + span < op.ncols ? c0 + span : op.ncols)};
        block_row_walk<kBmBlock, false, ITERS, 1, RUNS>(op, p0, p1, S, sc, [&](int key, double, double) {
            const unsigned rel = static_cast<unsigned>(key - c0i);   // one compare covers both ends
            if (rel < span32) atomicOr(bm32 + (rel >> 5), 1u << (rel & 31));
        }, &rsel);
        phase_end(1);
        // per-word prefix counts = rank of a word's first column in the
        // window. Warps own contiguous ranges of words and their lanes read
        // consecutive words (no bank conflicts): a warp scan per 32 words,
        // one block scan of the warp totals.
        const unsigned run = bitmap_ranks<kBmBlock>(bm, pre, nw, sw);
        phase_end(2);
        const int64_t cnt = run;
        if (done + cnt > n_expect) ok = false;   // uniform: cnt and done are block-wide
        if (ok) {
            int32_t *ccol = w.ccol + cbase + done;
            double *cval = w.cval + cbase + done;
            // Each warp takes a contiguous range of words of about equal
            // cost, a word costing its column count plus kWordCost for its
            // scan: the cost of the words before word i is pre[i] +
            // kWordCost * i, increasing in i, so a binary search over pre
            // finds a warp's range. (Equal word counts per warp put most
            // columns of a skewed row on a few warps: on R-MAT rows, whose
            // low columns are dense, one warp of 32 held about a quarter of
            // the row; cost ranges: 204 -> 194 ms on R-MAT n = 2^20.)
            // Lanes take consecutive words. A lane writes its own word's
            // columns (32-bit halves in turn: 32-bit bit scans are cheaper
            // than 64-bit ones) when the word holds fewer than kDenseWord of
            // them; denser words are written by the whole warp, one word at a
            // time with one lane per bit, so that each store covers one run
            // of consecutive entries of C.col (measured: 1.5% faster than
            // every lane writing its own word, on R-MAT n = 2^20). The
            // write is bound by instruction issue: a lane loop runs as often
            // as the fullest word of the 32 asks, so words of 12 columns or
            // more go to the whole warp (R-MAT n = 2^20 rows: 8.0 instead of
            // 9.2 loop trips per 32 words; this phase 3.6% faster than with
            // 24). Entry-parallel rounds (lane e finds the word of entry e by
            // a shuffle search) store fully coalesced but issue more: 27%
            // slower.
            constexpr int kDenseWord = 12;
            constexpr unsigned long long kWordCost = 2;
            const int lane = threadIdx.x & 31;
            const unsigned lt = (1u << lane) - 1u;
            const unsigned long long vtot =
                static_cast<unsigned long long>(cnt) + kWordCost * static_cast<unsigned long long>(nw);
            auto first_word = [&](unsigned long long cost) {   // first i in [0, nw] whose prefix cost >= cost
                int lo = 0, hi = nw;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (pre[mid] + kWordCost * static_cast<unsigned long long>(mid) >= cost) hi = mid;
                    else lo = mid + 1;
                }
                return lo;
            };
            const unsigned long long wq = static_cast<unsigned long long>(threadIdx.x >> 5);
            const int i_beg = first_word(vtot * wq / (kBmBlock / 32));
            const int i_end = first_word(vtot * (wq + 1) / (kBmBlock / 32));
            for (int ib = i_beg; ib < i_end; ib += 32) {   // uniform over the warp
                const int i = ib + lane;
                const unsigned long long x = i < i_end ? bm[i] : 0ull;
                const unsigned pos0 = i < i_end ? pre[i] : 0u;
                const bool dense = __popcll(x) >= kDenseWord;
                unsigned dm = __ballot_sync(0xffffffffu, dense);
                if (!dense) {
                    unsigned pos = pos0;
                    const int colbase = c0i + i * 64;
                    unsigned lo = static_cast<unsigned>(x), hi = static_cast<unsigned>(x >> 32);
                    while (lo) {
                        const int b = __ffs(lo) - 1;
                        lo &= lo - 1;
                        ccol[pos++] = colbase + b;
                    }
                    while (hi) {
                        const int b = __ffs(hi) - 1;
                        hi &= hi - 1;
                        ccol[pos++] = colbase + 32 + b;
                    }
                }
                while (dm) {
                    const int src = __ffs(dm) - 1;
                    dm &= dm - 1;
                    const unsigned long long xw = __shfl_sync(0xffffffffu, x, src);
                    const unsigned pw = __shfl_sync(0xffffffffu, pos0, src);
                    const int cb = c0i + (ib + src) * 64;
                    const unsigned lo = static_cast<unsigned>(xw), hi = static_cast<unsigned>(xw >> 32);
                    if ((lo >> lane) & 1u) ccol[pw + __popc(lo & lt)] = cb + lane;
                    if ((hi >> lane) & 1u) ccol[pw + __popc(lo) + __popc(hi & lt)] = cb + 32 + lane;
                }
            }
            phase_end(3);
            const unsigned long long pol = l2_evict_last_policy();
            const int nl = static_cast<int>(p1 - p0 < INT32_MAX ? p1 - p0 : INT32_MAX);
            // one thread per A entry: the row's A entries must fit the block
            if (w.bs && c0 == 0 && span >= op.ncols && nl <= w.wlists && nl <= kBmBlock) {
                // pass 2 by column windows of about w.wentries entries
                bool bad = false;
                if (threadIdx.x < nl) {
                    const int k = __ldg(op.acol + p0 + threadIdx.x);
                    rm->ks[threadIdx.x] = k;
                    rm->q0[threadIdx.x] = ld_rpt(op.brpt, op.b64, k);
                    rm->aval[threadIdx.x] = __ldg(op.aval + p0 + threadIdx.x);
                    rm->rs[threadIdx.x] = 0;
                }
                // rank of the first column of sub-range g (sub-ranges start on word boundaries)
                auto bnd_rank = [&](int g) -> unsigned {
                    const int64_t cb = static_cast<int64_t>(g) << w.gshift;
                    return cb >= op.ncols ? static_cast<unsigned>(cnt) : pre[cb >> 6];
                };
                for (int g = 0; g < w.G;) {
                    if (threadIdx.x == 0) {
                        const unsigned r0 = bnd_rank(g);
                        int g2 = g + 1;
                        while (g2 < w.G && bnd_rank(g2 + 1) - r0 <= static_cast<unsigned>(w.wentries)) ++g2;
                        rm->g2 = g2;
                    }
                    __syncthreads();
                    const int g2 = rm->g2;
                    const unsigned r_lo = bnd_rank(g), r_hi = bnd_rank(g2);
                    long long len = 0;
                    int re = 0;
                    if (threadIdx.x < nl) {
                        re = __ldg(w.bs + static_cast<int64_t>(rm->ks[threadIdx.x]) * (w.G + 1) + g2);
                        len = re - rm->rs[threadIdx.x];
                    }
                    for (unsigned t = r_lo + threadIdx.x; t < r_hi; t += kBmBlock) st_keep(cval + t, 0.0, pol);
                    long long total;
                    const long long ex = block_excl_scan_ll<kBmBlock>(len, total, rm->red);
                    if (threadIdx.x < nl) rm->lp[threadIdx.x] = ex;
                    if (threadIdx.x == 0) rm->lp[nl] = total;
                    __syncthreads();
                    if (total > 0)
                        run_walk<kBmBlock, kBmBlock == 1024 ? 8 : 4>(op, rm, nl, total,
                                                                      [&](int key, double a, double b) {
                            const unsigned rel = static_cast<unsigned>(key - c0i);
                            const unsigned wi = rel >> 6, bi = rel & 63u;
                            const unsigned rank = rel < span32 ? pre[wi] +
                                static_cast<unsigned>(__popcll(bm[wi] << (63u - bi))) - 1u : 0u;
                            if (rel < span32 && rank >= r_lo && rank < r_hi) red_add_keep(cval + rank, a * b, pol);
                            else bad = true;
                        });
                    __syncthreads();
                    const uintptr_t l0 = reinterpret_cast<uintptr_t>(cval + r_lo) & ~static_cast<uintptr_t>(127);
                    const uintptr_t l1 = reinterpret_cast<uintptr_t>(cval + r_hi);
                    for (uintptr_t l = l0 + 128 * static_cast<uintptr_t>(threadIdx.x); l < l1;
                         l += 128 * static_cast<uintptr_t>(kBmBlock))
                        l2_priority_normal(reinterpret_cast<const void *>(l));
                    if (threadIdx.x < nl) rm->rs[threadIdx.x] = re;
                    g = g2;
                    __syncthreads();
                }
                if (bad) set_error(w.err, DERR_WINDOW);
                done += cnt;
                __syncthreads();
                continue;
            }
            for (int64_t t = threadIdx.x; t < cnt; t += kBmBlock) st_keep(cval + t, 0.0, pol);
            __syncthreads();
            phase_end(4);
            // pass 2: each product lands on its column's rank (the walk
            // scratch of pass 1 is still in place)
            block_row_walk<kBmBlock, true, ITERS, 2, RUNS>(op, p0, p1, S, sc, [&](int key, double a, double b) {
                const unsigned rel = static_cast<unsigned>(key - c0i);
                if (rel < span32) {
                    const unsigned wi = rel >> 6, bi = rel & 63u;
                    // the column's own bit is set: bits 0..bi shifted to the
                    // top, counted, minus itself = columns before it in the word
                    const unsigned rank = pre[wi] +
                        static_cast<unsigned>(__popcll(bm[wi] << (63u - bi))) - 1u;
                    red_add_keep(cval + rank, a * b, pol);
                }
            }, &rsel);
            __syncthreads();
            phase_end(5);
            // back to normal priority: every 128-byte line the segment touches
            const uintptr_t l0 = reinterpret_cast<uintptr_t>(cval) & ~static_cast<uintptr_t>(127);
            const uintptr_t l1 = reinterpret_cast<uintptr_t>(cval + cnt);
            for (uintptr_t l = l0 + 128 * static_cast<uintptr_t>(threadIdx.x); l < l1;
                 l += 128 * static_cast<uintptr_t>(kBmBlock))
                l2_priority_normal(reinterpret_cast<const void *>(l));
            phase_end(6);
        }
        done += cnt;
        __syncthreads();
    }
    if (threadIdx.x == 0 && (!ok || done != n_expect)) set_error(w.err, DERR_COUNT_MISMATCH);
}

// --- kernel table ---------------------------------------------------------------
using NumFn = void (*)(Operands, BinWork);

#define NUM_TABLE(X)                 \
    X(8, 256, 32)                    \
    X(16, 256, 128)                  \
    X(32, 256, 256)                  \
    X(64, 64, 512)                   \
    X(128, 128, 1024)                \
    X(256, 256, 2048)                \
    X(512, 512, 4096)                \
    X(1024, 1024, 8192)              \
    X(1024, 1024, 18432)

struct NumEntry {
    KernelDesc d;
    NumFn fn;
};

// Largest row the table can sort in place: the bitonic network needs the
// next power of two of the row size to fit in the table.
constexpr long long pow2_floor(long long t) {
    long long p = 1;
    while (p * 2 <= t) p *= 2;
    return p;
}

// Row groups of a warp or less also get kStage B-piece slots per lane for
// the staged walk (12 bytes each).
#define NUM_ENTRY(TPR, BLOCK, T)                                                         \
    {{TPR, BLOCK, T, pow2_floor(T), 0,                                                   \
      (sizeof(int) + sizeof(double)) * (BLOCK / TPR) * (size_t)T +                       \
          (TPR > 32 ? sizeof(WalkScratch) : (sizeof(int) + sizeof(double)) * kStage * (size_t)BLOCK)}, \
     &num_hash_kernel<TPR, BLOCK, T>},

static NumEntry g_num[] = {NUM_TABLE(NUM_ENTRY)};

#define NUM_ONEPHASE_ENTRY(TPR, BLOCK, T) &num_hash_kernel<TPR, BLOCK, T, true>,
static NumFn g_num_onephase[] = {NUM_TABLE(NUM_ONEPHASE_ENTRY)};
// the plain kernels with the read-then-swap probe (BinWork::multi)
#define NUM_MULTI_ENTRY(TPR, BLOCK, T) &num_hash_kernel<TPR, BLOCK, T, false, true>,
static NumFn g_num_multi[] = {NUM_TABLE(NUM_MULTI_ENTRY)};
static constexpr int kNumHash = sizeof(g_num) / sizeof(g_num[0]);
static KernelDesc g_num_bitmap{1024, 1024, 0, LLONG_MAX, 1, 0};

using BmFn = void (*)(Operands, BinWork, int);
// bitmap kernel variants: (threads per block, products in flight per lane)
static const struct { int block, iters; BmFn fn; } g_num_bm[] = {
    {1024, 4, &num_bitmap_kernel<1024, 4>}, {1024, 8, &num_bitmap_kernel<1024, 8>},
    {512, 4, &num_bitmap_kernel<512, 4>},   {256, 4, &num_bitmap_kernel<256, 4>},
};
// the same walked by column windows over sorted B (BinWork::bidx set): two
// 512-thread blocks per SM when a window's bitmap takes half the SM
static const struct { int block; BmFn fn; } g_num_bm_runs[] = {
    {1024, &num_bitmap_kernel<1024, 4, true>}, {512, &num_bitmap_kernel<512, 4, true>},
};

int num_kernel_count() { return kNumHash + 1; }

const KernelDesc &num_kernel(int id) {
    return id < kNumHash ? g_num[id].d : g_num_bitmap;
}

cudaError_t num_prepare(int smem_optin) {
    // Opt in for every kernel: the 48 KB default covers static plus dynamic
    // shared memory, so a table of exactly 48 KB already needs it.
    for (int i = 0; i < kNumHash; ++i) {
        cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void *>(g_num[i].fn),
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(g_num[i].d.smem));
        if (e != cudaSuccess) return e;
    }
    for (int i = 0; i < kNumHash; ++i) {
        cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void *>(g_num_onephase[i]),
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(g_num[i].d.smem));
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(reinterpret_cast<const void *>(g_num_multi[i]),
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(g_num[i].d.smem));
        if (e != cudaSuccess) return e;
    }
    g_num_bitmap.table = static_cast<long long>((smem_optin - sizeof(WalkScratch)) / 12) * 64;
    for (const auto &v : g_num_bm) {
        cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void *>(v.fn),
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin);
        if (e != cudaSuccess) return e;
    }
    for (const auto &v : g_num_bm_runs) {
        cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void *>(v.fn),
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Bitmap kernel launch shape: the block size that keeps about 2048 threads
// per SM given how many blocks fit in shared memory (one 1024-thread block
// when a block needs most of the SM's 228 KB, as for a million columns;
// 256-thread blocks when the bitmap is small), and `iters` products in
// flight per lane (4 or 8; 0 = 4).
static int pick_bitmap_variant(size_t smem_total, int iters) {
    const size_t per_sm = 228 * 1024;
    const int fit = static_cast<int>(per_sm / (smem_total + 1024));
    int block = 1024;
    if (fit >= 8) block = 256;
    else if (fit >= 4) block = 512;
    if (iters == 8) block = 1024;
    for (int i = 0; i < static_cast<int>(sizeof(g_num_bm) / sizeof(g_num_bm[0])); ++i)
        if (g_num_bm[i].block == block && g_num_bm[i].iters == (iters == 8 ? 8 : 4)) return i;
    return 0;
}

cudaError_t launch_num_onephase(int id, const Operands &op, const BinWork &w, cudaStream_t s) {
    if (w.cnt <= 0) return cudaSuccess;
    if (id < 0 || id >= kNumHash) return cudaErrorInvalidValue;
    const KernelDesc &d = g_num[id].d;
    const int rpb = d.block / d.tpr;
    const int64_t grid = (w.cnt + rpb - 1) / rpb;
    g_num_onephase[id]<<<static_cast<unsigned>(grid), d.block, d.smem, s>>>(op, w);
    return cudaGetLastError();
}

// Copies the one-phase rows of a bin from their temporary slots into C: one
// warp per row, rows marked -1 in pred (mispredicted) are skipped.
__global__ void copy_rows_kernel(BinWork w) {
    const int64_t r = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= w.cnt) return;
    const int64_t row = w.bins ? static_cast<int64_t>(w.bins[w.off + r]) : w.off + r;
    if (w.pred[row] < 0) return;
    const int64_t base = w.crpt[row];
    const int64_t n = w.crpt[row + 1] - base;
    const int32_t *scol = w.tcol + w.tbase + r * w.tcap;
    const double *sval = w.tval + w.tbase + r * w.tcap;
    if (n > w.tcap || w.tbase + r * w.tcap + n > w.tlimit) {
        if (lane == 0) set_error(w.err, DERR_BOUNDS);
        return;
    }
    // four loads in flight per lane before the stores (the temporary rows
    // are read-only here)
    for (int64_t t0 = 0; t0 < n; t0 += 128) {
        int32_t c[4];
        double v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t t = t0 + u * 32 + lane;
            if (t < n) {
                c[u] = __ldg(scol + t);
                v[u] = __ldg(sval + t);
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t t = t0 + u * 32 + lane;
            if (t < n) {
                w.ccol[base + t] = c[u];
                w.cval[base + t] = v[u];
            }
        }
    }
}

cudaError_t launch_copy_rows(const BinWork &w, cudaStream_t s) {
    if (w.cnt <= 0) return cudaSuccess;
    const int64_t threads = w.cnt * 32;
    copy_rows_kernel<<<static_cast<unsigned>((threads + 255) / 256), 256, 0, s>>>(w);
    return cudaGetLastError();
}

cudaError_t launch_num(int id, const Operands &op, const BinWork &w, size_t smem_bitmap,
                       cudaStream_t s) {
    if (w.cnt <= 0) return cudaSuccess;
    if (id < kNumHash) {
        const KernelDesc &d = g_num[id].d;
        const int rpb = d.block / d.tpr;
        const int64_t grid = (w.cnt + rpb - 1) / rpb;
        const NumFn fn = w.multi ? g_num_multi[id] : g_num[id].fn;
        fn<<<static_cast<unsigned>(grid), d.block, d.smem, s>>>(op, w);
    } else {
        const int words = static_cast<int>(smem_bitmap / 12);
        BinWork wk = w;
        wk.head = static_cast<int>(num_bitmap_head_bytes(w.bs != nullptr));
        if (!w.bs) wk.wlists = 0;
        const size_t smem = smem_bitmap + static_cast<size_t>(wk.head);
        if (w.bidx && !w.bs) {
            // two blocks per SM when two windows fit the SM's shared memory
            const int two = (228 * 1024) / static_cast<int>(smem + 1024) >= 2;
            const auto &v = g_num_bm_runs[two ? 1 : 0];
            v.fn<<<static_cast<unsigned>(w.cnt), v.block, smem, s>>>(op, wk, words);
            return cudaGetLastError();
        }
        const auto &v = g_num_bm[pick_bitmap_variant(smem, w.unroll)];
        v.fn<<<static_cast<unsigned>(w.cnt), v.block, smem, s>>>(op, wk, words);
    }
    return cudaGetLastError();
}

}  // namespace ops
