// Device helpers shared by the SpGEMM kernels (sm_103a).
#pragma once

#include <climits>
#include <cstdint>
#include <cuda_runtime.h>

#include "internal.h"

namespace ops {

// Device error codes written to the handle's error word (first one wins).
enum : int {
    DERR_NONE = 0,
    DERR_TABLE_FULL = 1,      // a hash probe visited every slot
    DERR_COUNT_MISMATCH = 2,  // numeric row size differs from the symbolic count
    DERR_WINDOW = 3,          // bitmap window bookkeeping failed
    DERR_BOUNDS = 4,          // a learned-sizing index left its buffer (access skipped)
};

__device__ __forceinline__ void set_error(int *err, int code) {
    if (err) atomicCAS(err, 0, code);
}

// Row pointer load for int32 or int64 CSR row pointers (runtime flag, uniform
// across the grid, so the branch costs nothing measurable).
__device__ __forceinline__ int64_t ld_rpt(const void *rpt, int is64, int64_t i) {
    return is64 ? __ldg(static_cast<const long long *>(rpt) + i)
                : static_cast<int64_t>(__ldg(static_cast<const int *>(rpt) + i));
}

// Hash slot of a column key in a table of T slots. The paper multiplies the
// key by a constant and reduces modulo the table size (Sec. 5.2); here the
// product with a Fibonacci constant is reduced by its HIGH bits (a shift for
// a power-of-two T, a multiply-high otherwise). Low bits of stencil columns
// repeat with the grid stride, so taking low bits would pile keys that
// differ by a multiple of the stride onto one slot.
constexpr uint32_t kHashMul = 0x9E3779B1u;

template <int T>
__device__ __forceinline__ uint32_t hash_slot(int key) {
    const uint32_t x = static_cast<uint32_t>(key) * kHashMul;
    if constexpr ((T & (T - 1)) == 0) {
        constexpr int lg = __builtin_ctz(T);
        return lg == 0 ? 0u : (x >> (32 - lg));
    } else {
        return static_cast<uint32_t>((static_cast<uint64_t>(x) * T) >> 32);
    }
}

template <int T>
__device__ __forceinline__ uint32_t next_slot(uint32_t h) {
    if constexpr ((T & (T - 1)) == 0) return (h + 1) & (T - 1);
    else return (h + 1 == static_cast<uint32_t>(T)) ? 0u : h + 1;
}

// Products one lane loads together before using them (a piece of a B row
// is at most kPieceIters * S long for S lanes).
constexpr int kPieceIters = 4;

// Threads that walk one B row together: the smallest power of two S for
// which S * kPieceIters covers the mean length of the referenced B rows (so
// every lane keeps kPieceIters loads in flight), no larger than the row
// group or a warp, unless the configuration fixes it.
__device__ __forceinline__ int pick_lanes(int fixed, int64_t nprod, int64_t nnza, int group) {
    int cap = group < 32 ? group : 32;
    if (fixed > 0) return fixed < cap ? fixed : cap;
    if (nnza <= 0) return 1;
    int64_t mean = (nprod + nnza - 1) / nnza;
    int s = 1;
    while (static_cast<int64_t>(s) * kPieceIters < mean && s < cap) s <<= 1;
    return s;
}

// Threads per B row for the numeric phase: the smallest power of two that
// covers the mean referenced B-row length (capped at the row group or a
// warp), so one round of a sub-group holds the columns of one B row, which
// are distinct. Taking several overlapping B rows at once (stencil rows)
// sends lanes to the same table slot in the same round, and float64
// atomics on one address serialise.
__device__ __forceinline__ int pick_lanes_distinct(int fixed, int64_t nprod, int64_t nnza, int group) {
    int cap = group < 32 ? group : 32;
    if (fixed > 0) return fixed < cap ? fixed : cap;
    if (nnza <= 0) return 1;
    int64_t mean = (nprod + nnza - 1) / nnza;
    int s = 1;
    while (s < mean && s < cap) s <<= 1;
    return s;
}

// --- row-group synchronisation and reductions --------------------------------
// A row group is TPR consecutive threads. TPR <= 32: a slice of one warp;
// TPR > 32: the whole block (one row per block).

template <int TPR>
__device__ __forceinline__ unsigned group_mask() {
    if constexpr (TPR >= 32) return 0xffffffffu;
    else {
        const unsigned lane = threadIdx.x & 31u;
        const unsigned base = lane & ~static_cast<unsigned>(TPR - 1);
        return ((1u << TPR) - 1u) << base;
    }
}

template <int TPR>
__device__ __forceinline__ void group_sync() {
    if constexpr (TPR > 32) __syncthreads();
    else __syncwarp(group_mask<TPR>());
}

template <typename V>
__device__ __forceinline__ V warp_sum_xor(V v, int width) {
    for (int o = width >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the row group; every thread of the group gets the result.
// `red` must hold 32 values of V when TPR > 32.
template <int TPR, typename V>
__device__ __forceinline__ V group_sum(V v, V *red) {
    if constexpr (TPR <= 32) {
        return warp_sum_xor(v, TPR);
    } else {
        v = warp_sum_xor(v, 32);
        const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
        __syncthreads();  // earlier readers of `red` are done
        if (l == 0) red[w] = v;
        __syncthreads();
        V t = (l < (TPR >> 5)) ? red[l] : V(0);
        return warp_sum_xor(t, 32);  // every warp forms the same total
    }
}

// Minimum over a block of BLOCK threads (BLOCK a multiple of 32); every
// thread gets it. `red` holds 32 ints.
template <int BLOCK>
__device__ __forceinline__ int block_min(int v, int *red) {
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();   // earlier readers of `red` are done
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    int t = (threadIdx.x & 31) < (BLOCK >> 5) ? red[threadIdx.x & 31] : INT_MAX;
    for (int o = 16; o > 0; o >>= 1) t = min(t, __shfl_xor_sync(0xffffffffu, t, o));
    return t;
}

// Exclusive count of `flag` over the row group in thread order, plus the
// group total. `red` must hold 33 ints when TPR > 32.
template <int TPR>
__device__ __forceinline__ void group_excl_count(bool flag, int &prefix, int &total, int *red) {
    const unsigned lane = threadIdx.x & 31u;
    const unsigned bal = __ballot_sync(0xffffffffu, flag);
    if constexpr (TPR <= 32) {
        const unsigned gm = group_mask<TPR>();
        const unsigned mine = bal & gm;
        prefix = __popc(mine & ((1u << lane) - 1u));
        total = __popc(mine);
    } else {
        const int w = threadIdx.x >> 5;
        const int in_warp = __popc(bal & ((1u << lane) - 1u));
        __syncthreads();
        if (lane == 0) red[w] = __popc(bal);
        __syncthreads();
        if (w == 0) {
            int x = (lane < (TPR >> 5)) ? red[lane] : 0;
            int inc = x;
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= static_cast<unsigned>(o)) inc += y;
            }
            if (lane < (TPR >> 5)) red[lane] = inc - x;
            if (lane == 31) red[32] = inc;
        }
        __syncthreads();
        prefix = red[w] + in_warp;
        total = red[32];
    }
}

__device__ __forceinline__ int64_t upper_bound_rpt(const void *rpt, int is64, int64_t lo,
                                                   int64_t hi, int64_t p) {
    // largest r in [lo, hi) with rpt[r] <= p (rpt[lo] <= p assumed)
    while (hi - lo > 1) {
        int64_t mid = lo + ((hi - lo) >> 1);
        if (ld_rpt(rpt, is64, mid) <= p) lo = mid; else hi = mid;
    }
    return lo;
}

// *p = fma(a, b, *p) as one atomic update of a shared-memory float64: a
// compare-and-swap loop on the value's bits. One fused multiply-add per
// product instead of a multiply and an atomic add (whose add also runs on
// the float64 pipe, which this GPU has little of); fma rounds once, so the
// sum is at least as accurate. Some update succeeds in every round of
// competing threads, so the loop ends.
__device__ __forceinline__ void smem_fma_add(double *p, double a, double b) {
    unsigned long long *q = reinterpret_cast<unsigned long long *>(p);
    unsigned long long old = *reinterpret_cast<volatile unsigned long long *>(q);
    for (;;) {
        const unsigned long long want =
            static_cast<unsigned long long>(__double_as_longlong(fma(a, b, __longlong_as_double(
                static_cast<long long>(old)))));
        const unsigned long long got = atomicCAS(q, old, want);
        if (got == old) return;
        old = got;
    }
}

// Row pointers of the A rows that hold the entries [t0, t1) of a block's
// tile of A's non-zeros, staged in shared memory so that each thread finds
// the row of its entries with a short search there instead of a binary
// search over all of A.rpt in global memory: r[i] = A.rpt[rlo + i] for
// i < n. n = 0 when they do not fit (long runs of empty rows); the caller
// then searches global memory. Synchronises the block.
template <int CAP>
struct TileRpt {
    long long r[CAP + 1];
    long long rlo;
    int n;
};

template <int CAP>
__device__ __forceinline__ void stage_tile_rpt(const Operands &op, int64_t lo, int64_t hi, int64_t t0,
                                               int64_t t1, TileRpt<CAP> *tr) {
    __syncthreads();   // readers of the previous tile are done
    if (threadIdx.x == 0) {
        const int64_t rlo = upper_bound_rpt(op.arpt, op.a64, lo, hi, t0);
        const int64_t rhi = upper_bound_rpt(op.arpt, op.a64, rlo, hi, t1 - 1);
        tr->rlo = rlo;
        tr->n = rhi - rlo + 2 <= CAP + 1 ? static_cast<int>(rhi - rlo + 2) : 0;
    }
    __syncthreads();
    const int n = tr->n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) tr->r[i] = ld_rpt(op.arpt, op.a64, tr->rlo + i);
    __syncthreads();
}

// Largest i in [lo, n - 1) with r[i] <= p (r[lo] <= p assumed).
__device__ __forceinline__ int tile_row(const long long *r, int lo, int n, int64_t p) {
    int hi = n - 1;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (r[mid] <= p) lo = mid; else hi = mid;
    }
    return lo;
}

}  // namespace ops

namespace ops {

// --- block-level walk over the products of one output row -------------------
// A row's products are the entries of the B rows its A entries reference.
// Giving each A entry to one sub-group leaves most of a block idle when a row
// has few A entries with long B rows (common in power-law graphs). Instead,
// A entries are read CH at a time, every referenced B row is cut into pieces
// of at most W = S * kPieceIters products, and the block's sub-groups of S
// lanes take pieces round-robin; a sub-group's lanes read a piece with unit
// stride (coalesced). The piece -> A entry map is a binary search over the
// chunk's piece offsets in shared memory, paid once per piece.
constexpr int kWalkChunk = 256;

struct WalkScratch {
    long long q0[kWalkChunk];     // first B entry of each A entry's B row
    double a[kWalkChunk];         // A value
    int len[kWalkChunk];          // B row length
    long long pstart[kWalkChunk + 1];  // exclusive piece offsets
    long long warp_tot[33];
};

// Exclusive scan of one long long per thread over a block of BLOCK threads
// (BLOCK a multiple of 32); returns the thread's prefix, `total` the sum.
template <int BLOCK>
__device__ __forceinline__ long long block_excl_scan_ll(long long x, long long &total,
                                                        long long *sw) {
    const unsigned lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
    long long inc = x;
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= static_cast<unsigned>(o)) inc += y;
    }
    if constexpr (BLOCK == 32) {
        total = __shfl_sync(0xffffffffu, inc, 31);
        return inc - x;
    } else {
        __syncthreads();
        if (lane == 31) sw[w] = inc;
        __syncthreads();
        if (w == 0) {
            const long long t = lane < (BLOCK >> 5) ? sw[lane] : 0;
            long long ti = t;
            for (int o = 1; o < 32; o <<= 1) {
                const long long y = __shfl_up_sync(0xffffffffu, ti, o);
                if (lane >= static_cast<unsigned>(o)) ti += y;
            }
            if (lane < (BLOCK >> 5)) sw[lane] = ti - t;
            if (lane == 31) sw[32] = ti;
        }
        __syncthreads();
        total = sw[32];
        return sw[w] + inc - x;
    }
}

// L2 residency of a C.val segment that float64 reductions go into: its
// zeroing stores and the reductions carry an evict_last policy, so the B rows
// streaming through L2 evict other lines first; once the row is done its
// lines drop back to normal priority (applypriority, one 128-byte line).
__device__ __forceinline__ unsigned long long l2_evict_last_policy() {
    unsigned long long pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ void st_keep(double *p, double v, unsigned long long pol) {
    asm volatile("st.global.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(p), "d"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void red_add_keep(double *p, double v, unsigned long long pol) {
    asm volatile("red.global.add.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(p), "d"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void l2_priority_normal(const void *p) {
    asm volatile("applypriority.global.L2::evict_normal [%0], 128;" ::"l"(p) : "memory");
}

// Exclusive scan of one unsigned per thread over a block of BLOCK threads.
template <int BLOCK>
__device__ __forceinline__ unsigned block_excl_scan(unsigned x, unsigned &total, unsigned *sw) {
    const unsigned lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
    unsigned inc = x;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= static_cast<unsigned>(o)) inc += y;
    }
    __syncthreads();
    if (lane == 31) sw[w] = inc;
    __syncthreads();
    if (w == 0) {
        const unsigned t = lane < (BLOCK >> 5) ? sw[lane] : 0u;
        unsigned ti = t;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, ti, o);
            if (lane >= static_cast<unsigned>(o)) ti += y;
        }
        if (lane < (BLOCK >> 5)) sw[lane] = ti - t;
        if (lane == 31) sw[32] = ti;
    }
    __syncthreads();
    total = sw[32];
    return sw[w] + inc - x;
}

// Calls f(key, a_value, b_value) for every product of the row [p0, p1) of A
// (a_value and b_value only when NEED_VAL). Every thread of the block must
// call it (it synchronises the block). A lane's products of one piece (at
// most kPieceIters) are loaded together before any of them is used, so each
// thread keeps several L2 loads in flight.
// KEEP: a first walk of a row also stores the A values of its entries, and a
// later walk of the same row with the same S and ITERS and the scratch left
// untouched in between (KEEP = 2) reuses the entries' B-row offsets, lengths,
// A values and piece offsets when the row fits one chunk, instead of loading
// them and scanning again.
// Restriction of a walk to the columns [c0, c1) of a window, for rows of B
// sorted by column: each A entry's products are then one run of its B row,
// found in the cell index of the long B rows (bidx, slot from bslot; offsets
// of the first entry of each cell of 2^cs columns) or by binary search.
struct RunSel {
    const int32_t *bslot;
    const int32_t *bidx;
    int cs, ncells;
    int c0, c1;
};

__device__ __forceinline__ long long lower_col_in(const int32_t *bcol, long long lo, long long hi, int c) {
    while (lo < hi) {
        const long long mid = lo + ((hi - lo) >> 1);
        if (__ldg(bcol + mid) < c) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// [s, e) of B row k (entries [q0, q1)) inside the window's columns.
__device__ __forceinline__ void run_in(const Operands &op, const RunSel &rs, int k, long long q0, long long q1,
                                       long long &s, long long &e) {
    s = q0;
    e = q1;
    if (rs.c0 <= 0 && rs.c1 >= op.ncols) return;
    const int32_t slot = rs.bslot ? __ldg(rs.bslot + k) : -1;
    if (slot >= 0) {
        const int32_t *x = rs.bidx + static_cast<long long>(slot) * (rs.ncells + 1);
        if (rs.c0 > 0) s = q0 + __ldg(x + (rs.c0 >> rs.cs));
        if (rs.c1 < op.ncols) e = q0 + __ldg(x + (rs.c1 >> rs.cs));
    } else {
        if (rs.c0 > 0) s = lower_col_in(op.bcol, q0, q1, rs.c0);
        if (rs.c1 < op.ncols) e = lower_col_in(op.bcol, s, q1, rs.c1);
    }
    if (e < s) e = s;
}

// RUNS: only the products inside the columns of *rs (rows of B sorted).
template <int BLOCK, bool NEED_VAL, int ITERS = kPieceIters, int KEEP = 0, bool RUNS = false, typename F>
__device__ __forceinline__ void block_row_walk(const Operands &op, int64_t p0, int64_t p1, int S,
                                               WalkScratch *sc, F &&f, const RunSel *rs = nullptr) {
    static_assert(BLOCK >= 32 && BLOCK % 32 == 0, "block walk needs whole warps");
    constexpr int CH = BLOCK < kWalkChunk ? BLOCK : kWalkChunk;
    const int nsub = BLOCK / S, sub = threadIdx.x / S, ls = threadIdx.x % S;
    const long long W = static_cast<long long>(S) * ITERS;
    for (int64_t c = p0; c < p1; c += CH) {
        const int cnt = static_cast<int>(p1 - c < CH ? p1 - c : CH);
        long long total;
        if (KEEP == 2 && p1 - p0 <= CH) {
            total = sc->pstart[CH];
        } else {
            long long pieces = 0;
            if (threadIdx.x < CH) {
                const int t = threadIdx.x;
                if (t < cnt) {
                    const int k = __ldg(op.acol + c + t);
                    long long q0 = ld_rpt(op.brpt, op.b64, k);
                    long long len = ld_rpt(op.brpt, op.b64, k + 1) - q0;
                    if (RUNS) {
                        long long s0, e0;
                        run_in(op, *rs, k, q0, q0 + len, s0, e0);
                        q0 = s0;
                        len = e0 - s0;
                    }
                    sc->q0[t] = q0;
                    sc->len[t] = static_cast<int>(len);
                    if (NEED_VAL || KEEP == 1) sc->a[t] = __ldg(op.aval + c + t);
                    pieces = (len + W - 1) / W;
                }
            }
            const long long ex = block_excl_scan_ll<BLOCK>(pieces, total, sc->warp_tot);
            if (threadIdx.x < CH) sc->pstart[threadIdx.x] = ex;   // entries >= cnt hold `total`
            if (threadIdx.x == 0) sc->pstart[CH] = total;
            __syncthreads();
        }
        // sub-group `sub` takes a contiguous range of pieces: one binary
        // search finds its first entry, later entries follow by stepping
        const long long per = (total + nsub - 1) / nsub;
        const long long it0 = per * sub;
        const long long it1 = it0 + per < total ? it0 + per : total;
        int lo = 0;
        if (it0 < it1) {
            int hi = cnt;  // last e with pstart[e] <= it0
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (sc->pstart[mid] <= it0) lo = mid; else hi = mid;
            }
        }
        long long next = sc->pstart[lo + 1];
        for (long long it = it0; it < it1; ++it) {
            while (it >= next) {   // skips entries with empty B rows
                ++lo;
                next = sc->pstart[lo + 1];
            }
            const long long piece = it - sc->pstart[lo];
            const long long qb = sc->q0[lo] + piece * W + ls;
            const long long qe0 = sc->q0[lo] + sc->len[lo];
            const double a = NEED_VAL ? sc->a[lo] : 0.0;
            int key[ITERS];
            double bv[ITERS];
#pragma unroll
            for (int u = 0; u < ITERS; ++u) {
                const long long q = qb + static_cast<long long>(u) * S;
                key[u] = q < qe0 ? __ldg(op.bcol + q) : -1;
                bv[u] = (NEED_VAL && q < qe0) ? __ldg(op.bval + q) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < ITERS; ++u)
                if (key[u] >= 0) f(key[u], a, bv[u]);
        }
        __syncthreads();
    }
}

}  // namespace ops

namespace ops {

// Asynchronous global -> shared copies of 4 and 8 bytes (cp.async, cached
// in L1), their commit groups and waits. Each thread waits for its own
// copies only.
__device__ __forceinline__ void cp_async_4(void *sdst, const void *gsrc) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(
                     static_cast<unsigned>(__cvta_generic_to_shared(sdst))),
                 "l"(gsrc)
                 : "memory");
}
__device__ __forceinline__ void cp_async_8(void *sdst, const void *gsrc) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(
                     static_cast<unsigned>(__cvta_generic_to_shared(sdst))),
                 "l"(gsrc)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// B pieces a row group keeps in flight in group_row_walk_staged.
constexpr int kStage = 3;

// Row walk for a row group of TPR <= 32 lanes that takes one B row per step
// in pieces of TPR entries (lane l: entry l of the piece) and stages B's
// columns and values in shared memory with cp.async, kStage - 1 pieces
// ahead of the one being added, so that the loads of the next B rows overlap
// the hash updates of the current one. scol / sval: the group's
// kStage * TPR slots (slot k of lane l at k * TPR + l); a lane reads only
// the slots it copied itself. The group synchronises after every piece and
// every lane runs the same trip counts, as in group_row_walk with SYNC: a
// caller whose pieces hold distinct columns may update its table without
// atomics. The pipeline runs within one chunk of TPR A entries (the A data
// of a chunk sit one entry per lane) and drains at its end.
template <int TPR, typename F>
__device__ __forceinline__ void group_row_walk_staged(const Operands &op, int64_t p0, int64_t p1, int *scol,
                                                      double *sval, F &&f) {
    static_assert(TPR <= 32, "group walk is for sub-warp row groups");
    const unsigned gm = group_mask<TPR>();
    const int lg = threadIdx.x % TPR;
    const int gbase = (threadIdx.x & 31) - lg;     // first lane of this group in the warp
    const int64_t n = p1 - p0;
    for (int64_t c = 0; c < n; c += TPR) {
        const int cnt = static_cast<int>(n - c < TPR ? n - c : TPR);
        long long my_q0 = 0;
        int my_len = 0;
        double my_a = 0.0;
        if (lg < cnt) {
            const int k = __ldg(op.acol + p0 + c + lg);
            my_q0 = ld_rpt(op.brpt, op.b64, k);
            my_len = static_cast<int>(ld_rpt(op.brpt, op.b64, k + 1) - my_q0);
            my_a = __ldg(op.aval + p0 + c + lg);
        }
        // first non-empty entry at or after e (TPR: none); uniform over the group
        auto next_entry = [&](int e, long long &q0, int &len) {
            for (; e < TPR; ++e) {
                len = __shfl_sync(gm, my_len, gbase + e);
                if (len > 0) {
                    q0 = __shfl_sync(gm, my_q0, gbase + e);
                    return e;
                }
            }
            return TPR;
        };
        // issue cursor: the next piece to copy
        long long iq0 = 0;
        int ilen = 0, ioff = 0;
        int ie = next_entry(0, iq0, ilen);
        auto issue = [&](int slot) {
            if (ie < TPR) {
                const int o = ioff + lg;
                if (o < ilen) {
                    cp_async_4(scol + slot * TPR + lg, op.bcol + iq0 + o);
                    cp_async_8(sval + slot * TPR + lg, op.bval + iq0 + o);
                }
                ioff += TPR;
                if (ioff >= ilen) {
                    ioff = 0;
                    ie = next_entry(ie + 1, iq0, ilen);
                }
            }
            cp_async_commit();   // one group per slot, empty past the chunk's last piece
        };
#pragma unroll
        for (int k = 0; k < kStage - 1; ++k) issue(k);
        // processing cursor: the piece whose copies are the oldest group
        long long pq0 = 0;
        int plen = 0, poff = 0, slot = 0;
        int pe = next_entry(0, pq0, plen);
        while (pe < TPR) {   // uniform over the group
            issue(slot == 0 ? kStage - 1 : slot - 1);
            cp_async_wait<kStage - 1>();
            const double a = __shfl_sync(gm, my_a, gbase + pe);
            if (poff + lg < plen) f(scol[slot * TPR + lg], a, sval[slot * TPR + lg]);
            __syncwarp(gm);
            poff += TPR;
            if (poff >= plen) {
                poff = 0;
                pe = next_entry(pe + 1, pq0, plen);
            }
            slot = slot + 1 == kStage ? 0 : slot + 1;
        }
        cp_async_wait<0>();   // only empty groups remain; slots are free for the next chunk
    }
}

// Row walk for row groups of TPR <= 32 lanes (a slice of one warp). The
// group loads TPR A entries at once into registers (one per lane), then its
// sub-groups of S lanes take entries round-robin and read each B row in
// pieces of kPieceIters * S products, every lane loading its kPieceIters
// products before using them. Entry data moves between the group's lanes by
// shuffles under the group's own lane mask: groups of one warp may pick
// different S and run different trip counts. S must be the same on every
// lane of a group. Calls f(key, a_value, b_value).
// SYNC: the group synchronises after every piece, and its lanes run the
// same trip counts (pieces are stepped from 0 for the whole group), so a
// caller whose products of one piece are distinct (one B row per step,
// S == TPR, no repeated column in a B row) may update its table without
// atomics: no two lanes of a step touch the same entry, and a step sees the
// writes of the steps before it.
template <int TPR, bool NEED_VAL, bool SYNC = false, typename F>
__device__ __forceinline__ void group_row_walk(const Operands &op, int64_t p0, int64_t p1, int S,
                                               F &&f) {
    static_assert(TPR <= 32, "group walk is for sub-warp row groups");
    const unsigned gm = group_mask<TPR>();
    const int lg = threadIdx.x % TPR;
    const int gbase = (threadIdx.x & 31) - lg;     // first lane of this group in the warp
    const int nsub = TPR / S, sub = lg / S, ls = lg % S;
    const int64_t n = p1 - p0;
    for (int64_t c = 0; c < n; c += TPR) {
        long long my_q0 = 0;
        int my_len = 0;
        double my_a = 0.0;
        if (c + lg < n) {
            const int k = __ldg(op.acol + p0 + c + lg);
            my_q0 = ld_rpt(op.brpt, op.b64, k);
            my_len = static_cast<int>(ld_rpt(op.brpt, op.b64, k + 1) - my_q0);
            if (NEED_VAL) my_a = __ldg(op.aval + p0 + c + lg);
        }
        for (int e0 = 0; e0 < TPR; e0 += nsub) {
            const int src = gbase + e0 + sub;
            const long long q0 = __shfl_sync(gm, my_q0, src);
            const int len = __shfl_sync(gm, my_len, src);
            const double a = NEED_VAL ? __shfl_sync(gm, my_a, src) : 0.0;
            if constexpr (SYNC) {
                // the group's longest row sets the trip count (one B row per
                // step when S == TPR: every lane sees the same len)
                for (int off0 = 0; off0 < len; off0 += S * kPieceIters) {
                    int key[kPieceIters];
                    double bv[kPieceIters];
#pragma unroll
                    for (int u = 0; u < kPieceIters; ++u) {
                        const int o = off0 + ls + u * S;
                        key[u] = o < len ? __ldg(op.bcol + q0 + o) : -1;
                        bv[u] = (NEED_VAL && o < len) ? __ldg(op.bval + q0 + o) : 0.0;
                    }
#pragma unroll
                    for (int u = 0; u < kPieceIters; ++u)
                        if (key[u] >= 0) f(key[u], a, bv[u]);
                    __syncwarp(gm);
                }
            } else {
                for (int off = ls; off < len; off += S * kPieceIters) {
                    int key[kPieceIters];
                    double bv[kPieceIters];
#pragma unroll
                    for (int u = 0; u < kPieceIters; ++u) {
                        const int o = off + u * S;
                        key[u] = o < len ? __ldg(op.bcol + q0 + o) : -1;
                        bv[u] = (NEED_VAL && o < len) ? __ldg(op.bval + q0 + o) : 0.0;
                    }
#pragma unroll
                    for (int u = 0; u < kPieceIters; ++u)
                        if (key[u] >= 0) f(key[u], a, bv[u]);
                }
            }
        }
    }
}

}  // namespace ops
