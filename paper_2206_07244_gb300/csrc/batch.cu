// Batched SpGEMM: many products with small rows in one persistent launch.
//
// Row offsets without a serial scan: a symbolic tile also stores the sum
// of its rows' sizes (tsum[tile]); the scan item of a product scans only
// those tile sums; a numeric tile turns its own rows' sizes into offsets
// (tile prefix + block scan) and writes them to C.rpt before it multiplies.
//
// A batch is a list of products C_i = A_i * B_i in which B_i may be the C of
// an earlier product (a chain such as the Galerkin product P^T (A P) of
// algebraic multigrid). Per product the two-phase method of Sec. 2.2 runs as
// three kinds of work item: symbolic row tiles (distinct keys per row, into
// C.rpt), one scan (exclusive sum of C.rpt, Sec. 5.3), numeric row tiles
// (hash, condense, sort, store; Algorithm 5). Items sit in one queue in
// dependency order (all symbolic tiles of a level, its scans, its numeric
// tiles, then the next level) and the blocks of a persistent grid take them
// with one atomic each. A block that takes an item whose inputs are not
// complete yet waits on per-product counters; every wait is bounded and,
// when it runs out, records SPGEMM_ERR_TIMEOUT and stops the launch instead
// of spinning on. Data produced inside the launch (C.rpt, and the C of an
// earlier product used as B) is read with L2-coherent loads.
//
// Rows are small (the plan rejects rows with more intermediate products
// than the table holds), so a row group of G lanes owns a shared-memory
// table of T slots; products are walked with one lane per A entry.
#include <climits>

#include "common.cuh"
#include "internal.h"
#include "opsparse.h"

namespace ops {

constexpr int kBatchBlock = 256;

template <bool COHERENT>
__device__ __forceinline__ int64_t bload_rpt(const void *p, int is64, int64_t i) {
    if (COHERENT)
        return is64 ? __ldcg(static_cast<const long long *>(p) + i)
                    : static_cast<int64_t>(__ldcg(static_cast<const int *>(p) + i));
    return ld_rpt(p, is64, i);
}
template <bool COHERENT>
__device__ __forceinline__ int bload_col(const int32_t *p, int64_t i) {
    return COHERENT ? __ldcg(p + i) : __ldg(p + i);
}
template <bool COHERENT>
__device__ __forceinline__ double bload_val(const double *p, int64_t i) {
    return COHERENT ? __ldcg(p + i) : __ldg(p + i);
}

// Bounded wait for *ctr >= target (thread 0). false when the limit ran out.
__device__ __forceinline__ bool wait_at_least(const int *ctr, int target, long long limit) {
    for (long long k = 0; k < limit; ++k) {
        if (__ldcg(ctr) >= target) {
            __threadfence();
            return true;
        }
        __nanosleep(200);
    }
    return false;
}

template <int T>
__device__ __forceinline__ bool bsym_insert(int *tab, int key, int &cnt) {
    uint32_t h = hash_slot<T>(key);
    for (int it = 0; it < T; ++it) {
        const int old = atomicCAS(tab + h, -1, key);
        if (old == -1) { ++cnt; return true; }
        if (old == key) return true;
        h = next_slot<T>(h);
    }
    return false;
}

template <int T>
__device__ __forceinline__ bool bnum_insert(int *tk, double *tv, int key, double a, double b) {
    uint32_t h = hash_slot<T>(key);
    for (int it = 0; it < T; ++it) {
        const int old = atomicCAS(tk + h, -1, key);
        if (old == -1 || old == key) {
            smem_fma_add(tv + h, a, b);
            return true;
        }
        h = next_slot<T>(h);
    }
    return false;
}

// One row group (G lanes) multiplies row `row` of problem P into its table.
// NUMERIC: also accumulate values. Returns false if the table overflowed.
template <int G, int T, bool NUMERIC, bool COHERENT>
__device__ __forceinline__ bool batch_row(const BatchProb &P, int64_t row, int *tk, double *tv,
                                          int lg, int &cnt) {
    bool ok = true;
    const int64_t p0 = ld_rpt(P.arpt, P.a64, row), p1 = ld_rpt(P.arpt, P.a64, row + 1);
    for (int64_t p = p0 + lg; p < p1; p += G) {
        const int k = __ldg(P.acol + p);
        const double a = NUMERIC ? __ldg(P.aval + p) : 0.0;
        const int64_t q1 = bload_rpt<COHERENT>(P.brpt, P.b64, k + 1);
        for (int64_t q = bload_rpt<COHERENT>(P.brpt, P.b64, k); q < q1; ++q) {
            const int key = bload_col<COHERENT>(P.bcol, q);
            if (NUMERIC) ok &= bnum_insert<T>(tk, tv, key, a, bload_val<COHERENT>(P.bval, q));
            else ok &= bsym_insert<T>(tk, key, cnt);
        }
    }
    return ok;
}

// One thread per row: the thread keeps the row's distinct columns sorted
// in kBatchTiny shared slots of its own (slot j of thread t at
// j * kBatchBlock + t, so the threads of a warp hit distinct banks), adding
// equal columns in product order; the row is then stored as it stands,
// without condense or sort. Rows that do not fit (symbolic: a distinct
// column past kBatchTiny; numeric: a known size past kBatchTiny) are
// appended to `over` (tile-local row numbers) for the hash-table path.
template <bool NUMERIC, bool COHERENT>
__device__ __forceinline__ bool tiny_rows(const BatchProb &P, int64_t r0, int64_t r1, int *keys,
                                          double *vals, const long long *offs, const int *cnts,
                                          long long &tile_sum, int *over, int *nover) {
    bool ok = true;
    const int t = threadIdx.x;
    for (int64_t row = r0 + t; row < r1; row += kBatchBlock) {
        if (NUMERIC && cnts[row - r0] > kBatchTiny) {
            over[atomicAdd(nover, 1)] = static_cast<int>(row - r0);
            continue;
        }
        int n = 0;
        bool full = false;
        const int64_t p0 = ld_rpt(P.arpt, P.a64, row), p1 = ld_rpt(P.arpt, P.a64, row + 1);
        for (int64_t p = p0; p < p1 && !full; ++p) {
            const int k = __ldg(P.acol + p);
            const double a = NUMERIC ? __ldg(P.aval + p) : 0.0;
            const int64_t q1 = bload_rpt<COHERENT>(P.brpt, P.b64, k + 1);
            for (int64_t q = bload_rpt<COHERENT>(P.brpt, P.b64, k); q < q1; ++q) {
                const int key = bload_col<COHERENT>(P.bcol, q);
                const double b = NUMERIC ? bload_val<COHERENT>(P.bval, q) : 0.0;
                int pos = 0;
                while (pos < n && keys[pos * kBatchBlock + t] < key) ++pos;
                if (pos < n && keys[pos * kBatchBlock + t] == key) {
                    // one fused multiply-add per product (float64 is scarce here)
                    if (NUMERIC) vals[pos * kBatchBlock + t] = fma(a, b, vals[pos * kBatchBlock + t]);
                    continue;
                }
                if (n == kBatchTiny) {   // a ninth distinct column: the row goes to the tables
                    full = true;
                    break;
                }
                for (int m = n; m > pos; --m) {
                    keys[m * kBatchBlock + t] = keys[(m - 1) * kBatchBlock + t];
                    if (NUMERIC) vals[m * kBatchBlock + t] = vals[(m - 1) * kBatchBlock + t];
                }
                keys[pos * kBatchBlock + t] = key;
                if (NUMERIC) vals[pos * kBatchBlock + t] = fma(a, b, 0.0);   // 0 + a b, as the sum starts
                ++n;
            }
        }
        if (full) {
            if (NUMERIC) ok = false;   // its size said it fits: cannot happen
            else over[atomicAdd(nover, 1)] = static_cast<int>(row - r0);
            continue;
        }
        if (!NUMERIC) {
            P.crpt[row] = n;
            tile_sum += n;
        } else {
            const int64_t base = offs[row - r0];
            const int64_t want = cnts[row - r0];
            if (want != n || base + n > P.ccap) {
                ok = false;
            } else {
                for (int m = 0; m < n; ++m) {
                    P.ccol[base + m] = keys[m * kBatchBlock + t];
                    P.cval[base + m] = vals[m * kBatchBlock + t];
                }
            }
        }
    }
    return ok;
}

template <int G, int T>
__global__ void __launch_bounds__(kBatchBlock)
batch_kernel(const BatchProb *probs, const BatchItem *items, int nitems, BatchState *st,
             int *done_s, int *xflag, int *done_n, int tile_rows, long long spin_limit) {
    constexpr int RG = kBatchBlock / G;
    static_assert(RG * T >= kBatchTiny * kBatchBlock, "tiny rows reuse the tables");
    __shared__ int keys_all[RG * T];
    __shared__ double vals_all[RG * T];
    __shared__ long long offs[kBatchMaxTile];   // numeric tile: offset of each row in C
    __shared__ int cnts[kBatchMaxTile];         // numeric tile: size of each row
    __shared__ int over[kBatchMaxTile];         // rows left to the hash tables
    __shared__ int nover;
    __shared__ int red32[33];
    __shared__ long long red64[33];   // block scan: one slot per warp + the total
    __shared__ int s_item;
    __shared__ int s_ok;
    __shared__ long long s_run;
    const int g = threadIdx.x / G, lg = threadIdx.x % G;
    int *tk = keys_all + g * T;
    double *tv = vals_all + g * T;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const unsigned long long it = atomicAdd(&st->head, 1ull);
            s_item = (it < static_cast<unsigned long long>(nitems) && __ldcg(&st->err) == 0)
                         ? static_cast<int>(it) : -1;
        }
        __syncthreads();
        const int it = s_item;
        if (it < 0) return;
        const BatchItem I = items[it];
        const BatchProb &P = probs[I.prob];
        if (threadIdx.x == 0) {
            bool ok = true;
            if (I.type == 0 && P.dep >= 0) ok = wait_at_least(done_n + P.dep, probs[P.dep].ntiles, spin_limit);
            else if (I.type == 1) ok = wait_at_least(done_s + I.prob, P.ntiles, spin_limit);
            else if (I.type == 2) ok = wait_at_least(xflag + I.prob, 1, spin_limit);
            if (!ok && atomicCAS(&st->err, 0, SPGEMM_ERR_TIMEOUT) == 0) st->where = it;
            s_ok = ok;
        }
        __syncthreads();
        if (!s_ok) return;
        if (I.type == 1) {
            // exclusive scan of the tile sums in place; C.rpt[M] = total
            if (threadIdx.x == 0) s_run = 0;
            __syncthreads();
            for (int64_t b = 0; b < P.ntiles; b += kBatchBlock) {
                const int64_t i = b + threadIdx.x;
                const long long v = i < P.ntiles ? __ldcg(P.tsum + i) : 0;
                long long tot;
                const long long ex = block_excl_scan_ll<kBatchBlock>(v, tot, red64);
                if (i < P.ntiles) P.tsum[i] = s_run + ex;
                __syncthreads();
                if (threadIdx.x == 0) s_run += tot;
                __syncthreads();
            }
            if (threadIdx.x == 0) {
                P.crpt[P.M] = s_run;
                if (s_run > P.ccap && atomicCAS(&st->err, 0, SPGEMM_ERR_INTERNAL) == 0) st->where = it;
                __threadfence();
                atomicExch(xflag + I.prob, 1);
            }
            continue;
        }
        const int64_t r0 = static_cast<int64_t>(I.tile) * tile_rows;
        const int64_t r1 = r0 + tile_rows < P.M ? r0 + tile_rows : P.M;
        const bool coherent = P.dep >= 0;
        bool ok_all = true;
        long long tile_sum = 0;   // symbolic: this thread's share of the tile's n_nz
        if (I.type == 2) {
            // row offsets of the tile: its prefix from the scan plus a block
            // scan of its rows' sizes (each thread four consecutive rows)
            constexpr int kPer = kBatchMaxTile / kBatchBlock;
            const int64_t nrow = r1 - r0;
            long long c[kPer];
            long long part = 0;
#pragma unroll
            for (int q = 0; q < kPer; ++q) {
                const int64_t i = static_cast<int64_t>(threadIdx.x) * kPer + q;
                c[q] = i < nrow ? __ldcg(reinterpret_cast<const long long *>(P.crpt) + r0 + i) : 0;
                part += c[q];
            }
            long long tot;
            long long ex = block_excl_scan_ll<kBatchBlock>(part, tot, red64) + __ldcg(P.tsum + I.tile);
#pragma unroll
            for (int q = 0; q < kPer; ++q) {
                const int64_t i = static_cast<int64_t>(threadIdx.x) * kPer + q;
                if (i < nrow) {
                    offs[i] = ex;
                    cnts[i] = static_cast<int>(c[q]);
                    P.crpt[r0 + i] = ex;
                }
                ex += c[q];
            }
            __syncthreads();
        }
        // pass A: one thread per row; rows that do not fit are listed for pass B
        if (threadIdx.x == 0) nover = 0;
        __syncthreads();
        if (P.tiny >= 0) {
            if (I.type == 0)
                ok_all = coherent ? tiny_rows<false, true>(P, r0, r1, keys_all, vals_all, offs, cnts, tile_sum,
                                                           over, &nover)
                                  : tiny_rows<false, false>(P, r0, r1, keys_all, vals_all, offs, cnts, tile_sum,
                                                            over, &nover);
            else
                ok_all = coherent ? tiny_rows<true, true>(P, r0, r1, keys_all, vals_all, offs, cnts, tile_sum,
                                                          over, &nover)
                                  : tiny_rows<true, false>(P, r0, r1, keys_all, vals_all, offs, cnts, tile_sum,
                                                           over, &nover);
        } else {
            for (int i = threadIdx.x; i < r1 - r0; i += kBatchBlock) over[i] = i;
            if (threadIdx.x == 0) nover = static_cast<int>(r1 - r0);
        }
        __syncthreads();
        // pass B: the listed rows, a group of G lanes and a T-slot table each
        const int n_over = nover;
        for (int ob = 0; ob < n_over; ob += RG) {
            const bool valid = ob + g < n_over;
            const int64_t row = valid ? r0 + over[ob + g] : r0;
            for (int s = lg; s < T; s += G) {
                tk[s] = -1;
                tv[s] = 0.0;
            }
            group_sync<G>();
            int cnt = 0;
            bool ok = true;
            if (I.type == 0) {
                if (valid) ok = coherent ? batch_row<G, T, false, true>(P, row, tk, tv, lg, cnt)
                                         : batch_row<G, T, false, false>(P, row, tk, tv, lg, cnt);
                cnt = group_sum<G>(cnt, red32);
                if (valid && lg == 0) {
                    P.crpt[row] = cnt;
                    tile_sum += cnt;
                }
            } else {
                if (valid) ok = coherent ? batch_row<G, T, true, true>(P, row, tk, tv, lg, cnt)
                                         : batch_row<G, T, true, false>(P, row, tk, tv, lg, cnt);
                group_sync<G>();
                int n = 0;
                for (int c = 0; c < T; c += G) {
                    const int s = c + lg;
                    const int k = s < T ? tk[s] : -1;
                    const double v = s < T ? tv[s] : 0.0;
                    int pre, tot;
                    group_excl_count<G>(k >= 0, pre, tot, red32);
                    group_sync<G>();
                    if (k >= 0) {
                        tk[n + pre] = k;
                        tv[n + pre] = v;
                    }
                    n += tot;
                    group_sync<G>();
                }
                int Pn = 1;
                while (Pn < n) Pn <<= 1;
                if (Pn > T) { ok = false; Pn = 1; }
                for (int s = n + lg; s < Pn; s += G) tk[s] = INT_MAX;
                group_sync<G>();
                for (int k = 2; k <= Pn; k <<= 1) {
                    for (int j = k >> 1; j > 0; j >>= 1) {
                        for (int i = lg; i < Pn; i += G) {
                            const int ixj = i ^ j;
                            if (ixj > i) {
                                const int ka = tk[i], kb = tk[ixj];
                                if ((ka > kb) == ((i & k) == 0)) {
                                    tk[i] = kb;
                                    tk[ixj] = ka;
                                    const double va = tv[i];
                                    tv[i] = tv[ixj];
                                    tv[ixj] = va;
                                }
                            }
                        }
                        group_sync<G>();
                    }
                }
                if (valid) {
                    const int64_t base = offs[row - r0];
                    const int64_t want = cnts[row - r0];
                    if (want != n || base + n > P.ccap) ok = false;
                    else
                        for (int t = lg; t < n; t += G) {
                            P.ccol[base + t] = tk[t];
                            P.cval[base + t] = tv[t];
                        }
                }
            }
            ok_all &= ok;
            group_sync<G>();
        }
        if (!ok_all && atomicCAS(&st->err, 0, SPGEMM_ERR_INTERNAL) == 0) st->where = it;
        if (I.type == 0) {
            // the tile's n_nz for the product's scan
            long long tot;
            (void)block_excl_scan_ll<kBatchBlock>(tile_sum, tot, red64);
            if (threadIdx.x == 0) P.tsum[I.tile] = tot;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd((I.type == 0 ? done_s : done_n) + I.prob, 1);
        }
    }
}

using BatchFn = void (*)(const BatchProb *, const BatchItem *, int, BatchState *, int *, int *, int *,
                         int, long long);

// (threads per row, table slots) variants; the plan picks the smallest table
// that holds the batch's largest row bound
static const struct { int g, t; BatchFn fn; } g_batch[] = {
    {8, 64, &batch_kernel<8, 64>},
    {16, 128, &batch_kernel<16, 128>},
    {32, 256, &batch_kernel<32, 256>},
};

int batch_variant_count() { return sizeof(g_batch) / sizeof(g_batch[0]); }
int batch_variant_table(int v) { return g_batch[v].t; }
int batch_variant_lanes(int v) { return g_batch[v].g; }

cudaError_t launch_batch(int variant, int grid, const BatchProb *probs, const BatchItem *items,
                         int nitems, BatchState *st, int *done_s, int *xflag, int *done_n,
                         int tile_rows, long long spin_limit, cudaStream_t s) {
    g_batch[variant].fn<<<grid, kBatchBlock, 0, s>>>(probs, items, nitems, st, done_s, xflag, done_n,
                                                    tile_rows, spin_limit);
    return cudaGetLastError();
}

int batch_blocks_per_sm(int variant) {
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, reinterpret_cast<const void *>(g_batch[variant].fn),
                                                  kBatchBlock, 0);
    return n;
}

}  // namespace ops
