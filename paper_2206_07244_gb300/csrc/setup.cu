// Setup, binning and scan kernels (Sec. 5 steps 1, 2, 4; Sec. 5.1, 5.3).
//
//  - nprod_kernel: n_prod per output row (Sec. 5 step 1), written into the
//    int64 C.rpt array that later holds n_nz and then the row offsets
//    (the metadata reuse of Sec. 5.3). Work is split evenly over A's
//    non-zeros, not over rows, so power-law rows cannot stall a warp.
//  - bin_pass1_kernel: Algorithm 1. Per-bin counts gathered in shared memory
//    (one shared atomic per group of same-bin lanes, found with
//    __match_any_sync), one global atomic per bin per block; also the
//    maximum and the int64 total of the sizes, and per-tile sums that the
//    scan reuses.
//  - bin_pass2_kernel: Algorithm 2. Scatters row ids into one M-length
//    `bins` array at offsets the host computed from the pass-1 counts.
//  - scan kernels: exclusive sum of n_nz into C.rpt in place (Sec. 5.3),
//    from the tile sums of pass 1.
#include "common.cuh"
#include "internal.h"

namespace ops {

constexpr int kNprodBlock = 256;
constexpr int kNprodItems = 8;

__device__ __forceinline__ void flush_row(int64_t *nprod, int64_t row, long long acc) {
    if (acc) atomicAdd(reinterpret_cast<unsigned long long *>(nprod + row),
                       static_cast<unsigned long long>(acc));
}

__global__ void __launch_bounds__(kNprodBlock)
nprod_kernel(Operands op, int64_t *nprod) {
    constexpr int kTile = kNprodBlock * kNprodItems;
    __shared__ TileRpt<kTile> tr;
    const int64_t lo = op.row0, hi = op.row0 + op.mw;     // A rows of the window
    const int64_t pb = ld_rpt(op.arpt, op.a64, lo);
    const int64_t pe = ld_rpt(op.arpt, op.a64, hi);
    for (int64_t base = pb + static_cast<int64_t>(blockIdx.x) * kTile; base < pe;
         base += static_cast<int64_t>(gridDim.x) * kTile) {
        stage_tile_rpt<kTile>(op, lo, hi, base, base + kTile < pe ? base + kTile : pe, &tr);
        const int64_t p0 = base + static_cast<int64_t>(threadIdx.x) * kNprodItems;
        if (p0 >= pe) continue;
        const int n = tr.n;
        int ti = 0;
        int64_t row, next;
        if (n > 0) {
            ti = tile_row(tr.r, 0, n, p0);
            row = tr.rlo + ti;
            next = tr.r[ti + 1];
        } else {
            row = upper_bound_rpt(op.arpt, op.a64, lo, hi, p0);
            next = ld_rpt(op.arpt, op.a64, row + 1);
        }
        long long acc = 0;
#pragma unroll
        for (int j = 0; j < kNprodItems; ++j) {
            const int64_t p = p0 + j;
            if (p >= pe) break;
            if (p >= next) {
                flush_row(nprod, row - lo, acc);
                acc = 0;
                if (n > 0) {
                    ti = tile_row(tr.r, ti + 1, n, p);
                    row = tr.rlo + ti;
                    next = tr.r[ti + 1];
                } else {
                    row = upper_bound_rpt(op.arpt, op.a64, row + 1, hi, p);
                    next = ld_rpt(op.arpt, op.a64, row + 1);
                }
            }
            const int k = __ldg(op.acol + p);
            acc += ld_rpt(op.brpt, op.b64, k + 1) - ld_rpt(op.brpt, op.b64, k);
        }
        flush_row(nprod, row - lo, acc);
    }
}

cudaError_t launch_nprod(const Operands &op, int64_t *nprod, int grid, cudaStream_t s) {
    if (op.mw <= 0) return cudaSuccess;
    nprod_kernel<<<grid, kNprodBlock, 0, s>>>(op, nprod);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
constexpr int kBinBlock = 256;
constexpr int kBinItems = 4;                       // rows per thread
constexpr int kBinTile = kBinBlock * kBinItems;    // rows per block (tile)

int64_t bin_tile_rows() { return kBinTile; }

__device__ __forceinline__ int bin_of(long long v, const Ranges &rg) {
    // Algorithm 1: the first bin whose inclusive upper range holds v; a
    // negative range means "no bound".
    for (int j = 0; j < rg.nb; ++j)
        if (rg.r[j] < 0 || v <= rg.r[j]) return j;
    return rg.nb - 1;
}

__global__ void __launch_bounds__(kBinBlock)
bin_pass1_kernel(const int64_t *sizes, int64_t n, Ranges rg, Operands op, Counters *cnt,
                 long long *tile_sums) {
    __shared__ unsigned s_cnt[kMaxBins];
    __shared__ unsigned long long s_bsum[kMaxBins];
    __shared__ unsigned long long s_bnza[kMaxBins];
    __shared__ unsigned long long s_max;
    __shared__ long long s_sum;
    if (threadIdx.x < kMaxBins) {
        s_cnt[threadIdx.x] = 0;
        s_bsum[threadIdx.x] = 0;
        s_bnza[threadIdx.x] = 0;
    }
    if (threadIdx.x == 0) { s_max = 0; s_sum = 0; }
    __syncthreads();
    const int64_t tile0 = static_cast<int64_t>(blockIdx.x) * kBinTile;
    long long my_sum = 0;
    unsigned long long my_max = 0;
    const unsigned lane = threadIdx.x & 31u;
#pragma unroll
    for (int it = 0; it < kBinItems; ++it) {
        const int64_t i = tile0 + it * kBinBlock + threadIdx.x;
        const bool valid = i < n;
        const long long v = valid ? sizes[i] : 0;
        my_sum += v;
        if (static_cast<unsigned long long>(v) > my_max) my_max = v;
        const int j = valid ? bin_of(v, rg) : -1;
        const unsigned same = __match_any_sync(0xffffffffu, j);
        if (valid && lane == static_cast<unsigned>(__ffs(same) - 1))
            atomicAdd(&s_cnt[j], static_cast<unsigned>(__popc(same)));
        if (valid) {
            // per-bin totals for the diagnostics (sizes and A entries)
            const int64_t ar = op.row0 + i;
            const long long na = ld_rpt(op.arpt, op.a64, ar + 1) - ld_rpt(op.arpt, op.a64, ar);
            if (v) atomicAdd(&s_bsum[j], static_cast<unsigned long long>(v));
            if (na) atomicAdd(&s_bnza[j], static_cast<unsigned long long>(na));
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        my_sum += __shfl_xor_sync(0xffffffffu, my_sum, o);
        unsigned long long m = __shfl_xor_sync(0xffffffffu, my_max, o);
        if (m > my_max) my_max = m;
    }
    if (lane == 0) {
        atomicAdd(reinterpret_cast<unsigned long long *>(&s_sum),
                  static_cast<unsigned long long>(my_sum));
        atomicMax(&s_max, my_max);
    }
    __syncthreads();
    if (threadIdx.x < rg.nb && s_cnt[threadIdx.x]) {
        atomicAdd(&cnt->bin_cnt[threadIdx.x], static_cast<unsigned long long>(s_cnt[threadIdx.x]));
        atomicAdd(&cnt->bin_sum[threadIdx.x], s_bsum[threadIdx.x]);
        atomicAdd(&cnt->bin_nnza[threadIdx.x], s_bnza[threadIdx.x]);
    }
    if (threadIdx.x == 0) {
        atomicMax(&cnt->max_size, s_max);
        atomicAdd(&cnt->total, static_cast<unsigned long long>(s_sum));
        if (tile_sums) tile_sums[blockIdx.x] = s_sum;
    }
}

__global__ void __launch_bounds__(kBinBlock)
bin_pass2_kernel(const int64_t *sizes, int64_t n, Ranges rg, Counters *cnt, int32_t *bins,
                 Ranges off) {
    __shared__ unsigned s_cnt[kMaxBins];
    __shared__ long long s_base[kMaxBins];
    if (threadIdx.x < kMaxBins) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    const unsigned lane = threadIdx.x & 31u;
    const int64_t tile0 = static_cast<int64_t>(blockIdx.x) * kBinTile;
    int jv[kBinItems];
    unsigned pos[kBinItems];
#pragma unroll
    for (int it = 0; it < kBinItems; ++it) {
        const int64_t i = tile0 + it * kBinBlock + threadIdx.x;
        const bool valid = i < n;
        const int j = valid ? bin_of(sizes[i], rg) : -1;
        const unsigned same = __match_any_sync(0xffffffffu, j);
        const int leader = __ffs(same) - 1;
        unsigned wbase = 0;
        if (valid && static_cast<int>(lane) == leader)
            wbase = atomicAdd(&s_cnt[j], static_cast<unsigned>(__popc(same)));
        wbase = __shfl_sync(0xffffffffu, wbase, leader);
        jv[it] = j;
        pos[it] = wbase + __popc(same & ((1u << lane) - 1u));
    }
    __syncthreads();
    if (threadIdx.x < rg.nb) {
        const unsigned c = s_cnt[threadIdx.x];
        s_base[threadIdx.x] = off.r[threadIdx.x] +
            (c ? static_cast<long long>(atomicAdd(&cnt->cursor[threadIdx.x],
                                                  static_cast<unsigned long long>(c)))
               : 0);
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kBinItems; ++it) {
        const int64_t i = tile0 + it * kBinBlock + threadIdx.x;
        if (i < n) bins[s_base[jv[it]] + pos[it]] = static_cast<int32_t>(i);
    }
}

cudaError_t launch_bin_pass1(const int64_t *sizes, int64_t n, const Ranges &rg,
                             const Operands &op, Counters *cnt, long long *tile_sums,
                             cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int64_t grid = (n + kBinTile - 1) / kBinTile;
    bin_pass1_kernel<<<static_cast<unsigned>(grid), kBinBlock, 0, s>>>(sizes, n, rg, op, cnt,
                                                                       tile_sums);
    return cudaGetLastError();
}

cudaError_t launch_bin_pass2(const int64_t *sizes, int64_t n, const Ranges &rg,
                             const long long *offsets, Counters *cnt, int32_t *bins,
                             cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    Ranges off{};
    off.nb = rg.nb;
    for (int j = 0; j < rg.nb; ++j) off.r[j] = offsets[j];
    const int64_t grid = (n + kBinTile - 1) / kBinTile;
    bin_pass2_kernel<<<static_cast<unsigned>(grid), kBinBlock, 0, s>>>(sizes, n, rg, cnt, bins,
                                                                       off);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Is every row of B sorted by column (bit 0 of flags set when not), and
// are its columns distinct (bit 1 set when a row repeats a column)? The
// column-window kernels need non-decreasing rows; the warp-per-row numeric
// hash kernels update values without atomics when the columns of every B
// row are distinct. Work is split over
// B's non-zeros; each thread checks the pairs (e, e + 1) of its entries that
// lie in one row.
constexpr int kSortItems = 8;

__global__ void __launch_bounds__(kBinBlock)
sorted_check_kernel(Operands op, int64_t brows, int64_t bnnz, Counters *cnt) {
    const int64_t tile = static_cast<int64_t>(blockDim.x) * kSortItems;
    bool bad = false, dup = false;
    for (int64_t base = static_cast<int64_t>(blockIdx.x) * tile; base < bnnz - 1;
         base += static_cast<int64_t>(gridDim.x) * tile) {
        const int64_t e0 = base + static_cast<int64_t>(threadIdx.x) * kSortItems;
        if (e0 >= bnnz - 1) continue;
        int64_t row = upper_bound_rpt(op.brpt, op.b64, 0, brows, e0);
        int64_t next = ld_rpt(op.brpt, op.b64, row + 1);
        for (int j = 0; j < kSortItems; ++j) {
            const int64_t e = e0 + j;
            if (e >= bnnz - 1) break;
            while (e >= next) {
                row = upper_bound_rpt(op.brpt, op.b64, row + 1, brows, e);
                next = ld_rpt(op.brpt, op.b64, row + 1);
            }
            if (e + 1 < next) {
                const int c0 = __ldg(op.bcol + e), c1 = __ldg(op.bcol + e + 1);
                bad |= c1 < c0;
                dup |= c1 == c0;
            }
        }
    }
    const bool any_bad = __any_sync(0xffffffffu, bad), any_dup = __any_sync(0xffffffffu, dup);
    if ((threadIdx.x & 31u) == 0 && (any_bad || any_dup))
        atomicOr(&cnt->flags, (any_bad ? 1ull : 0ull) | (any_dup ? 2ull : 0ull));
}

cudaError_t launch_sorted_check(const Operands &op, int64_t brows, int64_t bnnz, Counters *cnt,
                                int grid, cudaStream_t s) {
    if (bnnz <= 1 || brows <= 0) return cudaSuccess;
    sorted_check_kernel<<<grid, kBinBlock, 0, s>>>(op, brows, bnnz, cnt);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Exclusive scan of the row sizes into C.rpt, in place (Sec. 5.3). Tile t
// covers rows [t*kBinTile, (t+1)*kBinTile), the same tiles whose sums
// bin_pass1_kernel stored.
constexpr int kScanBlock = 1024;

__global__ void __launch_bounds__(kScanBlock)
scan_tiles_kernel(long long *tile_sums, int64_t ntiles) {
    // Exclusive scan of tile_sums[0..ntiles) in place; tile_sums[ntiles] = total.
    __shared__ long long s_warp[32];
    __shared__ long long s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    const unsigned lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
    for (int64_t base = 0; base < ntiles; base += kScanBlock) {
        const int64_t i = base + threadIdx.x;
        const long long x = i < ntiles ? tile_sums[i] : 0;
        long long inc = x;
        for (int o = 1; o < 32; o <<= 1) {
            long long y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= static_cast<unsigned>(o)) inc += y;
        }
        if (lane == 31) s_warp[w] = inc;
        __syncthreads();
        if (w == 0) {
            long long t = s_warp[lane];
            long long ti = t;
            for (int o = 1; o < 32; o <<= 1) {
                long long y = __shfl_up_sync(0xffffffffu, ti, o);
                if (lane >= static_cast<unsigned>(o)) ti += y;
            }
            s_warp[lane] = ti - t;
        }
        __syncthreads();
        const long long carry = s_carry;
        const long long excl = carry + s_warp[w] + inc - x;
        if (i < ntiles) tile_sums[i] = excl;
        __syncthreads();
        if (threadIdx.x == kScanBlock - 1) s_carry = excl + x;
        __syncthreads();
    }
    if (threadIdx.x == 0) tile_sums[ntiles] = s_carry;
}

__global__ void __launch_bounds__(kBinBlock)
scan_apply_kernel(int64_t *crpt, int64_t n, const long long *tile_prefix, int64_t ntiles) {
    // One block per tile of kBinTile rows; each thread scans kBinItems
    // consecutive rows.
    __shared__ long long s_warp[kBinBlock / 32];
    const int64_t t = blockIdx.x;
    const int64_t r0 = t * kBinTile + static_cast<int64_t>(threadIdx.x) * kBinItems;
    long long v[kBinItems];
    long long local = 0;
#pragma unroll
    for (int k = 0; k < kBinItems; ++k) {
        v[k] = (r0 + k < n) ? crpt[r0 + k] : 0;
        local += v[k];
    }
    const unsigned lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
    long long inc = local;
    for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= static_cast<unsigned>(o)) inc += y;
    }
    if (lane == 31) s_warp[w] = inc;
    __syncthreads();
    if (w == 0) {
        long long x = lane < kBinBlock / 32 ? s_warp[lane] : 0;
        long long xi = x;
        for (int o = 1; o < 32; o <<= 1) {
            long long y = __shfl_up_sync(0xffffffffu, xi, o);
            if (lane >= static_cast<unsigned>(o)) xi += y;
        }
        if (lane < kBinBlock / 32) s_warp[lane] = xi - x;
    }
    __syncthreads();
    long long run = tile_prefix[t] + s_warp[w] + inc - local;
#pragma unroll
    for (int k = 0; k < kBinItems; ++k) {
        if (r0 + k < n) crpt[r0 + k] = run;
        run += v[k];
    }
    if (t == ntiles - 1 && threadIdx.x == 0) crpt[n] = tile_prefix[ntiles];
}

cudaError_t launch_scan(int64_t *crpt, int64_t n, long long *tile_sums, cudaStream_t s) {
    if (n <= 0) {
        return cudaMemsetAsync(crpt, 0, sizeof(int64_t), s);
    }
    const int64_t ntiles = (n + kBinTile - 1) / kBinTile;
    scan_tiles_kernel<<<1, kScanBlock, 0, s>>>(tile_sums, ntiles);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    scan_apply_kernel<<<static_cast<unsigned>(ntiles), kBinBlock, 0, s>>>(crpt, n, tile_sums, ntiles);
    return cudaGetLastError();
}

__global__ void iota_kernel(int32_t *out, int64_t n) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) out[i] = static_cast<int32_t>(i);
}

cudaError_t launch_iota(int32_t *out, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    iota_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(out, n);
    return cudaGetLastError();
}

}  // namespace ops
