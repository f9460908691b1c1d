// Symbolic phase (Sec. 2.2, Sec. 5.2, Algorithm 4): the number of distinct
// column keys of each output row, written over n_prod in C.rpt.
//
// Bins 0..8 use shared-memory hash tables. A row group of TPR threads owns one
// table of T int32 slots (-1 = empty). Each probe is one atomicCAS whose
// returned value decides everything (the paper's single-access probe, Sec.
// 5.2): -1 means the key was new, the key itself means it was already there,
// anything else moves to the next slot. Every probe loop is bounded by the
// table size, so a full table raises an error flag instead of spinning.
// New keys are counted in a register per thread and summed once per row
// instead of one shared atomicAdd per new key.
//
// Table sizes are chosen for GB300's 228 KB of shared memory and 2048 threads
// per SM: kernels 0-7 keep full occupancy (their table bytes per thread fit
// 228 KB / 2048), kernel 8 trades occupancy for a 128 KB table (the role of
// the paper's kernel 7).
//
// Rows past the largest table go to sym_bitmap_kernel: one 1024-thread block
// per row keeps a bitmap of the column space in shared memory (227 KB hold
// 1.86M columns; wider matrices are covered in several passes over column
// windows), sets one bit per product with atomicOr and counts bits with
// popc. It replaces the paper's kernel 7 -> kernel 8 global-hash recompute:
// no key ever leaves shared memory and nothing has to be recomputed.
#include <climits>

#include "common.cuh"
#include "internal.h"

namespace ops {

// One access per probe (Algorithm 4): the compare-and-swap itself returns
// the slot's key. MULTI: the access pattern the paper measures against
// (Sec. 6, the hashing comparison), a plain read of the slot first and the
// compare-and-swap only on an empty one.
template <int T, bool MULTI = false>
__device__ __forceinline__ int sym_insert(int *tab, int key, int *err) {
    uint32_t h = hash_slot<T>(key);
    for (int it = 0; it < T; ++it) {
        if (MULTI) {
            const int cur = *static_cast<volatile int *>(tab + h);
            if (cur == key) return 0;
            if (cur == -1) {
                const int old = atomicCAS(tab + h, -1, key);
                if (old == -1) return 1;
                if (old == key) return 0;
            }
        } else {
            const int old = atomicCAS(tab + h, -1, key);
            if (old == -1) return 1;
            if (old == key) return 0;
        }
        h = next_slot<T>(h);
    }
    set_error(err, DERR_TABLE_FULL);
    return 0;
}

// Minimum resident blocks: enough for 2048 threads per SM (<= 32 registers
// per thread, Sec. 5.6) unless the table is so large that one block fills
// the SM's shared memory anyway.
template <int TPR, int BLOCK, int T, bool MULTI = false>
__global__ void __launch_bounds__(BLOCK, (T * 4 * (BLOCK / TPR) > 110 * 1024) ? 1 : 2048 / BLOCK)
sym_hash_kernel(Operands op, BinWork w) {
    constexpr int RPB = BLOCK / TPR;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int *smem_tab = reinterpret_cast<int *>(smem_raw);
    __shared__ long long red[32];
    const int g = threadIdx.x / TPR, lg = threadIdx.x % TPR;
    int *tab = smem_tab + g * T;
    const int64_t r = static_cast<int64_t>(blockIdx.x) * RPB + g;
    const bool valid = r < w.cnt;
    const int64_t row = valid ? (w.bins ? static_cast<int64_t>(w.bins[w.off + r]) : w.off + r) : 0;
    for (int s = lg; s < T; s += TPR) tab[s] = -1;
    group_sync<TPR>();
    long long cnt = 0;
    if constexpr (TPR > 32) {
        // one row per block (grid = rows): flattened walk over B-row pieces
        WalkScratch *sc = reinterpret_cast<WalkScratch *>(smem_raw + sizeof(int) * (size_t)T);
        const int64_t ar = op.row0 + row;
        const int64_t p0 = ld_rpt(op.arpt, op.a64, ar);
        const int64_t p1 = ld_rpt(op.arpt, op.a64, ar + 1);
        const int S = pick_lanes(w.lanes, w.crpt[row], p1 - p0, 32);
        block_row_walk<BLOCK, false>(op, p0, p1, S, sc, [&](int key, double, double) {
            cnt += sym_insert<T, MULTI>(tab, key, w.err);
        });
    } else {
        int64_t p0 = 0, p1 = 0;
        int S = 1;
        if (valid) {
            const int64_t ar = op.row0 + row;
            p0 = ld_rpt(op.arpt, op.a64, ar);
            p1 = ld_rpt(op.arpt, op.a64, ar + 1);
            S = pick_lanes(w.lanes, w.crpt[row], p1 - p0, TPR);
        }
        // lanes of one group must agree on S: take the group's lane-0 value
        S = __shfl_sync(0xffffffffu, S, (threadIdx.x & 31) - lg);
        group_row_walk<TPR, false>(op, p0, p1, S, [&](int key, double, double) {
            cnt += sym_insert<T, MULTI>(tab, key, w.err);
        });
    }
    cnt = group_sum<TPR>(cnt, red);
    if (valid && lg == 0) w.crpt[row] = cnt;
}

// RUNS: several column passes over sorted B; each pass walks only the runs
// of B rows inside it (w.bslot / w.bidx), unless the device flag says some
// row of B is unsorted.
template <int BLOCK, int ITERS, bool RUNS = false>
__global__ void __launch_bounds__(BLOCK, BLOCK == 1024 ? 1 : 1536 / BLOCK)
sym_bitmap_kernel(Operands op, BinWork w, int words) {
    constexpr int kBmBlock = BLOCK;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    WalkScratch *sc = reinterpret_cast<WalkScratch *>(smem_raw);
    unsigned *bm = reinterpret_cast<unsigned *>(smem_raw + sizeof(WalkScratch));
    __shared__ long long red[32];
    const int64_t row = w.bins ? static_cast<int64_t>(w.bins[w.off + blockIdx.x])
                               : w.off + static_cast<int64_t>(blockIdx.x);
    const int64_t ar = op.row0 + row;
    const int64_t p0 = ld_rpt(op.arpt, op.a64, ar);
    const int64_t p1 = ld_rpt(op.arpt, op.a64, ar + 1);
    const int S = pick_lanes(w.lanes, w.crpt[row], p1 - p0, 32);
    const int64_t span = static_cast<int64_t>(words) * 32;
    long long total = 0;
    // cell counts for the column-window numeric kernel: the pass span is a
    // whole number of cells (the host rounds `words` down), so a cell never
    // straddles two passes
    uint16_t *cells = w.cells ? w.cells + static_cast<int64_t>(blockIdx.x) * w.ncells : nullptr;
    if (w.cslot && threadIdx.x == 0) w.cslot[row] = static_cast<int32_t>(blockIdx.x);
    for (int64_t c0 = 0; c0 < op.ncols; c0 += span) {
        const int nw = static_cast<int>(((op.ncols - c0 < span ? op.ncols - c0 : span) + 31) / 32);
        for (int i = threadIdx.x; i < nw; i += kBmBlock) bm[i] = 0u;
        __syncthreads();
        const int c0i = static_cast<int>(c0);
        const unsigned span32 = static_cast<unsigned>(span);
        RunSel rsel{w.bslot, w.bidx, w.cs, w.ncells, c0i,
                    static_cast<int>(c0 + span < op.ncols ? c0 + span : op.ncols)};
        if (RUNS && w.bflags && (*w.bflags & 1ull)) {   // unsorted B: whole rows, filtered
            rsel.c0 = 0;
            rsel.c1 = INT_MAX;
        }
        // column loads only: 8 per lane at once in 1024-thread blocks (one
        // block per SM, latency bound)
        constexpr int kIt = BLOCK == 1024 && ITERS < 8 ? 8 : ITERS;
        block_row_walk<kBmBlock, false, kIt, 0, RUNS>(op, p0, p1, S, sc, [&](int key, double, double) {
            const unsigned rel = static_cast<unsigned>(key - c0i);   // one compare covers both ends
            if (rel < span32) atomicOr(bm + (rel >> 5), 1u << (rel & 31));
        }, &rsel);
        if (cells) {
            // one warp per cell: its words' bits, summed over the warp
            const int cwords = 1 << (w.cs - 5);
            const int ncp = (nw + cwords - 1) / cwords;
            const int cell0 = static_cast<int>(c0 >> w.cs);
            const int lane = threadIdx.x & 31;
            for (int cc = threadIdx.x >> 5; cc < ncp; cc += kBmBlock / 32) {
                const int e = (cc + 1) * cwords < nw ? (cc + 1) * cwords : nw;
                unsigned v = 0;
                for (int i = cc * cwords + lane; i < e; i += 32) v += __popc(bm[i]);
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0) {
                    total += v;
                    if (cell0 + cc < w.ncells) cells[cell0 + cc] = static_cast<uint16_t>(v);
                }
            }
        } else {
            for (int i = threadIdx.x; i < nw; i += kBmBlock) total += __popc(bm[i]);
        }
        __syncthreads();
    }
    total = group_sum<kBmBlock>(total, red);
    if (threadIdx.x == 0) w.crpt[row] = total;
}

// --- kernel table ---------------------------------------------------------------
using SymFn = void (*)(Operands, BinWork);

#define SYM_TABLE(X)                 \
    X(8, 256, 64)                    \
    X(16, 256, 256)                  \
    X(32, 256, 512)                  \
    X(32, 128, 1024)                 \
    X(128, 128, 2048)                \
    X(256, 256, 4096)                \
    X(512, 512, 8192)                \
    X(1024, 1024, 16384)             \
    X(1024, 1024, 32768)

struct SymEntry {
    KernelDesc d;
    SymFn fn;
};

#define SYM_ENTRY(TPR, BLOCK, T)                                                        \
    {{TPR, BLOCK, T, T, 0,                                                              \
      sizeof(int) * (BLOCK / TPR) * (size_t)T + (TPR > 32 ? sizeof(WalkScratch) : 0)}, \
     &sym_hash_kernel<TPR, BLOCK, T>},

static SymEntry g_sym[] = {SYM_TABLE(SYM_ENTRY)};
static constexpr int kSymHash = sizeof(g_sym) / sizeof(g_sym[0]);
// the same kernels with the read-then-swap probe (BinWork::multi)
#define SYM_MULTI_ENTRY(TPR, BLOCK, T) &sym_hash_kernel<TPR, BLOCK, T, true>,
static SymFn g_sym_multi[] = {SYM_TABLE(SYM_MULTI_ENTRY)};
static KernelDesc g_sym_bitmap{1024, 1024, 0, LLONG_MAX, 1, 0};

using BmFn = void (*)(Operands, BinWork, int);
// bitmap kernel variants: (threads per block, products in flight per lane)
static const struct { int block, iters; BmFn fn; } g_sym_bm[] = {
    {1024, 4, &sym_bitmap_kernel<1024, 4>}, {1024, 8, &sym_bitmap_kernel<1024, 8>},
    {512, 4, &sym_bitmap_kernel<512, 4>},   {256, 4, &sym_bitmap_kernel<256, 4>},
};

int sym_kernel_count() { return kSymHash + 1; }

const KernelDesc &sym_kernel(int id) {
    return id < kSymHash ? g_sym[id].d : g_sym_bitmap;
}

// Default symbolic bins: every hash table at least 1.2x the largest n_prod
// of its bin (Sec. 5.7, the paper's "Sym_1.2x"), the bitmap kernel for the
// rest. The one rule both the handle's default configuration and the
// allocation-free entry point use.
int default_sym_bins(long long *range, int32_t *kernel) {
    for (int j = 0; j < kSymHash + 1; ++j) {
        kernel[j] = j;
        range[j] = j < kSymHash ? g_sym[j].d.table * 5 / 6 : -1;
    }
    return kSymHash + 1;
}

cudaError_t sym_prepare(int smem_optin) {
    // Opt in for every kernel: the 48 KB default covers static plus dynamic
    // shared memory, so a table of exactly 48 KB already needs it.
    for (int i = 0; i < kSymHash; ++i) {
        cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void *>(g_sym[i].fn),
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(g_sym[i].d.smem));
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(reinterpret_cast<const void *>(g_sym_multi[i]),
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(g_sym[i].d.smem));
        if (e != cudaSuccess) return e;
    }
    g_sym_bitmap.table = static_cast<long long>((smem_optin - sizeof(WalkScratch)) / 4) * 32;
    for (const auto &v : g_sym_bm) {
        cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void *>(v.fn),
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin);
        if (e != cudaSuccess) return e;
    }
    return cudaFuncSetAttribute(reinterpret_cast<const void *>(&sym_bitmap_kernel<1024, 4, true>),
                                cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin);
}

// Same launch-shape rule as the numeric bitmap kernel: about 2048 threads
// per SM given how many blocks fit in shared memory.
static int pick_sym_bitmap_variant(size_t smem_total, int iters) {
    const size_t per_sm = 228 * 1024;
    const int fit = static_cast<int>(per_sm / (smem_total + 1024));
    int block = 1024;
    if (fit >= 8) block = 256;
    else if (fit >= 4) block = 512;
    if (iters == 8) block = 1024;
    for (int i = 0; i < static_cast<int>(sizeof(g_sym_bm) / sizeof(g_sym_bm[0])); ++i)
        if (g_sym_bm[i].block == block && g_sym_bm[i].iters == (iters == 8 ? 8 : 4)) return i;
    return 0;
}

cudaError_t launch_sym(int id, const Operands &op, const BinWork &w, size_t smem_bitmap,
                       cudaStream_t s) {
    if (w.cnt <= 0) return cudaSuccess;
    if (id < kSymHash) {
        const KernelDesc &d = g_sym[id].d;
        const int rpb = d.block / d.tpr;
        const int64_t grid = (w.cnt + rpb - 1) / rpb;
        const SymFn fn = w.multi ? g_sym_multi[id] : g_sym[id].fn;
        fn<<<static_cast<unsigned>(grid), d.block, d.smem, s>>>(op, w);
    } else {
        const int words = static_cast<int>(smem_bitmap / 4);
        const size_t smem = smem_bitmap + sizeof(WalkScratch);
        if (w.bidx && static_cast<int64_t>(words) * 32 < op.ncols) {
            sym_bitmap_kernel<1024, 4, true><<<static_cast<unsigned>(w.cnt), 1024, smem, s>>>(op, w, words);
            return cudaGetLastError();
        }
        const auto &v = g_sym_bm[pick_sym_bitmap_variant(smem, w.unroll)];
        v.fn<<<static_cast<unsigned>(w.cnt), v.block, smem, s>>>(op, w, words);
    }
    return cudaGetLastError();
}

}  // namespace ops
