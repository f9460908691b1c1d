// Run boundaries of the rows of B at column sub-ranges.
//
// The numeric bitmap kernel can take pass 2 (the float64 sums) window by
// window over the column space, so that the C.val lines one window reduces
// into stay in L2 (num_bitmap_kernel). With every row of B sorted by column,
// the products of an output row that fall in columns [g * 2^s, g2 * 2^s) are,
// for each A entry, one contiguous run of its B row; bs gives the run bounds
// for every B row and every sub-range boundary:
//
//   bs[k * (G + 1) + g] = offset in row k of B of its first entry whose
//                         column is >= g * 2^s   (g = 0..G; bs[..G] = length)
//
// Work is split over B's non-zeros: entry e of row k writes the boundaries g
// in (sub-range of entry e - 1, sub-range of e]; the row's last entry writes
// the remaining ones; rows without entries are written all zero.
#include "common.cuh"
#include "internal.h"

namespace ops {

constexpr int kSplitBlock = 256;
constexpr int kSplitItems = 8;

__global__ void __launch_bounds__(kSplitBlock)
bsplit_kernel(Operands op, int64_t brows, int64_t bnnz, int gshift, int G, int32_t *bs) {
    const int64_t tile = static_cast<int64_t>(blockDim.x) * kSplitItems;
    for (int64_t base = static_cast<int64_t>(blockIdx.x) * tile; base < bnnz;
         base += static_cast<int64_t>(gridDim.x) * tile) {
        const int64_t e0 = base + static_cast<int64_t>(threadIdx.x) * kSplitItems;
        if (e0 >= bnnz) continue;
        int64_t row = upper_bound_rpt(op.brpt, op.b64, 0, brows, e0);
        int64_t rs = ld_rpt(op.brpt, op.b64, row);
        int64_t re = ld_rpt(op.brpt, op.b64, row + 1);
        for (int j = 0; j < kSplitItems; ++j) {
            const int64_t e = e0 + j;
            if (e >= bnnz) break;
            while (e >= re) {
                row = upper_bound_rpt(op.brpt, op.b64, row + 1, brows, e);
                rs = ld_rpt(op.brpt, op.b64, row);
                re = ld_rpt(op.brpt, op.b64, row + 1);
            }
            int32_t *b = bs + row * (G + 1);
            const int ge = __ldg(op.bcol + e) >> gshift;
            const int gp = e == rs ? -1 : (__ldg(op.bcol + e - 1) >> gshift);
            const int32_t off = static_cast<int32_t>(e - rs);
            for (int g = gp + 1; g <= ge && g <= G; ++g) b[g] = off;
            if (e + 1 == re)
                for (int g = ge + 1; g <= G; ++g) b[g] = off + 1;
        }
    }
}

__global__ void __launch_bounds__(kSplitBlock)
bsplit_empty_kernel(Operands op, int64_t brows, int G, int32_t *bs) {
    for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < brows;
         k += static_cast<int64_t>(gridDim.x) * blockDim.x)
        if (ld_rpt(op.brpt, op.b64, k + 1) == ld_rpt(op.brpt, op.b64, k))
            for (int g = 0; g <= G; ++g) bs[k * (G + 1) + g] = 0;
}

cudaError_t launch_bsplit(const Operands &op, int64_t brows, int64_t bnnz, int gshift, int G,
                          int32_t *bs, int grid, cudaStream_t s) {
    if (brows <= 0) return cudaSuccess;
    bsplit_empty_kernel<<<grid, kSplitBlock, 0, s>>>(op, brows, G, bs);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || bnnz <= 0) return e;
    bsplit_kernel<<<grid, kSplitBlock, 0, s>>>(op, brows, bnnz, gshift, G, bs);
    return cudaGetLastError();
}

}  // namespace ops
