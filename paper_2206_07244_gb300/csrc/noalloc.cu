// spgemm_rowptr_noalloc: the symbolic phase of C = A * B (row sizes and the
// exclusive-scanned row pointer of C) for callers that must not allocate
// device memory.
//
// Some callers cannot call cudaMalloc at run time: a serving loop that has
// handed every byte of device memory to another framework's allocator, an
// embedded runtime whose memory budget is fixed at start-up, or code that is
// itself part of an allocator. They can still size C with this entry point.
// Its scratch memory (binning counters, the row-id array of the bins, the
// scan's tile sums, the error word) lives in one file-scope __device__ array
// of fixed size, which every GPU that loads this library holds until the
// process exits. The caller passes the inputs and the output row pointer;
// nothing is allocated, and no handle, stream or event is created.
//
// Host code cannot use the array's name as a device address (on the host it
// names a stand-in object), so the address is looked up with
// cudaGetSymbolAddress once per device, with that device current, during the
// first call on that device.
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "internal.h"
#include "opsparse.h"

namespace ops {
namespace {

constexpr int64_t kNoAllocMaxRows = int64_t(1) << 20;  // SPGEMM_NOALLOC_MAX_ROWS
constexpr size_t kNaCounters = 2048;                    // 2 x Counters + error word
constexpr size_t kNaBins = sizeof(int32_t) * kNoAllocMaxRows;
constexpr size_t kNaTiles = sizeof(long long) * ((kNoAllocMaxRows + 1023) / 1024 + 2);
constexpr size_t kNoAllocBytes = kNaCounters + kNaBins + kNaTiles;

static_assert(2 * sizeof(Counters) + sizeof(int) <= kNaCounters, "counter block too small");

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_scratch_addr[kMaxDevices] = {};
bool g_prepared[kMaxDevices] = {};

// Per-device set-up: the array's device address and the kernels' shared
// memory opt-in. Runs with the caller's current device.
int setup_device(int dev, unsigned char **scratch, int *smem_dyn_max) {
    if (dev < 0 || dev >= kMaxDevices) return SPGEMM_ERR_INVALID;
    int optin = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return SPGEMM_ERR_CUDA;
    *smem_dyn_max = optin - 1024;
    // kernel attributes: the same once-per-device step as spgemm_create,
    // under its own lock
    if (prepare_device(dev, *smem_dyn_max) != cudaSuccess) return SPGEMM_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_prepared[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) return SPGEMM_ERR_CUDA;
        g_scratch_addr[dev] = static_cast<unsigned char *>(p);
        g_prepared[dev] = true;
    }
    *scratch = g_scratch_addr[dev];
    return SPGEMM_OK;
}

}  // namespace
}  // namespace ops

using namespace ops;

extern "C" int spgemm_rowptr_noalloc(const spgemm_csr_in *A, const spgemm_csr_in *B,
                                     int64_t *crpt, void *stream, int64_t *nnzC) {
    if (!A || !B || !crpt) return SPGEMM_ERR_INVALID;
    for (const spgemm_csr_in *m : {A, B}) {
        if (m->rows < 0 || m->cols < 0 || m->nnz < 0 || !m->rpt) return SPGEMM_ERR_INVALID;
        if (m->nnz > 0 && !m->col) return SPGEMM_ERR_INVALID;
        if (m->cols > INT32_MAX || m->rows > INT32_MAX) return SPGEMM_ERR_INVALID;
    }
    if (A->cols != B->rows) return SPGEMM_ERR_SHAPE;
    if (A->rows > kNoAllocMaxRows) return SPGEMM_ERR_INVALID;  // beyond the static scratch
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SPGEMM_ERR_CUDA;
    unsigned char *scratch = nullptr;
    int smem_dyn_max = 0;
    int rc = setup_device(dev, &scratch, &smem_dyn_max);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Counters *cnt = reinterpret_cast<Counters *>(scratch);
    int *err = reinterpret_cast<int *>(scratch + 2 * sizeof(Counters));
    int32_t *bins = reinterpret_cast<int32_t *>(scratch + kNaCounters);
    long long *tiles = reinterpret_cast<long long *>(scratch + kNaCounters + kNaBins);
    const int64_t mw = A->rows;
    Operands op;
    op.arpt = A->rpt; op.a64 = A->rpt_is_i64 ? 1 : 0; op.acol = A->col; op.aval = nullptr;
    op.brpt = B->rpt; op.b64 = B->rpt_is_i64 ? 1 : 0; op.bcol = B->col; op.bval = nullptr;
    op.row0 = 0; op.mw = mw; op.ncols = B->cols;
    // The array keeps the previous call's contents: clear everything that
    // must start at zero (counters and error word), and the output, which
    // collects n_prod by atomic adds.
    if (cudaMemsetAsync(scratch, 0, kNaCounters, s) != cudaSuccess ||
        cudaMemsetAsync(crpt, 0, sizeof(int64_t) * (size_t)(mw + 1), s) != cudaSuccess)
        return SPGEMM_ERR_CUDA;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (launch_nprod(op, crpt, sms * 8, s) != cudaSuccess) return SPGEMM_ERR_CUDA;
    // default symbolic bins: every hash table at least 1.2x its bin's
    // largest n_prod, the bitmap kernel for the rest
    Ranges rs{};
    int32_t kid[kMaxBins];
    rs.nb = default_sym_bins(rs.r, kid);
    if (launch_bin_pass1(crpt, mw, rs, op, cnt, nullptr, s) != cudaSuccess) return SPGEMM_ERR_CUDA;
    Counters host[2];
    int herr = 0;
    if (cudaMemcpyAsync(host, cnt, sizeof(Counters), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return SPGEMM_ERR_CUDA;
    long long size[kMaxBins] = {}, off[kMaxBins] = {};
    long long acc = 0;
    int nonempty = 0;
    for (int j = 0; j < rs.nb; ++j) {
        size[j] = static_cast<long long>(host[0].bin_cnt[j]);
        off[j] = acc;
        acc += size[j];
        nonempty += size[j] > 0;
    }
    const bool identity = nonempty <= 1;
    if (!identity && launch_bin_pass2(crpt, mw, rs, off, cnt, bins, s) != cudaSuccess)
        return SPGEMM_ERR_CUDA;
    // symbolic kernels, largest rows first, all on the caller's stream
    for (int j = rs.nb - 1; j >= 0; --j) {
        if (size[j] <= 0) continue;
        BinWork w{};   // every field the symbolic kernels do not use stays zero (one-access probes)
        w.bins = identity ? nullptr : bins;
        w.off = identity ? 0 : off[j];
        w.cnt = size[j];
        w.crpt = crpt; w.ccol = nullptr; w.cval = nullptr;
        w.lanes = 0;
        w.unroll = 0;
        w.err = err;
        size_t smem = 0;
        if (sym_kernel(kid[j]).bitmap) {
            const int64_t budget = smem_dyn_max - static_cast<int64_t>(sizeof(WalkScratch));
            const int64_t words = (op.ncols + 31) / 32 < budget / 4 ? (op.ncols + 31) / 32 : budget / 4;
            smem = static_cast<size_t>(words > 1 ? words : 1) * 4;
        }
        if (launch_sym(kid[j], op, w, smem, s) != cudaSuccess) return SPGEMM_ERR_CUDA;
    }
    // total and tile sums of n_nz, then the in-place exclusive scan
    Ranges all{};
    all.nb = 1;
    all.r[0] = -1;
    if (launch_bin_pass1(crpt, mw, all, op, cnt + 1, tiles, s) != cudaSuccess) return SPGEMM_ERR_CUDA;
    if (launch_scan(crpt, mw, tiles, s) != cudaSuccess) return SPGEMM_ERR_CUDA;
    if (cudaMemcpyAsync(&host[1], cnt + 1, sizeof(Counters), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return SPGEMM_ERR_CUDA;
    if (herr) return SPGEMM_ERR_INTERNAL;
    if (nnzC) *nnzC = static_cast<int64_t>(host[1].total);
    return SPGEMM_OK;
}
