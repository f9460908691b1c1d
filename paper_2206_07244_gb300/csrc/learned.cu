// Learned row sizing: per-row features, a 6 -> 64 -> 64 -> 1 multilayer
// perceptron (float32) that predicts log1p(n_nz) of each output row, its
// training kernels, and the one-phase numeric kernel that uses the
// prediction.
//
// The paper sizes every row with an exact symbolic pass (Sec. 2.2) and
// notes the alternative, a one-phase method with temporary storage and a
// final copy (Sec. 2.2, one-phase). Here a row predicted to fit a shared
// table is multiplied once into a table sized from the prediction; the
// exact size falls out of the table, the sorted row goes to temporary
// memory and is copied into C after the scan. A row whose distinct keys do
// not fit (a misprediction) is flagged and goes through the exact symbolic
// and numeric kernels, so C is the same as without the predictor.
#include <climits>

#include "common.cuh"
#include "internal.h"

namespace ops {

// ---------------------------------------------------------------------------
// Features (one flat pass over A's non-zeros, like nprod_kernel): per row
// n_prod, max and min referenced B-row length; then per row the six
// features: log1p(nnz A_i), log1p(n_prod), log1p(max), log1p(mean),
// log1p(min), log((i + 1) / M); empty A rows have max = mean = min = 0.
constexpr int kFeatBlock = 256;
constexpr int kFeatItems = 8;

__global__ void __launch_bounds__(kFeatBlock)
feature_scan_kernel(Operands op, long long *nprod, unsigned *maxlen, unsigned *minlen) {
    constexpr int kTile = kFeatBlock * kFeatItems;
    __shared__ TileRpt<kTile> tr;
    const int64_t lo = op.row0, hi = op.row0 + op.mw;
    const int64_t pb = ld_rpt(op.arpt, op.a64, lo);
    const int64_t pe = ld_rpt(op.arpt, op.a64, hi);
    for (int64_t base = pb + static_cast<int64_t>(blockIdx.x) * kTile; base < pe;
         base += static_cast<int64_t>(gridDim.x) * kTile) {
        stage_tile_rpt<kTile>(op, lo, hi, base, base + kTile < pe ? base + kTile : pe, &tr);
        const int64_t p0 = base + static_cast<int64_t>(threadIdx.x) * kFeatItems;
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
        unsigned mx = 0, mn = UINT_MAX;
        auto flush = [&]() {
            const int64_t r = row - lo;
            if (acc) atomicAdd(reinterpret_cast<unsigned long long *>(nprod + r),
                               static_cast<unsigned long long>(acc));
            atomicMax(maxlen + r, mx);
            atomicMin(minlen + r, mn);
        };
        for (int j = 0; j < kFeatItems; ++j) {
            const int64_t p = p0 + j;
            if (p >= pe) break;
            if (p >= next) {
                flush();
                acc = 0;
                mx = 0;
                mn = UINT_MAX;
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
            const long long len = ld_rpt(op.brpt, op.b64, k + 1) - ld_rpt(op.brpt, op.b64, k);
            acc += len;
            mx = max(mx, static_cast<unsigned>(len));
            mn = min(mn, static_cast<unsigned>(len));
        }
        flush();
    }
}

__global__ void feature_finish_kernel(Operands op, int64_t mrows, const long long *nprod,
                                      const unsigned *maxlen, const unsigned *minlen, float *X) {
    const int64_t r = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (r >= op.mw) return;
    const int64_t i = op.row0 + r;
    const long long na = ld_rpt(op.arpt, op.a64, i + 1) - ld_rpt(op.arpt, op.a64, i);
    const long long np = nprod[r];
    float *x = X + 6 * r;
    x[0] = log1pf(static_cast<float>(na));
    x[1] = log1pf(static_cast<float>(np));
    if (na > 0) {
        x[2] = log1pf(static_cast<float>(maxlen[r]));
        x[3] = log1pf(static_cast<float>(static_cast<double>(np) / static_cast<double>(na)));
        x[4] = log1pf(static_cast<float>(minlen[r]));
    } else {
        x[2] = x[3] = x[4] = 0.f;
    }
    x[5] = logf(static_cast<float>(static_cast<double>(i + 1) / static_cast<double>(mrows)));
}

cudaError_t launch_features(const Operands &op, int64_t mrows, long long *nprod, unsigned *maxlen,
                            unsigned *minlen, float *X, int grid, cudaStream_t s) {
    if (op.mw <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(nprod, 0, sizeof(long long) * (size_t)op.mw, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(maxlen, 0, sizeof(unsigned) * (size_t)op.mw, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(minlen, 0xff, sizeof(unsigned) * (size_t)op.mw, s);
    if (e != cudaSuccess) return e;
    feature_scan_kernel<<<grid, kFeatBlock, 0, s>>>(op, nprod, maxlen, minlen);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t g2 = (op.mw + 255) / 256;
    feature_finish_kernel<<<static_cast<unsigned>(g2), 256, 0, s>>>(op, mrows, nprod, maxlen, minlen, X);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// MLP 6 -> 64 -> 64 -> 1 with ReLU, parameters flat in this order:
// W1 (6x64 row-major), b1 (64), W2 (64x64 row-major), b2 (64), w3 (64), b3.
constexpr int kIn = 6, kH = 64;
constexpr int kOffW1 = 0, kOffB1 = kIn * kH, kOffW2 = kOffB1 + kH, kOffB2 = kOffW2 + kH * kH,
              kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + kH, kParams = kOffB3 + 1;
static_assert(kParams == 4673, "parameter count");

int mlp_param_count() { return kParams; }

// One row through the network. Weights are read from shared memory four at
// a time (16-byte broadcast loads: every thread of a warp reads the same
// address); each hidden unit sums its inputs in ascending order.
__device__ __forceinline__ float mlp_row(const float *w, const float *x) {
    float h1[kH];
#pragma unroll
    for (int a = 0; a < kH; a += 4) {
        float4 z = *reinterpret_cast<const float4 *>(w + kOffB1 + a);
#pragma unroll
        for (int f = 0; f < kIn; ++f) {
            const float4 wv = *reinterpret_cast<const float4 *>(w + kOffW1 + f * kH + a);
            z.x = fmaf(x[f], wv.x, z.x);
            z.y = fmaf(x[f], wv.y, z.y);
            z.z = fmaf(x[f], wv.z, z.z);
            z.w = fmaf(x[f], wv.w, z.w);
        }
        h1[a] = fmaxf(z.x, 0.f);
        h1[a + 1] = fmaxf(z.y, 0.f);
        h1[a + 2] = fmaxf(z.z, 0.f);
        h1[a + 3] = fmaxf(z.w, 0.f);
    }
    float y = w[kOffB3];
    for (int j = 0; j < kH; j += 4) {
        float4 z = *reinterpret_cast<const float4 *>(w + kOffB2 + j);
#pragma unroll
        for (int a = 0; a < kH; ++a) {
            const float4 wv = *reinterpret_cast<const float4 *>(w + kOffW2 + a * kH + j);
            z.x = fmaf(h1[a], wv.x, z.x);
            z.y = fmaf(h1[a], wv.y, z.y);
            z.z = fmaf(h1[a], wv.z, z.z);
            z.w = fmaf(h1[a], wv.w, z.w);
        }
        const float4 w3 = *reinterpret_cast<const float4 *>(w + kOffW3 + j);
        y = fmaf(fmaxf(z.x, 0.f), w3.x, y);
        y = fmaf(fmaxf(z.y, 0.f), w3.y, y);
        y = fmaf(fmaxf(z.z, 0.f), w3.z, y);
        y = fmaf(fmaxf(z.w, 0.f), w3.w, y);
    }
    return y;
}

// Inference: y[i] = MLP(X[i]); if sizes != nullptr also the predicted row
// size max(1, ceil(expm1(y) * (1 + margin))), capped at cap.
__global__ void __launch_bounds__(256)
mlp_forward_kernel(const float *theta, const float *X, int64_t n, float *y, long long *sizes,
                   float margin, long long cap) {
    __shared__ __align__(16) float w[kParams + 3];
    for (int i = threadIdx.x; i < kParams; i += blockDim.x) w[i] = theta[i];
    __syncthreads();
    const int64_t r = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (r >= n) return;
    float x[kIn];
#pragma unroll
    for (int f = 0; f < kIn; ++f) x[f] = X[kIn * r + f];
    const float out = mlp_row(w, x);
    if (y) y[r] = out;
    if (sizes) {
        const float e = expm1f(fminf(out, 40.f)) * (1.f + margin);
        long long s = static_cast<long long>(ceilf(e));
        if (s < 1) s = 1;
        if (s > cap) s = cap;
        sizes[r] = s;
    }
}

cudaError_t launch_mlp_forward(const float *theta, const float *X, int64_t n, float *y,
                               long long *sizes, float margin, long long cap, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    mlp_forward_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(theta, X, n, y, sizes,
                                                                              margin, cap);
    return cudaGetLastError();
}

// Training: mean squared error over n_total samples. One block handles up
// to kTrainBlock samples (one per thread): forward with the activations kept
// in shared memory, then the gradient of every parameter summed over the
// block's samples and added to grad with one float atomic per parameter per
// block. loss receives sum((y - t)^2) / n_total.
constexpr int kTrainBlock = 128;

struct TrainSmem {
    float w[kParams];
    float h1[kTrainBlock][kH + 1];    // +1: rows of one thread fall in different banks
    float h2[kTrainBlock][kH + 1];
    float dz2[kTrainBlock][kH + 1];
    float dz1[kTrainBlock][kH + 1];
    float x[kTrainBlock][kIn];
    float dy[kTrainBlock];
};

__global__ void __launch_bounds__(kTrainBlock)
mlp_train_kernel(const float *theta, const float *X, const float *t, int64_t n, int64_t n_total,
                 float *grad, float *loss) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TrainSmem &S = *reinterpret_cast<TrainSmem *>(smem_raw);
    for (int i = threadIdx.x; i < kParams; i += blockDim.x) S.w[i] = theta[i];
    __syncthreads();
    const int s = threadIdx.x;
    const int64_t r = static_cast<int64_t>(blockIdx.x) * kTrainBlock + s;
    const bool valid = r < n;
    const float inv_n = 1.f / static_cast<float>(n_total);
    // forward: sample s on thread s, activations kept for the backward pass
#pragma unroll
    for (int f = 0; f < kIn; ++f) S.x[s][f] = valid ? X[kIn * r + f] : 0.f;
    for (int a = 0; a < kH; ++a) {
        float z = S.w[kOffB1 + a];
#pragma unroll
        for (int f = 0; f < kIn; ++f) z = fmaf(S.x[s][f], S.w[kOffW1 + f * kH + a], z);
        S.h1[s][a] = fmaxf(z, 0.f);
    }
    float y = S.w[kOffB3];
    for (int j = 0; j < kH; ++j) {
        float z = S.w[kOffB2 + j];
#pragma unroll 8
        for (int a = 0; a < kH; ++a) z = fmaf(S.h1[s][a], S.w[kOffW2 + a * kH + j], z);
        const float h = fmaxf(z, 0.f);
        S.h2[s][j] = h;
        y = fmaf(h, S.w[kOffW3 + j], y);
    }
    // backward of mean((y - t)^2)
    const float d = valid ? (y - t[r]) : 0.f;
    const float dy = 2.f * d * inv_n;
    S.dy[s] = dy;
    float lsum = d * d * inv_n;
    for (int j = 0; j < kH; ++j) S.dz2[s][j] = S.h2[s][j] > 0.f ? dy * S.w[kOffW3 + j] : 0.f;
    for (int a = 0; a < kH; ++a) {
        float dh = 0.f;
#pragma unroll 8
        for (int j = 0; j < kH; ++j) dh = fmaf(S.w[kOffW2 + a * kH + j], S.dz2[s][j], dh);
        S.dz1[s][a] = S.h1[s][a] > 0.f ? dh : 0.f;
    }
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, lsum);
    __syncthreads();
    // every parameter's gradient summed over the block's samples
    for (int p = threadIdx.x; p < kParams; p += blockDim.x) {
        float g = 0.f;
        if (p < kOffB1) {                      // W1[f][a]: x[f] dz1[a]
            const int f = p / kH, a = p % kH;
            for (int q = 0; q < kTrainBlock; ++q) g = fmaf(S.x[q][f], S.dz1[q][a], g);
        } else if (p < kOffW2) {               // b1[a]: dz1[a]
            const int a = p - kOffB1;
            for (int q = 0; q < kTrainBlock; ++q) g += S.dz1[q][a];
        } else if (p < kOffB2) {               // W2[a][j]: h1[a] dz2[j]
            const int a = (p - kOffW2) / kH, j = (p - kOffW2) % kH;
            for (int q = 0; q < kTrainBlock; ++q) g = fmaf(S.h1[q][a], S.dz2[q][j], g);
        } else if (p < kOffW3) {               // b2[j]: dz2[j]
            const int j = p - kOffB2;
            for (int q = 0; q < kTrainBlock; ++q) g += S.dz2[q][j];
        } else if (p < kOffB3) {               // w3[j]: dy h2[j]
            const int j = p - kOffW3;
            for (int q = 0; q < kTrainBlock; ++q) g = fmaf(S.dy[q], S.h2[q][j], g);
        } else {                               // b3: dy
            for (int q = 0; q < kTrainBlock; ++q) g += S.dy[q];
        }
        atomicAdd(grad + p, g);
    }
}

cudaError_t launch_mlp_train(const float *theta, const float *X, const float *t, int64_t n,
                             int64_t n_total, float *grad, float *loss, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void *>(&mlp_train_kernel),
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(sizeof(TrainSmem)));
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    mlp_train_kernel<<<static_cast<unsigned>((n + kTrainBlock - 1) / kTrainBlock), kTrainBlock,
                       sizeof(TrainSmem), s>>>(theta, X, t, n, n_total, grad, loss);
    return cudaGetLastError();
}

// Adam (Kingma & Ba) with bias correction; step counts from 1.
__global__ void adam_kernel(float *theta, const float *grad, float *m, float *v, int n, int step,
                            float lr, float b1, float b2, float eps) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = grad[i];
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / (1.f - powf(b1, static_cast<float>(step)));
    const float vh = vi / (1.f - powf(b2, static_cast<float>(step)));
    theta[i] -= lr * mh / (sqrtf(vh) + eps);
}

cudaError_t launch_adam(float *theta, const float *grad, float *m, float *v, int n, int step,
                        float lr, float b1, float b2, float eps, cudaStream_t s) {
    adam_kernel<<<(n + 255) / 256, 256, 0, s>>>(theta, grad, m, v, n, step, lr, b1, b2, eps);
    return cudaGetLastError();
}

// Sizes for the learned binning: rows past the symbolic hash bins go to
// the exact path (a huge size); others get min(prediction, n_prod), since a
// row never has more distinct keys than products.
// Sizes for the binning by prediction: rows whose n_prod passes exact_above
// go to the exact path (huge); the others take their class's factor on the
// predicted size (class = bin of the prediction), at least 1 and at most
// n_prod (an upper bound of n_nz). Each block counts its rows per class that
// land in a hash bin (tried in one phase) into the feedback counters.
__global__ void __launch_bounds__(256)
learned_sizes_kernel(const int64_t *nprod, const long long *pred, int64_t n, long long exact_above,
                     long long huge, int64_t *sizes, SizeFactors sf, uint8_t *cls,
                     unsigned long long *fb) {
    __shared__ unsigned hist[kMaxBins];
    if (threadIdx.x < kMaxBins) hist[threadIdx.x] = 0u;
    __syncthreads();
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) {
        const long long np = nprod[i];
        const long long p = pred[i];
        int b = 0;
        while (b < sf.nb - 1 && p > sf.lim[b]) ++b;
        long long sz = huge;
        if (np <= exact_above) {
            const int k = sf.k[b];
            long long q = k >= 0 ? (p << k) : ((p + (1ll << -k) - 1) >> -k);
            if (q < 1) q = 1;
            sz = q < np ? q : np;
            if (b < sf.nb - 1 && sz <= sf.lim[sf.nb - 2]) atomicAdd(&hist[b], 1u);
        }
        sizes[i] = sz;
        cls[i] = static_cast<uint8_t>(b);
    }
    __syncthreads();
    if (fb && threadIdx.x < kMaxBins && hist[threadIdx.x] > 0u)
        atomicAdd(fb + threadIdx.x * kLoadSlots + blockIdx.x % kLoadSlots,
                  static_cast<unsigned long long>(hist[threadIdx.x]));
}

cudaError_t launch_learned_sizes(const int64_t *nprod, const long long *pred, int64_t n,
                                 long long exact_above, long long huge, int64_t *sizes,
                                 const SizeFactors &sf, uint8_t *cls, unsigned long long *fb,
                                 cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    if (sf.nb < 1 || sf.nb > kMaxBins) return cudaErrorInvalidValue;
    learned_sizes_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(
        nprod, pred, n, exact_above, huge, sizes, sf, cls, fb);
    return cudaGetLastError();
}

}  // namespace ops

// --- stateless C ABI of the predictor ------------------------------------------
#include "opsparse.h"

using namespace ops;

extern "C" {

int spgemm_mlp_param_count(void) { return kParams; }

int spgemm_features(const spgemm_csr_in *A, const spgemm_csr_in *B, int64_t row_begin,
                    int64_t row_end, float *X, void *workspace, void *stream) {
    if (!A || !B || !X || !workspace) return SPGEMM_ERR_INVALID;
    if (A->cols != B->rows) return SPGEMM_ERR_SHAPE;
    if (row_begin < 0 || row_end < row_begin || row_end > A->rows) return SPGEMM_ERR_INVALID;
    if (!A->rpt || !B->rpt || (A->nnz > 0 && !A->col)) return SPGEMM_ERR_INVALID;
    Operands op;
    op.arpt = A->rpt; op.a64 = A->rpt_is_i64 ? 1 : 0; op.acol = A->col; op.aval = nullptr;
    op.brpt = B->rpt; op.b64 = B->rpt_is_i64 ? 1 : 0; op.bcol = B->col; op.bval = nullptr;
    op.row0 = row_begin; op.mw = row_end - row_begin; op.ncols = B->cols;
    unsigned char *ws = static_cast<unsigned char *>(workspace);
    long long *np = reinterpret_cast<long long *>(ws);
    unsigned *mx = reinterpret_cast<unsigned *>(ws + sizeof(long long) * (size_t)op.mw);
    unsigned *mn = mx + op.mw;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return launch_features(op, A->rows, np, mx, mn, X, sms * 8, static_cast<cudaStream_t>(stream)) ==
                   cudaSuccess
               ? SPGEMM_OK
               : SPGEMM_ERR_CUDA;
}

int spgemm_mlp_forward(const float *theta, const float *X, int64_t n, float *y, void *stream) {
    if (!theta || (n > 0 && (!X || !y)) || n < 0) return SPGEMM_ERR_INVALID;
    return launch_mlp_forward(theta, X, n, y, nullptr, 0.f, 0, static_cast<cudaStream_t>(stream)) ==
                   cudaSuccess
               ? SPGEMM_OK
               : SPGEMM_ERR_CUDA;
}

int spgemm_mlp_train_step(const float *theta, const float *X, const float *t, int64_t n,
                          int64_t n_total, float *grad, float *loss, void *stream) {
    if (!theta || !grad || !loss || n < 0 || n_total < n || n_total <= 0) return SPGEMM_ERR_INVALID;
    if (n > 0 && (!X || !t)) return SPGEMM_ERR_INVALID;
    return launch_mlp_train(theta, X, t, n, n_total, grad, loss, static_cast<cudaStream_t>(stream)) ==
                   cudaSuccess
               ? SPGEMM_OK
               : SPGEMM_ERR_CUDA;
}

int spgemm_mlp_adam(float *theta, const float *grad, float *m, float *v, int step, float lr,
                    float beta1, float beta2, float eps, void *stream) {
    if (!theta || !grad || !m || !v || step < 1) return SPGEMM_ERR_INVALID;
    return launch_adam(theta, grad, m, v, kParams, step, lr, beta1, beta2, eps,
                       static_cast<cudaStream_t>(stream)) == cudaSuccess
               ? SPGEMM_OK
               : SPGEMM_ERR_CUDA;
}

}  // extern "C"
