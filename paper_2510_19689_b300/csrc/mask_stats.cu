// Per-feature statistics of aggregated feature masks over a window of rows,
// and the agreement of two aggregates' top-k feature sets: the audit signal
// of interpretability under load (Sec. V-C) -- which features carry the
// decisions, and whether their ranking holds when rows are served alone, in
// a mixed batch or at another precision.
//
// All of it reads the [rows][d] float32 aggregate that tabnet_forward writes
// and is memory-bound (one or two passes over it).  Means and variances are
// deterministic: each CTA sums a fixed block of rows per feature with
// compensated (Kahan) summation, and one CTA per feature adds the per-CTA
// partials in a fixed pairwise tree.  Top-k counts are integers.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "../../include/tabnet.h"

namespace tabnet {

int set_last_error(int code, const std::string& why);

namespace {

constexpr int kBlocks = 1184;     // partial sums per feature (8 per SM on 148 SMs)
constexpr int kMaxD = 1024;       // features per row the kernels take
constexpr int kMaxK = 32;         // largest top-k

struct Kahan {
    float s = 0.f, c = 0.f;
    __device__ void add(float x) {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

// Partial sums of agg[r][j] (center == nullptr) or of (agg[r][j] - center[j])^2
// over CTA b's rows, one thread per feature: a warp reads a row's features
// as one contiguous piece.
__global__ void partial_kernel(const float* __restrict__ agg, int64_t rows, int d,
                               const float* __restrict__ center, float* __restrict__ part) {
    const int j = threadIdx.x;
    const int64_t per = (rows + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = (int64_t)blockIdx.x * per, r1 = min(rows, r0 + per);
    if (j >= d) return;
    const float mu = center ? center[j] : 0.f;
    Kahan k;
    for (int64_t r = r0; r < r1; ++r) {
        const float x = __ldg(agg + r * d + j);
        if (center) {
            const float e = x - mu;
            k.add(e * e);
        } else {
            k.add(x);
        }
    }
    part[(size_t)blockIdx.x * d + j] = k.s;
}

// out[j] = (sum over the kBlocks partials of feature j) / rows, pairwise in a
// fixed order (one CTA of 1024 threads per feature).
__global__ void finish_kernel(const float* __restrict__ part, int d, int64_t rows, float* __restrict__ out) {
    __shared__ float s[1024];
    const int j = blockIdx.x, t = threadIdx.x;
    float v = 0.f;
    for (int b = t; b < kBlocks; b += 1024) v += part[(size_t)b * d + j];  // at most two terms
    s[t] = v;
    __syncthreads();
    for (int h = 512; h > 0; h >>= 1) {
        if (t < h) s[t] += s[t + h];
        __syncthreads();
    }
    if (t == 0) out[j] = s[0] / (float)rows;
}

// The k largest entries of row x (ties: the lower index first), as a bit set
// over d <= kMaxD features in `sel` (kMaxD / 32 words).
__device__ void topk_row(const float* __restrict__ x, int d, int k, uint32_t* sel) {
    for (int w = 0; w < kMaxD / 32; ++w) sel[w] = 0u;
    for (int i = 0; i < k; ++i) {
        int best = -1;
        float bv = 0.f;
        for (int j = 0; j < d; ++j) {
            if ((sel[j >> 5] >> (j & 31)) & 1u) continue;
            const float v = __ldg(x + j);
            if (best < 0 || v > bv) { best = j; bv = v; }  // strict: an equal later entry does not win
        }
        sel[best >> 5] |= 1u << (best & 31);
    }
}

// counts[j] += number of rows whose top-k holds j (a row per thread).
__global__ void topk_count_kernel(const float* __restrict__ agg, int64_t rows, int d, int k,
                                  unsigned long long* __restrict__ counts) {
    __shared__ unsigned int c[kMaxD];
    for (int j = threadIdx.x; j < d; j += blockDim.x) c[j] = 0u;
    __syncthreads();
    uint32_t sel[kMaxD / 32];
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x) {
        topk_row(agg + r * d, d, k, sel);
        for (int w = 0; w < (d + 31) / 32; ++w) {
            uint32_t m = sel[w];
            while (m) {
                const int b = __ffs(m) - 1;
                m &= m - 1;
                atomicAdd(&c[w * 32 + b], 1u);
            }
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < d; j += blockDim.x)
        if (c[j]) atomicAdd(counts + j, (unsigned long long)c[j]);
}

// hits += sum over rows of |topk(a_r) & topk(b_r)|.
__global__ void topk_agree_kernel(const float* __restrict__ a, const float* __restrict__ b, int64_t rows, int d,
                                  int k, unsigned long long* __restrict__ hits) {
    uint32_t sa[kMaxD / 32], sb[kMaxD / 32];
    unsigned long long h = 0;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x) {
        topk_row(a + r * d, d, k, sa);
        topk_row(b + r * d, d, k, sb);
        for (int w = 0; w < (d + 31) / 32; ++w) h += __popc(sa[w] & sb[w]);
    }
    if (h) atomicAdd(hits, h);
}

__global__ void frac_kernel(const unsigned long long* __restrict__ counts, int n, double denom, float* __restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) out[j] = (float)((double)counts[j] / denom);
}

int check_common(const void* agg, int64_t rows, int d, int k) {
    if (!agg) return set_last_error(TABNET_ERR_ARG, "aggregate pointer is NULL");
    if (rows < 1) return set_last_error(TABNET_ERR_ARG, "rows must be >= 1");
    if (d < 1 || d > kMaxD) return set_last_error(TABNET_ERR_ARG, "d must be in [1, 1024]");
    if (k < 1 || k > d || k > kMaxK) return set_last_error(TABNET_ERR_ARG, "k must be in [1, min(d, 32)]");
    return TABNET_OK;
}

int cuda_fail(cudaError_t e, const char* where) {
    return set_last_error(TABNET_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

}  // namespace

}  // namespace tabnet

using namespace tabnet;

extern "C" int tabnet_mask_stats(const float* agg, int64_t rows, int d, int k, float* mean, float* var,
                                 float* topk_frac, void* stream) {
    int rc = check_common(agg, rows, d, k);
    if (rc != TABNET_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    float* part = nullptr;
    float* mu = nullptr;
    unsigned long long* counts = nullptr;
    const size_t part_bytes = sizeof(float) * (size_t)kBlocks * d;
    const int threads = (d + 31) / 32 * 32;
    if (mean || var) {
        if ((e = cudaMallocAsync((void**)&part, part_bytes, s)) != cudaSuccess) return cuda_fail(e, "cudaMallocAsync");
        mu = mean;
        if (!mu && (e = cudaMallocAsync((void**)&mu, sizeof(float) * d, s)) != cudaSuccess) {
            cudaFreeAsync(part, s);
            return cuda_fail(e, "cudaMallocAsync");
        }
        partial_kernel<<<kBlocks, threads, 0, s>>>(agg, rows, d, nullptr, part);
        finish_kernel<<<d, 1024, 0, s>>>(part, d, rows, mu);
        if (var) {
            partial_kernel<<<kBlocks, threads, 0, s>>>(agg, rows, d, mu, part);
            finish_kernel<<<d, 1024, 0, s>>>(part, d, rows, var);
        }
        e = cudaGetLastError();
        if (mu != mean) cudaFreeAsync(mu, s);
        cudaFreeAsync(part, s);
        if (e != cudaSuccess) return cuda_fail(e, "mask statistics launch");
    }
    if (topk_frac) {
        if ((e = cudaMallocAsync((void**)&counts, sizeof(unsigned long long) * d, s)) != cudaSuccess)
            return cuda_fail(e, "cudaMallocAsync");
        cudaMemsetAsync(counts, 0, sizeof(unsigned long long) * d, s);
        const int blocks = (int)std::min<int64_t>((rows + 255) / 256, 148 * 8);
        topk_count_kernel<<<blocks, 256, 0, s>>>(agg, rows, d, k, counts);
        frac_kernel<<<(d + 255) / 256, 256, 0, s>>>(counts, d, (double)rows, topk_frac);
        e = cudaGetLastError();
        cudaFreeAsync(counts, s);
        if (e != cudaSuccess) return cuda_fail(e, "top-k count launch");
    }
    return TABNET_OK;
}

extern "C" int tabnet_topk_agreement(const float* agg_a, const float* agg_b, int64_t rows, int d, int k,
                                     float* out, void* stream) {
    int rc = check_common(agg_a, rows, d, k);
    if (rc != TABNET_OK) return rc;
    if (!agg_b || !out) return set_last_error(TABNET_ERR_ARG, "NULL pointer");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned long long* hits = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&hits, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync");
    cudaMemsetAsync(hits, 0, sizeof(unsigned long long), s);
    const int blocks = (int)std::min<int64_t>((rows + 255) / 256, 148 * 8);
    topk_agree_kernel<<<blocks, 256, 0, s>>>(agg_a, agg_b, rows, d, k, hits);
    frac_kernel<<<1, 32, 0, s>>>(hits, 1, (double)rows * k, out);
    e = cudaGetLastError();
    cudaFreeAsync(hits, s);
    if (e != cudaSuccess) return cuda_fail(e, "top-k agreement launch");
    return TABNET_OK;
}
