// Segmented launches: prefix sums of the segments' row counts, computed on
// the device so that a launch over device-resident descriptors needs no host
// round trip (and can be captured in a CUDA graph).
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/tabnet.h"

namespace tabnet {

namespace {

constexpr int kScanThreads = 1024;

// prefix[i] = sum of max(rows, 0) over segments [0, i), for i = 0..n.
// One CTA: each thread sums a contiguous range, a shared-memory scan over the
// thread totals, then each thread writes its range.
__global__ void __launch_bounds__(kScanThreads) seg_prefix_kernel(const tabnet_segment* __restrict__ segs, int n,
                                                                  int64_t* __restrict__ prefix) {
    __shared__ int64_t part[kScanThreads];
    const int t = threadIdx.x;
    const int per = (n + kScanThreads - 1) / kScanThreads;
    const int lo = min(n, t * per), hi = min(n, lo + per);
    int64_t s = 0;
    for (int i = lo; i < hi; ++i) {
        const int64_t r = segs[i].rows;
        s += r > 0 ? r : 0;
    }
    part[t] = s;
    __syncthreads();
    // Hillis-Steele inclusive scan over the thread totals
    for (int off = 1; off < kScanThreads; off <<= 1) {
        const int64_t v = t >= off ? part[t - off] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int64_t run = part[t] - s;  // exclusive prefix of this thread's range
    for (int i = lo; i < hi; ++i) {
        prefix[i] = run;
        const int64_t r = segs[i].rows;
        run += r > 0 ? r : 0;
    }
    if (t == kScanThreads - 1) prefix[n] = part[t];
}

}  // namespace

cudaError_t seg_prefix_launch(const tabnet_segment* segs, int n, int64_t* prefix, cudaStream_t stream) {
    seg_prefix_kernel<<<1, kScanThreads, 0, stream>>>(segs, n, prefix);
    return cudaGetLastError();
}

}  // namespace tabnet
