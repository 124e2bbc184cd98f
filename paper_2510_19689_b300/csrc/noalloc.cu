// Segmented launch that allocates nothing: the only scratch the segmented
// path needs -- the prefix sums of the segments' row counts -- lives in a
// file-scope device array instead of memory the library would cudaMalloc.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/tabnet.h"
#include "kernel_params.h"
#include "model_handle.h"

namespace tabnet {

// tabnet_abi.cu
int forward_impl(tabnet_model* m, const float* x_num, const int32_t* x_cat, int64_t rows, float* logits,
                 float* masks, float* agg, cudaStream_t stream, const SegTable* seg);
int set_last_error(int code, const std::string& why);
// segments.cu
cudaError_t seg_prefix_launch(const tabnet_segment* segs, int n, int64_t* prefix, cudaStream_t stream);

namespace {

// (TABNET_NOALLOC_MAX_SEGMENTS + 1) prefix sums.  Every GPU that loads the
// library holds this array (512 KB) until the process exits.  All calls on a
// device share it; the scan kernel rewrites every entry a launch reads, so no
// entry has to start at zero.
static __device__ __align__(256) int64_t g_noalloc_prefix[TABNET_NOALLOC_MAX_SEGMENTS + 1];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
int64_t* g_prefix_ptr[kMaxDevices] = {};  // device address of the array, looked up once per device

// The array's device address on `device`, which must be the current device.
// The name g_noalloc_prefix in host code is only a host-side stand-in, so the
// address is taken from the runtime the first time a device is used.
int prefix_address(int device, int64_t** out) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (device < 0 || device >= kMaxDevices) return set_last_error(TABNET_ERR_ARG, "device ordinal out of range");
    if (!g_prefix_ptr[device]) {
        int64_t* ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void**>(&ptr), g_noalloc_prefix);
        if (e != cudaSuccess || ptr == nullptr)
            return set_last_error(TABNET_ERR_CUDA, std::string("cudaGetSymbolAddress(prefix scratch): ") +
                                                       cudaGetErrorString(e));
        g_prefix_ptr[device] = ptr;
    }
    *out = g_prefix_ptr[device];
    return TABNET_OK;
}

}  // namespace

}  // namespace tabnet

using namespace tabnet;

extern "C" int tabnet_forward_segments_noalloc(tabnet_model* m, const tabnet_segment* segs, int n_segs,
                                               void* stream) {
    if (!m || n_segs < 0) return set_last_error(TABNET_ERR_ARG, "null model or negative count");
    if (n_segs == 0) return TABNET_OK;
    if (!segs) return set_last_error(TABNET_ERR_ARG, "segs is NULL");
    if (n_segs > TABNET_NOALLOC_MAX_SEGMENTS)
        return set_last_error(TABNET_ERR_ARG, "n_segs " + std::to_string(n_segs) +
                                                  " exceeds the fixed scratch of TABNET_NOALLOC_MAX_SEGMENTS = " +
                                                  std::to_string(TABNET_NOALLOC_MAX_SEGMENTS) + " segments");
    int prev = -1;
    cudaError_t e = cudaGetDevice(&prev);
    if (e != cudaSuccess) return set_last_error(TABNET_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (prev != m->device && (e = cudaSetDevice(m->device)) != cudaSuccess)
        return set_last_error(TABNET_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    int64_t* prefix = nullptr;
    int rc = prefix_address(m->device, &prefix);
    if (rc == TABNET_OK) {
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        e = seg_prefix_launch(segs, n_segs, prefix, s);
        if (e != cudaSuccess) {
            rc = set_last_error(TABNET_ERR_CUDA, std::string("segment prefix launch: ") + cudaGetErrorString(e));
        } else {
            const SegTable t{segs, prefix, n_segs};
            rc = forward_impl(m, nullptr, nullptr, 0, nullptr, nullptr, nullptr, s, &t);
        }
    }
    if (prev != m->device) cudaSetDevice(prev);
    return rc;
}
