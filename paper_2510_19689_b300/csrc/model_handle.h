// The opaque tabnet_model handle and the pieces shared by the ABI and the
// per-precision packers/launchers.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "host_model.h"
#include "kernel_params.h"
#include "tc_params.h"

namespace tabnet {

// Host image of the device arena: every constant array of a model is laid
// out here first, then copied with one cudaMemcpy.
struct Arena {
    std::vector<uint8_t> image;
    size_t add(const void* data, size_t bytes, size_t align = 16);
};

struct ConstOffsets {
    size_t s0, t0, emb, cat_off, cat_card, cat_base, feat_col, feat_len, wf, bf;
};

// Launch shape of the tensor-core kernel (chosen by the host heuristics or
// by the autotuner through tabnet_set_tile_config).
struct TcLaunch {
    int nwg = 1;          // epilogue warpgroups per CTA (1 or 2)
    int n_slots = 2;      // weight-staging ring depth
    int ctas_per_sm = 1;  // resident CTAs per SM
    size_t smem = 0;      // dynamic shared memory per CTA
    bool zreg = false;    // sparsemax input held in registers
    bool lean = false;    // everything staged: the specialised kernel instantiation
};

}  // namespace tabnet

struct tabnet_model {
    tabnet::HostModel host;
    int device = 0;
    int precision = 0;
    int num_sms = 0;
    size_t smem_optin = 0;
    void* d_arena = nullptr;
    size_t arena_bytes = 0;
    unsigned* d_status = nullptr;
    tabnet::ConstOffsets consts_off{};
    tabnet::ModelConsts consts{};
    // FP32 path
    tabnet::SimtParams simt{};
    int simt_rows = 0;
    int simt_max_ctas = 0;
    int64_t simt_row_max = 0;  // calls of at most this many rows take the warp-per-row kernel
    // tensor-core path
    tabnet::TcParams tc{};
    tabnet::TcLaunch tc_launch_cfg{};
    // Set while the model is served next to other models (tabnet_server):
    // every tensor-core launch then takes shared memory in proportion to its
    // tensor-memory columns, so that CTAs of different kernels placed on one
    // SM always fit in its 512 columns.
    bool tmem_shared = false;
    size_t tc_off_chunks = 0, tc_off_epi = 0, tc_off_colinfo = 0, tc_off_colfeat = 0;
    std::vector<size_t> tc_chunk_off;          // arena offsets of the weight chunks, stream order
    std::vector<uint32_t> tc_chunk_bytes;
    // host-buffer forward workspace, and the streams that pipeline its
    // copies and launches over row chunks (created on first use)
    void* d_ws = nullptr;
    size_t ws_bytes = 0;
    static constexpr int kHostStreams = 4;
    cudaStream_t host_streams[kHostStreams] = {};
    cudaEvent_t host_done[kHostStreams] = {};
    cudaEvent_t host_start = nullptr;
    // segmented launches: device descriptors (host-staged calls) + prefix sums
    void* d_seg = nullptr;
    int seg_cap = 0;
    tabnet_segment* h_seg_stage = nullptr;  // pinned staging for host descriptors
    int seg_stage_cap = 0;
    cudaEvent_t seg_stage_done = nullptr;
};

namespace tabnet {

int tc_build(tabnet_model* m, Arena& a, std::string* why);
int tc_patch(tabnet_model* m, Arena& a, const uint8_t* base, std::string* why);
cudaError_t tc_launch(tabnet_model* m, const float* x_num, const int* x_cat, int64_t rows,
                      float* logits, float* masks, float* agg, cudaStream_t stream,
                      const SegTable* seg = nullptr);
void tc_release(tabnet_model* m);
int forward_interleaved(tabnet_model* m, const void* rows_in, int64_t rows, float* logits, float* step_masks,
                        float* agg_mask, cudaStream_t stream);
int tc_choose_launch(tabnet_model* m, int nwg, int n_slots, int ctas_per_sm, std::string* why);

}  // namespace tabnet
