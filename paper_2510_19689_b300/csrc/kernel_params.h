// Parameter blocks shared by the host launcher and the device kernels.
// Every pointer is device memory owned by the model handle.
#pragma once

#include <cstdint>

#include "../../include/tabnet.h"

namespace tabnet {

// Rows of several requests packed back to back (segmented launch); segs ==
// nullptr means one contiguous batch given by the kernel arguments.
struct SegTable {
    const tabnet_segment* segs;  // [n] device copy of the descriptors
    const int64_t* prefix;       // [n + 1] exclusive prefix sums of the rows
    int n;
};

// Where one packed row reads its inputs and writes its outputs.
struct RowIO {
    const float* x_num;
    const int* x_cat;
    float* logits;
    float* masks;  // the row's [n_steps, de] block, or null
    float* agg;    // the row's [d] block, or null
    bool valid;
};

// Per-model constants used by every kernel variant.  BN is already folded:
// input BN becomes (s0, t0) for numeric columns and is baked into the
// embedding tables for categorical ones.
struct ModelConsts {
    int n_num, n_cat, de, d, n_d, n_a, N, n_steps, layers_per_ft, n_classes;
    float gamma;
    const float* s0;        // [de] input-BN scale
    const float* t0;        // [de] input-BN shift (also the value of an out-of-range
                            //      categorical index, whose embedding row is taken as 0)
    const float* emb;       // folded embedding tables, concatenated
    const int* cat_off;     // [n_cat] float offset of table j in emb
    const int* cat_card;    // [n_cat]
    const int* cat_base;    // [n_cat] raw code of each column's index 0 (the caller's
                            //      label/ordinal encoding, tabnet_set_input_transform)
    const int* feat_col;    // [d] first embedded column of feature j
    const int* feat_len;    // [d] embedded width of feature j
    const float* wf;        // [n_classes, n_d]
    const float* bf;        // [n_classes]
    unsigned* status;       // device status: [0] TABNET_STATUS_* bits, [1] first timeout
                            // location (kind << 24 | index), [2] its block
};

// FP32 SIMT path: one layer = transposed weights plus folded BN.
struct SimtLayer {
    const float* wt;     // [k][n_out] (k-major: output index fastest)
    const float* scale;  // [n_out]
    const float* shift;  // [n_out]
    int k, n_out;
};

struct SimtParams {
    ModelConsts m;
    SegTable seg;
    const SimtLayer* ft;   // [(n_steps + 1) * layers_per_ft], FT s layer l at s * lpf + l
    const SimtLayer* att;  // [n_steps]
};

#ifdef __CUDACC__
// Total rows of a launch: the batch size, or the last prefix sum.
__device__ __forceinline__ int64_t total_rows(const SegTable& t, int64_t rows) {
    return t.segs ? t.prefix[t.n] : rows;
}

// Resolve packed row gr to its buffers (binary search over the prefix sums
// for a segmented launch).
__device__ __forceinline__ RowIO row_io(const SegTable& t, const ModelConsts& m, int64_t gr, int64_t total,
                                        const float* x_num, const int* x_cat, float* logits, float* masks,
                                        float* agg) {
    RowIO io;
    io.valid = gr < total;
    int64_t r = io.valid ? gr : 0;
    if (t.segs) {
        int lo = 0, hi = t.n;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (t.prefix[mid] <= r) lo = mid; else hi = mid;
        }
        const tabnet_segment sg = t.segs[lo];
        r -= t.prefix[lo];
        if (!io.valid) r = 0;
        x_num = sg.x_num;
        x_cat = sg.x_cat;
        logits = sg.logits;
        masks = sg.step_masks;
        agg = sg.agg_mask;
    }
    io.x_num = x_num ? x_num + r * m.n_num : nullptr;
    io.x_cat = x_cat ? x_cat + r * m.n_cat : nullptr;
    io.logits = logits + r * m.n_classes;
    io.masks = masks ? masks + r * (int64_t)m.n_steps * m.de : nullptr;
    io.agg = agg ? agg + r * m.d : nullptr;
    return io;
}
#endif

}  // namespace tabnet
