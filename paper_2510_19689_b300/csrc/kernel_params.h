// Parameter blocks shared by the host launcher and the device kernels.
// Every pointer is device memory owned by the model handle.
#pragma once

#include <cstdint>

namespace tabnet {

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
    const SimtLayer* ft;   // [(n_steps + 1) * layers_per_ft], FT s layer l at s * lpf + l
    const SimtLayer* att;  // [n_steps]
};

}  // namespace tabnet
