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
    // 4-byte words from one input row to the next, for x_num and x_cat
    // alike (rows whose numeric and categorical columns are interleaved in
    // one buffer); 0: dense, n_num and n_cat words
    int in_stride = 0;
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
    // The warp-per-row kernel's copy of the layers: one unit per layer use
    // in forward order (feature transformer 0's layers, then for each step
    // its attentive layer and the next feature transformer's layers), unit u
    // at row_units + u * row_slot: the weight output-major, [ld][kp] (output
    // o's k weights contiguous, ld = n_out and kp = k rounded up as
    // row_r4 / row_kp give, zero-padded), then the BN scale [ld] and shift
    // [ld].
    const float* row_units;
    int row_slot;
};

#if defined(__CUDACC__)
#define TABNET_HD __host__ __device__
#else
#define TABNET_HD
#endif

TABNET_HD inline int row_r4(int n) { return (n + 3) & ~3; }
TABNET_HD inline int row_n_units(int lpf, int n_steps) { return lpf + n_steps * (1 + lpf); }
// Shape of unit u; *att_step = the step of an attentive unit, else -1, and
// *ft_layer = the index into SimtParams::ft of a feature-transformer unit.
TABNET_HD inline void row_unit_shape(int u, int lpf, int de, int N, int n_a, int* k, int* n_out, int* att_step,
                                     int* ft_layer) {
    int s = 0, l = u;
    if (u >= lpf) {
        const int v = u - lpf, j = v % (1 + lpf);
        s = v / (1 + lpf) + 1;
        if (j == 0) {
            *k = n_a;
            *n_out = de;
            *att_step = s - 1;
            *ft_layer = -1;
            return;
        }
        l = j - 1;
    }
    *k = l == 0 ? de : N;
    *n_out = 2 * N;
    *att_step = -1;
    *ft_layer = s * lpf + l;
}
// Floats of one unit slot: the largest unit.
// Row stride of a unit's weight: k rounded up to 4 floats, and to an odd
// number of 16-byte groups, so that eight consecutive outputs' float4 reads
// fall in eight different bank groups.
TABNET_HD inline int row_kp(int k) {
    const int kp = row_r4(k);
    return ((kp >> 2) & 1) ? kp : kp + 4;
}
// Floats of unit (k, n_out), and of one slot: the largest unit.
TABNET_HD inline int row_unit_floats(int k, int n_out) { return row_r4(n_out) * (row_kp(k) + 2); }
TABNET_HD inline int row_slot_floats(int de, int N, int n_a) {
    const int f0 = row_unit_floats(de, 2 * N), f1 = row_unit_floats(N, 2 * N), fa = row_unit_floats(n_a, de);
    const int ft = f0 > f1 ? f0 : f1;
    return ft > fa ? ft : fa;
}

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
    io.x_num = x_num ? x_num + r * (t.in_stride ? t.in_stride : m.n_num) : nullptr;
    io.x_cat = x_cat ? x_cat + r * (t.in_stride ? t.in_stride : m.n_cat) : nullptr;
    io.logits = logits + r * m.n_classes;
    io.masks = masks ? masks + r * (int64_t)m.n_steps * m.de : nullptr;
    io.agg = agg ? agg + r * m.d : nullptr;
    return io;
}
#endif

}  // namespace tabnet
