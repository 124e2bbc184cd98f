// Parameter block of the tensor-core (tcgen05) forward kernel.
#pragma once

#include <cstdint>

#include "kernel_params.h"

namespace tabnet {

// Shared-memory layout of one CTA, byte offsets from a 1024-aligned base;
// an offset of -1 means the part is not staged (read from global instead).
struct TcSmem {
    int a_hi;   // A operand (activations, bf16, SW128 K-major, 16 KB per 64 K-columns)
    int a_lo;   // low halves of the split-bf16 A operand (-1 unless split)
    int ring;   // weight-staging ring: n_slots x slot_bytes
    int agg;    // aggregate per original feature, float [d][128] (-1: kept in TMEM)
    int xch;    // cross-warpgroup exchange, float2 [2][2][128] (-1 with one warpgroup)
    int wf;     // final linear weights, float [n_classes][n_d]
    int epi;    // every layer's folded BN scale/shift (-1: read from global)
    int fcache; // embedded, BN'd input of the tile, float [de][129] (-1: recomputed)
    int rowp;   // with fcache: the tile's row pointers, [128] x_num, [128] x_cat, [128] masks
    int mstage; // per-warp mask staging, float [warps][32][17] (-1: direct stores)
    int chunks; // the weight-chunk table, uint2 [chunks_per_tile]
    int colf;   // original feature of each embedded column, int [dp]
    int bar;    // mbarriers: n_slots full, n_slots empty, 1 accumulator; TMEM address; abort flag
    int total;  // bytes used (without the alignment slack)
};

struct TcParams {
    ModelConsts m;
    SegTable seg;              // segmented launch (seg.segs != nullptr) or one batch
    const uint8_t* wbase;      // packed weight chunks (device)
    const uint2* chunks;       // [chunks_per_tile] {byte offset from wbase, bytes}, stream order
    int chunks_per_tile;
    // Every layer's BN shift (the scale is folded into the packed weights) as
    // one float block: feature-transformer layer L = s * layers_per_ft + l at
    // L * 2N (shift[2N]), then the attentive layer of step i at
    // n_ft_layers * 2N + i * dp (shift[dp]).
    const float* epi;
    int epi_floats;
    const int2* col_info;      // [dp]: {-1, numeric column} | {categorical j, element e} | {-2, 0} pad
    const int* col_feat;       // [dp]: original feature of each embedded column (-1 for pad)
    int dp;                    // mask width padded to a multiple of 16
    int att_k0;                // first K step of the attentive layer (n_d / K step; the decision
                               // half's weights before it are zero)
    int ks_0;                  // K steps of a feature transformer's first layer (K = dp)
    int ks_n;                  // K steps of the other layers (K = N); a K step is 16 bf16 or
                               // 32 e4m3 elements
    int epi_sc;                // FP8: float offset in epi of the per-output-channel weight
                               // scales (laid out like the shifts); 0 otherwise
    int tmem_cols;             // TMEM columns allocated per CTA
    // P, the step mask and the aggregate are fp32 regions of dp columns, or
    // dp - 8 when the last 16-column chunk holds at most 8 mask columns (tail8)
    int tail8;
    int m16;                   // the step mask kept as fp16 pairs (dp / 2 columns): set only
                               // when the fp32 regions exceed the 512 TMEM columns
    int tm_p;                  // TMEM column of the prior P
    int tm_m;                  // TMEM column of the current step mask
    int tm_agg;                // TMEM column of the aggregate (-1: in shared memory)
    int n_slots;
    int slot_bytes;
    TcSmem sm;
};

}  // namespace tabnet
