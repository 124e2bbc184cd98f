// Host-side model: the weight blob parsed into plain arrays, plus the
// folding of inference-mode batch norm into per-channel scale/shift pairs.
//
// Blob format version 1 (little-endian): a 96-byte header
//   u32 magic "TABN", u32 version, u32 header_bytes, u32 flags,
//   u64 payload_bytes, u64 payload_hash,
//   i32 n_num, n_cat, n_d, n_a, n_steps, n_shared, n_indep, n_classes,
//   f64 gamma, f64 bn_eps, 16 reserved bytes,
// then the payload: cat_card[n_cat], cat_emb_dim[n_cat] (i32), and float32
// arrays in this order: embedding tables, input BN {mean, var, weight, bias},
// shared FC weights [2N, K], per feature transformer s = 0..n_steps its
// shared-layer BNs and its (FC [2N, K], BN) step layers, per decision step
// the attentive FC [D_e, n_a] and BN, the final W_f [C, n_d] and b_f [C].
#pragma once

#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/tabnet.h"

namespace tabnet {

struct BN {
    std::vector<float> mean, var, weight, bias;
};

// One GLU layer of one feature transformer: weights [n_out, k] and its BN.
struct GluLayer {
    const std::vector<float>* w = nullptr;  // points into HostModel storage
    int k = 0;
    const BN* bn = nullptr;
};

struct HostModel {
    tabnet_dims dims{};
    std::vector<int32_t> cat_card, cat_emb_dim;
    std::vector<std::vector<float>> emb;       // [card_j * emb_dim_j]
    BN bn0;                                    // [D_e]
    std::vector<std::vector<float>> shared_fc; // [2N * K_l]
    std::vector<std::vector<BN>> ft_shared_bn; // [n_steps+1][n_shared]
    std::vector<std::vector<std::vector<float>>> ft_indep_fc;  // [n_steps+1][n_indep]
    std::vector<std::vector<BN>> ft_indep_bn;  // [n_steps+1][n_indep]
    std::vector<std::vector<float>> att_fc;    // [n_steps][D_e * n_a]
    std::vector<BN> att_bn;                    // [n_steps]
    std::vector<float> final_w, final_b;       // [C * n_d], [C]

    int n_hidden() const { return dims.n_d + dims.n_a; }
    // Layer l (0-based) of feature transformer s, in execution order.
    GluLayer layer(int s, int l) const;
    int layers_per_ft() const { return dims.n_shared + dims.n_indep; }
    // First embedded column of every original feature, and its width.
    void feature_columns(std::vector<int>& col, std::vector<int>& len) const;
};

// Payload hash: sum over u32 words w_i (i from 1) of mix64(w_i ^ i * golden).
uint64_t payload_hash(const uint8_t* p, size_t bytes);

// Parse and validate.  Returns TABNET_OK or a TABNET_ERR_* code; `why`
// receives a one-line reason on failure.
int parse_blob(const void* blob, size_t bytes, HostModel* out, std::string* why);

// Inference BN as y = scale * x + shift, computed in double and rounded to
// float once: scale = w / sqrt(var + eps), shift = b - mean * scale.
void fold_bn(const BN& bn, double eps, std::vector<float>& scale, std::vector<float>& shift);

}  // namespace tabnet
