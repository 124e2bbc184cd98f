// Weight-blob parser and BN folding (host only, no CUDA).
#include "host_model.h"

#include <cmath>

namespace tabnet {

namespace {

constexpr uint32_t kMagic = 0x4E424154u;  // "TABN"
constexpr uint32_t kVersion = 1;
constexpr uint32_t kHeaderBytes = 96;
constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;

uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

struct Reader {
    const uint8_t* p;
    size_t left;
    bool ok = true;
    template <typename T>
    void take(std::vector<T>& v, size_t n) {
        if (!ok || n * sizeof(T) > left) { ok = false; return; }
        v.resize(n);
        if (n) std::memcpy(v.data(), p, n * sizeof(T));
        p += n * sizeof(T);
        left -= n * sizeof(T);
    }
    void bn(BN& b, size_t n) { take(b.mean, n); take(b.var, n); take(b.weight, n); take(b.bias, n); }
};

}  // namespace

uint64_t payload_hash(const uint8_t* p, size_t bytes) {
    uint64_t h = 0;
    size_t words = bytes / 4;
    for (size_t i = 0; i < words; ++i) {
        uint32_t w;
        std::memcpy(&w, p + 4 * i, 4);
        h += mix64((uint64_t)w ^ ((uint64_t)(i + 1) * kGolden));
    }
    return h;
}

GluLayer HostModel::layer(int s, int l) const {
    GluLayer g;
    const int N = n_hidden();
    if (l < dims.n_shared) {
        g.w = &shared_fc[l];
        g.k = (l == 0) ? dims.d_emb : N;
        g.bn = &ft_shared_bn[s][l];
    } else {
        int j = l - dims.n_shared;
        g.w = &ft_indep_fc[s][j];
        g.k = (l == 0) ? dims.d_emb : N;
        g.bn = &ft_indep_bn[s][j];
    }
    return g;
}

void HostModel::feature_columns(std::vector<int>& col, std::vector<int>& len) const {
    col.clear();
    len.clear();
    for (int c = 0; c < dims.n_num; ++c) { col.push_back(c); len.push_back(1); }
    int c = dims.n_num;
    for (int j = 0; j < dims.n_cat; ++j) { col.push_back(c); len.push_back(cat_emb_dim[j]); c += cat_emb_dim[j]; }
}

int parse_blob(const void* blob, size_t bytes, HostModel* m, std::string* why) {
    if (!blob || !m) { if (why) *why = "null pointer"; return TABNET_ERR_ARG; }
    const uint8_t* b = static_cast<const uint8_t*>(blob);
    if (bytes < 16) { if (why) *why = "blob shorter than a header"; return TABNET_ERR_BLOB_SIZE; }
    uint32_t magic, version, header_bytes;
    std::memcpy(&magic, b, 4);
    std::memcpy(&version, b + 4, 4);
    std::memcpy(&header_bytes, b + 8, 4);
    if (magic != kMagic) { if (why) *why = "bad magic"; return TABNET_ERR_BLOB_MAGIC; }
    if (version != kVersion) { if (why) *why = "unsupported blob version"; return TABNET_ERR_BLOB_VERSION; }
    if (header_bytes != kHeaderBytes || bytes < kHeaderBytes) {
        if (why) *why = "bad header size"; return TABNET_ERR_BLOB_SIZE;
    }
    uint64_t payload_bytes, hash;
    std::memcpy(&payload_bytes, b + 16, 8);
    std::memcpy(&hash, b + 24, 8);
    int32_t f[8];
    std::memcpy(f, b + 32, 32);
    double gamma, eps;
    std::memcpy(&gamma, b + 64, 8);
    std::memcpy(&eps, b + 72, 8);
    if (payload_bytes != bytes - kHeaderBytes || payload_bytes % 4) {
        if (why) *why = "payload size does not match the header"; return TABNET_ERR_BLOB_SIZE;
    }
    tabnet_dims& d = m->dims;
    d.n_num = f[0]; d.n_cat = f[1]; d.n_d = f[2]; d.n_a = f[3]; d.n_steps = f[4];
    d.n_shared = f[5]; d.n_indep = f[6]; d.n_classes = f[7];
    d.gamma = gamma; d.bn_eps = eps;
    d.content_hash = hash;
    if (d.n_num < 0 || d.n_cat < 0 || d.n_num + d.n_cat < 1 || d.n_num > 4096 || d.n_cat > 4096 ||
        d.n_d < 1 || d.n_a < 1 || d.n_d > 4096 || d.n_a > 4096 || d.n_steps < 1 || d.n_steps > 256 ||
        d.n_shared < 0 || d.n_indep < 0 || d.n_shared + d.n_indep < 1 || d.n_shared + d.n_indep > 64 ||
        d.n_classes < 1 || d.n_classes > 4096 || !(gamma >= 1.0 && gamma < 1e6) || !(eps >= 0.0 && eps < 1.0)) {
        if (why) *why = "shape field out of range";
        return TABNET_ERR_UNSUPPORTED_DIMS;
    }
    if (payload_hash(b + kHeaderBytes, payload_bytes) != hash) {
        if (why) *why = "payload hash mismatch"; return TABNET_ERR_BLOB_HASH;
    }
    Reader r{b + kHeaderBytes, (size_t)payload_bytes};
    r.take(m->cat_card, d.n_cat);
    r.take(m->cat_emb_dim, d.n_cat);
    if (!r.ok) { if (why) *why = "payload truncated"; return TABNET_ERR_BLOB_SIZE; }
    int64_t de = d.n_num;
    for (int j = 0; j < d.n_cat; ++j) {
        if (m->cat_card[j] < 1 || m->cat_card[j] > (1 << 24) || m->cat_emb_dim[j] < 1 || m->cat_emb_dim[j] > 64) {
            if (why) *why = "categorical cardinality or embedding dim out of range";
            return TABNET_ERR_UNSUPPORTED_DIMS;
        }
        de += m->cat_emb_dim[j];
    }
    if (de > 8192) { if (why) *why = "embedded width too large"; return TABNET_ERR_UNSUPPORTED_DIMS; }
    d.d_emb = (int32_t)de;
    d.n_feat = d.n_num + d.n_cat;
    const int N = d.n_d + d.n_a;
    m->emb.resize(d.n_cat);
    for (int j = 0; j < d.n_cat; ++j) r.take(m->emb[j], (size_t)m->cat_card[j] * m->cat_emb_dim[j]);
    r.bn(m->bn0, de);
    m->shared_fc.resize(d.n_shared);
    for (int l = 0; l < d.n_shared; ++l) r.take(m->shared_fc[l], (size_t)2 * N * (l == 0 ? de : N));
    const int nft = d.n_steps + 1;
    m->ft_shared_bn.assign(nft, {});
    m->ft_indep_fc.assign(nft, {});
    m->ft_indep_bn.assign(nft, {});
    for (int s = 0; s < nft; ++s) {
        m->ft_shared_bn[s].resize(d.n_shared);
        for (int l = 0; l < d.n_shared; ++l) r.bn(m->ft_shared_bn[s][l], 2 * N);
        m->ft_indep_fc[s].resize(d.n_indep);
        m->ft_indep_bn[s].resize(d.n_indep);
        for (int l = 0; l < d.n_indep; ++l) {
            int k = (d.n_shared == 0 && l == 0) ? (int)de : N;
            r.take(m->ft_indep_fc[s][l], (size_t)2 * N * k);
            r.bn(m->ft_indep_bn[s][l], 2 * N);
        }
    }
    m->att_fc.resize(d.n_steps);
    m->att_bn.resize(d.n_steps);
    for (int i = 0; i < d.n_steps; ++i) {
        r.take(m->att_fc[i], (size_t)de * d.n_a);
        r.bn(m->att_bn[i], de);
    }
    r.take(m->final_w, (size_t)d.n_classes * d.n_d);
    r.take(m->final_b, d.n_classes);
    if (!r.ok) { if (why) *why = "payload truncated"; return TABNET_ERR_BLOB_SIZE; }
    if (r.left != 0) { if (why) *why = "trailing bytes after the payload"; return TABNET_ERR_BLOB_SIZE; }
    return TABNET_OK;
}

void fold_bn(const BN& bn, double eps, std::vector<float>& scale, std::vector<float>& shift) {
    size_t n = bn.mean.size();
    scale.resize(n);
    shift.resize(n);
    for (size_t i = 0; i < n; ++i) {
        double s = (double)bn.weight[i] / std::sqrt((double)bn.var[i] + eps);
        scale[i] = (float)s;
        shift[i] = (float)((double)bn.bias[i] - (double)bn.mean[i] * s);
    }
}

}  // namespace tabnet
