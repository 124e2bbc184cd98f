// The C ABI: argument checks, model loading (parse, BN folding, packing,
// upload) and kernel dispatch.  No exception crosses the extern "C" edge.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/tabnet.h"
#include "host_model.h"
#include "kernel_params.h"
#include "model_handle.h"

namespace tabnet {

// simt_forward.cu
size_t simt_smem_bytes(const ModelConsts& m, int rows_per_cta);
cudaError_t simt_configure(int rows_per_cta, size_t smem);
cudaError_t simt_launch(const SimtParams& p, int rows_per_cta, const float* x_num, const int* x_cat,
                        int64_t rows, float* logits, float* masks, float* agg, cudaStream_t stream,
                        int max_ctas);
int simt_occupancy(int rows_per_cta, size_t smem);
cudaError_t simt_row_configure(size_t smem);
bool simt_row_plan(const ModelConsts& m, int64_t rows, int num_sms, int w_max, size_t smem_max, int* W, int* nbuf);
cudaError_t simt_row_launch(const SimtParams& p, const float* x_num, const int* x_cat, int64_t rows, float* logits,
                            float* masks, float* agg, cudaStream_t stream, int num_sms, int w_max, size_t smem_max);
// rows per CTA of the warp-per-row kernel at most (one warp each; the kernel
// caps it at what its launch bounds allow)
constexpr int kFp32RowWarpsMax = 16;
// A float32 call of at most this many rows per SM takes the warp-per-row
// kernel (4,736 rows on 148 SMs).  Measured on B300 at 14, 35 and 100
// inputs, the warp-per-row kernel is the faster one up to 4-6 K rows and
// the four-lanes-per-row kernel beyond.
constexpr int kFp32RowRowsPerSm = 32;
// segments.cu
cudaError_t seg_prefix_launch(const tabnet_segment* segs, int n, int64_t* prefix, cudaStream_t stream);

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& why) {
    g_last_error = why;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? TABNET_ERR_OOM : TABNET_ERR_CUDA;
}

// Keeps the caller's current device across a call that needs another one.
struct DeviceGuard {
    int prev = -1;
    bool switched = false;
    cudaError_t err = cudaSuccess;
    explicit DeviceGuard(int dev) {
        err = cudaGetDevice(&prev);
        if (err == cudaSuccess && prev != dev) {
            err = cudaSetDevice(dev);
            switched = (err == cudaSuccess);
        }
    }
    ~DeviceGuard() {
        if (switched) cudaSetDevice(prev);
    }
};

}  // namespace

int set_last_error(int code, const std::string& why) { return fail(code, why); }

size_t Arena::add(const void* data, size_t bytes, size_t align) {
    size_t off = (image.size() + align - 1) / align * align;
    image.resize(off + bytes, 0);
    if (data && bytes) std::memcpy(image.data() + off, data, bytes);
    return off;
}

namespace {

// Common per-model constants (input BN, embeddings, final linear, tables).
void build_consts(const HostModel& hm, Arena& a, ConstOffsets& o) {
    const tabnet_dims& d = hm.dims;
    std::vector<float> s0, t0;
    fold_bn(hm.bn0, d.bn_eps, s0, t0);
    o.s0 = a.add(s0.data(), s0.size() * 4);
    o.t0 = a.add(t0.data(), t0.size() * 4);
    // Input BN folded into the tables: emb'[v][e] = s0[c+e] * emb[v][e] + t0[c+e].
    std::vector<float> emb;
    std::vector<int> cat_off(d.n_cat);
    int col = d.n_num;
    for (int j = 0; j < d.n_cat; ++j) {
        cat_off[j] = (int)emb.size();
        const int e = hm.cat_emb_dim[j];
        for (int v = 0; v < hm.cat_card[j]; ++v)
            for (int k = 0; k < e; ++k)
                emb.push_back((float)((double)s0[col + k] * hm.emb[j][(size_t)v * e + k] + t0[col + k]));
        col += e;
    }
    if (emb.empty()) emb.push_back(0.f);
    o.emb = a.add(emb.data(), emb.size() * 4);
    if (cat_off.empty()) cat_off.push_back(0);
    o.cat_off = a.add(cat_off.data(), cat_off.size() * 4);
    std::vector<int> card(hm.cat_card.begin(), hm.cat_card.end());
    if (card.empty()) card.push_back(1);
    o.cat_card = a.add(card.data(), card.size() * 4);
    std::vector<int> cbase(card.size(), 0);
    o.cat_base = a.add(cbase.data(), cbase.size() * 4);
    std::vector<int> fcol, flen;
    hm.feature_columns(fcol, flen);
    o.feat_col = a.add(fcol.data(), fcol.size() * 4);
    o.feat_len = a.add(flen.data(), flen.size() * 4);
    o.wf = a.add(hm.final_w.data(), hm.final_w.size() * 4);
    o.bf = a.add(hm.final_b.data(), hm.final_b.size() * 4);
}

void fill_consts(const HostModel& hm, const ConstOffsets& o, const uint8_t* base, unsigned* status,
                 ModelConsts& m) {
    const tabnet_dims& d = hm.dims;
    m.n_num = d.n_num; m.n_cat = d.n_cat; m.de = d.d_emb; m.d = d.n_feat;
    m.n_d = d.n_d; m.n_a = d.n_a; m.N = d.n_d + d.n_a; m.n_steps = d.n_steps;
    m.layers_per_ft = d.n_shared + d.n_indep; m.n_classes = d.n_classes;
    m.gamma = (float)d.gamma;
    m.s0 = (const float*)(base + o.s0);
    m.t0 = (const float*)(base + o.t0);
    m.emb = (const float*)(base + o.emb);
    m.cat_off = (const int*)(base + o.cat_off);
    m.cat_card = (const int*)(base + o.cat_card);
    m.cat_base = (const int*)(base + o.cat_base);
    m.feat_col = (const int*)(base + o.feat_col);
    m.feat_len = (const int*)(base + o.feat_len);
    m.wf = (const float*)(base + o.wf);
    m.bf = (const float*)(base + o.bf);
    m.status = status;
}

std::vector<float> transpose(const std::vector<float>& w, int rows, int cols) {
    std::vector<float> t((size_t)rows * cols);
    for (int r = 0; r < rows; ++r)
        for (int c = 0; c < cols; ++c) t[(size_t)c * rows + r] = w[(size_t)r * cols + c];
    return t;
}

// FP32 path: transposed weights and folded BN per layer; layer tables are
// patched with device addresses once the arena is allocated.
struct SimtLayout {
    struct L { size_t wt, scale, shift; int k, n_out; };
    std::vector<L> ft, att;
    size_t ft_table = 0, att_table = 0;
    size_t row_units = 0;
    int row_slot = 0;
};

void build_simt(const HostModel& hm, Arena& a, SimtLayout& lay) {
    const tabnet_dims& d = hm.dims;
    const int N = d.n_d + d.n_a;
    std::vector<size_t> shared_wt(d.n_shared);
    for (int l = 0; l < d.n_shared; ++l) {
        const int k = (l == 0) ? d.d_emb : N;
        auto t = transpose(hm.shared_fc[l], 2 * N, k);
        shared_wt[l] = a.add(t.data(), t.size() * 4, 16);
    }
    for (int s = 0; s <= d.n_steps; ++s) {
        for (int l = 0; l < d.n_shared + d.n_indep; ++l) {
            GluLayer g = hm.layer(s, l);
            SimtLayout::L L{};
            L.k = g.k;
            L.n_out = 2 * N;
            if (l < d.n_shared) {
                L.wt = shared_wt[l];
            } else {
                auto t = transpose(*g.w, 2 * N, g.k);
                L.wt = a.add(t.data(), t.size() * 4, 16);
            }
            std::vector<float> sc, sh;
            fold_bn(*g.bn, d.bn_eps, sc, sh);
            L.scale = a.add(sc.data(), sc.size() * 4);
            L.shift = a.add(sh.data(), sh.size() * 4);
            lay.ft.push_back(L);
        }
    }
    for (int i = 0; i < d.n_steps; ++i) {
        SimtLayout::L L{};
        L.k = d.n_a;
        L.n_out = d.d_emb;
        auto t = transpose(hm.att_fc[i], d.d_emb, d.n_a);
        L.wt = a.add(t.data(), t.size() * 4, 16);
        std::vector<float> sc, sh;
        fold_bn(hm.att_bn[i], d.bn_eps, sc, sh);
        L.scale = a.add(sc.data(), sc.size() * 4);
        L.shift = a.add(sh.data(), sh.size() * 4);
        lay.att.push_back(L);
    }
    // the warp-per-row kernel's unit image (layout in SimtParams)
    const int lpf = d.n_shared + d.n_indep, n_units = row_n_units(lpf, d.n_steps);
    const int slot = row_slot_floats(d.d_emb, N, d.n_a);
    std::vector<float> img((size_t)n_units * slot, 0.f);
    bool shapes_ok = true;
    for (int u = 0; u < n_units && shapes_ok; ++u) {
        int k, n_out, att_step, ft_layer;
        row_unit_shape(u, lpf, d.d_emb, N, d.n_a, &k, &n_out, &att_step, &ft_layer);
        const SimtLayout::L& L = att_step >= 0 ? lay.att[att_step] : lay.ft[ft_layer];
        shapes_ok = L.k == k && L.n_out == n_out;
        if (!shapes_ok) break;
        const int ld = row_r4(n_out), kp = row_kp(k);
        const float* wt = reinterpret_cast<const float*>(a.image.data() + L.wt);
        const float* sc = reinterpret_cast<const float*>(a.image.data() + L.scale);
        const float* sh = reinterpret_cast<const float*>(a.image.data() + L.shift);
        float* dst = img.data() + (size_t)u * slot;
        for (int o = 0; o < n_out; ++o)
            for (int kk = 0; kk < k; ++kk) dst[(size_t)o * kp + kk] = wt[(size_t)kk * n_out + o];
        std::memcpy(dst + (size_t)ld * kp, sc, n_out * sizeof(float));
        std::memcpy(dst + (size_t)ld * kp + ld, sh, n_out * sizeof(float));
    }
    // (row_slot stays 0, and the kernel unused, if a layer had another shape)
    if (shapes_ok) {
        lay.row_units = a.add(img.data(), img.size() * sizeof(float), 16);
        lay.row_slot = slot;
    }
    lay.ft_table = a.add(nullptr, lay.ft.size() * sizeof(SimtLayer), 16);
    lay.att_table = a.add(nullptr, lay.att.size() * sizeof(SimtLayer), 16);
}

void patch_simt(const SimtLayout& lay, Arena& a, const uint8_t* base, SimtParams& p) {
    auto fill = [&](const std::vector<SimtLayout::L>& src, size_t table) {
        for (size_t i = 0; i < src.size(); ++i) {
            SimtLayer L;
            L.wt = (const float*)(base + src[i].wt);
            L.scale = (const float*)(base + src[i].scale);
            L.shift = (const float*)(base + src[i].shift);
            L.k = src[i].k;
            L.n_out = src[i].n_out;
            std::memcpy(a.image.data() + table + i * sizeof(SimtLayer), &L, sizeof(L));
        }
    };
    fill(lay.ft, lay.ft_table);
    fill(lay.att, lay.att_table);
    p.ft = (const SimtLayer*)(base + lay.ft_table);
    p.att = (const SimtLayer*)(base + lay.att_table);
    p.row_units = (const float*)(base + lay.row_units);
    p.row_slot = lay.row_slot;
}

int check_ptr(const void* p, bool required, const char* name) {
    if (!p) return required ? fail(TABNET_ERR_ARG, std::string(name) + " is NULL") : TABNET_OK;
    if (reinterpret_cast<uintptr_t>(p) % 4) return fail(TABNET_ERR_ARG, std::string(name) + " is not 4-byte aligned");
    return TABNET_OK;
}

}  // namespace

int forward_impl(tabnet_model* m, const float* x_num, const int32_t* x_cat, int64_t rows,
                 float* logits, float* masks, float* agg, cudaStream_t stream, const SegTable* seg = nullptr) {
    cudaError_t e;
    if (m->precision == TABNET_FP32) {
        SimtParams p = m->simt;
        p.seg = seg ? *seg : SegTable{nullptr, nullptr, 0};
        // a call of few rows (known on the host) takes a warp per row, with
        // results bit for bit those of the four-lanes-per-row kernel
        if (!(seg && seg->segs) && rows <= m->simt_row_max)
            e = simt_row_launch(p, x_num, x_cat, rows, logits, masks, agg, stream, m->num_sms, kFp32RowWarpsMax,
                                m->smem_optin);
        else
            e = simt_launch(p, m->simt_rows, x_num, x_cat, rows, logits, masks, agg, stream, m->simt_max_ctas);
    } else {
        e = tc_launch(m, x_num, x_cat, rows, logits, masks, agg, stream, seg);
    }
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    return TABNET_OK;
}

// One batch whose input row i is n_num floats then n_cat int32 codes at
// rows_in + 4 (n_num + n_cat) i (the server's input ring); outputs as in
// tabnet_forward.  Not part of the C ABI.
int forward_interleaved(tabnet_model* m, const void* rows_in, int64_t rows, float* logits, float* step_masks,
                                float* agg_mask, cudaStream_t stream) {
    if (!m || !rows_in) return fail(TABNET_ERR_ARG, "null model or inputs");
    if (rows <= 0) return rows < 0 ? fail(TABNET_ERR_ARG, "rows < 0") : TABNET_OK;
    const tabnet_dims& d = m->host.dims;
    int rc;
    if ((rc = check_ptr(rows_in, true, "rows_in")) || (rc = check_ptr(logits, true, "logits")) ||
        (rc = check_ptr(step_masks, false, "step_masks")) || (rc = check_ptr(agg_mask, false, "agg_mask")))
        return rc;
    DeviceGuard guard(m->device);
    if (guard.err != cudaSuccess) return cuda_fail(guard.err, "cudaSetDevice");
    SegTable t{nullptr, nullptr, 0};
    t.in_stride = d.n_num + d.n_cat;
    const float* xn = static_cast<const float*>(rows_in);
    return forward_impl(m, d.n_num ? xn : nullptr, d.n_cat ? reinterpret_cast<const int32_t*>(xn + d.n_num) : nullptr,
                        rows, logits, step_masks, agg_mask, stream, &t);
}

}  // namespace tabnet

using namespace tabnet;

extern "C" {

int tabnet_abi_version(void) { return TABNET_ABI_VERSION; }

const char* tabnet_last_error(void) { return g_last_error.c_str(); }

const char* tabnet_status_string(int code) {
    switch (code) {
        case TABNET_OK: return "ok";
        case TABNET_ERR_ARG: return "invalid argument";
        case TABNET_ERR_BLOB_MAGIC: return "blob: bad magic";
        case TABNET_ERR_BLOB_VERSION: return "blob: unsupported version";
        case TABNET_ERR_BLOB_SIZE: return "blob: size mismatch";
        case TABNET_ERR_BLOB_HASH: return "blob: payload hash mismatch";
        case TABNET_ERR_UNSUPPORTED_DIMS: return "model shape not supported";
        case TABNET_ERR_CUDA: return "CUDA error";
        case TABNET_ERR_OOM: return "out of device memory";
        case TABNET_ERR_TIMEOUT: return "device wait timed out";
        case TABNET_ERR_DEVICE: return "device reported a fault";
    }
    return "unknown status";
}

int tabnet_blob_inspect(const void* blob, size_t blob_bytes, tabnet_dims* out) {
    if (!blob || !out) return fail(TABNET_ERR_ARG, "null pointer");
    try {
        HostModel hm;
        std::string why;
        int rc = parse_blob(blob, blob_bytes, &hm, &why);
        if (rc != TABNET_OK) return fail(rc, why);
        *out = hm.dims;
        return TABNET_OK;
    } catch (const std::bad_alloc&) {
        return fail(TABNET_ERR_OOM, "host allocation failed");
    } catch (...) {
        return fail(TABNET_ERR_ARG, "unexpected error while parsing");
    }
}

int tabnet_create(const void* blob, size_t blob_bytes, int precision, int device, tabnet_model** out) {
    if (!blob || !out) return fail(TABNET_ERR_ARG, "null pointer");
    *out = nullptr;
    if (precision < TABNET_FP32 || precision > TABNET_BF16X6) return fail(TABNET_ERR_ARG, "unknown precision");
    tabnet_model* m = nullptr;
    try {
        m = new tabnet_model();
        std::string why;
        int rc = parse_blob(blob, blob_bytes, &m->host, &why);
        if (rc != TABNET_OK) { delete m; return fail(rc, why); }
        m->device = device;
        m->precision = precision;
        int ndev = 0;
        cudaError_t e = cudaGetDeviceCount(&ndev);
        if (e != cudaSuccess || device < 0 || device >= ndev) {
            delete m;
            return fail(TABNET_ERR_CUDA, e != cudaSuccess ? std::string("no CUDA device: ") + cudaGetErrorString(e)
                                                          : std::string("device ordinal out of range"));
        }
        DeviceGuard guard(device);
        if (guard.err != cudaSuccess) { delete m; return cuda_fail(guard.err, "cudaSetDevice"); }
        cudaDeviceProp prop;
        if ((e = cudaGetDeviceProperties(&prop, device)) != cudaSuccess) { delete m; return cuda_fail(e, "cudaGetDeviceProperties"); }
        if (prop.major != 10 || prop.minor != 3) {
            delete m;
            return fail(TABNET_ERR_CUDA, "kernels are built for sm_103a (B300); device is sm_" +
                                             std::to_string(prop.major) + std::to_string(prop.minor));
        }
        m->num_sms = prop.multiProcessorCount;
        m->smem_optin = prop.sharedMemPerBlockOptin;

        Arena arena;
        build_consts(m->host, arena, m->consts_off);
        SimtLayout simt_lay;
        if (precision == TABNET_FP32) {
            build_simt(m->host, arena, simt_lay);
        } else {
            rc = tc_build(m, arena, &why);
            if (rc != TABNET_OK) { delete m; return fail(rc, why); }
        }
        if ((e = cudaMalloc(&m->d_arena, arena.image.size())) != cudaSuccess) {
            int r2 = cuda_fail(e, "cudaMalloc(weights)");
            delete m;
            return r2;
        }
        if ((e = cudaMalloc(&m->d_status, 4 * sizeof(unsigned))) != cudaSuccess) {
            int r2 = cuda_fail(e, "cudaMalloc(status)");
            cudaFree(m->d_arena);
            delete m;
            return r2;
        }
        const uint8_t* base = static_cast<const uint8_t*>(m->d_arena);
        fill_consts(m->host, m->consts_off, base, m->d_status, m->consts);
        if (precision == TABNET_FP32) {
            m->simt.m = m->consts;
            patch_simt(simt_lay, arena, base, m->simt);
            // rows per CTA: the most rows resident per SM (CTAs per SM x rows
            // per CTA, registers and shared memory permitting), more rows per
            // CTA on a tie
            m->simt_rows = 0;
            int best_resident = 0;
            for (int r : {32, 16, 8}) {
                const size_t sm = simt_smem_bytes(m->consts, r);
                if (sm > m->smem_optin) continue;
                if ((e = simt_configure(r, sm)) != cudaSuccess) {
                    tabnet_destroy(m);
                    return cuda_fail(e, "cudaFuncSetAttribute");
                }
                const int resident = simt_occupancy(r, sm) * r;
                if (resident > best_resident) {
                    best_resident = resident;
                    m->simt_rows = r;
                }
            }
            if (m->simt_rows == 0) {
                tabnet_destroy(m);
                return fail(TABNET_ERR_UNSUPPORTED_DIMS, "model state does not fit in shared memory");
            }
            m->simt_max_ctas = m->num_sms * simt_occupancy(m->simt_rows, simt_smem_bytes(m->consts, m->simt_rows));
            // warp-per-row form for calls of up to simt_row_max rows (none if
            // one row and one weight slot exceed shared memory)
            m->simt_row_max = 0;
            int row_w = 0, row_nbuf = 0;
            if (m->simt.row_slot > 0 &&
                simt_row_plan(m->consts, 1, m->num_sms, kFp32RowWarpsMax, m->smem_optin, &row_w, &row_nbuf)) {
                if ((e = simt_row_configure(m->smem_optin)) != cudaSuccess) {
                    tabnet_destroy(m);
                    return cuda_fail(e, "cudaFuncSetAttribute");
                }
                m->simt_row_max = (int64_t)kFp32RowRowsPerSm * m->num_sms;
            }
        } else {
            rc = tc_patch(m, arena, base, &why);
            if (rc != TABNET_OK) { tabnet_destroy(m); return fail(rc, why); }
        }
        m->arena_bytes = arena.image.size();
        if ((e = cudaMemcpy(m->d_arena, arena.image.data(), arena.image.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
            (e = cudaMemset(m->d_status, 0, 4 * sizeof(unsigned))) != cudaSuccess) {
            tabnet_destroy(m);
            return cuda_fail(e, "upload");
        }
        *out = m;
        return TABNET_OK;
    } catch (const std::bad_alloc&) {
        delete m;
        return fail(TABNET_ERR_OOM, "host allocation failed");
    } catch (...) {
        delete m;
        return fail(TABNET_ERR_ARG, "unexpected error in create");
    }
}

int tabnet_dims_of(const tabnet_model* m, tabnet_dims* out) {
    if (!m || !out) return fail(TABNET_ERR_ARG, "null pointer");
    *out = m->host.dims;
    return TABNET_OK;
}

int tabnet_precision_of(const tabnet_model* m) {
    if (!m) return fail(TABNET_ERR_ARG, "null pointer");
    return m->precision;
}

int tabnet_forward(tabnet_model* m, const float* x_num, const int32_t* x_cat, int64_t rows,
                   float* logits, float* step_masks, float* agg_mask, void* stream) {
    if (!m) return fail(TABNET_ERR_ARG, "null model");
    if (rows < 0) return fail(TABNET_ERR_ARG, "rows < 0");
    if (rows == 0) return TABNET_OK;
    const tabnet_dims& d = m->host.dims;
    int rc;
    if ((rc = check_ptr(x_num, d.n_num > 0, "x_num")) || (rc = check_ptr(x_cat, d.n_cat > 0, "x_cat")) ||
        (rc = check_ptr(logits, true, "logits")) || (rc = check_ptr(step_masks, false, "step_masks")) ||
        (rc = check_ptr(agg_mask, false, "agg_mask")))
        return rc;
    DeviceGuard guard(m->device);
    if (guard.err != cudaSuccess) return cuda_fail(guard.err, "cudaSetDevice");
    return forward_impl(m, x_num, x_cat, rows, logits, step_masks, agg_mask, (cudaStream_t)stream);
}

int tabnet_forward_host(tabnet_model* m, const float* x_num, const int32_t* x_cat, int64_t rows,
                        float* logits, float* step_masks, float* agg_mask, void* stream) {
    if (!m) return fail(TABNET_ERR_ARG, "null model");
    if (rows < 0) return fail(TABNET_ERR_ARG, "rows < 0");
    if (rows == 0) return TABNET_OK;
    const tabnet_dims& d = m->host.dims;
    int rc;
    if ((rc = check_ptr(x_num, d.n_num > 0, "x_num")) || (rc = check_ptr(x_cat, d.n_cat > 0, "x_cat")) ||
        (rc = check_ptr(logits, true, "logits")) || (rc = check_ptr(step_masks, false, "step_masks")) ||
        (rc = check_ptr(agg_mask, false, "agg_mask")))
        return rc;
    DeviceGuard guard(m->device);
    if (guard.err != cudaSuccess) return cuda_fail(guard.err, "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    // bytes per row of each buffer
    const size_t r_num = (size_t)d.n_num * 4, r_cat = (size_t)d.n_cat * 4, r_lg = (size_t)d.n_classes * 4;
    const size_t r_mk = step_masks ? (size_t)d.n_steps * d.d_emb * 4 : 0, r_ag = agg_mask ? (size_t)d.n_feat * 4 : 0;
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t need = up(rows * r_num) + up(rows * r_cat) + up(rows * r_lg) + up(rows * r_mk) + up(rows * r_ag);
    cudaError_t e;
    if (need > m->ws_bytes) {
        if (m->d_ws) {
            cudaStreamSynchronize(s);
            cudaFree(m->d_ws);
            m->d_ws = nullptr;
            m->ws_bytes = 0;
        }
        if ((e = cudaMalloc(&m->d_ws, need)) != cudaSuccess) return cuda_fail(e, "cudaMalloc(workspace)");
        m->ws_bytes = need;
    }
    uint8_t* w = static_cast<uint8_t*>(m->d_ws);
    uint8_t* dn = w;  w += up(rows * r_num);
    uint8_t* dc = w;  w += up(rows * r_cat);
    uint8_t* dl = w;  w += up(rows * r_lg);
    uint8_t* dm = w;  w += up(rows * r_mk);
    uint8_t* da = w;
    // Row chunks of about 8 MB of outputs (whole 128-row tiles), each copied
    // in, run and copied out on one of the handle's streams in turn: the
    // input copy of a chunk, the kernels of others and the output copy of an
    // earlier one overlap (the two copy directions and the SMs work at once).
    const size_t r_out = r_lg + r_mk + r_ag;
    int64_t chunk = (int64_t)((8u << 20) / r_out);
    chunk = std::max<int64_t>(2048, chunk / 128 * 128);
    const int64_t n_chunks = (rows + chunk - 1) / chunk;
    const int n_str = (int)std::min<int64_t>(n_chunks, tabnet_model::kHostStreams);
    if (n_chunks > 1 && !m->host_start) {
        // all or nothing: host_start marks a complete set
        for (int i = 0; i < tabnet_model::kHostStreams; ++i) {
            if (!m->host_streams[i] &&
                (e = cudaStreamCreateWithFlags(&m->host_streams[i], cudaStreamNonBlocking)) != cudaSuccess)
                return cuda_fail(e, "pipeline streams");
            if (!m->host_done[i] && (e = cudaEventCreateWithFlags(&m->host_done[i], cudaEventDisableTiming)) != cudaSuccess)
                return cuda_fail(e, "pipeline events");
        }
        if ((e = cudaEventCreateWithFlags(&m->host_start, cudaEventDisableTiming)) != cudaSuccess)
            return cuda_fail(e, "pipeline events");
    }
    if (n_chunks > 1) {
        // the chunks start after the work already on the caller's stream
        if ((e = cudaEventRecord(m->host_start, s)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
        for (int i = 0; i < n_str; ++i)
            if ((e = cudaStreamWaitEvent(m->host_streams[i], m->host_start, 0)) != cudaSuccess)
                return cuda_fail(e, "cudaStreamWaitEvent");
    }
    // A failure part-way leaves no chunk running that a later call's copies
    // into the workspace could overtake.
    auto drain = [&](int rc_) {
        if (n_chunks > 1)
            for (int i = 0; i < n_str; ++i) cudaStreamSynchronize(m->host_streams[i]);
        return rc_;
    };
    auto h2d = [&](uint8_t* dst, const void* src, size_t b, cudaStream_t st) {
        return b ? cudaMemcpyAsync(dst, src, b, cudaMemcpyHostToDevice, st) : cudaSuccess;
    };
    auto d2h = [&](void* dst, const uint8_t* src, size_t b, cudaStream_t st) {
        return b ? cudaMemcpyAsync(dst, src, b, cudaMemcpyDeviceToHost, st) : cudaSuccess;
    };
    for (int64_t c = 0; c < n_chunks; ++c) {
        cudaStream_t st = n_chunks > 1 ? m->host_streams[c % n_str] : s;
        const int64_t r0 = c * chunk, nr = std::min(chunk, rows - r0);
        if ((e = h2d(dn + r0 * r_num, reinterpret_cast<const uint8_t*>(x_num) + r0 * r_num, nr * r_num, st)) !=
            cudaSuccess)
            return drain(cuda_fail(e, "H2D x_num"));
        if ((e = h2d(dc + r0 * r_cat, reinterpret_cast<const uint8_t*>(x_cat) + r0 * r_cat, nr * r_cat, st)) !=
            cudaSuccess)
            return drain(cuda_fail(e, "H2D x_cat"));
        rc = forward_impl(m, r_num ? reinterpret_cast<float*>(dn + r0 * r_num) : nullptr,
                          r_cat ? reinterpret_cast<int32_t*>(dc + r0 * r_cat) : nullptr, nr,
                          reinterpret_cast<float*>(dl + r0 * r_lg),
                          step_masks ? reinterpret_cast<float*>(dm + r0 * r_mk) : nullptr,
                          agg_mask ? reinterpret_cast<float*>(da + r0 * r_ag) : nullptr, st);
        if (rc != TABNET_OK) return drain(rc);
        if ((e = d2h(reinterpret_cast<uint8_t*>(logits) + r0 * r_lg, dl + r0 * r_lg, nr * r_lg, st)) != cudaSuccess)
            return drain(cuda_fail(e, "D2H logits"));
        if (step_masks &&
            (e = d2h(reinterpret_cast<uint8_t*>(step_masks) + r0 * r_mk, dm + r0 * r_mk, nr * r_mk, st)) != cudaSuccess)
            return drain(cuda_fail(e, "D2H masks"));
        if (agg_mask &&
            (e = d2h(reinterpret_cast<uint8_t*>(agg_mask) + r0 * r_ag, da + r0 * r_ag, nr * r_ag, st)) != cudaSuccess)
            return drain(cuda_fail(e, "D2H agg"));
    }
    if (n_chunks > 1) {
        // the caller's stream continues after every chunk
        for (int i = 0; i < n_str; ++i) {
            if ((e = cudaEventRecord(m->host_done[i], m->host_streams[i])) != cudaSuccess ||
                (e = cudaStreamWaitEvent(s, m->host_done[i], 0)) != cudaSuccess)
                return drain(cuda_fail(e, "stream join"));
        }
    }
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    return TABNET_OK;
}

namespace {

// Scratch of the segmented launches: [descriptors: cap][prefix: cap + 1].
int seg_reserve(tabnet_model* m, int n, cudaStream_t stream) {
    if (n <= m->seg_cap) return TABNET_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
        return fail(TABNET_ERR_OOM, "segment scratch too small during stream capture: reserve it first");
    int cap = std::max(n, std::max(256, 2 * m->seg_cap));
    void* p = nullptr;
    const size_t bytes = (size_t)cap * sizeof(tabnet_segment) + ((size_t)cap + 1) * sizeof(int64_t);
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(segment scratch)");
    if (m->d_seg) {
        cudaDeviceSynchronize();  // the old scratch may still be read by a launch in flight
        cudaFree(m->d_seg);
    }
    m->d_seg = p;
    m->seg_cap = cap;
    return TABNET_OK;
}

int segments_device(tabnet_model* m, const tabnet_segment* segs, int n, cudaStream_t s) {
    int rc = seg_reserve(m, n, s);
    if (rc != TABNET_OK) return rc;
    int64_t* prefix = reinterpret_cast<int64_t*>(static_cast<uint8_t*>(m->d_seg) +
                                                 (size_t)m->seg_cap * sizeof(tabnet_segment));
    cudaError_t e = seg_prefix_launch(segs, n, prefix, s);
    if (e != cudaSuccess) return cuda_fail(e, "segment prefix launch");
    const SegTable t{segs, prefix, n};
    return forward_impl(m, nullptr, nullptr, 0, nullptr, nullptr, nullptr, s, &t);
}

}  // namespace

int tabnet_reserve_segments(tabnet_model* m, int max_segs) {
    if (!m || max_segs < 0) return fail(TABNET_ERR_ARG, "null model or negative count");
    DeviceGuard guard(m->device);
    if (guard.err != cudaSuccess) return cuda_fail(guard.err, "cudaSetDevice");
    return seg_reserve(m, max_segs, nullptr);
}

int tabnet_forward_segments_device(tabnet_model* m, const tabnet_segment* segs, int n_segs, void* stream) {
    if (!m || n_segs < 0) return fail(TABNET_ERR_ARG, "null model or negative count");
    if (n_segs == 0) return TABNET_OK;
    if (!segs) return fail(TABNET_ERR_ARG, "segs is NULL");
    DeviceGuard guard(m->device);
    if (guard.err != cudaSuccess) return cuda_fail(guard.err, "cudaSetDevice");
    return segments_device(m, segs, n_segs, (cudaStream_t)stream);
}

int tabnet_forward_segments(tabnet_model* m, const tabnet_segment* segs, int n_segs, void* stream) {
    if (!m || n_segs < 0) return fail(TABNET_ERR_ARG, "null model or negative count");
    if (n_segs == 0) return TABNET_OK;
    if (!segs) return fail(TABNET_ERR_ARG, "segs is NULL");
    const tabnet_dims& d = m->host.dims;
    for (int i = 0; i < n_segs; ++i) {
        const tabnet_segment& g = segs[i];
        if (g.rows < 0) return fail(TABNET_ERR_ARG, "segment " + std::to_string(i) + " has rows < 0");
        if (g.rows == 0) continue;
        int rc;
        if ((rc = check_ptr(g.x_num, d.n_num > 0, "segment x_num")) || (rc = check_ptr(g.x_cat, d.n_cat > 0, "segment x_cat")) ||
            (rc = check_ptr(g.logits, true, "segment logits")) || (rc = check_ptr(g.step_masks, false, "segment step_masks")) ||
            (rc = check_ptr(g.agg_mask, false, "segment agg_mask")))
            return rc;
    }
    DeviceGuard guard(m->device);
    if (guard.err != cudaSuccess) return cuda_fail(guard.err, "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    int rc = seg_reserve(m, n_segs, s);
    if (rc != TABNET_OK) return rc;
    if (n_segs > m->seg_stage_cap) {
        if (m->h_seg_stage) {
            if (m->seg_stage_done) cudaEventSynchronize(m->seg_stage_done);
            cudaFreeHost(m->h_seg_stage);
            m->h_seg_stage = nullptr;
            m->seg_stage_cap = 0;
        }
        if ((e = cudaHostAlloc((void**)&m->h_seg_stage, sizeof(tabnet_segment) * (size_t)m->seg_cap,
                               cudaHostAllocDefault)) != cudaSuccess)
            return cuda_fail(e, "cudaHostAlloc(segment staging)");
        m->seg_stage_cap = m->seg_cap;
    }
    if (!m->seg_stage_done && (e = cudaEventCreateWithFlags(&m->seg_stage_done, cudaEventDisableTiming)) != cudaSuccess)
        return cuda_fail(e, "cudaEventCreate");
    // the previous call's upload must have left the staging buffer
    if ((e = cudaEventSynchronize(m->seg_stage_done)) != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
    std::memcpy(m->h_seg_stage, segs, sizeof(tabnet_segment) * (size_t)n_segs);
    tabnet_segment* d_segs = static_cast<tabnet_segment*>(m->d_seg);
    if ((e = cudaMemcpyAsync(d_segs, m->h_seg_stage, sizeof(tabnet_segment) * (size_t)n_segs,
                             cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return cuda_fail(e, "upload segment descriptors");
    if ((e = cudaEventRecord(m->seg_stage_done, s)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    return segments_device(m, d_segs, n_segs, s);
}

int tabnet_set_tile_config(tabnet_model* m, int nwg, int n_slots, int ctas_per_sm) {
    if (!m) return fail(TABNET_ERR_ARG, "null model");
    if (m->precision == TABNET_FP32)
        return fail(TABNET_ERR_UNSUPPORTED_DIMS, "tile shapes apply to the tensor-core precisions");
    DeviceGuard guard(m->device);
    if (guard.err != cudaSuccess) return cuda_fail(guard.err, "cudaSetDevice");
    const TcParams saved_p = m->tc;
    const TcLaunch saved_l = m->tc_launch_cfg;
    std::string why;
    int rc = tc_choose_launch(m, nwg, n_slots, ctas_per_sm, &why);
    if (rc != TABNET_OK) {
        m->tc = saved_p;
        m->tc_launch_cfg = saved_l;
        return fail(rc, why);
    }
    return TABNET_OK;
}

int tabnet_get_tile_config(const tabnet_model* m, int* nwg, int* n_slots, int* ctas_per_sm) {
    if (!m) return fail(TABNET_ERR_ARG, "null model");
    if (m->precision == TABNET_FP32)
        return fail(TABNET_ERR_UNSUPPORTED_DIMS, "tile shapes apply to the tensor-core precisions");
    if (nwg) *nwg = m->tc_launch_cfg.nwg;
    if (n_slots) *n_slots = m->tc_launch_cfg.n_slots;
    if (ctas_per_sm) *ctas_per_sm = m->tc_launch_cfg.ctas_per_sm;
    return TABNET_OK;
}

int tabnet_set_input_transform(tabnet_model* m, const float* num_mean, const float* num_scale,
                               const int32_t* cat_base) {
    if (!m) return fail(TABNET_ERR_ARG, "null model");
    const tabnet_dims& d = m->host.dims;
    std::vector<float> s0, t0;
    fold_bn(m->host.bn0, d.bn_eps, s0, t0);
    // (x - mean) * scale through input BN s0 x + t0:  s0' = s0 scale, t0' = t0 - s0 scale mean
    for (int c = 0; c < d.n_num; ++c) {
        const double sc = num_scale ? (double)num_scale[c] : 1.0, mu = num_mean ? (double)num_mean[c] : 0.0;
        if (!std::isfinite(sc) || !std::isfinite(mu)) return fail(TABNET_ERR_ARG, "non-finite scaler value");
        const double s = (double)s0[c] * sc;
        t0[c] = (float)((double)t0[c] - s * mu);
        s0[c] = (float)s;
    }
    std::vector<int> cb(std::max(d.n_cat, 1), 0);
    for (int j = 0; j < d.n_cat; ++j) cb[j] = cat_base ? cat_base[j] : 0;
    DeviceGuard guard(m->device);
    if (guard.err != cudaSuccess) return cuda_fail(guard.err, "cudaSetDevice");
    uint8_t* base = static_cast<uint8_t*>(m->d_arena);
    cudaError_t e;
    if ((e = cudaDeviceSynchronize()) != cudaSuccess ||
        (d.n_num > 0 && (e = cudaMemcpy(base + m->consts_off.s0, s0.data(), sizeof(float) * d.n_num,
                                        cudaMemcpyHostToDevice)) != cudaSuccess) ||
        (d.n_num > 0 && (e = cudaMemcpy(base + m->consts_off.t0, t0.data(), sizeof(float) * d.n_num,
                                        cudaMemcpyHostToDevice)) != cudaSuccess) ||
        (e = cudaMemcpy(base + m->consts_off.cat_base, cb.data(), sizeof(int) * cb.size(),
                        cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_fail(e, "upload input transform");
    return TABNET_OK;
}

int tabnet_poll_status(tabnet_model* m, void* stream, uint32_t* status) {
    if (!m || !status) return fail(TABNET_ERR_ARG, "null pointer");
    DeviceGuard guard(m->device);
    if (guard.err != cudaSuccess) return cuda_fail(guard.err, "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    unsigned w[4] = {0, 0, 0, 0};
    cudaError_t e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    if ((e = cudaMemcpy(w, m->d_status, sizeof(w), cudaMemcpyDeviceToHost)) != cudaSuccess) return cuda_fail(e, "read status");
    if ((e = cudaMemset(m->d_status, 0, sizeof(w))) != cudaSuccess) return cuda_fail(e, "clear status");
    const unsigned v = w[0];
    *status = v;
    if (v & TABNET_STATUS_TIMEOUT) {
        // word 1: where the first wait ran out (kind << 24 | index), word 2: CTA
        char buf[160];
        std::snprintf(buf, sizeof(buf), "a bounded device wait ran out (kind %u, index %u, block %u)", w[1] >> 24,
                      w[1] & 0xFFFFFFu, w[2]);
        return fail(TABNET_ERR_TIMEOUT, buf);
    }
    if (v) return fail(TABNET_ERR_DEVICE, "device status bits set");
    return TABNET_OK;
}

void tabnet_destroy(tabnet_model* m) {
    if (!m) return;
    {
        DeviceGuard guard(m->device);
        cudaDeviceSynchronize();
        if (m->d_arena) cudaFree(m->d_arena);
        if (m->d_status) cudaFree(m->d_status);
        if (m->d_ws) cudaFree(m->d_ws);
        if (m->d_seg) cudaFree(m->d_seg);
        if (m->h_seg_stage) cudaFreeHost(m->h_seg_stage);
        if (m->seg_stage_done) cudaEventDestroy(m->seg_stage_done);
        for (int i = 0; i < tabnet_model::kHostStreams; ++i) {
            if (m->host_streams[i]) cudaStreamDestroy(m->host_streams[i]);
            if (m->host_done[i]) cudaEventDestroy(m->host_done[i]);
        }
        if (m->host_start) cudaEventDestroy(m->host_start);
        tc_release(m);
    }
    delete m;
}

}  // extern "C"
