// FP32 TabNet forward on the CUDA cores (FFMA, no TF32): the float32
// precision mode of the library.
//
// Layout.  A CTA owns ROWS rows; four consecutive lanes own one row, so the
// whole life of a row (embedding, every feature transformer, attentive
// transformer, sparsemax, prior, aggregation) stays inside one warp and the
// only synchronisation is __syncwarp.  Per-row state lives in shared memory
// as [column][row] arrays, which makes the four lanes of a row read the
// same word (broadcast) and different rows hit different banks.  Weights
// are read through the read-only cache, transposed to [k][n_out] so that the
// four lanes of a row read consecutive outputs.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/tabnet.h"
#include "kernel_params.h"

namespace tabnet {

namespace {

constexpr int TPR = 4;  // threads per row
constexpr float kSqrtHalf = 0.70710678118654752440f;

// The four lanes of one row: rows of a warp leave data-dependent loops
// (sparsemax) at different iterations, so shuffles name only this group.
__device__ __forceinline__ unsigned row_mask() { return 0xFu << (threadIdx.x & 28); }

__device__ __forceinline__ float sum4(float v) {
    const unsigned mk = row_mask();
    v += __shfl_xor_sync(mk, v, 1);
    v += __shfl_xor_sync(mk, v, 2);
    return v;
}

__device__ __forceinline__ int sum4i(int v) {
    const unsigned mk = row_mask();
    v += __shfl_xor_sync(mk, v, 1);
    v += __shfl_xor_sync(mk, v, 2);
    return v;
}

__device__ __forceinline__ float sigmoid_exact(float x) { return 1.0f / (1.0f + expf(-x)); }

// One GLU layer for the calling row: nxt[c] = GLU(BN(W cur))[c] (+ residual).
// The gate product and the residual are rounded separately (__fmul_rn,
// __fadd_rn): whether the compiler would contract them into an FMA depends
// on the surrounding code, and the two forms differ in the last bits.
template <int ROWS>
__device__ __forceinline__ void glu_layer(const SimtLayer& L, const float* cur, float* nxt,
                                          bool first, int N, int r, int q) {
    constexpr int NB = 4;
    const float* __restrict__ wt = L.wt;
    const int two_n = 2 * N;
    for (int c0 = q; c0 < N; c0 += TPR * NB) {
        float lin[NB], gate[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) { lin[b] = 0.f; gate[b] = 0.f; }
        for (int k = 0; k < L.k; ++k) {
            const float x = cur[k * ROWS + r];
            const float* w = wt + (size_t)k * two_n;
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                const int c = c0 + TPR * b;
                if (c < N) {
                    lin[b] = fmaf(__ldg(w + c), x, lin[b]);
                    gate[b] = fmaf(__ldg(w + N + c), x, gate[b]);
                }
            }
        }
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int c = c0 + TPR * b;
            if (c < N) {
                const float ul = fmaf(lin[b], __ldg(L.scale + c), __ldg(L.shift + c));
                const float ug = fmaf(gate[b], __ldg(L.scale + N + c), __ldg(L.shift + N + c));
                const float g = __fmul_rn(ul, sigmoid_exact(ug));
                nxt[c * ROWS + r] = first ? g : __fmul_rn(__fadd_rn(cur[c * ROWS + r], g), kSqrtHalf);
            }
        }
    }
}

template <int CT>
__device__ __forceinline__ void load_w(const float* __restrict__ w, float (&o)[CT]) {
    if constexpr (CT % 4 == 0) {
#pragma unroll
        for (int j = 0; j < CT; j += 4) {
            const float4 v = __ldg(reinterpret_cast<const float4*>(w + j));
            o[j] = v.x; o[j + 1] = v.y; o[j + 2] = v.z; o[j + 3] = v.w;
        }
    } else if constexpr (CT == 2) {
        const float2 v = __ldg(reinterpret_cast<const float2*>(w));
        o[0] = v.x; o[1] = v.y;
    } else {
#pragma unroll
        for (int j = 0; j < CT; ++j) o[j] = __ldg(w + j);
    }
}

// The same layer for all ROWS rows of the CTA at once, N = 16 CT: thread t
// takes rows 4 (t mod ROWS/4) + [0, 4) and outputs CT (t div ROWS/4) + [0, CT)
// (with their gates), so each weight it loads serves four rows and each
// input value CT outputs.  Every output is the same sequential FMA chain over
// k as in glu_layer, so the results are identical.  The caller synchronises
// the CTA before (cur complete) and after (nxt complete).
template <int ROWS, int CT>
__device__ __forceinline__ void glu_layer_tiled(const SimtLayer& L, const float* cur, float* nxt, bool first,
                                                int N) {
    constexpr int RG = ROWS / 4;
    const int rg = (int)threadIdx.x % RG, c0 = ((int)threadIdx.x / RG) * CT;
    const float* __restrict__ wt = L.wt;
    const int two_n = 2 * N;
    float lin[4][CT], gate[4][CT];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < CT; ++j) { lin[i][j] = 0.f; gate[i][j] = 0.f; }
#pragma unroll 4
    for (int k = 0; k < L.k; ++k) {
        const float4 xv = *reinterpret_cast<const float4*>(cur + k * ROWS + 4 * rg);
        const float x[4] = {xv.x, xv.y, xv.z, xv.w};
        float wl[CT], wg[CT];
        load_w<CT>(wt + (size_t)k * two_n + c0, wl);
        load_w<CT>(wt + (size_t)k * two_n + N + c0, wg);
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < CT; ++j) {
                lin[i][j] = fmaf(wl[j], x[i], lin[i][j]);
                gate[i][j] = fmaf(wg[j], x[i], gate[i][j]);
            }
    }
#pragma unroll
    for (int j = 0; j < CT; ++j) {
        const int c = c0 + j;
        const float sl = __ldg(L.scale + c), tl = __ldg(L.shift + c);
        const float sg = __ldg(L.scale + N + c), tg = __ldg(L.shift + N + c);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = 4 * rg + i;
            const float ul = fmaf(lin[i][j], sl, tl);
            const float ug = fmaf(gate[i][j], sg, tg);
            // separately rounded, as in glu_layer (no contraction into an FMA)
            const float g = __fmul_rn(ul, sigmoid_exact(ug));
            nxt[c * ROWS + r] = first ? g : __fmul_rn(__fadd_rn(cur[c * ROWS + r], g), kSqrtHalf);
        }
    }
}

// The attentive layer for all ROWS rows of the CTA at once, as the tiled GLU
// layer: thread t takes rows 4 (t mod ROWS/4) + [0, 4) and the columns
// c = t div ROWS/4 + 16 j (j < ceil(de / 16) <= kAttMaxCt).  Each output is
// the same sequential FMA chain over k as the per-row form.  The caller
// synchronises the CTA afterwards (z complete); a (the transformer output's
// attention part) and P are complete before (the feature transformer ends
// with a CTA barrier).
constexpr int kAttMaxCt = 16;

template <int ROWS>
__device__ __forceinline__ void attentive_tiled(const SimtLayer& A, const float* a, const float* P, float* Z,
                                                int de, int n_a) {
    constexpr int RG = ROWS / 4;
    const int rg = (int)threadIdx.x % RG, cg = (int)threadIdx.x / RG;
    const int ct = (de + 15) / 16;
    float acc[4][kAttMaxCt];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < kAttMaxCt; ++j) acc[i][j] = 0.f;
#pragma unroll 2
    for (int k = 0; k < n_a; ++k) {
        const float4 xv = *reinterpret_cast<const float4*>(a + k * ROWS + 4 * rg);
        const float x[4] = {xv.x, xv.y, xv.z, xv.w};
        const float* w = A.wt + (size_t)k * de;
#pragma unroll
        for (int j = 0; j < kAttMaxCt; ++j) {
            const int c = cg + 16 * j;
            if (j < ct && c < de) {
                const float wv = __ldg(w + c);
#pragma unroll
                for (int i = 0; i < 4; ++i) acc[i][j] = fmaf(wv, x[i], acc[i][j]);
            }
        }
    }
#pragma unroll
    for (int j = 0; j < kAttMaxCt; ++j) {
        const int c = cg + 16 * j;
        if (j < ct && c < de) {
            const float sc = __ldg(A.scale + c), sh = __ldg(A.shift + c);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int r = 4 * rg + i;
                Z[c * ROWS + r] = fmaf(acc[i][j], sc, sh) * P[c * ROWS + r];
            }
        }
    }
}

// Feature transformer s on `in` (k = de for the first layer).  Returns the
// buffer holding its N outputs.  Widths 16, 32, 64 and 128 run the
// CTA-wide tiled layer, others the per-row one.
template <int ROWS>
__device__ __forceinline__ float* feature_transformer(const SimtParams& p, int s, const float* in,
                                                      float* b0, float* b1, int r, int q) {
    const int lpf = p.m.layers_per_ft, N = p.m.N;
    const float* cur = in;
    float* nxt = b1;
    __syncthreads();  // every row's input is in place
    for (int l = 0; l < lpf; ++l) {
        const SimtLayer& L = p.ft[s * lpf + l];
        switch (N) {
            case 16: glu_layer_tiled<ROWS, 1>(L, cur, nxt, l == 0, N); break;
            case 32: glu_layer_tiled<ROWS, 2>(L, cur, nxt, l == 0, N); break;
            case 64: glu_layer_tiled<ROWS, 4>(L, cur, nxt, l == 0, N); break;
            case 128: glu_layer_tiled<ROWS, 8>(L, cur, nxt, l == 0, N); break;
            default: glu_layer<ROWS>(L, cur, nxt, l == 0, N, r, q);
        }
        __syncthreads();
        cur = nxt;
        nxt = (nxt == b1) ? b0 : b1;
    }
    return const_cast<float*>(cur);
}

template <int ROWS>
__global__ void __launch_bounds__(ROWS * TPR)
simt_forward_kernel(const SimtParams p, const float* __restrict__ x_num,
                    const int* __restrict__ x_cat, int64_t rows, float* __restrict__ logits,
                    float* __restrict__ masks, float* __restrict__ agg_out) {
    extern __shared__ float sm[];
    const ModelConsts& m = p.m;
    const int de = m.de, N = m.N, D = m.d, n_d = m.n_d;
    const int kmax = de > N ? de : N;
    float* F = sm;                    // [de]   BN'd embedded input
    float* P = F + de * ROWS;         // [de]   prior
    float* Z = P + de * ROWS;         // [de]   attentive output, then the mask
    float* B0 = Z + de * ROWS;        // [kmax] layer buffer
    float* B1 = B0 + kmax * ROWS;     // [N]    layer buffer
    float* AGG = B1 + N * ROWS;       // [D]    aggregate per feature
    float* ACC = AGG + D * ROWS;      // [n_d]  decision accumulator

    const int r = threadIdx.x / TPR, q = threadIdx.x % TPR;
    const int64_t total = total_rows(p.seg, rows);
    const int64_t num_tiles = (total + ROWS - 1) / ROWS;
  for (int64_t tile = blockIdx.x; tile < num_tiles; tile += gridDim.x) {
    const RowIO io = row_io(p.seg, m, tile * ROWS + r, total, x_num, x_cat, logits, masks, agg_out);
    const bool valid = io.valid;
    __syncwarp(row_mask());

    // Embedding lookup and input BN (features j = q mod 4).
    for (int j = q; j < D; j += TPR) {
        const int c0 = m.feat_col[j];
        if (j < m.n_num) {
            const float x = valid ? io.x_num[j] : 0.f;
            F[c0 * ROWS + r] = fmaf(__ldg(m.s0 + c0), x, __ldg(m.t0 + c0));
        } else {
            const int jc = j - m.n_num;
            const int len = m.feat_len[j];
            const int idx = valid ? io.x_cat[jc] - m.cat_base[jc] : 0;
            const bool oob = idx < 0 || idx >= m.cat_card[jc];
            if (oob) atomicOr(m.status, TABNET_STATUS_CAT_OOB);
            const float* t = m.emb + m.cat_off[jc] + (size_t)(oob ? 0 : idx) * len;
            for (int e = 0; e < len; ++e)
                F[(c0 + e) * ROWS + r] = oob ? __ldg(m.t0 + c0 + e) : __ldg(t + e);
        }
    }
    for (int c = q; c < de; c += TPR) P[c * ROWS + r] = 1.f;
    for (int j = q; j < D; j += TPR) AGG[j * ROWS + r] = 0.f;
    for (int c = q; c < n_d; c += TPR) ACC[c * ROWS + r] = 0.f;
    __syncwarp(row_mask());

    float* out = feature_transformer<ROWS>(p, 0, F, B0, B1, r, q);

    for (int i = 0; i < m.n_steps; ++i) {
        // Attentive transformer: z = BN(W_att a) * P.
        const SimtLayer& A = p.att[i];
        if (de <= 16 * kAttMaxCt) {
            attentive_tiled<ROWS>(A, out + n_d * ROWS, P, Z, de, m.n_a);
            __syncthreads();  // every row's z is in place
        } else {
            for (int c = q; c < de; c += TPR) {
                float acc = 0.f;
                for (int k = 0; k < m.n_a; ++k)
                    acc = fmaf(__ldg(A.wt + (size_t)k * de + c), out[(n_d + k) * ROWS + r], acc);
                const float u = fmaf(acc, __ldg(A.scale + c), __ldg(A.shift + c));
                Z[c * ROWS + r] = u * P[c * ROWS + r];
            }
            __syncwarp(row_mask());
        }
        // Sparsemax by Michelot's fixed point: tau = (sum_S z - 1) / |S| over
        // S = {z > tau}, starting from S = all columns, until S stops shrinking.
        float s = 0.f;
        for (int c = q; c < de; c += TPR) s += Z[c * ROWS + r];
        s = sum4(s);
        float tau = (s - 1.f) / (float)de;
        int prev = de;
        for (int it = 0; it < de; ++it) {
            float ss = 0.f;
            int cnt = 0;
            for (int c = q; c < de; c += TPR) {
                const float z = Z[c * ROWS + r];
                if (z > tau) { ss += z; ++cnt; }
            }
            ss = sum4(ss);
            cnt = sum4i(cnt);
            if (cnt == prev || cnt == 0) break;
            prev = cnt;
            tau = (ss - 1.f) / (float)cnt;
        }
        // Mask, prior update, masked input, mask output.
        float* mrow = (io.masks && valid) ? io.masks + (size_t)i * de : nullptr;
        for (int c = q; c < de; c += TPR) {
            const float mk = fmaxf(Z[c * ROWS + r] - tau, 0.f);
            Z[c * ROWS + r] = mk;
            P[c * ROWS + r] *= (m.gamma - mk);
            B0[c * ROWS + r] = mk * F[c * ROWS + r];
            if (mrow) mrow[c] = mk;
        }
        __syncwarp(row_mask());
        out = feature_transformer<ROWS>(p, i + 1, B0, B0, B1, r, q);
        // Decision output: acc += ReLU(d), eta = sum ReLU(d), agg += eta * M.
        float eta = 0.f;
        for (int c = q; c < n_d; c += TPR) {
            const float dv = fmaxf(out[c * ROWS + r], 0.f);
            ACC[c * ROWS + r] += dv;
            eta += dv;
        }
        eta = sum4(eta);
        for (int j = q; j < D; j += TPR) {
            const int c0 = m.feat_col[j], len = m.feat_len[j];
            float a = AGG[j * ROWS + r];
            for (int e = 0; e < len; ++e) a = fmaf(eta, Z[(c0 + e) * ROWS + r], a);
            AGG[j * ROWS + r] = a;
        }
        __syncwarp(row_mask());
    }

    // Final linear and the normalised aggregate.
    for (int k = q; k < m.n_classes; k += TPR) {
        float acc = __ldg(m.bf + k);
        for (int c = 0; c < n_d; ++c) acc = fmaf(__ldg(m.wf + (size_t)k * n_d + c), ACC[c * ROWS + r], acc);
        if (valid) io.logits[k] = acc;
    }
    float tot = 0.f;
    for (int j = q; j < D; j += TPR) tot += AGG[j * ROWS + r];
    tot = sum4(tot);
    if (io.agg && valid) {
        const float inv = tot > 0.f ? 1.f / tot : 0.f;
        for (int j = q; j < D; j += TPR) io.agg[j] = tot > 0.f ? AGG[j * ROWS + r] * inv : 0.f;
    }
  }
}

}  // namespace

size_t simt_smem_bytes(const ModelConsts& m, int rows_per_cta) {
    const int kmax = m.de > m.N ? m.de : m.N;
    return (size_t)(3 * m.de + kmax + m.N + m.d + m.n_d) * rows_per_cta * sizeof(float);
}

int simt_occupancy(int rows_per_cta, size_t smem) {
    int n = 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (rows_per_cta) {
        case 32: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, simt_forward_kernel<32>, 32 * TPR, smem); break;
        case 16: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, simt_forward_kernel<16>, 16 * TPR, smem); break;
        case 8: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, simt_forward_kernel<8>, 8 * TPR, smem); break;
    }
    return (e == cudaSuccess && n > 0) ? n : 1;
}

cudaError_t simt_configure(int rows_per_cta, size_t smem) {
    switch (rows_per_cta) {
        case 32: return cudaFuncSetAttribute(simt_forward_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        case 16: return cudaFuncSetAttribute(simt_forward_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        case 8:  return cudaFuncSetAttribute(simt_forward_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
    return cudaErrorInvalidValue;
}

cudaError_t simt_launch(const SimtParams& p, int rows_per_cta, const float* x_num, const int* x_cat,
                        int64_t rows, float* logits, float* masks, float* agg, cudaStream_t stream,
                        int max_ctas) {
    const size_t smem = simt_smem_bytes(p.m, rows_per_cta);
    // persistent: at most max_ctas CTAs loop over the tiles (a segmented
    // launch learns its row count on the device and takes all of them)
    int64_t grid = p.seg.segs ? max_ctas : std::min<int64_t>((rows + rows_per_cta - 1) / rows_per_cta, max_ctas);
    if (grid < 1) grid = 1;
    const dim3 block(rows_per_cta * TPR);
    switch (rows_per_cta) {
        case 32: simt_forward_kernel<32><<<(unsigned)grid, block, smem, stream>>>(p, x_num, x_cat, rows, logits, masks, agg); break;
        case 16: simt_forward_kernel<16><<<(unsigned)grid, block, smem, stream>>>(p, x_num, x_cat, rows, logits, masks, agg); break;
        case 8:  simt_forward_kernel<8><<<(unsigned)grid, block, smem, stream>>>(p, x_num, x_cat, rows, logits, masks, agg); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace tabnet
