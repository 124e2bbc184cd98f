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

// ------------------------------------------------------------------
// Latency form for small batches: one warp per row, the layers' weights
// staged in shared memory.
//
// A call of few rows leaves the four-lanes-per-row kernel with few CTAs
// (1,024 rows at 32 rows a CTA are 32 CTAs on 148 SMs), and each row's chain
// is then bound by the latency of its weight reads: one dependent L2 round
// trip every few FMAs, since L1 starts cold at every launch.  Here a CTA
// holds W rows, one warp each, and reads the layers from shared memory.  The
// host lays the layers out as "units" in forward order (SimtParams::row_units);
// a model whose units all fit is copied whole at the start, with no CTA
// barrier after that, and a larger one streams through a ring of nbuf slots
// with cp.async, nbuf - 1 units ahead of the one being computed.  Lane t of
// a row's warp computes the pre-activations 4t .. 4t + 3 (+ 128 j) of a
// layer from float4 reads.
//
// The arithmetic is the four-lane kernel's, so the results are bit for bit
// those of simt_forward_kernel whatever the batch size: every pre-activation
// is the same sequential FMA chain over k from the same weights, the GLU and
// attentive epilogues are the same expressions, and every row-level sum
// (the sparsemax sums and counts, eta, the aggregate total) is formed as the
// partial sums over the columns q, q + 4, q + 8, ... in order (q < 4),
// combined as (p0 + p1) + (p2 + p3).

__device__ __forceinline__ void cp_async16(float* dst, const float* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(__cvta_generic_to_global(src)) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// Wait until at most n (capped at 7) of this thread's groups are pending:
// waiting for more than asked is still correct.
__device__ __forceinline__ void cp_async_wait(int n) {
    switch (n < 7 ? n : 7) {
        case 0: asm volatile("cp.async.wait_group 0;\n" ::: "memory"); break;
        case 1: asm volatile("cp.async.wait_group 1;\n" ::: "memory"); break;
        case 2: asm volatile("cp.async.wait_group 2;\n" ::: "memory"); break;
        case 3: asm volatile("cp.async.wait_group 3;\n" ::: "memory"); break;
        case 4: asm volatile("cp.async.wait_group 4;\n" ::: "memory"); break;
        case 5: asm volatile("cp.async.wait_group 5;\n" ::: "memory"); break;
        case 6: asm volatile("cp.async.wait_group 6;\n" ::: "memory"); break;
        default: asm volatile("cp.async.wait_group 7;\n" ::: "memory"); break;
    }
}

// n floats (a multiple of 4) from global src to shared dst, both 16-byte
// aligned, spread over the CTA's threads.
__device__ __forceinline__ void copy_async(float* dst, const float* src, int n) {
    for (int i = 4 * (int)threadIdx.x; i < n; i += 4 * (int)blockDim.x) cp_async16(dst + i, src + i);
}

// Unit u into its ring slot (nothing past the last unit), then one commit,
// so that every thread commits exactly one group per unit index.
__device__ __forceinline__ void row_issue(const SimtParams& p, int u, int n_units, float* ring, int nbuf) {
    if (u < n_units) {
        const ModelConsts& m = p.m;
        int k, n_out, a, f;
        row_unit_shape(u, m.layers_per_ft, m.de, m.N, m.n_a, &k, &n_out, &a, &f);
        copy_async(ring + (size_t)(u % nbuf) * p.row_slot, p.row_units + (size_t)u * p.row_slot,
                   row_unit_floats(k, n_out));
    }
    cp_async_commit();
}

// y[o] = sum_k w[o][k] x[k] as one sequential FMA chain per o (k = 0, 1,
// ...), for the outputs o = lane + 32 (j0 + j), j < J, o < ld: a lane reads
// four k steps of its output's weights as one float4 (X4: and of x, which
// must then be 16-byte aligned).
template <int J, bool X4>
__device__ __forceinline__ void preact_chunk(const float* w, int k, int kp, int ld, const float* x, float* y,
                                             int lane, int j0) {
    float acc[J];
    const float* wo[J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
        acc[j] = 0.f;
        wo[j] = w + (size_t)(lane + 32 * (j0 + j)) * kp;
    }
    int kk = 0;
    if (X4) {
#pragma unroll 4
        for (; kk + 4 <= k; kk += 4) {
            const float4 xv = *reinterpret_cast<const float4*>(x + kk);
#pragma unroll
            for (int j = 0; j < J; ++j)
                if (lane + 32 * (j0 + j) < ld) {
                    const float4 wv = *reinterpret_cast<const float4*>(wo[j] + kk);
                    acc[j] = fmaf(wv.x, xv.x, acc[j]);
                    acc[j] = fmaf(wv.y, xv.y, acc[j]);
                    acc[j] = fmaf(wv.z, xv.z, acc[j]);
                    acc[j] = fmaf(wv.w, xv.w, acc[j]);
                }
        }
    }
    for (; kk < k; ++kk) {
        const float xs = x[kk];
#pragma unroll
        for (int j = 0; j < J; ++j)
            if (lane + 32 * (j0 + j) < ld) acc[j] = fmaf(wo[j][kk], xs, acc[j]);
    }
#pragma unroll
    for (int j = 0; j < J; ++j)
        if (lane + 32 * (j0 + j) < ld) y[lane + 32 * (j0 + j)] = acc[j];
}

template <bool X4>
__device__ __forceinline__ void preact_rows(const float* w, int k, int ld, const float* x, float* y, int lane) {
    const int kp = row_kp(k), jn = (ld + 31) >> 5;
    if (jn == 1) preact_chunk<1, X4>(w, k, kp, ld, x, y, lane, 0);
    else if (jn == 2) preact_chunk<2, X4>(w, k, kp, ld, x, y, lane, 0);
    else
        for (int j0 = 0; j0 < jn; j0 += 4) preact_chunk<4, X4>(w, k, kp, ld, x, y, lane, j0);
}

// y[0 .. ld) for the calling warp's row from unit weights w ([ld][kp]).
// (Two call sites, the feature-transformer layer and the attentive layer.)
__device__ __forceinline__ void preact_row(const float* w, int k, int ld, const float* x, float* y, int lane) {
    if ((reinterpret_cast<uintptr_t>(x) & 15) == 0) preact_rows<true>(w, k, ld, x, y, lane);
    else preact_rows<false>(w, k, ld, x, y, lane);
}

// sum4 over lanes 0..3 (each holding its partial), the result in every lane
__device__ __forceinline__ float warp_sum4(float v) {
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    return __shfl_sync(0xffffffffu, v, 0);
}
__device__ __forceinline__ int warp_sum4i(int v) {
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    return __shfl_sync(0xffffffffu, v, 0);
}

// Start of unit u: issue unit u + nbuf - 1 into the slot that unit u - 1
// left, wait for unit u's copies (this thread's, then the CTA's), and
// return its slot.  The CTA barrier at the end of the previous unit is what
// frees that slot.  With every unit resident (whole) there is nothing to
// wait for.
__device__ __forceinline__ const float* unit_begin(const SimtParams& p, int u, int n_units, float* ring, int nbuf,
                                                   bool whole) {
    if (!whole) {
        row_issue(p, u + nbuf - 1, n_units, ring, nbuf);
        cp_async_wait(nbuf - 1);
        __syncthreads();
    }
    return ring + (size_t)(whole ? u : u % nbuf) * p.row_slot;
}
__device__ __forceinline__ void unit_end(bool whole) {
    if (whole) __syncwarp();
    else __syncthreads();
}

// Sparsemax sums over z > tau (over all of z when `all`), as lanes 0..3 of
// the four-lane kernel form them: partial sums p_q over the columns
// q, q + 4, q + 8, ... in order, total (p0 + p1) + (p2 + p3).  Up to 64
// columns every lane forms all four from broadcast reads (no shuffles);
// wider rows take lanes 0..3 and two shuffle rounds.
__device__ __forceinline__ void thresh_add(float z, float tau, bool all, float& p, int& cnt) {
    if (all || z > tau) {
        p += z;
        ++cnt;
    }
}

// sum over c < n of v[c] as lanes 0..3 of the four-lane kernel form it
// (partials over c = q mod 4 in order, then (p0 + p1) + (p2 + p3)), formed
// by every lane from broadcast reads when n <= 64
template <typename F>
__device__ __forceinline__ float row_sum4(int n, int lane, F v) {
    if (n <= 64) {
        float p0 = 0.f, p1 = 0.f, p2 = 0.f, p3 = 0.f;
        int c = 0;
        for (; c + 4 <= n; c += 4) {
            p0 += v(c);
            p1 += v(c + 1);
            p2 += v(c + 2);
            p3 += v(c + 3);
        }
        if (c < n) p0 += v(c);
        if (c + 1 < n) p1 += v(c + 1);
        if (c + 2 < n) p2 += v(c + 2);
        return __fadd_rn(__fadd_rn(p0, p1), __fadd_rn(p2, p3));
    }
    float t = 0.f;
    if (lane < 4)
        for (int c = lane; c < n; c += 4) t += v(c);
    return warp_sum4(t);
}

// Michelot's threshold for a row of de <= R columns held in registers (every
// lane the same), with the sums formed as in row_thresh_sum.
template <int R>
__device__ __forceinline__ float sparsemax_tau_reg(const float* Z, int de) {
    float z[R];
#pragma unroll
    for (int c = 0; c < R; ++c) z[c] = c < de ? Z[c] : 0.f;
    auto sum = [&](float tau, bool all, int& cnt) {
        float p[4] = {0.f, 0.f, 0.f, 0.f};
        cnt = 0;
#pragma unroll
        for (int c = 0; c < R; ++c)
            if (c < de && (all || z[c] > tau)) {
                p[c & 3] += z[c];
                ++cnt;
            }
        return __fadd_rn(__fadd_rn(p[0], p[1]), __fadd_rn(p[2], p[3]));
    };
    int cnt = 0;
    float tau = (sum(0.f, true, cnt) - 1.f) / (float)de;
    int prev = de;
    for (int it = 0; it < de; ++it) {
        const float ss = sum(tau, false, cnt);
        if (cnt == prev || cnt == 0) break;
        prev = cnt;
        tau = (ss - 1.f) / (float)cnt;
    }
    return tau;
}

__device__ __forceinline__ float row_thresh_sum(const float* Z, int de, float tau, bool all, int lane, int* cnt_out) {
    if (de <= 64) {
        float p0 = 0.f, p1 = 0.f, p2 = 0.f, p3 = 0.f;
        int cnt = 0, c = 0;
        for (; c + 4 <= de; c += 4) {
            thresh_add(Z[c], tau, all, p0, cnt);
            thresh_add(Z[c + 1], tau, all, p1, cnt);
            thresh_add(Z[c + 2], tau, all, p2, cnt);
            thresh_add(Z[c + 3], tau, all, p3, cnt);
        }
        if (c < de) thresh_add(Z[c], tau, all, p0, cnt);
        if (c + 1 < de) thresh_add(Z[c + 1], tau, all, p1, cnt);
        if (c + 2 < de) thresh_add(Z[c + 2], tau, all, p2, cnt);
        *cnt_out = cnt;
        return __fadd_rn(__fadd_rn(p0, p1), __fadd_rn(p2, p3));
    }
    float ss = 0.f;
    int cnt = 0;
    if (lane < 4)
        for (int c = lane; c < de; c += 4) thresh_add(Z[c], tau, all, ss, cnt);
    *cnt_out = warp_sum4i(cnt);
    return warp_sum4(ss);
}

// Per-row shared-memory floats of the warp-per-row kernel: F, P, Z [de],
// B0 [max(de, N)], B1 [N], AGG [D], ACC [n_d], Y [max(2N, de)], each
// rounded up to 4 floats so that every buffer is 16-byte aligned.
__host__ __device__ __forceinline__ int row_state_floats(const ModelConsts& m) {
    const int kmax = m.de > m.N ? m.de : m.N;
    const int ymax = 2 * m.N > m.de ? 2 * m.N : m.de;
    return 3 * row_r4(m.de) + row_r4(kmax) + row_r4(m.N) + row_r4(m.d) + row_r4(m.n_d) + row_r4(ymax);
}

// Shared-memory words of the model's small tables, copied per CTA: input BN
// scale and shift [de], final linear [n_classes n_d] and bias [n_classes],
// feature column and width [D], categorical base, cardinality and table
// offset [n_cat].
__host__ __device__ __forceinline__ int row_const_words(const ModelConsts& m) {
    return 2 * row_r4(m.de) + row_r4(m.n_classes * m.n_d) + row_r4(m.n_classes) + 2 * row_r4(m.d) +
           3 * row_r4(m.n_cat);
}

__device__ __forceinline__ void load_table(float* dst, const float* src, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = __ldg(src + i);
}
__device__ __forceinline__ void load_table(int* dst, const int* src, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = __ldg(src + i);
}

constexpr int kRowWarpsMax = 16;  // rows (warps) per CTA at most: 128 registers a thread

__global__ void __launch_bounds__(32 * kRowWarpsMax)
simt_row_kernel(const SimtParams p, const float* __restrict__ x_num, const int* __restrict__ x_cat, int64_t rows,
                float* __restrict__ logits, float* __restrict__ masks, float* __restrict__ agg_out, int nbuf) {
    extern __shared__ __align__(16) float sm[];
    const ModelConsts& m = p.m;
    const int de = m.de, N = m.N, D = m.d, n_d = m.n_d, lpf = m.layers_per_ft, nc = m.n_classes;
    const int kmax = de > N ? de : N;
    const int n_units = row_n_units(lpf, m.n_steps);
    const int W = blockDim.x >> 5, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int ld_ft = row_r4(2 * N), ld_att = row_r4(de);
    float* ring = sm;  // [nbuf][row_slot]
    // the model's small tables
    float* s0 = ring + (size_t)nbuf * p.row_slot;
    float* t0 = s0 + row_r4(de);
    float* wf = t0 + row_r4(de);
    float* bf = wf + row_r4(nc * n_d);
    int* feat_col = reinterpret_cast<int*>(bf + row_r4(nc));
    int* feat_len = feat_col + row_r4(D);
    int* cat_base = feat_len + row_r4(D);
    int* cat_card = cat_base + row_r4(m.n_cat);
    int* cat_off = cat_card + row_r4(m.n_cat);
    // this warp's row
    float* F = s0 + row_const_words(m) + (size_t)w * row_state_floats(m);  // BN'd embedded input
    float* P = F + row_r4(de);      // prior
    float* Z = P + row_r4(de);      // attentive output, then the mask
    float* B0 = Z + row_r4(de);     // layer buffer
    float* B1 = B0 + row_r4(kmax);  // layer buffer
    float* AGG = B1 + row_r4(N);    // aggregate per feature
    float* ACC = AGG + row_r4(D);   // decision accumulator
    float* Y = ACC + row_r4(n_d);   // pre-activations
    const int64_t total = total_rows(p.seg, rows);
    // every unit resident: copied once, then no CTA barrier at all
    const bool whole = nbuf >= n_units;
    if (whole) {
        copy_async(ring, p.row_units, n_units * p.row_slot);
        cp_async_commit();
    }
    load_table(s0, m.s0, de);
    load_table(t0, m.t0, de);
    load_table(wf, m.wf, nc * n_d);
    load_table(bf, m.bf, nc);
    load_table(feat_col, m.feat_col, D);
    load_table(feat_len, m.feat_len, D);
    load_table(cat_base, m.cat_base, m.n_cat);
    load_table(cat_card, m.cat_card, m.n_cat);
    load_table(cat_off, m.cat_off, m.n_cat);
    bool first = true;
    // every warp takes part in every pass (a row past the end computes on
    // row 0's inputs and writes nothing), so the CTA barriers line up
    for (int64_t base = (int64_t)blockIdx.x * W; base < total; base += (int64_t)gridDim.x * W) {
        if (!whole)
            for (int u = 0; u < nbuf - 1; ++u) row_issue(p, u, n_units, ring, nbuf);
        const RowIO io = row_io(p.seg, m, base + w, total, x_num, x_cat, logits, masks, agg_out);
        const bool valid = io.valid;
        // the row's raw inputs of features lane + 32 q (q < 4) are read
        // before the first wait for the tables and units, so that the two
        // global round trips overlap
        float xr[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int j = lane + 32 * q;
            xr[q] = !valid || j >= D ? 0.f
                    : j < m.n_num    ? io.x_num[j]
                                     : __int_as_float(io.x_cat[j - m.n_num]);
        }
        if (first) {
            if (whole) cp_async_wait(0);
            __syncthreads();
            first = false;
        }
        // embedding lookup and input BN
        for (int j = lane; j < D; j += 32) {
            const int q = (j - lane) >> 5;
            const float xq = q == 0 ? xr[0] : q == 1 ? xr[1] : q == 2 ? xr[2] : q == 3 ? xr[3]
                           : !valid ? 0.f : j < m.n_num ? io.x_num[j] : __int_as_float(io.x_cat[j - m.n_num]);
            const int c0 = feat_col[j];
            if (j < m.n_num) {
                F[c0] = fmaf(s0[c0], xq, t0[c0]);
            } else {
                const int jc = j - m.n_num;
                const int len = feat_len[j];
                const int idx = valid ? __float_as_int(xq) - cat_base[jc] : 0;
                const bool oob = idx < 0 || idx >= cat_card[jc];
                if (oob) atomicOr(m.status, TABNET_STATUS_CAT_OOB);
                const float* t = m.emb + cat_off[jc] + (size_t)(oob ? 0 : idx) * len;
                for (int e = 0; e < len; ++e) F[c0 + e] = oob ? t0[c0 + e] : __ldg(t + e);
            }
        }
        for (int c = lane; c < de; c += 32) P[c] = 1.f;
        for (int j = lane; j < D; j += 32) AGG[j] = 0.f;
        for (int c = lane; c < n_d; c += 32) ACC[c] = 0.f;
        __syncwarp();

        int u = 0;
        const float* out = F;
        // step s = 0 is the initial feature transformer; each later step is
        // attentive transformer, sparsemax mask, feature transformer and
        // decision output (one call site for the feature transformer)
        for (int s = 0; s <= m.n_steps; ++s) {
            const int i = s - 1;
            const float* in = F;
            if (s > 0) {
                // attentive transformer: z = BN(W_att a) * P
                const float* sl = unit_begin(p, u, n_units, ring, nbuf, whole);
                preact_row(sl, m.n_a, ld_att, out + n_d, Y, lane);
                __syncwarp();
                const float* sc = sl + (size_t)ld_att * row_kp(m.n_a);
                const float* sh = sc + ld_att;
                for (int c = lane; c < de; c += 32) Z[c] = fmaf(Y[c], sc[c], sh[c]) * P[c];
                unit_end(whole);
                ++u;
                // sparsemax: Michelot's fixed point, the sums as the four-lane kernel forms them
                float tau;
                if (de <= 16) {
                    tau = sparsemax_tau_reg<16>(Z, de);
                } else if (de <= 32) {
                    tau = sparsemax_tau_reg<32>(Z, de);
                } else {
                    int cnt = 0;
                    const float zs = row_thresh_sum(Z, de, 0.f, true, lane, &cnt);
                    tau = (zs - 1.f) / (float)de;
                    int prev = de;
                    for (int it = 0; it < de; ++it) {
                        const float ss = row_thresh_sum(Z, de, tau, false, lane, &cnt);
                        if (cnt == prev || cnt == 0) break;
                        prev = cnt;
                        tau = (ss - 1.f) / (float)cnt;
                    }
                }
                // mask, prior update, masked input, mask output
                float* mrow = (io.masks && valid) ? io.masks + (size_t)i * de : nullptr;
                for (int c = lane; c < de; c += 32) {
                    const float mk = fmaxf(Z[c] - tau, 0.f);
                    Z[c] = mk;
                    P[c] *= (m.gamma - mk);
                    B0[c] = mk * F[c];
                    if (mrow) mrow[c] = mk;
                }
                __syncwarp();
                in = B0;
            }
            // feature transformer s on `in`, ping-ponging B1 / B0
            const float* cur = in;
            float* nxt = B1;
            for (int l = 0; l < lpf; ++l, ++u) {
                const float* sl = unit_begin(p, u, n_units, ring, nbuf, whole);
                const int k = l == 0 ? de : N;
                preact_row(sl, k, ld_ft, cur, Y, lane);
                __syncwarp();
                const float* sc = sl + (size_t)ld_ft * row_kp(k);
                const float* sh = sc + ld_ft;
                for (int c = lane; c < N; c += 32) {
                    const float ul = fmaf(Y[c], sc[c], sh[c]);
                    const float ug = fmaf(Y[N + c], sc[N + c], sh[N + c]);
                    const float g = __fmul_rn(ul, sigmoid_exact(ug));
                    nxt[c] = l == 0 ? g : __fmul_rn(__fadd_rn(cur[c], g), kSqrtHalf);
                }
                unit_end(whole);  // the slot is free, nxt complete
                cur = nxt;
                nxt = (nxt == B1) ? B0 : B1;
            }
            out = cur;
            if (s > 0) {
                // decision output: acc += ReLU(d), eta = sum ReLU(d), agg += eta * M
                const float eta = row_sum4(n_d, lane, [&](int c) { return fmaxf(out[c], 0.f); });
                for (int c = lane; c < n_d; c += 32) ACC[c] += fmaxf(out[c], 0.f);
                for (int j = lane; j < D; j += 32) {
                    const int c0 = feat_col[j], len = feat_len[j];
                    float a = AGG[j];
                    for (int e = 0; e < len; ++e) a = fmaf(eta, Z[c0 + e], a);
                    AGG[j] = a;
                }
                __syncwarp();
            }
        }
        // final linear and the normalised aggregate
        for (int k = lane; k < nc; k += 32) {
            float acc = bf[k];
            for (int c = 0; c < n_d; ++c) acc = fmaf(wf[k * n_d + c], ACC[c], acc);
            if (valid) io.logits[k] = acc;
        }
        const float tot = row_sum4(D, lane, [&](int j) { return AGG[j]; });
        if (io.agg && valid) {
            const float inv = tot > 0.f ? 1.f / tot : 0.f;
            for (int j = lane; j < D; j += 32) io.agg[j] = tot > 0.f ? AGG[j] * inv : 0.f;
        }
        __syncwarp();
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

static int slot_floats_of(const ModelConsts& m) { return row_slot_floats(m.de, m.N, m.n_a); }

// Bytes of shared memory for W rows a CTA and nbuf unit slots.
size_t simt_row_smem_bytes(const ModelConsts& m, int W, int nbuf) {
    return ((size_t)nbuf * slot_floats_of(m) + row_const_words(m) + (size_t)W * row_state_floats(m)) * sizeof(float);
}

cudaError_t simt_row_configure(size_t smem) {
    return cudaFuncSetAttribute(simt_row_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

// Rows per CTA (W) and unit slots for a call of `rows` rows: W spreads the
// rows over the SMs (at most w_max, and at most what leaves room for one
// slot), then as many slots as fit in smem_max, up to one per unit.
// Returns false when not even one row and one slot fit.
bool simt_row_plan(const ModelConsts& m, int64_t rows, int num_sms, int w_max, size_t smem_max, int* W, int* nbuf) {
    const size_t slot = (size_t)slot_floats_of(m) * sizeof(float);
    const size_t per_row = (size_t)row_state_floats(m) * sizeof(float);
    const size_t fixed0 = simt_row_smem_bytes(m, 0, 0);
    if (fixed0 + slot + per_row > smem_max) return false;
    const int64_t w_fit = (int64_t)((smem_max - fixed0 - slot) / per_row);
    const int64_t w = (rows + num_sms - 1) / num_sms;
    *W = (int)std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(w, w_max), w_fit));
    const size_t fixed = simt_row_smem_bytes(m, *W, 0);
    *nbuf = (int)std::min<size_t>((smem_max - fixed) / slot, (size_t)row_n_units(m.layers_per_ft, m.n_steps));
    return true;
}

cudaError_t simt_row_launch(const SimtParams& p, const float* x_num, const int* x_cat, int64_t rows, float* logits,
                            float* masks, float* agg, cudaStream_t stream, int num_sms, int w_max, size_t smem_max) {
    int W = 0, nbuf = 0;
    if (!simt_row_plan(p.m, rows, num_sms, std::min(w_max, kRowWarpsMax), smem_max, &W, &nbuf))
        return cudaErrorInvalidConfiguration;
    const size_t smem = simt_row_smem_bytes(p.m, W, nbuf);
    int64_t grid = (rows + W - 1) / W;
    if (grid < 1) grid = 1;
    if (grid > 65535) grid = 65535;
    simt_row_kernel<<<(unsigned)grid, 32 * W, smem, stream>>>(p, x_num, x_cat, rows, logits, masks, agg, nbuf);
    return cudaGetLastError();
}

}  // namespace tabnet
