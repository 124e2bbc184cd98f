// TabNet forward with the fully connected layers on the 5th-generation
// tensor cores (tcgen05, sm_103a): the bf16, split-bf16, three-part
// (float32-accurate) and FP8 E4M3 precision modes.
//
// One CTA owns a tile of 128 rows for the whole forward pass: the embedding
// and input BN, the step-0 feature transformer, then per decision step the
// attentive FC, sparsemax, prior update, masked input and the step's feature
// transformer, and finally the logits and the aggregated mask (TabNet as
// deployed in Sec. IV-A; masks as returned per call, Sec. III-B).  Only the
// inputs, the weights and the outputs touch global memory.  CTAs are
// persistent over tiles; a segmented launch finds each row's request.
//
//   * Tile start: the warps gather the tile's inputs together (each warp
//     32 rows, all of their loads in flight per column), fold the input BN
//     and keep f in shared memory; the next tile's rows are prefetched to L2.
//   * Every FC is a 128 x n x K tcgen05.mma chain (M = 128 rows; n = 2N for a
//     GLU layer, the padded mask width for the attentive layer) reading the
//     activations (A) and the layer's weights (B) from shared memory in the
//     128-byte-swizzled K-major layout and accumulating in fp32 in tensor
//     memory (TMEM lane = row).  In split mode both operands are carried as
//     hi + lo bf16 pairs and each K step issues hi*hi, hi*lo and lo*hi; with
//     three parts (hi, lo, lo2) the five products down to 2^-16 of hi*hi go
//     first and hi*hi last.  In FP8 mode (kind::f8f6f4, 32-element K steps)
//     the weights are E4M3 scaled per output channel (amax / 448, quantized
//     on the host) and every FC input is E4M3 scaled per row (amax / 448 of
//     the row's K inputs -- of the attention half for the attentive layer);
//     the epilogue multiplies the accumulator by both scales.  One phase
//     loop walks a tile's layers, so there is one MMA issue site.
//   * Weights stream from L2 through a ring of shared-memory slots filled by
//     1-D bulk async copies (TMA engine), one part of a K block (128 bytes a
//     row: 64 bf16 or 128 e4m3 elements) per slot, pre-swizzled by the host;
//     a K block's parts sit in consecutive slots and arrive by one copy (a
//     copy costs the issuing thread a few hundred cycles when every SM is
//     copying).  Warp 0 keeps the ring's bookkeeping in every lane (warp-
//     uniform descriptors and loop state) and its lane 0 issues copies and
//     MMAs; each such unit has a
//     "full" barrier (copy landed); a unit read by a layer's last K block is
//     free once the accumulator barrier fires, earlier blocks' units get
//     their own "empty" commit.
//   * Epilogue threads read the accumulator with tcgen05.ld (thread = row),
//     add the BN shift (the BN scale, -log2(e) for the gate and sqrt(1/2)
//     for the residual are folded into the packed weights), apply the GLU
//     and the residual (kept in fp32 registers), and write the next layer's
//     A operand straight into shared memory.
//   * Sparsemax runs in fp32, row per thread, by Michelot's fixed point on
//     the threshold (the sort-free exact projection); the prior P and the
//     current mask live in TMEM in fp32 (the mask is read again for the
//     aggregate once the step's decision output is known), the per-feature
//     aggregate in TMEM or shared memory.  Only when those fp32 regions do
//     not fit next to a 256-column accumulator (128 hidden units with a
//     160-column mask) is the mask kept as fp16 pairs.
//   * The attentive layer's MMA chain starts at K step n_d / 16: its weights
//     on the decision half of the feature transformer's output are zero.
//   * Masks and the aggregate leave through per-warp staging blocks as
//     64-byte row pieces.
//   * With NWG = 2 two warpgroups split the columns of each row and combine
//     partial sums through shared memory.
//
// Every wait is bounded: a wait that runs out sets TABNET_STATUS_TIMEOUT,
// the CTA stops at the next barrier, drains its copies and MMAs, frees its
// TMEM and exits.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "../../include/tabnet.h"
#include "model_handle.h"
#include "tc_ptx.cuh"

namespace tabnet {

namespace {

constexpr uint64_t kWaitLimit = 1000000000ull;  // 1 s per wait
constexpr float kSqrtHalf = 0.70710678118654752440f;
constexpr int kMaxClasses = 4;
constexpr int kFStride = 129;  // row stride (floats) of the input cache: transposed writes hit distinct banks
// sparsemax input kept in registers: up to this many 16-column chunks per thread
// (two warpgroups per row keep z in TMEM: their register budget is 128)
__host__ __device__ constexpr int zreg_chunks(int nwg) { return nwg == 1 ? 3 : 0; }

// Record a wait that ran out: the status bit, and the first location.
__device__ __forceinline__ void note_timeout(unsigned* status, unsigned kind, unsigned index) {
    atomicOr(status, TABNET_STATUS_TIMEOUT);
    if (atomicCAS(status + 1, 0u, (kind << 24) | (index & 0xFFFFFFu)) == 0u) status[2] = blockIdx.x;
}

// sigmoid(x) = 1 / (1 + 2^(-x log2 e)) with the ex2/rcp approximations
// (about 2^-21 relative): the gate of every tensor-core mode, so that a mode
// differs from float32 arithmetic only by its operand rounding.  The
// argument is y = -x log2 e, already scaled by the packed gate weights and
// shifts.
__device__ __forceinline__ float sigmoid_from_log2(float y) {
    float e, r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(y));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(1.0f + e));
    return r;
}

// Byte offset of 16-byte unit q (0..7) of row r inside a 128-row x 64-column
// bf16 block in the 128B-swizzled K-major layout.
__device__ __forceinline__ uint32_t sw128_off(int r, int q) {
    return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((q ^ (r & 7)) << 4));
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}

// Row r, K columns [16 ch, 16 ch + 16) of the A operand as NP bf16 parts:
// part 0 = bf16(v) into sA, and each further part the bf16 rounding of what
// the earlier parts leave (v - hi, then v - hi - mid) into sAlo, one part
// every `part_bytes`.  The remainders are exact in float32.
template <int NP>
__device__ __forceinline__ void store_a16(uint8_t* sA, uint8_t* sAlo, uint32_t part_bytes, int r, int ch,
                                          const float (&v)[16]) {
    uint32_t w[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) w[j] = pack_bf16(v[2 * j], v[2 * j + 1]);
    const uint32_t o0 = (uint32_t)((ch >> 2) * 16384) + sw128_off(r, (ch & 3) * 2);
    const uint32_t o1 = (uint32_t)((ch >> 2) * 16384) + sw128_off(r, (ch & 3) * 2 + 1);
    *reinterpret_cast<uint4*>(sA + o0) = make_uint4(w[0], w[1], w[2], w[3]);
    *reinterpret_cast<uint4*>(sA + o1) = make_uint4(w[4], w[5], w[6], w[7]);
    if constexpr (NP >= 2) {
        float rem[16];
        uint32_t l[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float2 hf = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w[j]));
            rem[2 * j] = v[2 * j] - hf.x;
            rem[2 * j + 1] = v[2 * j + 1] - hf.y;
            l[j] = pack_bf16(rem[2 * j], rem[2 * j + 1]);
        }
        *reinterpret_cast<uint4*>(sAlo + o0) = make_uint4(l[0], l[1], l[2], l[3]);
        *reinterpret_cast<uint4*>(sAlo + o1) = make_uint4(l[4], l[5], l[6], l[7]);
        if constexpr (NP >= 3) {
            uint32_t q[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float2 mf = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&l[j]));
                q[j] = pack_bf16(rem[2 * j] - mf.x, rem[2 * j + 1] - mf.y);
            }
            *reinterpret_cast<uint4*>(sAlo + part_bytes + o0) = make_uint4(q[0], q[1], q[2], q[3]);
            *reinterpret_cast<uint4*>(sAlo + part_bytes + o1) = make_uint4(q[4], q[5], q[6], q[7]);
        }
    }
}

// Row r, K columns [8 u, 8 u + 8) of the A operand (u = 8-column unit).
template <int NP>
__device__ __forceinline__ void store_a8(uint8_t* sA, uint8_t* sAlo, uint32_t part_bytes, int r, int u,
                                         const float (&v)[8]) {
    static_assert(NP <= 2, "the three-part split runs with one warpgroup (16-column pieces)");
    uint32_t w[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) w[j] = pack_bf16(v[2 * j], v[2 * j + 1]);
    const uint32_t o = (uint32_t)((u >> 3) * 16384) + sw128_off(r, u & 7);
    *reinterpret_cast<uint4*>(sA + o) = make_uint4(w[0], w[1], w[2], w[3]);
    if constexpr (NP >= 2) {
        uint32_t l[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float2 hf = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w[j]));
            l[j] = pack_bf16(v[2 * j] - hf.x, v[2 * j + 1] - hf.y);
        }
        *reinterpret_cast<uint4*>(sAlo + o) = make_uint4(l[0], l[1], l[2], l[3]);
    }
    (void)part_bytes;
}

// Row r, K columns [16 ch, 16 ch + 16) of an FP8 E4M3 A operand: v * inv
// rounded to nearest even and saturated at +-448, one byte per element (a
// 128-element K block is one 128-byte row of the 128B-swizzled layout).
__device__ __forceinline__ void store_a16_e4m3(uint8_t* sA, int r, int ch, const float (&v)[16], float inv) {
    uint32_t w[4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
        w[j] = (uint32_t)ptx::cvt_e4m3x2(v[4 * j] * inv, v[4 * j + 1] * inv) |
               ((uint32_t)ptx::cvt_e4m3x2(v[4 * j + 2] * inv, v[4 * j + 3] * inv) << 16);
    *reinterpret_cast<uint4*>(sA + (uint32_t)((ch >> 3) * 16384) + sw128_off(r, ch & 7)) = make_uint4(w[0], w[1], w[2], w[3]);
}

// Zero K columns [16 ch, 16 ch + 16) of row r of an FP8 A operand (the
// padding a 32-element K step reads past a width that is 16 mod 32).
__device__ __forceinline__ void zero_a16_e4m3(uint8_t* sA, int r, int ch) {
    *reinterpret_cast<uint4*>(sA + (uint32_t)((ch >> 3) * 16384) + sw128_off(r, ch & 7)) = make_uint4(0u, 0u, 0u, 0u);
}

// Folded-BN vectors: staged in shared memory (epi_s != 0, a shared address)
// or read through the read-only path from global memory.
template <bool STAGED>
__device__ __forceinline__ float4 ld_epi(const float* g, uint32_t epi_s, int idx) {
    if (STAGED || epi_s) return ptx::ld_shared_f4(epi_s + 4u * (uint32_t)idx);
    return __ldg(reinterpret_cast<const float4*>(g + idx));
}

// LEAN: the launch shape stages the BN shifts and the input cache in shared
// memory and keeps the aggregate in TMEM, so the kernel is compiled with only
// those paths (smaller code, fewer instruction misses).
template <int N, int NWG, int NP, bool ZREG, bool LEAN>
__global__ void __launch_bounds__(128 * NWG, (NWG == 2 && N <= 64) ? 2 : 1)
tc_forward_kernel(const TcParams p, const float* __restrict__ x_num, const int* __restrict__ x_cat,
                  int64_t rows, float* __restrict__ logits, float* __restrict__ masks,
                  float* __restrict__ agg_out) {
    constexpr int THREADS = 128 * NWG;
    constexpr int CPW = N / NWG;  // GLU output columns per warpgroup
    constexpr int RCH = CPW / 16;  // 16-column chunks per thread
    constexpr bool FP8 = NP == 0;         // FP8 E4M3 operands (one 8-bit part, per-row and per-channel scales)
    constexpr bool SPLIT = NP >= 2;       // operands carried in several bf16 parts
    constexpr int PARTS = FP8 ? 1 : NP;   // weight chunks (parts) per K block
    constexpr int kZregChunks = zreg_chunks(NWG);
    static_assert(CPW % 16 == 0, "each warpgroup takes whole 16-column chunks");

    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const ModelConsts& m = p.m;
    const int tid = threadIdx.x, wg = tid >> 7, lt = tid & 127, warp = tid >> 5;
    const uint32_t lane_off = (uint32_t)((warp & 3) * 32) << 16;

    uint8_t* sA = smem + p.sm.a_hi;
    uint8_t* sAlo = SPLIT ? smem + p.sm.a_lo : nullptr;
    const uint32_t a_part = SPLIT ? (uint32_t)(p.sm.a_lo - p.sm.a_hi) : 0u;  // bytes per operand part
    float* sAgg = reinterpret_cast<float*>(smem + (p.sm.agg >= 0 ? p.sm.agg : 0));
    float2* sX = reinterpret_cast<float2*>(smem + (p.sm.xch >= 0 ? p.sm.xch : 0));
    float* sWf = reinterpret_cast<float*>(smem + p.sm.wf);
    const uint32_t wf_s = ptx::smem_u32(sWf);
    const bool has_f = LEAN || p.sm.fcache >= 0;
    const uint32_t f_s = has_f ? ptx::smem_u32(smem + p.sm.fcache) : 0u;  // f cache (shared address)
    const uint32_t epi_s = (LEAN || p.sm.epi >= 0) ? ptx::smem_u32(smem + p.sm.epi) : 0u;  // BN vectors
    const float* epi = p.epi;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + p.sm.bar);
    const int S = p.n_slots;
    volatile uint32_t* sTmem = reinterpret_cast<volatile uint32_t*>(bars + 2 * S + 1);
    // Stop flags, one per layer parity: a thread that finds during layer L
    // that the CTA has to stop sets the flag of layer L + 1, which every
    // thread reads after that layer's CTA barrier -- never the flag of the
    // layer whose flag other threads may still be reading.
    volatile int* sAbort = reinterpret_cast<volatile int*>(bars + 2 * S + 2);
    const uint32_t bar_full = ptx::smem_u32(bars);
    const uint32_t bar_empty = ptx::smem_u32(bars + S);
    const uint32_t bar_acc = ptx::smem_u32(bars + 2 * S);
    const uint32_t a_base = ptx::smem_u32(sA);
    const uint32_t ring_base = ptx::smem_u32(smem + p.sm.ring);

    if (tid == 0) {
        for (int s = 0; s < 2 * S + 1; ++s) ptx::mbar_init(bar_full + 8 * s, 1);
        sAbort[0] = 0;
        sAbort[1] = 0;
        ptx::fence_mbar_init();
    }
    if (warp == 0) {
        ptx::tmem_alloc(ptx::smem_u32((const void*)sTmem), (uint32_t)p.tmem_cols);
        ptx::tmem_relinquish();
    }
    // model constants staged once per CTA
    int* sColf = reinterpret_cast<int*>(smem + p.sm.colf);
    for (int i = tid; i < p.dp; i += THREADS) sColf[i] = __ldg(p.col_feat + i);
    uint2* sChunks = reinterpret_cast<uint2*>(smem + p.sm.chunks);
    for (int i = tid; i < p.chunks_per_tile; i += THREADS) sChunks[i] = __ldg(p.chunks + i);
    for (int i = tid; i < m.n_classes * N; i += THREADS) {
        const int k = i / N, c = i % N;
        sWf[i] = c < m.n_d ? __ldg(m.wf + k * m.n_d + c) : 0.f;
    }
    if (p.sm.epi >= 0)
        for (int i = tid; i < p.epi_floats / 4; i += THREADS)
            reinterpret_cast<float4*>(smem + p.sm.epi)[i] = __ldg(reinterpret_cast<const float4*>(p.epi) + i);
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = *sTmem;
    const uint32_t t_acc = tmem + lane_off;
    const uint32_t t_p = t_acc + (uint32_t)p.tm_p;
    const uint32_t t_m = t_acc + (uint32_t)p.tm_m;
    const bool agg_tmem = LEAN || p.tm_agg >= 0;
    const uint32_t t_agg = t_acc + (uint32_t)(agg_tmem ? p.tm_agg : 0);
    // the last 16-column chunk of the P / mask / aggregate regions holds 8
    // columns when the mask width leaves at most 8 in it
    const bool tail8 = p.tail8 != 0;
    // step mask kept as fp16 pairs (TMEM budget); never in a LEAN launch,
    // whose aggregate fits in TMEM next to fp32 P and mask regions
    const bool m16 = !LEAN && p.m16 != 0;
    const int dchunks = p.dp / 16;
    // 16 columns of a P / mask / aggregate region (8 in a half chunk, the
    // rest read as 0); the caller waits with tmem_wait_ld
    auto tm_ld = [&](uint32_t taddr, int ch, uint32_t (&r)[16]) {
        if (tail8 && ch == dchunks - 1) {
#pragma unroll
            for (int j = 8; j < 16; ++j) r[j] = 0u;
            ptx::tmem_ld8_lo(taddr, r);
        } else {
            ptx::tmem_ld16(taddr, r);
        }
    };
    auto tm_st = [&](uint32_t taddr, int ch, const uint32_t (&r)[16]) {
        if (tail8 && ch == dchunks - 1) {
            uint32_t h[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) h[j] = r[j];
            ptx::tmem_st8(taddr, h);
        } else {
            ptx::tmem_st16(taddr, r);
        }
    };

    const int64_t total = total_rows(p.seg, rows);
    const int64_t num_tiles = (total + 127) / 128;
    const int64_t my_tiles =
        (int64_t)blockIdx.x < num_tiles ? (num_tiles - 1 - (int64_t)blockIdx.x) / gridDim.x + 1 : 0;
    // The ring holds SU units of PARTS consecutive slots; a unit is one K
    // block of one layer with all its parts, brought in by one bulk copy (the
    // parts are contiguous in the weight stream), with one full and one empty
    // barrier.
    const int SU = S / PARTS;
    const int64_t total_chunks = my_tiles * p.chunks_per_tile;
    // Ring bookkeeping (every lane of warp 0), incremental so that no 64-bit
    // division sits on the MMA critical path: unit g of the CTA's stream
    // goes to ring unit g mod SU in round g / SU, and is unit g mod
    // chunks_per_tile of a tile's sequence.
    int64_t g_issue = 0, g_cons = 0;  // units issued / consumed so far
    int is_slot = 0, is_chunk = 0;    // ring unit and per-tile index of unit g_issue
    int cs_slot = 0;                  // ring unit of unit g_cons
    uint32_t cs_round = 0;            // round of unit g_cons
    // Ring units whose release is signalled on their own "empty" barrier (a
    // K block followed by more blocks of the same layer) and the parity to
    // wait for; the last block's unit is released by the accumulator barrier.
    uint32_t empty_pending = 0, empty_par = 0;
    bool acc_outstanding = false;
    uint32_t acc_phase = 0;
    int xc = 0;
    int lc = 0;  // layers run by this CTA

    // Warp 0 drives the ring and the MMAs: every lane runs the bookkeeping
    // (so the descriptors and loop state are warp-uniform) and lane 0 issues
    // the copies, MMAs and commits.  A wait's outcome is lane 0's.
    const int lane_id = tid & 31;
    auto warp_wait = [&](uint32_t bar, uint32_t parity) -> bool {
        const bool w = ptx::mbar_wait(bar, parity, kWaitLimit);
        return __shfl_sync(0xffffffffu, w ? 1 : 0, 0) != 0;
    };
    // Start the copy of unit g_issue once its ring unit is free (the MMAs
    // that read its previous occupant have completed).
    auto issue_next = [&]() -> bool {
        const int slot = is_slot;
        if (empty_pending & (1u << slot)) {
            if (!warp_wait(bar_empty + 8 * slot, (empty_par >> slot) & 1u)) {
                if (lane_id == 0) note_timeout(m.status, 5, (unsigned)g_issue);
                return false;
            }
            empty_par ^= 1u << slot;
            empty_pending &= ~(1u << slot);
        }
        const uint2 ck = sChunks[is_chunk];
        if (lane_id == 0) {
            ptx::mbar_arrive_expect_tx(bar_full + 8 * slot, ck.y);
            ptx::bulk_g2s(ring_base + (uint32_t)(slot * PARTS * p.slot_bytes), p.wbase + ck.x, ck.y,
                          bar_full + 8 * slot);
        }
        ++g_issue;
        if (++is_chunk == p.chunks_per_tile) is_chunk = 0;
        if (++is_slot == SU) is_slot = 0;
        return true;
    };
    if (warp == 0)
        while (g_issue < total_chunks && g_issue < SU) issue_next();

    // Publish this thread's A-operand writes and TMEM reads, then let warp 0
    // run one layer's MMA chain (K steps of 16 columns [kbeg, kend) over the
    // 64-wide K blocks that hold them) and wait for the accumulator.
    // Returns false when the CTA has to stop.
    // nout: the layer's output rows (its weight block has nout rows of 128
    // bytes, and the parts of a unit follow each other at that stride).
    auto run_mma = [&](int kbeg, int kend, uint32_t idesc, int nout) -> bool {
        ptx::fence_proxy_async();
        ptx::tc_fence_before();
        __syncthreads();
        if (sAbort[lc & 1]) return false;
        if (warp == 0) {
            ptx::tc_fence_after();
            bool ok = true;
#pragma unroll 1
            for (int b = kbeg >> 2; 4 * b < kend && ok; ++b) {
                while (ok && g_issue < g_cons + 1) ok = issue_next();
                // this K block's unit: its parts in consecutive slots
                if (ok && !warp_wait(bar_full + 8 * cs_slot, cs_round & 1u)) {
                    if (lane_id == 0) note_timeout(m.status, 1, (unsigned)g_cons);
                    ok = false;
                }
                if (!ok) break;
                // descriptors of the block's first K step; a K step of 16
                // bf16 (32 bytes) adds 2 to the encoded start address
                uint64_t d_b[PARTS], d_a[PARTS];  // part k of W and of A for this K block
#pragma unroll
                for (int part = 0; part < PARTS; ++part) {
                    d_b[part] = ptx::sw128_desc(ring_base + (uint32_t)(cs_slot * PARTS * p.slot_bytes + part * nout * 128));
                    d_a[part] = ptx::sw128_desc(a_base + (uint32_t)part * a_part + (uint32_t)(b * 16384));
                }
                const int k0 = max(kbeg - 4 * b, 0), k1 = min(kend - 4 * b, 4);
                if (lane_id == 0) {  // the block's MMAs, then release its unit if more blocks follow
                    if constexpr (NP == 3) {
                        // Products whose parts' significance reaches 2^-16 of hi hi:
                        // the five small ones first, so that most additions into
                        // the accumulator happen while it is still small (each
                        // rounds relative to the running sum), then hi hi.
#pragma unroll
                        for (int k4 = 0; k4 < 4; ++k4) {
                            if (k4 >= k0 && k4 < k1) {
                                const uint64_t step = 2u * (uint32_t)k4;
                                ptx::mma_f16(tmem, d_a[0] + step, d_b[1] + step, idesc, (4 * b + k4) > kbeg ? 1u : 0u);
                                ptx::mma_f16(tmem, d_a[1] + step, d_b[0] + step, idesc, 1u);
                                ptx::mma_f16(tmem, d_a[0] + step, d_b[2] + step, idesc, 1u);
                                ptx::mma_f16(tmem, d_a[1] + step, d_b[1] + step, idesc, 1u);
                                ptx::mma_f16(tmem, d_a[2] + step, d_b[0] + step, idesc, 1u);
                            }
                        }
#pragma unroll
                        for (int k4 = 0; k4 < 4; ++k4) {
                            if (k4 >= k0 && k4 < k1) {
                                const uint64_t step = 2u * (uint32_t)k4;
                                ptx::mma_f16(tmem, d_a[0] + step, d_b[0] + step, idesc, 1u);
                            }
                        }
                    } else if constexpr (FP8) {
                        // 32 e4m3 elements (32 bytes) per K step
#pragma unroll
                        for (int k4 = 0; k4 < 4; ++k4) {
                            if (k4 >= k0 && k4 < k1) {
                                const uint64_t step = 2u * (uint32_t)k4;
                                ptx::mma_f8(tmem, d_a[0] + step, d_b[0] + step, idesc, (4 * b + k4) > kbeg ? 1u : 0u);
                            }
                        }
                    } else {
#pragma unroll
                        for (int k4 = 0; k4 < 4; ++k4) {
                            if (k4 >= k0 && k4 < k1) {
                                // hi hi; with two parts also hi lo and lo hi
                                const uint64_t step = 2u * (uint32_t)k4;
                                ptx::mma_f16(tmem, d_a[0] + step, d_b[0] + step, idesc, (4 * b + k4) > kbeg ? 1u : 0u);
                                if constexpr (NP >= 2) {
                                    ptx::mma_f16(tmem, d_a[0] + step, d_b[1] + step, idesc, 1u);
                                    ptx::mma_f16(tmem, d_a[1] + step, d_b[0] + step, idesc, 1u);
                                }
                            }
                        }
                    }
                    if (4 * (b + 1) < kend) ptx::mma_commit(bar_empty + 8 * cs_slot);
                }
                if (4 * (b + 1) < kend) empty_pending |= 1u << cs_slot;
                g_cons += 1;
                if (++cs_slot == SU) { cs_slot = 0; ++cs_round; }
            }
            if (lane_id == 0) ptx::mma_commit(bar_acc);
            acc_outstanding = true;
            if (!ok) sAbort[(lc + 1) & 1] = 1;
        }
        __syncwarp();
        // With two warpgroups every thread waits for the accumulator itself,
        // suspended in the barrier's try-wait (no issue slots spent), so each
        // warp's epilogue starts as soon as the MMAs complete rather than
        // after warp 0 has woken, refilled the ring and released a 256-thread
        // barrier (+2 % on the 100-input model).  With one warpgroup warp 0
        // waits alone and the others park on the CTA barrier (the all-thread
        // wait measured 1 % slower there).  No thread can fall a phase behind:
        // the next commit needs every thread at the next layer's CTA barrier.
        constexpr bool kAllWait = NWG == 2;
        bool got = true;
        if (warp == 0) got = warp_wait(bar_acc, acc_phase);
        else if (kAllWait) got = ptx::mbar_wait(bar_acc, acc_phase, kWaitLimit);
        if (!got) {
            sAbort[(lc + 1) & 1] = 1;
            if (warp != 0 || lane_id == 0) note_timeout(m.status, 2, (unsigned)lc);
        }
        if (warp == 0) {
            if (got) acc_outstanding = false;
            // every MMA so far has completed: refill the free slots
            if (__shfl_sync(0xffffffffu, sAbort[(lc + 1) & 1], 0) == 0)
                while (g_issue < total_chunks && g_issue < g_cons + SU)
                    if (!issue_next()) { sAbort[(lc + 1) & 1] = 1; break; }
        }
        acc_phase ^= 1;
        ++lc;
        if constexpr (!kAllWait) __syncthreads();
        ptx::tc_fence_after();
        return true;
    };

    // With two warpgroups, warps w and w + 4 hold the same 32 rows (the same
    // TMEM lanes) and are the only threads that exchange row data: they meet
    // at a barrier of their own (ids 1..4, 64 threads), so the other pairs
    // run on.
    auto pair_sync = [&]() {
        if constexpr (NWG == 2) ptx::named_bar_sync(1 + (warp & 3), 64);
    };

    // Sum of (a, b) over the warpgroups sharing a row, same order everywhere.
    auto xsum = [&](float a, float b) -> float2 {
        if constexpr (NWG == 1) {
            return make_float2(a, b);
        } else {
            float2* slot = sX + (xc & 1) * 256;
            slot[wg * 128 + lt] = make_float2(a, b);
            pair_sync();
            const float2 o = slot[(wg ^ 1) * 128 + lt];
            ++xc;
            return wg == 0 ? make_float2(a + o.x, b + o.y) : make_float2(o.x + a, o.y + b);
        }
    };

    // Row-wise outputs leave through the warp's 32 x 16 staging block: this
    // thread's values v of its row go to columns [base, base + ncol) of
    // rowptr[row] (a null pointer skips the row), written as 64-byte row
    // pieces -- two rows per warp store instead of 32 scattered words.
    float* const mstw = p.sm.mstage >= 0 ? reinterpret_cast<float*>(smem + p.sm.mstage) + warp * (32 * 17) : nullptr;
    auto stage_store = [&](float* const* rowptr, size_t base, int ncol, const float (&v)[16]) {
        const int lane = tid & 31;
#pragma unroll
        for (int j = 0; j < 16; ++j) mstw[lane * 17 + j] = v[j];
        __syncwarp();
        // fully unrolled the row pointers and values of all pieces load
        // together (+3 % at 35 inputs); by 4 with two warpgroups, whose
        // 128-register budget it would otherwise spill.  A piece of at most
        // 8 (4) columns -- the last of a row -- takes 4 (8) rows a store.
        constexpr int kStageUnroll = NWG == 1 ? 16 : 4;
        if (ncol > 8) {
            const int c = lane & 15;
#pragma unroll kStageUnroll
            for (int i = 0; i < 16; ++i) {
                const int r = 2 * i + (lane >> 4);
                float* dst = rowptr[(warp & 3) * 32 + r];
                if (dst && c < ncol) dst[base + c] = mstw[r * 17 + c];
            }
        } else if (ncol > 4) {
            const int c = lane & 7;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int r = 4 * i + (lane >> 3);
                float* dst = rowptr[(warp & 3) * 32 + r];
                if (dst && c < ncol) dst[base + c] = mstw[r * 17 + c];
            }
        } else {
            const int c = lane & 3;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int r = 8 * i + (lane >> 2);
                float* dst = rowptr[(warp & 3) * 32 + r];
                if (dst && c < ncol) dst[base + c] = mstw[r * 17 + c];
            }
        }
        __syncwarp();
    };

    // (sum of a, max of b) over the warpgroups sharing a row
    auto xsummax = [&](float a, float b) -> float2 {
        if constexpr (NWG == 1) {
            return make_float2(a, b);
        } else {
            float2* slot = sX + (xc & 1) * 256;
            slot[wg * 128 + lt] = make_float2(a, b);
            pair_sync();
            const float2 o = slot[(wg ^ 1) * 128 + lt];
            ++xc;
            return make_float2(wg == 0 ? a + o.x : o.x + a, fmaxf(b, o.y));
        }
    };

    const int de = m.de, dch = p.dp / 16, n_d = m.n_d, n_cls = m.n_classes;
    const float gamma = m.gamma;
    const uint32_t idesc_ft = FP8 ? ptx::idesc_e4m3(2 * N) : ptx::idesc_bf16(2 * N);
    const uint32_t idesc_att = FP8 ? ptx::idesc_e4m3(p.dp) : ptx::idesc_bf16(p.dp);
    // FP8: per-output-channel weight scales, indexed like the BN shifts
    const int esc = p.epi_sc;
    const int lpf = m.layers_per_ft;
    const int n_ft_layers = (m.n_steps + 1) * lpf;

    // FP8: scale of the current A operand's row (amax / 448 of what was stored)
    float sa = 1.f;
    bool alive = true;
    for (int64_t tile = blockIdx.x; tile < num_tiles && alive; tile += gridDim.x) {
        const RowIO io = row_io(p.seg, m, tile * 128 + lt, total, x_num, x_cat, logits, masks, agg_out);
        const bool valid = io.valid;
        // warm L2 with this thread's row of the CTA's next tile: that tile's
        // input gather then waits on L2 rather than DRAM
        if (tile + gridDim.x < num_tiles) {
            const RowIO nx = row_io(p.seg, m, (tile + gridDim.x) * 128 + lt, total, x_num, x_cat, logits, nullptr,
                                    nullptr);
            if (nx.valid) {
                if (nx.x_num && m.n_num > 0) {
                    ptx::prefetch_l2(nx.x_num);
                    ptx::prefetch_l2(nx.x_num + m.n_num - 1);
                }
                if (nx.x_cat && m.n_cat > 0) {
                    ptx::prefetch_l2(nx.x_cat);
                    ptx::prefetch_l2(nx.x_cat + m.n_cat - 1);
                }
            }
        }

        // Embedded, BN'd input value of column c for this row.
        auto f_value = [&](int c, bool check) -> float {
            const int2 ci = __ldg(p.col_info + c);
            if (ci.x == -1) {
                const float x = valid ? __ldg(io.x_num + ci.y) : 0.f;
                return fmaf(__ldg(m.s0 + c), x, __ldg(m.t0 + c));
            }
            if (ci.x >= 0) {
                const int idx = valid ? __ldg(io.x_cat + ci.x) - __ldg(m.cat_base + ci.x) : 0;
                if (idx < 0 || idx >= __ldg(m.cat_card + ci.x)) {
                    if (check) atomicOr(m.status, TABNET_STATUS_CAT_OOB);
                    return __ldg(m.t0 + c);
                }
                const int len = __ldg(m.feat_len + m.n_num + ci.x);
                return __ldg(m.emb + __ldg(m.cat_off + ci.x) + (size_t)idx * len + ci.y);
            }
            return 0.f;
        };

        // ---- tile start: f -> A (K = dp), P = 1, aggregate = 0
        float* fc = reinterpret_cast<float*>(smem + (has_f ? p.sm.fcache : 0));
        if (has_f) {
            // Gather the tile's inputs cooperatively: warp w takes 128/(4 NWG)
            // rows, its lanes walk the columns (coalesced reads of a row),
            // all rows' loads in flight before any use.
            constexpr int RPW = 128 / (4 * NWG);
            const float** sRowX = reinterpret_cast<const float**>(smem + p.sm.rowp);
            const int** sRowC = reinterpret_cast<const int**>(smem + p.sm.rowp + 128 * 8);
            float** sRowM = reinterpret_cast<float**>(smem + p.sm.rowp + 128 * 16);
            float** sRowA = reinterpret_cast<float**>(smem + p.sm.rowp + 128 * 24);
            if (wg == 0) {
                sRowX[lt] = valid ? io.x_num : nullptr;
                sRowC[lt] = valid ? io.x_cat : nullptr;
                sRowM[lt] = valid ? io.masks : nullptr;
                sRowA[lt] = valid ? io.agg : nullptr;
            }
            __syncthreads();
            const int lane = tid & 31, r0 = warp * RPW;
#pragma unroll 1
            for (int cb = 0; cb < m.n_num; cb += 32) {
                const int c = cb + lane;
                if (c < m.n_num) {
                    const float s0 = __ldg(m.s0 + c), t0 = __ldg(m.t0 + c);
                    // every row of the warp's share in flight at once
                    float xv[RPW];
#pragma unroll
                    for (int i = 0; i < RPW; ++i) {
                        const float* xr = sRowX[r0 + i];
                        xv[i] = xr ? __ldg(xr + c) : 0.f;
                    }
#pragma unroll
                    for (int i = 0; i < RPW; ++i) fc[c * kFStride + r0 + i] = fmaf(s0, xv[i], t0);
                }
            }
#pragma unroll 1
            for (int jb = 0; jb < m.n_cat; jb += 32) {
                const int j = jb + lane;
                if (j < m.n_cat) {
                    const int card = __ldg(m.cat_card + j), cbase = __ldg(m.cat_base + j);
                    const int c0 = __ldg(m.feat_col + m.n_num + j), len = __ldg(m.feat_len + m.n_num + j);
                    const float* tab = m.emb + __ldg(m.cat_off + j);
                    constexpr int G = RPW;  // every row of the warp's share in flight at once
#pragma unroll 1
                    for (int i0 = r0; i0 < r0 + RPW; i0 += G) {
                        int iv[G];
#pragma unroll
                        for (int i = 0; i < G; ++i) {
                            const int* cr = sRowC[i0 + i];
                            iv[i] = cr ? __ldg(cr + j) - cbase : 0;
                        }
                        unsigned oob = 0;  // bit i: row i0 + i has an out-of-range index
#pragma unroll
                        for (int i = 0; i < G; ++i) {
                            if (iv[i] < 0 || iv[i] >= card) {
                                oob |= 1u << i;
                                if (sRowC[i0 + i]) atomicOr(m.status, TABNET_STATUS_CAT_OOB);
                            }
                        }
                        // the rows' embedding values are loaded together, one
                        // embedding column at a time
#pragma unroll 1
                        for (int e = 0; e < len; ++e) {
                            const float t0e = __ldg(m.t0 + c0 + e);
                            float v[G];
#pragma unroll
                            for (int i = 0; i < G; ++i)
                                v[i] = ((oob >> i) & 1u) ? t0e : __ldg(tab + (size_t)iv[i] * len + e);
#pragma unroll
                            for (int i = 0; i < G; ++i) fc[(c0 + e) * kFStride + i0 + i] = v[i];
                        }
                    }
                }
            }
            __syncthreads();
        }
        // FP8: the row's scale is amax(f) / 448 (the first pass), then f is
        // stored scaled by its inverse
        float inv = 1.f;
        if constexpr (FP8) {
            float amax = 0.f;
#pragma unroll 1
            for (int ch = wg; ch < dch; ch += NWG) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int c = ch * 16 + j;
                    amax = fmaxf(amax, fabsf(has_f ? (c < de ? fc[c * kFStride + lt] : 0.f) : f_value(c, valid)));
                }
            }
            amax = xsummax(0.f, amax).y;
            sa = amax > 0.f ? amax / 448.f : 1.f;
            inv = amax > 0.f ? 448.f / amax : 1.f;
            if (wg == 0 && (dch & 1)) zero_a16_e4m3(sA, lt, dch);
        }
#pragma unroll 1
        for (int ch = wg; ch < dch; ch += NWG) {
            float v[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int c = ch * 16 + j;
                v[j] = has_f ? (c < de ? fc[c * kFStride + lt] : 0.f) : f_value(c, valid && !FP8);
            }
            if constexpr (FP8) store_a16_e4m3(sA, lt, ch, v, inv);
            else store_a16<NP>(sA, sAlo, a_part, lt, ch, v);
            uint32_t ones[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) ones[j] = 0x3f800000u;
            tm_st(t_p + ch * 16, ch, ones);
            if (agg_tmem) {
                uint32_t zeros[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) zeros[j] = 0u;
                tm_st(t_agg + ch * 16, ch, zeros);
            }
        }
        if (!agg_tmem) {
            // the partner warp may still be reading the last tile's aggregate
            // of these rows (it stages 16-feature blocks, not this thread's
            // interleaved subset)
            pair_sync();
            for (int j = wg; j < m.d; j += NWG) sAgg[j * 128 + lt] = 0.f;
        }
        ptx::tmem_wait_st();
        float lacc[kMaxClasses];
#pragma unroll 1
        for (int k = 0; k < n_cls; ++k) lacc[k] = 0.f;
        float res[RCH][16];

#pragma unroll
        for (int cc = 0; cc < RCH; ++cc)
#pragma unroll
            for (int j = 0; j < 16; ++j) res[cc][j] = 0.f;

        // The tile's MMA chains in order: the step-0 feature transformer's
        // layers, then per decision step its attentive layer and its feature
        // transformer's layers (one call site keeps the issue code compact).
        int s = 0, l = 0;
        bool att = false;
#pragma unroll 1
        while (true) {
            const bool first = !att && l == 0;
            // K steps: a feature transformer's first layer reads the dp masked
            // inputs, the others the N outputs of the layer before; the
            // attentive layer reads only the attention half (its weights on
            // the decision half are 0)
            if (!run_mma(att ? p.att_k0 : 0, (att || !first) ? p.ks_n : p.ks_0, att ? idesc_att : idesc_ft,
                         att ? p.dp : 2 * N)) {
                alive = false;
                break;
            }
            if (att) {
                // ---- attentive transformer of step s: z = (W_att a) * scale + shift, times P
                const int ash = n_ft_layers * 2 * N + (s - 1) * p.dp;  // float index of the BN shift
                auto load_z = [&](int ch, float (&z)[16], uint32_t (&pr)[16]) {
                    uint32_t acc[16];
                    ptx::tmem_ld16(t_acc + ch * 16, acc);
                    tm_ld(t_p + ch * 16, ch, pr);
                    ptx::tmem_wait_ld(acc, pr);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float4 b = ld_epi<LEAN>(epi, epi_s, ash + ch * 16 + 4 * q);
                        const float bv[4] = {b.x, b.y, b.z, b.w};
                        float wv[4] = {1.f, 1.f, 1.f, 1.f};
                        if constexpr (FP8) {
                            const float4 w = ld_epi<LEAN>(epi, epi_s, esc + ash + ch * 16 + 4 * q);
                            wv[0] = sa * w.x; wv[1] = sa * w.y; wv[2] = sa * w.z; wv[3] = sa * w.w;
                        }
#pragma unroll
                        for (int t = 0; t < 4; ++t) {
                            const int j = 4 * q + t;
                            const float u = FP8 ? fmaf(__uint_as_float(acc[j]), wv[t], bv[t]) : __uint_as_float(acc[j]) + bv[t];
                            z[j] = (ch * 16 + j < de) ? u * __uint_as_float(pr[j]) : -INFINITY;
                        }
                    }
                };
                // Sparsemax: Michelot's fixed point tau = (sum_{z > tau} z - 1) / #{z > tau}
                // until the support stops changing, started from the larger of two
                // lower bounds of the threshold, (sum z - 1) / de and max z - 1 (the
                // mask's mass 1 is at least max z - tau): sparse masks, i.e. most,
                // then converge in a pass or two.  From any start the iterates reach
                // the same support, so the threshold and mask do not depend on it.
                float zr[(ZREG && kZregChunks > 0) ? kZregChunks : 1][16];
                float zs = 0.f, zmax = -INFINITY;
                if constexpr (ZREG) {
#pragma unroll
                    for (int il = 0; il < kZregChunks; ++il) {
                        const int ch = wg + il * NWG;
                        if (ch < dch) {
                            uint32_t pr[16];
                            load_z(ch, zr[il], pr);
#pragma unroll
                            for (int j = 0; j < 16; ++j) {
                                if (ch * 16 + j < de) zs += zr[il][j];
                                zmax = fmaxf(zmax, zr[il][j]);
                            }
                        }
                    }
                } else {
                    // z replaces the consumed accumulator columns in TMEM
#pragma unroll 1
                    for (int ch = wg; ch < dch; ch += NWG) {
                        float z[16];
                        uint32_t pr[16], zu[16];
                        load_z(ch, z, pr);
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            if (ch * 16 + j < de) zs += z[j];
                            zmax = fmaxf(zmax, z[j]);
                            zu[j] = __float_as_uint(z[j]);
                        }
                        ptx::tmem_st16(t_acc + ch * 16, zu);
                    }
                    ptx::tmem_wait_st();
                }
                const float2 zsm = xsummax(zs, zmax);
                float tau = fmaxf((zsm.x - 1.f) / (float)de, zsm.y - 1.f);
                int prev = de;
                bool done = false;
                // Rows converge after different numbers of passes, but TMEM
                // loads and the warpgroup exchange are collective: every thread
                // runs every pass until the last row of its warp (of its warp
                // pair, with two warpgroups) has converged; a converged row
                // keeps its threshold.
#pragma unroll 1
                for (int it = 0; it < de; ++it) {
                    float ss = 0.f, cnt = 0.f;
                    if constexpr (ZREG) {
#pragma unroll
                        for (int il = 0; il < kZregChunks; ++il) {
                            if (wg + il * NWG < dch) {
#pragma unroll
                                for (int j = 0; j < 16; ++j)
                                    if (zr[il][j] > tau) { ss += zr[il][j]; cnt += 1.f; }
                            }
                        }
                    } else {
#pragma unroll 1
                        for (int ch = wg; ch < dch; ch += NWG) {
                            uint32_t zu[16];
                            ptx::tmem_ld16(t_acc + ch * 16, zu);
                            ptx::tmem_wait_ld(zu);
#pragma unroll
                            for (int j = 0; j < 16; ++j) {
                                const float z = __uint_as_float(zu[j]);
                                if (z > tau) { ss += z; cnt += 1.f; }
                            }
                        }
                    }
                    const float2 t = xsum(ss, cnt);
                    if (!done) {
                        const int c = (int)t.y;
                        if (c == prev || c == 0) {
                            done = true;
                        } else {
                            prev = c;
                            tau = (t.x - 1.f) / t.y;
                        }
                    }
                    // the two warps holding these rows see the same totals,
                    // hence the same flags, and leave together
                    if (!__any_sync(0xffffffffu, !done)) break;
                }
                // Mask, prior, masked input (A for the step's first FC), outputs.
                float* mrow = (io.masks && valid) ? io.masks + (size_t)(s - 1) * de : nullptr;
                float vamax = 0.f;  // FP8: amax of the row's masked input
                float* const* sRowM = reinterpret_cast<float* const*>(smem + p.sm.rowp + 128 * 16);
#pragma unroll 1
                for (int il = 0; wg + il * NWG < dch; ++il) {
                    const int ch = wg + il * NWG;
                    float z[16];
                    uint32_t pr[16];
                    if constexpr (ZREG) {
                        tm_ld(t_p + ch * 16, ch, pr);
                        ptx::tmem_wait_ld(pr);
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            float zz = zr[0][j];
#pragma unroll
                            for (int q = 1; q < kZregChunks; ++q)
                                if (il == q) zz = zr[q][j];
                            z[j] = zz;
                        }
                    } else {
                        uint32_t zu[16];
                        ptx::tmem_ld16(t_acc + ch * 16, zu);
                        tm_ld(t_p + ch * 16, ch, pr);
                        ptx::tmem_wait_ld(zu, pr);
#pragma unroll
                        for (int j = 0; j < 16; ++j) z[j] = __uint_as_float(zu[j]);
                    }
                    float mk[16], v[16];
                    uint32_t pn[16], mu[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        mk[j] = fmaxf(z[j] - tau, 0.f);
                        pn[j] = __float_as_uint(__uint_as_float(pr[j]) * (gamma - mk[j]));
                        mu[j] = __float_as_uint(mk[j]);
                    }
                    tm_st(t_p + ch * 16, ch, pn);
                    if (!m16) {
                        tm_st(t_m + ch * 16, ch, mu);  // the mask, kept in fp32 for the aggregate
                    } else {
                        uint32_t mh[8];
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            __half2 h = __floats2half2_rn(mk[2 * j], mk[2 * j + 1]);
                            mh[j] = *reinterpret_cast<uint32_t*>(&h);
                        }
                        ptx::tmem_st8(t_m + ch * 8, mh);
                    }
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int c = ch * 16 + j;
                        if (has_f) {
                            v[j] = c < de ? mk[j] * ptx::ld_shared_f32(f_s + 4u * (uint32_t)(c * kFStride + lt)) : 0.f;
                        } else {
                            v[j] = (c < de && mk[j] > 0.f) ? mk[j] * f_value(c, false) : 0.f;
                        }
                    }
                    if constexpr (FP8) {
#pragma unroll
                        for (int j = 0; j < 16; ++j) vamax = fmaxf(vamax, fabsf(v[j]));
                        if constexpr (!ZREG) {
                            // v replaces this chunk's z in TMEM until the row's scale is known
                            uint32_t vu[16];
#pragma unroll
                            for (int j = 0; j < 16; ++j) vu[j] = __float_as_uint(v[j]);
                            ptx::tmem_st16(t_acc + ch * 16, vu);
                        }
                    }
                    if (mstw) {
                        stage_store(sRowM, (size_t)(s - 1) * de + ch * 16, min(16, de - ch * 16), mk);
                    } else if (mrow) {
                        if (((de & 3) == 0) && ((reinterpret_cast<uintptr_t>(mrow) & 15) == 0) && ch * 16 + 16 <= de) {
                            float4* d4 = reinterpret_cast<float4*>(mrow + ch * 16);
#pragma unroll
                            for (int q = 0; q < 4; ++q)
                                d4[q] = make_float4(mk[4 * q], mk[4 * q + 1], mk[4 * q + 2], mk[4 * q + 3]);
                        } else {
#pragma unroll
                            for (int j = 0; j < 16; ++j)
                                if (ch * 16 + j < de) mrow[ch * 16 + j] = mk[j];
                        }
                    }
                    if constexpr (!FP8) store_a16<NP>(sA, sAlo, a_part, lt, ch, v);
                }
                ptx::tmem_wait_st();
                if constexpr (FP8) {
                    // the masked input scaled by its row's amax / 448
                    vamax = xsummax(0.f, vamax).y;
                    sa = vamax > 0.f ? vamax / 448.f : 1.f;
                    const float vinv = vamax > 0.f ? 448.f / vamax : 1.f;
#pragma unroll 1
                    for (int il = 0; wg + il * NWG < dch; ++il) {
                        const int ch = wg + il * NWG;
                        float v[16];
                        if constexpr (ZREG) {
#pragma unroll
                            for (int j = 0; j < 16; ++j) {
                                float zz = zr[0][j];
#pragma unroll
                                for (int q = 1; q < kZregChunks; ++q)
                                    if (il == q) zz = zr[q][j];
                                const int c = ch * 16 + j;
                                const float mkj = fmaxf(zz - tau, 0.f);
                                v[j] = c < de ? mkj * ptx::ld_shared_f32(f_s + 4u * (uint32_t)(c * kFStride + lt)) : 0.f;
                            }
                        } else {
                            uint32_t vu[16];
                            ptx::tmem_ld16(t_acc + ch * 16, vu);
                            ptx::tmem_wait_ld(vu);
#pragma unroll
                            for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(vu[j]);
                        }
                        store_a16_e4m3(sA, lt, ch, v, vinv);
                    }
                    if (wg == 0 && (dch & 1)) zero_a16_e4m3(sA, lt, dch);
                }
                att = false;
                continue;
            }

            // ---- layer l of feature transformer s
            const int sh = (s * lpf + l) * 2 * N;  // float index of the layer's BN shift
            // x = sqrt(1/2) (x_prev + g): the linear half of every layer but an
            // FT's first is scaled by sqrt(1/2), so x = x_prev sqrt(1/2) + g;
            // the gate half by -log2(e), the sigmoid's argument.  The shifts
            // are stored scaled; with several bf16 parts the packed weights
            // are too (the parts then carry the scaled weight to ~2^-24), with
            // one part the weights are rounded unscaled and the accumulator
            // takes the constant (cl, cg)
            const float cres = first ? 0.f : kSqrtHalf;
            const float cl = (SPLIT || first) ? 1.f : kSqrtHalf;
            const float cg = SPLIT ? 1.f : -1.44269504088896340736f;
            // One warpgroup alone on a row (NWG = 1) takes 16-column pieces and
            // requests piece k+1 from TMEM before computing piece k; with two
            // warpgroups per row, 8-column pieces loaded one at a time keep
            // the register count within the two-CTAs-per-SM budget.
            constexpr int SW = NWG == 1 ? 16 : 8;
            constexpr int NSUB = CPW / SW;
            uint32_t lin[NWG == 1 ? 2 : 1][SW], gat[NWG == 1 ? 2 : 1][SW];
            ptx::tmem_ld_cols<SW>(t_acc + wg * CPW, lin[0]);
            ptx::tmem_ld_cols<SW>(t_acc + N + wg * CPW, gat[0]);
            ptx::tmem_wait_ld(lin[0], gat[0]);
#pragma unroll
            for (int sc = 0; sc < NSUB; ++sc) {
                const int c0 = wg * CPW + sc * SW;
                const int cur = NWG == 1 ? (sc & 1) : 0;
                if constexpr (NWG == 1) {
                    if (sc + 1 < NSUB) {
                        ptx::tmem_ld_cols<SW>(t_acc + c0 + SW, lin[cur ^ 1]);
                        ptx::tmem_ld_cols<SW>(t_acc + N + c0 + SW, gat[cur ^ 1]);
                    }
                } else if (sc > 0) {
                    ptx::tmem_ld_cols<SW>(t_acc + c0, lin[0]);
                    ptx::tmem_ld_cols<SW>(t_acc + N + c0, gat[0]);
                    ptx::tmem_wait_ld(lin[0], gat[0]);
                }
                float out[SW];
#pragma unroll
                for (int q = 0; q < SW / 4; ++q) {
                    const float4 hl = ld_epi<LEAN>(epi, epi_s, sh + c0 + 4 * q);
                    const float4 hg = ld_epi<LEAN>(epi, epi_s, sh + N + c0 + 4 * q);
                    const float hlv[4] = {hl.x, hl.y, hl.z, hl.w};
                    const float hgv[4] = {hg.x, hg.y, hg.z, hg.w};
                    // accumulator multipliers: the constant pre-scales (the weights
                    // are packed as BN-folded and rounded, unscaled); in FP8 the row
                    // and channel scales, which carry the pre-scales
                    float wl[4] = {cl, cl, cl, cl}, wgt[4] = {cg, cg, cg, cg};
                    if constexpr (FP8) {
                        const float4 a = ld_epi<LEAN>(epi, epi_s, esc + sh + c0 + 4 * q);
                        const float4 b = ld_epi<LEAN>(epi, epi_s, esc + sh + N + c0 + 4 * q);
                        wl[0] = sa * a.x; wl[1] = sa * a.y; wl[2] = sa * a.z; wl[3] = sa * a.w;
                        wgt[0] = sa * b.x; wgt[1] = sa * b.y; wgt[2] = sa * b.z; wgt[3] = sa * b.w;
                    }
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const int j = 4 * q + t;
                        float& r = res[(sc * SW + j) / 16][(sc * SW + j) % 16];
                        const float ul = fmaf(__uint_as_float(lin[cur][j]), wl[t], hlv[t]);
                        const float ug = fmaf(__uint_as_float(gat[cur][j]), wgt[t], hgv[t]);
                        const float g = ul * sigmoid_from_log2(ug);
                        const float x = fmaf(r, cres, g);
                        r = x;
                        out[j] = x;
                    }
                }
                if constexpr (NWG == 1) {
                    if (sc + 1 < NSUB) ptx::tmem_wait_ld(lin[cur ^ 1], gat[cur ^ 1]);
                }
                if constexpr (!FP8) {
                    if constexpr (SW == 16) store_a16<NP>(sA, sAlo, a_part, lt, c0 / 16, out);
                    else store_a8<NP>(sA, sAlo, a_part, lt, c0 / 8, out);
                }
            }
            if constexpr (FP8) {
                // the layer's outputs scaled by the row's amax / 448; the last
                // layer of a feature transformer feeds only the attentive
                // layer, which reads the attention half: its amax alone
                const bool att_next = l == lpf - 1;
                float amax = 0.f;
#pragma unroll
                for (int cc = 0; cc < RCH; ++cc)
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        if (!att_next || wg * CPW + cc * 16 + j >= n_d) amax = fmaxf(amax, fabsf(res[cc][j]));
                amax = xsummax(0.f, amax).y;
                sa = amax > 0.f ? amax / 448.f : 1.f;
                const float ginv = amax > 0.f ? 448.f / amax : 1.f;
#pragma unroll
                for (int cc = 0; cc < RCH; ++cc) store_a16_e4m3(sA, lt, wg * RCH + cc, res[cc], ginv);
                if (wg == 0 && ((N / 16) & 1)) zero_a16_e4m3(sA, lt, N / 16);
            }
            if (++l < lpf) continue;
            l = 0;
            if (s > 0) {
                // ---- decision output: acc += ReLU(d) (folded into the logits), eta, aggregate
                // res becomes ReLU(d) (zero on the attention columns): the next
                // step's feature transformer starts from its own first layer.
                // Where TMEM holds the step mask as fp16 pairs and the caller
                // takes the masks, the aggregate is summed from the fp32 mask
                // row this row wrote to the output (several CTA barriers ago);
                // its chunks are loaded one ahead of their use, the first one
                // here, before the decision's arithmetic.  Not in FP8, whose
                // masks carry E4M3's error (2^-4) far above fp16's (2^-11),
                // and whose kernel has no registers to spare for the chunk.
                const float* mrow32 = (!FP8 && m16 && io.masks && valid) ? io.masks + (size_t)(s - 1) * de : nullptr;
                const bool mrow32_v4 = mrow32 && (de & 3) == 0 && (reinterpret_cast<uintptr_t>(mrow32) & 15) == 0;
                float mnext[16];
                auto load_mrow = [&](int ch) {
                    if (!mrow32 || ch >= dch) return;
                    if (mrow32_v4 && ch * 16 + 16 <= de) {
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const float4 v4 = *reinterpret_cast<const float4*>(mrow32 + ch * 16 + 4 * q);
                            mnext[4 * q] = v4.x; mnext[4 * q + 1] = v4.y; mnext[4 * q + 2] = v4.z; mnext[4 * q + 3] = v4.w;
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; ++j) mnext[j] = ch * 16 + j < de ? mrow32[ch * 16 + j] : 0.f;
                    }
                };
                load_mrow(wg);
                float eta = 0.f;
#pragma unroll
                for (int cc = 0; cc < RCH; ++cc) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int c = wg * CPW + cc * 16 + j;
                        const float dv = c < n_d ? fmaxf(res[cc][j], 0.f) : 0.f;
                        res[cc][j] = dv;
                        eta += dv;
                    }
                }
                // logits += W_f ReLU(d), W_f staged as [class][N] with zero columns
                // past n_d; one class per pass (the per-class sums live in local memory)
#pragma unroll 1
                for (int k = 0; k < n_cls; ++k) {
                    float a0 = 0.f, a1 = 0.f;
#pragma unroll
                    for (int cc = 0; cc < RCH; ++cc) {
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const float4 w = ptx::ld_shared_f4(wf_s + 4u * (uint32_t)(k * N + wg * CPW + cc * 16 + 4 * q));
                            a0 = fmaf(w.x, res[cc][4 * q], a0);
                            a1 = fmaf(w.y, res[cc][4 * q + 1], a1);
                            a0 = fmaf(w.z, res[cc][4 * q + 2], a0);
                            a1 = fmaf(w.w, res[cc][4 * q + 3], a1);
                        }
                    }
                    lacc[k] += a0 + a1;
                }
                eta = xsum(eta, 0.f).x;
                // aggregate += eta * M (the step's mask as kept in TMEM, or the
                // fp32 mask row loaded above)
#pragma unroll 1
                for (int ch = wg; ch < dch; ch += NWG) {
                    float mv[16];
                    if (!m16) {
                        uint32_t mu[16];
                        tm_ld(t_m + ch * 16, ch, mu);
                        ptx::tmem_wait_ld(mu);
#pragma unroll
                        for (int j = 0; j < 16; ++j) mv[j] = __uint_as_float(mu[j]);
                    } else {
                        uint32_t mh[8];
                        ptx::tmem_ld8(t_m + ch * 8, mh);  // collective: every lane of the warp
                        ptx::tmem_wait_ld8(mh);
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const float2 mm = __half22float2(*reinterpret_cast<__half2*>(&mh[j]));
                            mv[2 * j] = mm.x;
                            mv[2 * j + 1] = mm.y;
                        }
                        if (mrow32) {
#pragma unroll
                            for (int j = 0; j < 16; ++j) mv[j] = mnext[j];
                            load_mrow(ch + NWG);
                        }
                    }
                    if (agg_tmem) {
                        uint32_t ag[16];
                        tm_ld(t_agg + ch * 16, ch, ag);
                        ptx::tmem_wait_ld(ag);
#pragma unroll
                        for (int j = 0; j < 16; ++j) ag[j] = __float_as_uint(fmaf(eta, mv[j], __uint_as_float(ag[j])));
                        tm_st(t_agg + ch * 16, ch, ag);
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const int c = ch * 16 + j;
                            if (c < de && mv[j] > 0.f) {
                                float* dst = sAgg + sColf[c] * 128 + lt;
                                if constexpr (NWG == 1) *dst = fmaf(eta, mv[j], *dst);
                                else atomicAdd(dst, eta * mv[j]);
                            }
                        }
                    }
                }
                if (agg_tmem) ptx::tmem_wait_st();
            }
            if (++s > m.n_steps) break;
            att = true;
        }
        if (!alive) break;

        // ---- logits and the normalised aggregate
#pragma unroll 1
        for (int k = 0; k < n_cls; ++k) {
            const float v = xsum(lacc[k], 0.f).x;
            if (wg == 0 && valid) io.logits[k] = v + __ldg(m.bf + k);
        }
        if (agg_tmem) {
            // one column per feature: normalise the TMEM aggregate directly
            float tot = 0.f;
#pragma unroll 1
            for (int ch = wg; ch < dch; ch += NWG) {
                uint32_t ag[16];
                tm_ld(t_agg + ch * 16, ch, ag);
                ptx::tmem_wait_ld(ag);
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    if (ch * 16 + j < de) tot += __uint_as_float(ag[j]);
            }
            tot = xsum(tot, 0.f).x;
            const float inv = tot > 0.f ? 1.f / tot : 0.f;
            float* const* sRowA = reinterpret_cast<float* const*>(smem + p.sm.rowp + 128 * 24);
#pragma unroll 1
            for (int ch = wg; ch < dch; ch += NWG) {
                uint32_t ag[16];
                tm_ld(t_agg + ch * 16, ch, ag);
                ptx::tmem_wait_ld(ag);
                if (mstw) {
                    float v[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) v[j] = tot > 0.f ? __uint_as_float(ag[j]) * inv : 0.f;
                    stage_store(sRowA, ch * 16, min(16, de - ch * 16), v);
                } else if (io.agg && valid) {
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        if (ch * 16 + j < de) io.agg[ch * 16 + j] = tot > 0.f ? __uint_as_float(ag[j]) * inv : 0.f;
                }
            }
        } else {
            pair_sync();  // both warpgroups' aggregate updates of these rows are in shared memory
            float tot = 0.f;
            for (int j = wg; j < m.d; j += NWG) tot += sAgg[j * 128 + lt];
            tot = xsum(tot, 0.f).x;
            const float inv = tot > 0.f ? 1.f / tot : 0.f;
            if (mstw) {
                float* const* sRowA = reinterpret_cast<float* const*>(smem + p.sm.rowp + 128 * 24);
#pragma unroll 1
                for (int cb = wg * 16; cb < m.d; cb += 16 * NWG) {
                    float v[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) v[j] = (cb + j < m.d && tot > 0.f) ? sAgg[(cb + j) * 128 + lt] * inv : 0.f;
                    stage_store(sRowA, cb, min(16, m.d - cb), v);
                }
            } else if (io.agg && valid) {
                for (int j = wg; j < m.d; j += NWG) io.agg[j] = tot > 0.f ? sAgg[j * 128 + lt] * inv : 0.f;
            }
        }
    }

    // ---- teardown: no copy or MMA may still target this CTA's memory
    __syncthreads();
    if (warp == 0) {
        int sl = cs_slot;
        uint32_t rd = cs_round;
        for (int64_t g = g_cons; g < g_issue; ++g) {
            if (!warp_wait(bar_full + 8 * sl, rd & 1u) && lane_id == 0) note_timeout(m.status, 3, (unsigned)g);
            if (++sl == SU) { sl = 0; ++rd; }
        }
        if (acc_outstanding && !warp_wait(bar_acc, acc_phase ^ 1) && lane_id == 0)
            note_timeout(m.status, 4, (unsigned)lc);
        for (int sl2 = 0; sl2 < SU; ++sl2)
            if ((empty_pending >> sl2) & 1u)
                if (!warp_wait(bar_empty + 8 * sl2, (empty_par >> sl2) & 1u) && lane_id == 0)
                    note_timeout(m.status, 6, (unsigned)sl2);
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    if (warp == 0) ptx::tmem_dealloc(tmem, (uint32_t)p.tmem_cols);
}

// ---------------------------------------------------------------- host side

uint16_t f32_to_bf16_rne(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return (uint16_t)((u >> 16) | ((u & 0xffffu) ? 0x40u : 0u));
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

float bf16_to_f32(uint16_t h) {
    const uint32_t u = (uint32_t)h << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

// Pack W [n_out, k_valid] (row-major; input column j lands at K index
// j + col_shift) into ceil(k_pad / 64) blocks of n_out x 64 bf16 in the
// 128B-swizzled K-major layout.  part 0: bf16(w); part 1: bf16(w - bf16(w)).
void pack_sw128(const float* W, int n_out, int k_valid, int col_shift, int k_pad, int part,
                std::vector<uint8_t>& out) {
    const int n_blocks = (k_pad + 63) / 64;
    out.assign((size_t)n_blocks * n_out * 128, 0);
    for (int b = 0; b < n_blocks; ++b) {
        uint8_t* blk = out.data() + (size_t)b * n_out * 128;
        for (int n = 0; n < n_out; ++n) {
            for (int kk = 0; kk < 64; ++kk) {
                const int k = b * 64 + kk;
                const int src = k - col_shift;
                const float w = (src >= 0 && src < k_valid) ? W[(size_t)n * k_valid + src] : 0.f;
                // part 0: bf16(w); each further part: bf16 of what the earlier parts leave
                float rem = w;
                uint16_t h = f32_to_bf16_rne(rem);
                for (int q = 1; q <= part; ++q) {
                    rem -= bf16_to_f32(h);
                    h = f32_to_bf16_rne(rem);
                }
                const size_t off = (size_t)(n >> 3) * 1024 + (n & 7) * 128 + ((((kk >> 3) ^ (n & 7)) & 7) << 4) +
                                   (kk & 7) * 2;
                std::memcpy(blk + off, &h, 2);
            }
        }
    }
}

// FP8 E4M3 (1 sign, 4 exponent bits with bias 7, 3 mantissa bits; no
// infinities, largest finite 448) nearest to x, ties to even, saturating.
uint8_t e4m3_rne(double x) {
    const uint8_t sign = x < 0 ? 0x80 : 0x00;
    double a = std::fabs(x);
    if (!(a < 448.0)) return sign | 0x7E;  // saturate (NaN inputs do not occur: weights are finite)
    int e;
    std::frexp(a, &e);                 // a = m 2^e, m in [0.5, 1)
    const int binade = std::max(e - 1, -6);  // subnormals share the 2^-6 binade's spacing
    const double step = std::ldexp(1.0, binade - 3);
    const double q = std::nearbyint(a / step);  // round-half-even in the default mode
    double v = q * step;
    if (v >= 448.0) return sign | 0x7E;
    if (v == 0.0) return sign;
    int ev;
    const double mv = std::frexp(v, &ev);  // v = mv 2^ev
    const int E = ev - 1 + 7;               // biased exponent of 1.f x 2^(ev-1)
    if (E <= 0) return sign | (uint8_t)std::lround(v / std::ldexp(1.0, -9));  // subnormal: v / 2^-9
    const int mant = (int)std::lround((mv * 2.0 - 1.0) * 8.0);
    return sign | (uint8_t)((E << 3) | mant);
}

// Pack W [n_out, k_valid] (row-major doubles; input column j at K index
// j + col_shift) into ceil(k_pad / 128) blocks of n_out x 128 e4m3 bytes in
// the 128B-swizzled K-major layout, each row scaled by its own amax / 448;
// scale[n] = amax / 448 (1 for an all-zero row).
void pack_e4m3(const double* W, int n_out, int k_valid, int col_shift, int k_pad, std::vector<uint8_t>& out,
               std::vector<double>& scale) {
    const int n_blocks = (k_pad + 127) / 128;
    out.assign((size_t)n_blocks * n_out * 128, 0);
    scale.assign(n_out, 1.0);
    for (int n = 0; n < n_out; ++n) {
        double amax = 0.0;
        for (int j = 0; j < k_valid; ++j) amax = std::max(amax, std::fabs(W[(size_t)n * k_valid + j]));
        if (amax > 0.0) scale[n] = amax / 448.0;
        for (int k = 0; k < n_blocks * 128; ++k) {
            const int src = k - col_shift;
            if (src < 0 || src >= k_valid) continue;
            const int b = k / 128, kk = k % 128;
            const size_t off = (size_t)b * n_out * 128 + (size_t)(n >> 3) * 1024 + (n & 7) * 128 +
                               ((((kk >> 4) ^ (n & 7)) & 7) << 4) + (kk & 15);
            out[off] = e4m3_rne(W[(size_t)n * k_valid + src] / scale[n]);
        }
    }
}

int round_up(int x, int a) { return (x + a - 1) / a * a; }

struct Variant {
    int N, nwg;
    int np;  // bf16 parts per operand: 1 (bf16), 2 (split-bf16), 3 (three-part split); 0: FP8 E4M3
    bool zreg, lean;
};

// Run f on the kernel instantiation of a variant; false when none exists.
template <typename F>
bool with_kernel(const Variant& v, F&& f) {
#define TC_VAR4(NN, WW, NP, ZR)                                                      \
    if (v.np == NP && v.zreg == ZR) {                                                \
        if (v.lean) f(tc_forward_kernel<NN, WW, NP, ZR, true>);                       \
        else f(tc_forward_kernel<NN, WW, NP, ZR, false>);                            \
        return true;                                                                 \
    }
// one warpgroup: 1, 2 or 3 parts, z in registers or TMEM
#define TC_VARIANT(NN, WW)              \
    if (v.N == NN && v.nwg == WW) {     \
        TC_VAR4(NN, WW, 3, true)        \
        TC_VAR4(NN, WW, 3, false)       \
        TC_VAR4(NN, WW, 2, true)        \
        TC_VAR4(NN, WW, 2, false)       \
        TC_VAR4(NN, WW, 1, true)        \
        TC_VAR4(NN, WW, 1, false)       \
        TC_VAR4(NN, WW, 0, true)        \
        TC_VAR4(NN, WW, 0, false)       \
    }
// two warpgroups: FP8, 1 or 2 parts, z in TMEM
#define TC_VARIANT_NOZ(NN, WW)          \
    if (v.N == NN && v.nwg == WW) {     \
        TC_VAR4(NN, WW, 2, false)       \
        TC_VAR4(NN, WW, 1, false)       \
        TC_VAR4(NN, WW, 0, false)       \
    }
    TC_VARIANT(16, 1)
    TC_VARIANT(32, 1)
    TC_VARIANT_NOZ(32, 2)
    TC_VARIANT(64, 1)
    TC_VARIANT_NOZ(64, 2)
    TC_VARIANT_NOZ(128, 2)
#undef TC_VARIANT
#undef TC_VARIANT_NOZ
#undef TC_VAR4
    return false;
}

TcSmem smem_layout(int N, int dp, int de, int d, int n_cls, int n_d, int n_slots, int slot_bytes, int np,
                   int nwg, int epi_floats, int n_chunks, bool agg_tmem, bool with_epi, bool with_f, bool with_mst) {
    TcSmem s{};
    const int a_blocks = (std::max(dp, N) + 63) / 64;
    int o = 0;
    s.a_hi = o; o += a_blocks * 16384;
    s.a_lo = -1;  // the further parts follow the first, a_blocks * 16 KB each
    if (np > 1) { s.a_lo = o; o += (np - 1) * a_blocks * 16384; }
    s.ring = o; o += n_slots * slot_bytes;
    s.agg = -1;
    if (!agg_tmem) { s.agg = o; o += round_up(d * 128 * 4, 16); }
    s.xch = -1;
    if (nwg > 1) { s.xch = o; o += 2 * 2 * 128 * 8; }
    s.wf = o; o += round_up(n_cls * N * 4, 16);
    s.epi = -1;
    if (with_epi) { s.epi = o; o += round_up(epi_floats * 4, 16); }
    s.fcache = -1;
    s.rowp = -1;
    s.mstage = -1;
    if (with_f) {
        s.fcache = o; o += round_up(de * kFStride * 4, 16);
        s.rowp = o; o += 128 * 32;
        if (with_mst) { s.mstage = o; o += 4 * nwg * 32 * 17 * 4; }
    }
    s.colf = o; o += round_up(dp * 4, 16);
    s.chunks = o; o += round_up(n_chunks * 8, 16);
    s.bar = o; o += round_up((2 * n_slots + 3) * 8, 16);
    s.total = o;
    return s;
}

}  // namespace

// bf16 parts per operand of a tensor-core precision, 0 for FP8 E4M3 (-1:
// not a tensor-core precision).
int precision_parts(int precision) {
    switch (precision) {
        case TABNET_BF16: return 1;
        case TABNET_BF16X3: return 2;
        case TABNET_BF16X6: return 3;
        case TABNET_FP8_E4M3: return 0;
    }
    return -1;
}

int tc_build(tabnet_model* m, Arena& a, std::string* why) {
    const tabnet_dims& d = m->host.dims;
    const int N = d.n_d + d.n_a;
    const int dp = round_up(d.d_emb, 16);
    const int np = precision_parts(m->precision);
    const bool fp8 = np == 0;
    if (np < 0) {
        *why = "not a tensor-core precision";
        return TABNET_ERR_UNSUPPORTED_DIMS;
    }
    if (N != 16 && N != 32 && N != 64 && N != 128) {
        *why = "tensor-core path needs n_d + n_a in {16, 32, 64, 128}";
        return TABNET_ERR_UNSUPPORTED_DIMS;
    }
    if (np == 3 && N > 64) {
        *why = "the three-part split (TABNET_BF16X6) needs n_d + n_a <= 64 (one warpgroup per row)";
        return TABNET_ERR_UNSUPPORTED_DIMS;
    }
    if (dp > 256) { *why = "tensor-core path needs d_emb <= 256"; return TABNET_ERR_UNSUPPORTED_DIMS; }
    if (d.n_classes > kMaxClasses) { *why = "tensor-core path needs n_classes <= 4"; return TABNET_ERR_UNSUPPORTED_DIMS; }
    // TMEM: the accumulator, then P and the step mask in fp32 (the last
    // 16-column chunk cut to 8 columns when it holds at most 8 mask columns),
    // then the aggregate when every feature is one embedded column
    const int accw = std::max(2 * N, dp);
    const bool tail8 = (d.d_emb % 16) != 0 && (d.d_emb % 16) <= 8;
    const int pw = tail8 ? dp - 8 : dp;
    auto pow2 = [](int need) { int c = 32; while (c < need) c *= 2; return c; };
    bool m16 = false;
    int need = accw + 2 * pw;
    if (need > 512) {
        // the step mask as fp16 pairs: the only layout that fits 128 hidden
        // units with a 160-column mask
        m16 = true;
        need = accw + pw + dp / 2;
    }
    int cols = pow2(need);
    if (cols > 512) { *why = "TMEM budget exceeded"; return TABNET_ERR_UNSUPPORTED_DIMS; }
    TcParams& p = m->tc;
    p.dp = dp;
    p.tail8 = tail8 ? 1 : 0;
    p.m16 = m16 ? 1 : 0;
    p.tm_p = accw;
    p.tm_m = accw + pw;
    // K steps: 16 bf16 or 32 e4m3 elements
    const int kstep = fp8 ? 32 : 16;
    p.att_k0 = d.n_d / kstep;
    p.ks_0 = (dp + kstep - 1) / kstep;
    p.ks_n = (N + kstep - 1) / kstep;
    // the aggregate lives in TMEM when every feature is one embedded column
    // and its region fits in the allocation (or the next, <= 256)
    p.tm_agg = -1;
    if (d.d_emb == d.n_feat) {
        const int c2 = pow2(need + pw);
        if (c2 <= std::max(cols, 256)) { p.tm_agg = need; cols = c2; }
    }
    p.tmem_cols = cols;

    const HostModel& hm = m->host;
    const int parts = fp8 ? 1 : np;
    const int kblock = fp8 ? 128 : 64;  // elements of a K block (128 bytes a row)
    // Every 64-wide K block of W (its parts in order: hi, then lo or mid, lo) becomes a chunk.
    // Blocks before first_block are not streamed (all their weights are 0).
    bool parts_contiguous = true;
    auto push_layer = [&](const float* W, int n_out, int k_valid, int col_shift, int k_pad, int first_block,
                          std::vector<std::pair<size_t, uint32_t>>* keep) {
        const uint32_t cb = (uint32_t)n_out * 128;
        std::vector<std::vector<uint8_t>> pk(parts);
        for (int part = 0; part < parts; ++part) pack_sw128(W, n_out, k_valid, col_shift, k_pad, part, pk[part]);
        const int blocks = (k_pad + 63) / 64;
        for (int b = first_block; b < blocks; ++b) {
            // one ring unit: the block's parts back to back (cb is a multiple
            // of 1024, so the arena keeps them contiguous)
            size_t off0 = 0;
            for (int part = 0; part < parts; ++part) {
                const size_t off = a.add(pk[part].data() + (size_t)b * cb, cb, 1024);
                if (part == 0) off0 = off;
                else if (off != off0 + (size_t)part * cb) parts_contiguous = false;
            }
            keep->push_back({off0, cb * (uint32_t)parts});
        }
    };
    // FP8: W' = diag(BN scale) W in double (as the rounding study folds it),
    // quantized per output channel; the kernel's per-channel scale also
    // carries the row's constant pre-scale c (sqrt(1/2) or -log2 e), which
    // leaves the quantized bytes unchanged.
    std::vector<float> wsc;  // per-channel dequantization scales, laid out like epi
    auto push_layer_e4m3 = [&](const std::vector<float>& W, const BN& bn, int n_out, int k_valid, int col_shift,
                               int k_pad, int first_block, const std::vector<double>& c,
                               std::vector<std::pair<size_t, uint32_t>>* keep, std::vector<float>* scales) {
        std::vector<double> wd((size_t)n_out * k_valid, 0.0);
        const int n_bn = (int)bn.mean.size();
        for (int r = 0; r < n_out && r < n_bn; ++r) {
            const double sbn = (double)bn.weight[r] / std::sqrt((double)bn.var[r] + d.bn_eps);
            for (int k = 0; k < k_valid; ++k) wd[(size_t)r * k_valid + k] = sbn * (double)W[(size_t)r * k_valid + k];
        }
        std::vector<uint8_t> pk;
        std::vector<double> sc;
        pack_e4m3(wd.data(), n_out, k_valid, col_shift, k_pad, pk, sc);
        for (int r = 0; r < n_out; ++r) scales->push_back((float)(sc[r] * (r < (int)c.size() ? c[r] : 1.0)));
        const uint32_t cb = (uint32_t)n_out * 128;
        const int blocks = (k_pad + 127) / 128;
        for (int b = first_block; b < blocks; ++b) {
            const size_t off = a.add(pk.data() + (size_t)b * cb, cb, 1024);
            keep->push_back({off, cb});
        }
    };
    // BN scale is folded into the packed weights (W' = diag(scale) W, rounded
    // after scaling, so a shared layer gets one packed copy per feature
    // transformer); the epilogue adds the BN shift only.
    auto scaled = [](const std::vector<float>& W, const std::vector<float>& sc, int rows, int k) {
        std::vector<float> w((size_t)rows * k);
        for (int r = 0; r < rows; ++r)
            for (int c = 0; c < k; ++c) w[(size_t)r * k + c] = (float)((double)sc[r] * W[(size_t)r * k + c]);
        return w;
    };
    std::vector<std::pair<size_t, uint32_t>> stream;
    std::vector<float> epi, att_epi, att_wsc;
    for (int s = 0; s <= d.n_steps; ++s) {
        if (s > 0) {
            // attentive FC [de, n_a] acting on the whole FT output [N] as
            // [dp, N]: columns [0, n_d) (the decision part) and rows beyond
            // de (padding) carry zero weight
            std::vector<float> sc, sh;
            fold_bn(hm.att_bn[s - 1], d.bn_eps, sc, sh);
            // the MMA chain starts at K step att_k0: blocks wholly inside the
            // decision half are not streamed
            if (fp8) {
                std::vector<float> wraw((size_t)dp * d.n_a, 0.f);
                std::memcpy(wraw.data(), hm.att_fc[s - 1].data(), sizeof(float) * d.d_emb * d.n_a);
                push_layer_e4m3(wraw, hm.att_bn[s - 1], dp, d.n_a, d.n_d, N, p.att_k0 / 4, {}, &stream, &att_wsc);
            } else {
                std::vector<float> wp((size_t)dp * d.n_a, 0.f);
                const std::vector<float> ws = scaled(hm.att_fc[s - 1], sc, d.d_emb, d.n_a);
                std::memcpy(wp.data(), ws.data(), sizeof(float) * d.d_emb * d.n_a);
                push_layer(wp.data(), dp, d.n_a, d.n_d, N, p.att_k0 / 4, &stream);
            }
            sh.resize(dp, 0.f);
            att_epi.insert(att_epi.end(), sh.begin(), sh.end());
        }
        for (int l = 0; l < d.n_shared + d.n_indep; ++l) {
            GluLayer g = hm.layer(s, l);
            std::vector<float> sc, sh;
            fold_bn(*g.bn, d.bn_eps, sc, sh);
            // The kernel scales the linear half of every layer but an FT's
            // first by sqrt(1/2) (it forms the residual sqrt(1/2) (x + g) as
            // x sqrt(1/2) + g) and the gate half by -log2(e) (its sigmoid takes
            // 2^(-x log2 e)): the shifts are stored pre-scaled.  With several
            // bf16 parts the weights are pre-scaled too; with one part (bf16,
            // FP8) they are packed unscaled, BN-folded and then rounded, so the
            // rounding is that of the BN-folded weight, and the kernel applies
            // the constant to the accumulator.
            const bool prescale_w = np >= 2;
            for (int n = 0; n < N && l > 0; ++n) {
                sh[n] = (float)((double)sh[n] * 0.70710678118654752440);
                if (prescale_w) sc[n] = (float)((double)sc[n] * 0.70710678118654752440);
            }
            for (int n = N; n < 2 * N; ++n) {
                sh[n] = (float)((double)sh[n] * -1.4426950408889634);
                if (prescale_w) sc[n] = (float)((double)sc[n] * -1.4426950408889634);
            }
            if (fp8) {
                std::vector<double> c(2 * N, 1.0);
                for (int n = 0; n < N; ++n) c[n] = l > 0 ? 0.70710678118654752440 : 1.0;
                for (int n = N; n < 2 * N; ++n) c[n] = -1.4426950408889634;
                push_layer_e4m3(*g.w, *g.bn, 2 * N, g.k, 0, l == 0 ? dp : N, 0, c, &stream, &wsc);
            } else {
                const std::vector<float> ws = scaled(*g.w, sc, 2 * N, g.k);
                push_layer(ws.data(), 2 * N, g.k, 0, l == 0 ? dp : N, 0, &stream);
            }
            epi.insert(epi.end(), sh.begin(), sh.end());
        }
    }
    epi.insert(epi.end(), att_epi.begin(), att_epi.end());
    p.epi_sc = 0;
    if (fp8) {
        // the per-channel weight scales follow the shifts, in the same layout
        wsc.insert(wsc.end(), att_wsc.begin(), att_wsc.end());
        p.epi_sc = (int)epi.size();
        epi.insert(epi.end(), wsc.begin(), wsc.end());
    }
    m->tc_chunk_off.clear();
    m->tc_chunk_bytes.clear();
    for (auto& c : stream) {
        m->tc_chunk_off.push_back(c.first);
        m->tc_chunk_bytes.push_back(c.second);
    }
    if (!parts_contiguous) { *why = "weight stream layout: a K block's parts are not contiguous"; return TABNET_ERR_UNSUPPORTED_DIMS; }
    p.chunks_per_tile = (int)stream.size();
    p.epi_floats = (int)epi.size();
    m->tc_off_epi = a.add(epi.data(), epi.size() * 4, 16);
    m->tc_off_chunks = a.add(nullptr, sizeof(uint2) * stream.size(), 16);
    std::vector<int2> ci(dp);
    std::vector<int> cf(dp, -1);
    for (int c = 0; c < dp; ++c) ci[c] = make_int2(-2, 0);
    for (int c = 0; c < d.n_num; ++c) { ci[c] = make_int2(-1, c); cf[c] = c; }
    int col = d.n_num;
    for (int j = 0; j < d.n_cat; ++j)
        for (int e = 0; e < hm.cat_emb_dim[j]; ++e, ++col) { ci[col] = make_int2(j, e); cf[col] = d.n_num + j; }
    m->tc_off_colinfo = a.add(ci.data(), sizeof(int2) * dp, 16);
    m->tc_off_colfeat = a.add(cf.data(), sizeof(int) * dp, 16);
    return TABNET_OK;
}

// Pick warpgroups, ring depth, CTAs per SM and what to stage in shared memory.
int tc_choose_launch(tabnet_model* m, int nwg, int n_slots, int ctas_per_sm, std::string* why) {
    const tabnet_dims& d = m->host.dims;
    const int N = d.n_d + d.n_a;
    TcParams& p = m->tc;
    const int np = precision_parts(m->precision);
    if (nwg <= 0) nwg = (N == 128) ? 2 : 1;
    if (N == 128 && nwg != 2) { *why = "N = 128 needs two warpgroups"; return TABNET_ERR_UNSUPPORTED_DIMS; }
    if (N == 16 && nwg != 1) { *why = "N = 16 takes one warpgroup"; return TABNET_ERR_UNSUPPORTED_DIMS; }
    if (nwg != 1 && nwg != 2) { *why = "one or two warpgroups"; return TABNET_ERR_UNSUPPORTED_DIMS; }
    if (np == 3 && nwg != 1) { *why = "the three-part split takes one warpgroup"; return TABNET_ERR_UNSUPPORTED_DIMS; }
    const int dch = p.dp / 16;
    const bool zreg = (dch + nwg - 1) / nwg <= zreg_chunks(nwg);
    Variant v{N, nwg, np, zreg, false};
    cudaFuncAttributes fa{}, fa_lean{};
    if (!with_kernel(v, [&](auto fn) { cudaFuncGetAttributes(&fa, fn); })) {
        *why = "no kernel for this shape";
        return TABNET_ERR_UNSUPPORTED_DIMS;
    }
    v.lean = true;
    with_kernel(v, [&](auto fn) { cudaFuncGetAttributes(&fa_lean, fn); });
    v.lean = false;
    // either instantiation may run: size the CTA count for the larger register file
    const int regs = std::max({fa.numRegs, fa_lean.numRegs, 1});
    int dev_smem_sm = 0;
    cudaDeviceGetAttribute(&dev_smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, m->device);
    const int reserved = 1024;
    const int threads = 128 * nwg;
    const int reg_limit = 65536 / (((regs * 32 + 255) / 256 * 256) * (threads / 32));
    const int tmem_limit = 512 / p.tmem_cols;
    const int slot_bytes = std::max(2 * N, p.dp) * 128;
    const int min_slots = std::max(np, 1);  // one K block's parts
    int cps_max = std::max(1, std::min({tmem_limit, reg_limit, 4}));
    int best_cps = 0, best_slots = 0;
    bool best_epi = false, best_f = false, best_mst = false;
    // Per CTA count (most first): stage the BN shifts and the tile's input in
    // shared memory when they fit, then take the deepest ring (<= 6) left.
    for (int cps = cps_max; cps >= 1 && !best_cps; --cps) {
        if (ctas_per_sm > 0 && cps != ctas_per_sm) continue;
        const size_t per_cta = (size_t)dev_smem_sm / cps - reserved;
        const size_t budget = std::min((size_t)m->smem_optin, per_cta) - 1024;
        const bool stage_opts[6][3] = {{true, true, true},  {true, true, false},  {true, false, false},
                                       {false, true, true}, {false, true, false}, {false, false, false}};
        for (const auto& st : stage_opts) {
            int found = 0;
            for (int sl = 6; sl >= min_slots; --sl) {
                if (n_slots > 0 && sl != n_slots) continue;
                if (sl % min_slots) continue;  // whole ring units (a K block's parts)
                TcSmem sm = smem_layout(N, p.dp, d.d_emb, d.n_feat, d.n_classes, d.n_d, sl, slot_bytes, np, nwg,
                                        p.epi_floats, p.chunks_per_tile, p.tm_agg >= 0, st[0], st[1], st[2]);
                if ((size_t)sm.total <= budget) { found = sl; break; }
            }
            if (found) {
                best_cps = cps;
                best_slots = found;
                best_epi = st[0];
                best_f = st[1];
                best_mst = st[2];
                break;
            }
        }
    }
    if (!best_cps) { *why = "no launch shape fits shared memory"; return TABNET_ERR_UNSUPPORTED_DIMS; }
    p.n_slots = best_slots;
    p.slot_bytes = slot_bytes;
    p.sm = smem_layout(N, p.dp, d.d_emb, d.n_feat, d.n_classes, d.n_d, best_slots, slot_bytes, np, nwg,
                       p.epi_floats, p.chunks_per_tile, p.tm_agg >= 0, best_epi, best_f, best_mst);
    size_t smem = (size_t)p.sm.total + 1024;
    // request enough shared memory that no more than best_cps CTAs share an SM
    const size_t floor_smem = (size_t)dev_smem_sm / (best_cps + 1) + 1;
    if (smem < floor_smem) smem = std::min(floor_smem, (size_t)m->smem_optin);
    // The CTA scheduler places CTAs by shared memory, registers and threads,
    // not by tensor memory, and a CTA whose tcgen05.alloc finds too few free
    // columns waits until a CTA holding them exits -- after all of that CTA's
    // tiles, when kernels of other models share the SM.  When the model is
    // served next to others, a CTA that asks for T of the 512 columns also
    // takes at least T / 512 of the SM's shared memory (with its reserved
    // share): then any set of such CTAs the scheduler co-locates fits in
    // tensor memory.  (Alone, the smaller request leaves more L1 to the
    // kernels that gather their inputs from global memory: 8 % on the
    // 100-input FP8 kernel.)
    if (m->tmem_shared) {
        const size_t tmem_smem = ((size_t)p.tmem_cols * (size_t)dev_smem_sm + 511) / 512 - (size_t)reserved;
        if (smem < tmem_smem) smem = std::min(tmem_smem, (size_t)m->smem_optin);
    }
    m->tc_launch_cfg.nwg = nwg;
    m->tc_launch_cfg.n_slots = best_slots;
    m->tc_launch_cfg.ctas_per_sm = best_cps;
    m->tc_launch_cfg.smem = smem;
    m->tc_launch_cfg.zreg = zreg;
    m->tc_launch_cfg.lean = p.tm_agg >= 0 && best_epi && best_f;
    v.lean = m->tc_launch_cfg.lean;
    cudaError_t e = cudaSuccess;
    with_kernel(v, [&](auto fn) { e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); });
    if (e != cudaSuccess) { *why = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e); return TABNET_ERR_CUDA; }
    return TABNET_OK;
}

int tc_patch(tabnet_model* m, Arena& a, const uint8_t* base, std::string* why) {
    TcParams& p = m->tc;
    p.m = m->consts;
    p.wbase = base;
    std::vector<uint2> ck(m->tc_chunk_off.size());
    for (size_t i = 0; i < ck.size(); ++i) ck[i] = make_uint2((uint32_t)m->tc_chunk_off[i], m->tc_chunk_bytes[i]);
    std::memcpy(a.image.data() + m->tc_off_chunks, ck.data(), sizeof(uint2) * ck.size());
    p.chunks = (const uint2*)(base + m->tc_off_chunks);
    p.epi = (const float*)(base + m->tc_off_epi);
    p.col_info = (const int2*)(base + m->tc_off_colinfo);
    p.col_feat = (const int*)(base + m->tc_off_colfeat);
    return tc_choose_launch(m, 0, 0, 0, why);
}

cudaError_t tc_launch(tabnet_model* m, const float* x_num, const int* x_cat, int64_t rows, float* logits,
                      float* masks, float* agg, cudaStream_t stream, const SegTable* seg) {
    TcParams p = m->tc;
    p.seg = seg ? *seg : SegTable{nullptr, nullptr, 0};
    const TcLaunch& L = m->tc_launch_cfg;
    const int64_t slots = (int64_t)m->num_sms * L.ctas_per_sm;
    // a segmented launch learns its row count on the device: one CTA per slot
    const unsigned grid = (unsigned)(seg && seg->segs ? slots : std::min<int64_t>((rows + 127) / 128, slots));
    const dim3 block(128 * L.nwg);
    const Variant v{p.m.N, L.nwg, precision_parts(m->precision), L.zreg, L.lean};
    const bool found = with_kernel(v, [&](auto fn) {
        fn<<<grid, block, L.smem, stream>>>(p, x_num, x_cat, rows, logits, masks, agg);
    });
    if (!found) return cudaErrorInvalidValue;
    return cudaGetLastError();
}

void tc_release(tabnet_model*) {}


}  // namespace tabnet
