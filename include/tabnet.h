/*
 * tabnet.h -- C ABI of the B300 TabNet inference library (libtabnet.so).
 *
 * The paper (Sec. III-B) serves a pre-trained TabNet from a GPU function:
 * each call takes a batch of records and returns the predictions together
 * with the feature-attribution masks, the batch size being chosen per call;
 * the model is loaded into GPU memory once, on cold start.  This library is
 * that compute core: tabnet_create loads a weight blob into device memory,
 * tabnet_forward runs the whole TabNet forward pass (Sec. IV-A: n_d = n_a,
 * several decision steps, sparsemax masks; TabNet of Arik & Pfister 2021)
 * for `rows` records in hand-written sm_103a kernels on the caller's stream.
 *
 * Conventions for every function below:
 *   - Return value: TABNET_OK (0) or a negative TABNET_ERR_* code.  No C++
 *     exception and no abort crosses this boundary.  Argument checks are
 *     synchronous; faults found by a kernel (an out-of-range categorical
 *     index, a wait that ran out) are reported asynchronously through
 *     tabnet_poll_status.
 *   - "device pointer" means memory of the model's device (cudaMalloc,
 *     cudaMallocAsync, or torch tensors); "host pointer" means CPU memory.
 *   - Streams are passed as `void*` holding a cudaStream_t (NULL = legacy
 *     default stream).  Calls are stream-ordered and return before the work
 *     finishes; the caller synchronises.
 *   - All floating-point tensors are row-major float32, integers int32.
 *   - A handle may be used from several host threads and streams at once
 *     for forward calls (the weights are read-only); create/destroy must not
 *     race with other calls on the same handle.
 */
#ifndef TABNET_H
#define TABNET_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TABNET_ABI_VERSION 1

/* Status codes. */
#define TABNET_OK                    0
#define TABNET_ERR_ARG              -1  /* null pointer, negative size, misaligned buffer */
#define TABNET_ERR_BLOB_MAGIC       -2  /* blob does not start with the TABN magic */
#define TABNET_ERR_BLOB_VERSION     -3  /* blob format version not supported */
#define TABNET_ERR_BLOB_SIZE        -4  /* blob shorter/longer than its header says */
#define TABNET_ERR_BLOB_HASH        -5  /* payload hash mismatch (corrupt blob) */
#define TABNET_ERR_UNSUPPORTED_DIMS -6  /* model shape outside the kernels' limits */
#define TABNET_ERR_CUDA             -7  /* a CUDA runtime call failed (no device, bad stream...) */
#define TABNET_ERR_OOM              -8  /* device allocation failed */
#define TABNET_ERR_TIMEOUT          -9  /* a bounded device wait ran out (see poll_status) */
#define TABNET_ERR_DEVICE           -10 /* poll_status found a device-side fault bit */

/* Device status bits (tabnet_poll_status). */
#define TABNET_STATUS_CAT_OOB  0x1u  /* a categorical index was outside [0, card): a zero
                                        embedding row was used for it */
#define TABNET_STATUS_TIMEOUT  0x2u  /* a bounded barrier wait ran out; outputs of that
                                        launch are undefined */

/* Arithmetic of the fully connected layers.  In every mode the sparsemax
 * threshold, the prior, the masks and their aggregation are float32. */
typedef enum {
    TABNET_FP32 = 0,      /* float32 FMA everywhere (no TF32), on the CUDA cores;
                             a call of at most 32 rows per SM runs one warp
                             per row (the latency form), a larger one four
                             lanes per row, with bit-identical results */
    TABNET_BF16 = 1,      /* bf16 x bf16 -> fp32 tensor-core FCs (tcgen05): every
                             BN-folded weight and every FC input rounded once
                             to bf16; the rest in fp32 */
    TABNET_FP8_E4M3 = 2,  /* e4m3 x e4m3 -> fp32 tensor-core FCs (tcgen05
                             kind::f8f6f4): every BN-folded weight row scaled
                             by its amax / 448 (per output channel) and every
                             FC input row by its amax / 448 (per row; the
                             attentive layer's input over its attention half),
                             rounded to nearest even, saturating at 448; the
                             accumulator is multiplied back by both scales.
                             E4M3's 3 mantissa bits move the sparsemax masks
                             of most rows: against float64 the mean per-row
                             mask L1 is about 0.2 / 0.8 / 1.0 and the argmax
                             agreement 99.9 / 100 / 94.7 % on the 14-, 35- and
                             100-input models (the rounding's own error) */
    TABNET_BF16X3 = 3,    /* split bf16 on the same tensor cores: each operand
                             carried as hi + lo bf16 (lo = bf16(x - hi)), three
                             bf16 MMAs per K step (hi*hi + hi*lo + lo*hi) into
                             one fp32 accumulator, accurate sigmoid; about
                             16 significant bits per operand */
    TABNET_BF16X6 = 4     /* float32-accurate FCs on the tensor cores: each
                             operand as hi + mid + lo bf16 (exact for float32
                             values), six bf16 MMAs per K step (every product
                             down to 2^-16 of hi*hi) into one fp32 accumulator;
                             meets the float32 tolerances.  Needs
                             n_d + n_a <= 64 and a launch shape within shared
                             memory (three A-operand parts and three ring
                             slots: wide embeddings with multi-column
                             features may not fit); tabnet_create returns
                             TABNET_ERR_UNSUPPORTED_DIMS otherwise */
} tabnet_precision;

/* Model shape, as read from a blob. */
typedef struct {
    int32_t n_num;      /* numeric input columns */
    int32_t n_cat;      /* categorical input columns */
    int32_t d_emb;      /* D_e: width after embedding = n_num + sum of embedding dims;
                           width of each per-step mask */
    int32_t n_feat;     /* D = n_num + n_cat: width of the aggregated mask */
    int32_t n_d, n_a;   /* decision / attention widths */
    int32_t n_steps;    /* decision steps (= masks per row) */
    int32_t n_shared;   /* GLU layers shared by every feature transformer */
    int32_t n_indep;    /* GLU layers specific to each feature transformer */
    int32_t n_classes;  /* logits per row */
    double gamma;       /* prior relaxation */
    double bn_eps;
    uint64_t content_hash;  /* payload hash stored in (and checked against) the blob */
} tabnet_dims;

typedef struct tabnet_model tabnet_model;

/* Returns TABNET_ABI_VERSION. */
int tabnet_abi_version(void);

/* Validate a weight blob and read its shape without touching a GPU.
 * blob: host pointer to blob_bytes bytes (format version 1: 96-byte header
 * then the parameter arrays; written by paper_2510_19689_b300.synth.to_blob).
 * out: filled on success.  Errors: ARG, BLOB_MAGIC, BLOB_VERSION, BLOB_SIZE,
 * BLOB_HASH, UNSUPPORTED_DIMS (shape fields out of range). */
int tabnet_blob_inspect(const void* blob, size_t blob_bytes, tabnet_dims* out);

/* Load a model onto `device` for the given precision (a tabnet_precision).
 * The blob is validated, its BN statistics are folded into per-channel
 * scale/shift pairs (input BN also into the embedding tables), its weights
 * are converted and packed for the kernels of that precision and copied to
 * device memory owned by the handle.  The blob is only read during the call;
 * the caller may free it afterwards.  On success *out holds a new handle.
 * Errors: any of tabnet_blob_inspect, UNSUPPORTED_DIMS (shape outside what
 * the kernels of that precision handle), CUDA (no such device), OOM. */
int tabnet_create(const void* blob, size_t blob_bytes, int precision, int device,
                  tabnet_model** out);

/* Shape of a loaded model.  Errors: ARG. */
int tabnet_dims_of(const tabnet_model* model, tabnet_dims* out);

/* Precision the handle was created with, or ARG. */
int tabnet_precision_of(const tabnet_model* model);

/* Batched inference, stream-ordered on `stream`.
 *   x_num      device, [rows, n_num] float32 (may be NULL when n_num == 0)
 *   x_cat      device, [rows, n_cat] int32   (may be NULL when n_cat == 0)
 *   logits     device, [rows, n_classes] float32, raw logits (no softmax)
 *   step_masks device, [rows, n_steps, d_emb] float32: sparsemax mask of
 *              every decision step (each sums to 1), or NULL to skip
 *   agg_mask   device, [rows, n_feat] float32: step masks weighted by each
 *              step's decision strength, summed over each feature's embedding
 *              columns and normalised to sum 1 (all zero when every step's
 *              decision output is zero), or NULL to skip
 * All buffers are owned by the caller, 4-byte aligned, and must not overlap.
 * rows == 0 returns TABNET_OK without launching.  Rows are independent:
 * a row's outputs do not depend on the other rows of the call.
 * Errors: ARG (null handle or required pointer, rows < 0), CUDA (launch). */
int tabnet_forward(tabnet_model* model, const float* x_num, const int32_t* x_cat,
                   int64_t rows, float* logits, float* step_masks, float* agg_mask,
                   void* stream);

/* One request of a segmented launch: its own device buffers, laid out as in
 * tabnet_forward (rows may be 0; step_masks / agg_mask may be NULL). */
typedef struct {
    const float* x_num;     /* device [rows, n_num] */
    const int32_t* x_cat;   /* device [rows, n_cat] */
    int64_t rows;
    float* logits;          /* device [rows, n_classes] */
    float* step_masks;      /* device [rows, n_steps, d_emb] or NULL */
    float* agg_mask;        /* device [rows, n_feat] or NULL */
} tabnet_segment;

/* Many independent request batches of uneven size in ONE persistent kernel
 * launch (the paper's per-invocation batch size, Sec. III-B, served for many
 * invocations at once).  The rows of all segments are packed back to back
 * into 128-row tiles (a tile may span segments, so small requests waste no
 * tile); every row reads and writes its own segment's buffers.
 *   segs   HOST array of n_segs descriptors (copied before return; the call
 *          may wait for the previous call's copy of the same handle)
 * The device side needs (n_segs + 1) 8-byte prefix sums of scratch, owned by
 * the handle and grown on demand.  Not for stream capture (it stages through
 * host memory): use tabnet_forward_segments_device for CUDA graphs.
 * Errors: ARG (null, n_segs < 0, a segment with rows < 0 or a NULL required
 * pointer), OOM, CUDA. */
int tabnet_forward_segments(tabnet_model* model, const tabnet_segment* segs, int n_segs, void* stream);

/* As tabnet_forward_segments with the descriptors already in DEVICE memory
 * (caller-owned, read by the kernels on `stream`, never written).  A scan
 * kernel computes the prefix sums on the device, so the call makes no host
 * round trip and can be captured in a CUDA graph, provided the scratch was
 * reserved beforehand (tabnet_reserve_segments) for at least n_segs; a
 * capture that would need more scratch fails with OOM instead of allocating.
 * Segment rows are not validated on the host (a negative count is treated
 * as 0 by the scan).  Errors: ARG, OOM, CUDA. */
int tabnet_forward_segments_device(tabnet_model* model, const tabnet_segment* segs, int n_segs,
                                   void* stream);

/* Reserve the segmented launches' scratch for up to max_segs segments
 * (device memory owned by the handle, freed by tabnet_destroy).
 * Errors: ARG, OOM. */
int tabnet_reserve_segments(tabnet_model* model, int max_segs);

/* tabnet_forward_segments_device for callers that cannot allocate device
 * memory.  (The paper has no counterpart: this is a deployment convenience of
 * this library.)  Some callers must not call cudaMalloc once they are
 * running: serving processes that fix their device memory at start-up so
 * that no request can fail or stall on an allocation, and hosts that give a
 * plug-in only memory they allocated themselves.  This entry point allocates nothing: the prefix sums
 * of the segments' row counts (its only scratch) live in a fixed array in the
 * library's device image, TABNET_NOALLOC_MAX_SEGMENTS + 1 entries (512 KB),
 * held by every GPU that loads the library until the process exits.
 *   segs    DEVICE array of n_segs descriptors (caller-owned, only read)
 * The first call on a device looks up that array's device address (once per
 * device, with the model's device made current for the call); make that
 * first call before any stream capture.  Every call on a device shares the
 * array: calls whose work overlaps on the GPU (other streams, other handles
 * on the same device) race on it, so serialise them.  Nothing in the array
 * has to start at zero: each launch rewrites the entries it reads.
 * Errors: ARG (null, n_segs < 0 or > TABNET_NOALLOC_MAX_SEGMENTS), CUDA. */
#define TABNET_NOALLOC_MAX_SEGMENTS 65536
int tabnet_forward_segments_noalloc(tabnet_model* model, const tabnet_segment* segs, int n_segs,
                                    void* stream);

/* Same computation with HOST buffers (pinned or pageable): the inputs are
 * copied into a device workspace owned by the handle, the forward runs, and
 * the outputs are copied back; the call returns after the copies have
 * finished (synchronous).  A call with more than about 8 MB of outputs is
 * split into row chunks (whole 128-row tiles) that run on four streams owned
 * by the handle, so that input copies, kernels and output copies of
 * different chunks overlap; those streams start after the work already
 * queued on `stream`, and `stream` waits for them before the call returns.
 * Every row's results are the same as in one tabnet_forward launch.  This is the paper's
 * function invocation (records in, predictions and masks out, Sec. III-B)
 * seen from a host caller.  Workspace grows on demand and is freed by
 * tabnet_destroy.  Not thread-safe per handle.  Errors: as tabnet_forward,
 * OOM. */
int tabnet_forward_host(tabnet_model* model, const float* x_num, const int32_t* x_cat,
                        int64_t rows, float* logits, float* step_masks, float* agg_mask,
                        void* stream);

/* Launch shape of the tensor-core kernels (bf16, split-bf16 precisions):
 *   nwg          epilogue warpgroups per 128-row tile (1 or 2; 2 is required
 *                when n_d + n_a = 128, 1 when it is 16)
 *   n_slots      depth of the shared-memory ring that stages weight blocks
 *                (>= 1, >= 2 for split-bf16)
 *   ctas_per_sm  tiles resident per SM (bounded by tensor memory, registers
 *                and shared memory)
 * Values <= 0 let the library choose.  What does not fit is reported as
 * UNSUPPORTED_DIMS and leaves the previous shape in place.  Results may
 * differ between shapes in the last bits (sums split across warpgroups).
 * Not thread-safe against concurrent forward calls on the same handle.
 * This is the hook of the autotuner (paper_2510_19689_b300.autotune).
 * Errors: ARG, UNSUPPORTED_DIMS (also for the fp32 precision), CUDA. */
int tabnet_set_tile_config(tabnet_model* model, int nwg, int n_slots, int ctas_per_sm);

/* The launch shape in use (each output may be NULL).  Errors: ARG,
 * UNSUPPORTED_DIMS for the fp32 precision. */
int tabnet_get_tile_config(const tabnet_model* model, int* nwg, int* n_slots, int* ctas_per_sm);

/* ---------------------------------------------------------------- serving
 * A continuous-batching request server over resident models on one GPU (the
 * paper's GPU functions keep the model in GPU memory and serve batches of
 * records per invocation, Sec. III-B, measured by p50/p95/p99 latency,
 * Sec. IV-C).  A request's inputs are copied at submission into its
 * model's pinned input ring (rows in submission order).  An engine thread
 * owned by the server packs every staged request that has arrived for a
 * model into one batch (admission by memory: a request waits while a ring is
 * full), runs it as one forward launch with one copy in and one copy out
 * on one of the model's streams, and forms the next batch without waiting,
 * so requests arriving while others run are admitted as memory frees and
 * overlap on the device.  Latency = completion observed on the host -
 * arrival (the submission, or a replayed request's scheduled arrival). */
typedef struct tabnet_server tabnet_server;

typedef struct {
    size_t device_bytes;       /* device memory for all rings (0: 1 GiB), split by bytes per row */
    int max_batch_rows;        /* rows per batch at most (0: 65536) */
    int max_inflight_batches;  /* batches per model running on the GPU at once (0: 32); finished
                                  but unreleased results hold ring memory, not a slot */
    int streams_per_model;     /* CUDA streams per model (0: 8, at most 64): small batches of
                                  one model run side by side on different SMs */
    int batch_min_rows;        /* adaptive batching: once batch_busy of a model's batches are
                                  running, a batch of fewer rows than this (0: 2048; < 0: off)
                                  waits ... */
    int batch_wait_us;         /* ... for more requests, at most this long for its oldest
                                  (0: 200 us), so that one launch serves more rows under load */
    int batch_busy;            /* adaptive batching engages once this many of a model's batches are
                                  running (0: 2) */
    int mask_slots;            /* step masks go to the host compact: per (row, step) the count of
                                  nonzero columns and up to this many (column, value) pairs,
                                  exact; a batch with a row-step over the limit is sent densely.
                                  0: max(16, d_emb / 5) rounded up to 8 where that saves a quarter
                                  of the bytes, else dense; < 0: always dense; at most 254 */
} tabnet_server_config;

typedef struct {
    uint64_t submitted, completed, rejected, rows_completed, batches;
    double mean_batch_rows;
    double p50_ms, p95_ms, p99_ms, mean_ms, max_ms;  /* latency of completed requests: completion seen
                                                        on the host - arrival (submission, or a replayed
                                                        request's scheduled arrival); every percentile
                                                        of these stats is over the most recent 1,048,576
                                                        requests completed since the reset */
    double rows_per_s;                               /* completed rows / time since reset */
    int64_t queue_depth, inflight_batches;
    size_t device_bytes_in_use;
    uint64_t engine_staged;  /* requests whose inputs the engine copied (the input ring
                                was full when they were submitted) */
    double p50_queue_ms, p99_queue_ms;  /* of completed requests: arrival -> their batch's launch */
    double engine_busy;      /* fraction of the time since the reset the engine thread was not
                                asleep waiting for work */
    double engine_max_pass_ms;  /* longest single engine pass (completions + launches) */
    double replay_max_late_ms;  /* tabnet_server_replay: latest submission behind its arrival */
    double p50_submit_ms, p99_submit_ms;  /* latency counted from the submission call instead (the
                                             server's share when a replay client fell behind) */
} tabnet_server_stats;

/* One request of a replayed trace (tabnet_server_replay). */
typedef struct {
    int model;              /* index into the server's models */
    const float* x_num;     /* host [rows, n_num] */
    const int32_t* x_cat;   /* host [rows, n_cat] */
    int64_t rows;
    double arrival_s;       /* offset from the start of the replay */
} tabnet_server_request;

/* Create a server over n_models loaded handles (all on one device; the
 * handles must outlive the server).  cfg may be NULL.  Allocates the device
 * rings and their pinned host mirrors and starts the engine thread.  The
 * handles' tensor-core launches are resized (same launch shape, more shared
 * memory where needed) so that CTAs of the different models that the GPU
 * places on one SM always fit in its tensor memory; this stays in effect for
 * the handles after the server is destroyed.
 * Errors: ARG, OOM. */
int tabnet_server_create(tabnet_model* const* models, int n_models, const tabnet_server_config* cfg,
                         tabnet_server** out);

/* Queue a request: host inputs [rows, n_num] / [rows, n_cat] of model
 * `model`, which must stay valid until the request is complete.  Copies the
 * inputs into the model's input ring when it has room (on the calling
 * thread; otherwise the engine copies them once room frees) and returns with
 * a ticket without waiting for the GPU.  A request larger than the model's
 * rings is rejected by the engine (counted in stats.rejected; it never
 * completes).  Thread-safe.  Errors: ARG, OOM. */
int tabnet_server_submit(tabnet_server* server, int model, const float* x_num, const int32_t* x_cat,
                         int64_t rows, uint64_t* ticket);

/* Tickets completed since the last poll (at most max_tickets).  Returns the
 * engine's sticky error (TABNET_OK normally). */
int tabnet_server_poll(tabnet_server* server, uint64_t* tickets, int max_tickets, int* n_done);

/* Block until the request is complete or timeout_s passes (TIMEOUT). */
int tabnet_server_wait(tabnet_server* server, uint64_t ticket, double timeout_s);

/* Pointers to a completed request's outputs (host memory owned by the
 * server, laid out as in tabnet_forward), valid until it is released.  Step
 * masks that came compact are expanded on the first call, on the calling
 * thread (call result and release of one ticket from one thread). */
int tabnet_server_result(tabnet_server* server, uint64_t ticket, const float** logits,
                         const float** step_masks, const float** agg_mask, int64_t* rows);

/* The step masks of a completed request in the compact form they came in:
 * for (row i, step s) at k = i n_steps + s, counts[k] nonzero columns, the
 * first min(counts[k], slots) of them at cols[k slots + j] (ascending) with
 * values vals[k slots + j]; every other entry is +0.  *slots = 0 and NULL
 * pointers when the request's batch was sent densely (read it through
 * tabnet_server_result).  Valid until the request is released.
 * Errors: ARG. */
int tabnet_server_result_compact(tabnet_server* server, uint64_t ticket, const uint8_t** counts,
                                 const uint16_t** cols, const float** vals, int* slots, int64_t* rows);

/* Give a completed request's result memory back (ring space is reused once
 * every request of its batch and of older batches is released). */
int tabnet_server_release(tabnet_server* server, uint64_t ticket);

/* Counters and latency percentiles since the last reset. */
int tabnet_server_get_stats(tabnet_server* server, tabnet_server_stats* stats);
int tabnet_server_reset_stats(tabnet_server* server);

/* Load driver: submit reqs[i] at its arrival offset (busy-waiting on the
 * host clock) from `threads` submitting threads (<= 0: 1, at most 64;
 * thread j takes requests j, j + threads, ... in order), standing for that
 * many clients; a replayed request's latency counts from its scheduled
 * arrival, so a submission that comes late counts too.  The first `warmup`
 * requests are served but left out of the latency statistics (the counts
 * and row totals include them).  With `release` != 0 completed requests are
 * released as they finish (polled every 20 us, between submissions too when
 * a thread is behind schedule) and the call returns when all are done.
 * Errors: as tabnet_server_submit. */
int tabnet_server_replay(tabnet_server* server, const tabnet_server_request* reqs, int n, int release,
                         int threads, int warmup);

/* Stop the engine, wait for the GPU, free everything. */
void tabnet_server_destroy(tabnet_server* server);

/* Preprocessing folded into the model (the upstream step of the paper's
 * data pipeline, Sec. III-A): numeric column c is fed as
 * (x_num[c] - num_mean[c]) * num_scale[c] (a fitted standard scaler:
 * scale = 1 / std) and categorical column j as x_cat[j] - cat_base[j]
 * (raw ordinal or label codes whose first category is cat_base[j]).  The
 * scaler is folded into the input BN on the host (no work per row); the base
 * is one subtraction in the gather.  Host arrays of n_num, n_num and n_cat
 * entries; NULL means identity (mean 0, scale 1, base 0), and each call
 * replaces the previous transform.  Synchronises the device first; no
 * forward on this model may run concurrently with the call.  Errors: ARG
 * (NULL model, a non-finite mean or scale), CUDA. */
int tabnet_set_input_transform(tabnet_model* model, const float* num_mean, const float* num_scale,
                               const int32_t* cat_base);

/* Read and clear the handle's device status word (TABNET_STATUS_* bits) after
 * synchronising `stream`.  *status receives the bits; returns TABNET_OK when
 * no bit was set, TABNET_ERR_TIMEOUT when the timeout bit was set, else
 * TABNET_ERR_DEVICE.  Errors: ARG, CUDA. */
int tabnet_poll_status(tabnet_model* model, void* stream, uint32_t* status);

/* Free the handle and its device memory (synchronises the device first).
 * NULL is accepted. */
void tabnet_destroy(tabnet_model* model);

/* Static description of a status code. */
const char* tabnet_status_string(int code);

/* ---- audit statistics of aggregated masks (Sec. V-C: interpretability
 * under load -- which features carry the decisions and whether their
 * ranking holds).  Both read a [rows][d] float32 device array laid out as
 * tabnet_forward's agg_mask output (any row-major [rows][d] float32 array
 * works), need no model, run on `stream` and return once launched; they
 * allocate their small scratch stream-ordered (cudaMallocAsync).  Errors:
 * TABNET_ERR_ARG for a NULL input, rows < 1, d outside [1, 1024] or k
 * outside [1, min(d, 32)]; TABNET_ERR_CUDA if an allocation or launch fails. */

/* Per feature j over the rows (float32 device outputs, each may be NULL):
 *   mean[j]      = (1/rows) sum_r agg[r][j]
 *   var[j]       = (1/rows) sum_r (agg[r][j] - mean[j])^2   (population)
 *   topk_frac[j] = fraction of rows whose k largest entries include j,
 *                  equal entries ranked by the lower index first.
 * Sums are compensated and combined in a fixed order (deterministic). */
int tabnet_mask_stats(const float* agg, int64_t rows, int d, int k, float* mean, float* var,
                      float* topk_frac, void* stream);

/* Agreement of two aggregates' top-k feature sets, row by row (e.g. the same
 * rows served alone and inside a mixed batch, or at two precisions):
 *   *out = (1/(rows k)) sum_r |topk(agg_a[r]) intersect topk(agg_b[r])|
 * with the tie rule above; out is one float32 in device memory. */
int tabnet_topk_agreement(const float* agg_a, const float* agg_b, int64_t rows, int d, int k, float* out,
                          void* stream);

/* One-line reason for the last failing call made by this host thread
 * ("" when none).  The pointer stays valid until the thread's next call. */
const char* tabnet_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* TABNET_H */
