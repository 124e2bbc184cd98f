// Continuous-batching request server over resident models.
//
// The paper serves TabNet from GPU functions that keep the model in GPU
// memory after a cold start and take a batch of records per invocation
// (Sec. III-B), reporting p50/p95/p99 latency beside throughput (Sec. IV-C).
// This engine does that for many concurrent requests on one GPU:
//
//   * every model has two device rings with pinned host mirrors (its share
//     of the memory budget, split so both hold about as many rows): an
//     input ring of rows, filled in submission order, and an output ring of
//     bytes with one contiguous region per batch;
//   * a request's inputs are copied into the input ring by the submitting
//     thread when the ring has room (and no older request of the model is
//     still waiting for room), otherwise by the engine later, in order --
//     admission is by memory: a request waits while a ring is full and is
//     rejected only if it could never fit.  The copies stay off the engine
//     thread, whose time per request is what bounds the request rate;
//   * an engine thread takes, per model, every staged request that has
//     arrived (up to max_batch_rows; consecutive requests are consecutive
//     input rows) into one batch: one host-to-device copy of its rows, ONE
//     forward launch over them, and one device-to-host copy of the outputs,
//     on one of the model's streams (the copy engines, not the kernels, are
//     what saturates first at high request rates: each copy counts); the
//     engine never waits for a batch before forming the next one, so
//     requests that arrive while others are on the GPU are admitted as soon
//     as ring space frees and their batches overlap on the device (streams
//     of other batches and of the other models);
//   * completion is observed by polling the batch's event (a batch found
//     running is asked again 10 us later); its input rows go back at once,
//     the request's results stay in the pinned output mirror until the
//     caller releases it, and an output region is reused once its batch and
//     every older batch of the ring are released.
// Latency of a request = completion observed on the host - submission time.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <pthread.h>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/tabnet.h"
#include "model_handle.h"

namespace tabnet {
int set_last_error(int code, const std::string& why);
cudaError_t mask_compact_launch(const float* masks, int64_t row_steps, int de, int slots, uint8_t* counts,
                                uint16_t* cols, float* vals, cudaStream_t stream);
}

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket = 0;
    int model = 0;
    const float* x_num = nullptr;
    const int32_t* x_cat = nullptr;
    int64_t rows = 0;
    // arrival: the submission time, or a replayed request's scheduled
    // arrival (a late submission then counts in its latency)
    Clock::time_point t_arrival;
    Clock::time_point t_submit;  // when the submission call ran
    bool measured = true;        // in the latency statistics (a replay's warm-up requests are not)
    // rows of the model's input ring holding the inputs (-1: not staged
    // yet), and whether they are copied there
    int64_t in_row0 = -1;
    std::atomic<bool> ready{false};
    // the dense step masks, expanded from the compact form on first request
    std::vector<float> dense_masks;
    // filled when batched
    int64_t row0 = 0;       // first row inside its batch
    struct Batch* batch = nullptr;
};

struct Batch {
    int model;
    int stream_idx;
    size_t off = 0, bytes = 0;  // output ring region
    int64_t rows = 0;
    int64_t in_row0 = 0;        // input ring rows [in_row0, in_row0 + rows)
    Clock::time_point next_query;  // no completion query before this
    // offsets inside the output region: logits, aggregate, then (compact
    // transfer) counts, columns and values, then the dense step masks; the
    // first copy_bytes go to the host, the dense masks too when dense
    size_t out_lg = 0, out_ag = 0, out_cnt = 0, out_col = 0, out_val = 0, out_mk = 0, copy_bytes = 0;
    bool dense = true;          // the host mirror holds the dense step masks
    bool dense_pending = false; // a row-step overflowed its slots: the dense copy is on its way
    std::vector<uint64_t> tickets;
    cudaEvent_t done = nullptr;
    Clock::time_point t_launch;
    bool complete = false;
    int released = 0;
};

// A ring of `cap` units: allocate at head, free at tail, in order.
struct Ring {
    size_t cap = 0, head = 0, tail = 0, used = 0;
};

struct ModelCtx {
    tabnet_model* model;
    tabnet_dims d;
    size_t in_row, out_row;        // bytes per row (inputs, outputs)
    // outputs: a ring of bytes, one region per batch
    uint8_t* dev = nullptr;        // device ring
    uint8_t* host = nullptr;       // pinned mirror
    Ring out;
    // inputs: a ring of rows, requests in submission order (so a batch of
    // consecutive requests is one row range, one copy); row i at
    // in_* + i in_row: its n_num floats, then its n_cat codes
    uint8_t* in_dev = nullptr;
    uint8_t* in_host = nullptr;
    Ring in;
    int slots = 0;                 // compact mask slots per (row, step); 0: dense transfer
    int64_t stage_max = 0;         // rows a request may have to be staged (fits both rings)
    // queued requests whose inputs are not in the input ring yet, in
    // submission order (all of them after every staged request)
    std::deque<Request*> unstaged;
    std::deque<Batch*> in_order;   // batches holding input rows, in ring order
    std::deque<Batch*> inflight;   // in output-ring order
    std::deque<Request*> pending;
    std::vector<cudaStream_t> streams;
    int next_stream = 0;
    int running = 0;               // batches launched and not yet complete
    // running estimate of a batch's time from launch to its completion being
    // seen (us; 0 until the first): a batch is not asked before most of it
    // has passed, so the engine's event queries stay few per batch
    double est_us = 0;
    int64_t pending_rows = 0;      // rows of the pending requests
};

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

constexpr size_t kRegionSlack = 6 * 256;  // alignment of the six arrays of an output region

}  // namespace

namespace {
// Latency samples for the percentiles: the most recent kCap values (a ring
// once full), so that a server that runs for hours without a reset keeps a
// bounded record.
struct Samples {
    static constexpr size_t kCap = (size_t)1 << 20;
    std::vector<double> v;
    size_t n = 0;  // values pushed since the last clear
    void push(double x) {
        if (v.size() < kCap) v.push_back(x);
        else v[n % kCap] = x;
        ++n;
    }
    void clear() { v.clear(); n = 0; }
};

// The server lock: a pthread mutex of the adaptive kind, which spins
// briefly before it sleeps.  Its critical sections are short and taken
// hundreds of thousands of times a second by the clients and the engine; a
// plain mutex puts every contender to sleep at once, and the wake-ups queue
// submissions behind each other.
class ServerMutex {
public:
    ServerMutex() {
        pthread_mutexattr_t a;
        pthread_mutexattr_init(&a);
        pthread_mutexattr_settype(&a, PTHREAD_MUTEX_ADAPTIVE_NP);
        pthread_mutex_init(&m_, &a);
        pthread_mutexattr_destroy(&a);
    }
    ~ServerMutex() { pthread_mutex_destroy(&m_); }
    ServerMutex(const ServerMutex&) = delete;
    ServerMutex& operator=(const ServerMutex&) = delete;
    void lock() { pthread_mutex_lock(&m_); }
    bool try_lock() { return pthread_mutex_trylock(&m_) == 0; }
    void unlock() { pthread_mutex_unlock(&m_); }

private:
    pthread_mutex_t m_;
};
}  // namespace

struct tabnet_server {
    std::vector<ModelCtx> models;
    tabnet_server_config cfg{};
    ServerMutex mu;                      // guards pending queues, requests, stats
    std::condition_variable_any cv;
    std::unordered_map<uint64_t, Request*> reqs;
    std::atomic<uint64_t> next_ticket{1};
    std::deque<uint64_t> completed;      // tickets completed, not yet returned by poll
    Samples lat_ms;                      // completed requests' latencies since the last reset
    Samples queue_ms;                    // their arrival -> batch launch times
    Samples sub_ms;                      // their submission call -> completion times
    double engine_sleep_s = 0;           // engine time asleep on cv since the last reset
    double engine_max_pass_ms = 0;       // longest engine pass (completions + launches) since the reset
    std::atomic<int64_t> replay_max_late_ns{0};  // latest replayed submission behind its arrival
    uint64_t submitted = 0, n_completed = 0, rejected = 0, rows_done = 0, batches = 0, batch_rows = 0;
    uint64_t engine_staged = 0;
    Clock::time_point t_reset = Clock::now();
    std::thread engine;
    std::atomic<bool> stop{false};
    std::atomic<bool> engine_idle{false};  // the engine sleeps on cv: submit and release wake it
    int device = 0;
    int error = TABNET_OK;
    std::vector<cudaEvent_t> free_events;  // completion events of freed batches, reused (engine thread only)
};

namespace {

// Offsets of a batch's output region (see Batch).
void layout_region(const ModelCtx& mc, Batch* b) {
    const tabnet_dims& d = mc.d;
    const size_t rs = (size_t)b->rows * d.n_steps;
    b->out_lg = 0;
    b->out_ag = b->out_lg + align256((size_t)b->rows * d.n_classes * 4);
    b->out_cnt = b->out_ag + align256((size_t)b->rows * d.n_feat * 4);
    b->out_col = b->out_cnt + (mc.slots ? align256(rs) : 0);
    b->out_val = b->out_col + (mc.slots ? align256(rs * mc.slots * 2) : 0);
    b->out_mk = b->out_val + (mc.slots ? align256(rs * mc.slots * 4) : 0);
    b->copy_bytes = mc.slots ? b->out_mk : b->out_mk + rs * d.d_emb * 4;
    b->dense = mc.slots == 0;
}

// Reserve n contiguous units at the ring head (wrapping to 0 when the tail
// leaves room there).  Returns false when the ring cannot hold them now.
bool ring_alloc(Ring& g, size_t n, size_t* off) {
    if (n > g.cap) return false;
    if (g.used == 0) g.head = g.tail = 0;
    if (g.head >= g.tail && g.used < g.cap) {
        if (g.cap - g.head >= n) { *off = g.head; g.head += n; g.used += n; return true; }
        if (g.tail >= n) {  // wrap: waste the end of the ring
            g.used += (g.cap - g.head) + n;
            *off = 0;
            g.head = n;
            return true;
        }
        return false;
    }
    if (g.head < g.tail && g.tail - g.head >= n) { *off = g.head; g.head += n; g.used += n; return true; }
    return false;
}

// Free the oldest allocation, [off, off + n) (allocations are freed in ring
// order).
void ring_free_front(Ring& g, size_t off, size_t n) {
    if (off < g.tail) {  // this allocation wrapped: the waste before it goes too
        g.used -= (g.cap - g.tail);
        g.tail = 0;
    }
    g.used -= n;
    g.tail = off + n;
    if (g.used == 0) g.head = g.tail = 0;
}

// Copy a request's inputs into its input-ring rows (pinned host memory),
// each row's numeric columns then its categorical codes.
void stage_inputs(ModelCtx& mc, Request* r) {
    const tabnet_dims& d = mc.d;
    const size_t nb = (size_t)d.n_num * 4, cb = (size_t)d.n_cat * 4;
    uint8_t* dst = mc.in_host + (size_t)r->in_row0 * mc.in_row;
    const uint8_t* xn = reinterpret_cast<const uint8_t*>(r->x_num);
    const uint8_t* xc = reinterpret_cast<const uint8_t*>(r->x_cat);
    for (int64_t i = 0; i < r->rows; ++i, dst += mc.in_row) {
        if (nb) std::memcpy(dst, xn + i * nb, nb);
        if (cb) std::memcpy(dst + nb, xc + i * cb, cb);
    }
    r->ready.store(true, std::memory_order_release);
}

void engine_loop(tabnet_server* S) {
    cudaSetDevice(S->device);
    std::vector<Request*> take, stage_now;
    while (!S->stop.load(std::memory_order_relaxed)) {
        bool did = false;
        const auto t_pass = Clock::now();
        // 1. completions: batches of one stream finish in order, batches of
        // different streams in any order, so each stream's oldest unfinished
        // batch is asked and a stream is skipped once one of its batches is
        // still running (a short batch is not held behind a long one on
        // another stream)
        for (auto& mc : S->models) {
            uint64_t blocked = 0;  // bit i: stream i has a batch still running
            const auto t_now = Clock::now();
            for (Batch* b : mc.inflight) {
                if (b->complete) continue;
                const uint64_t bit = 1ull << (b->stream_idx & 63);
                if (blocked & bit) continue;
                // a batch is first asked once 3/4 of the model's recent
                // launch-to-completion time (at least 20 us) has passed, and
                // one found running is asked again 10 us later: a query costs
                // the engine about a microsecond, and asking every running
                // batch of three models every 10 us took most of its time
                if (t_now < b->next_query) {
                    blocked |= bit;
                    continue;
                }
                const cudaError_t q = cudaEventQuery(b->done);
                if (q == cudaErrorNotReady) {
                    b->next_query = t_now + std::chrono::microseconds(10);
                    blocked |= bit;
                    continue;
                }
                if (q == cudaSuccess && !b->dense_pending) {
                    const double obs = std::chrono::duration<double, std::micro>(t_now - b->t_launch).count();
                    mc.est_us = mc.est_us > 0 ? 0.9 * mc.est_us + 0.1 * obs : obs;
                }
                if (q == cudaSuccess && !b->dense) {
                    if (b->dense_pending) {
                        b->dense = true;  // the dense copy has arrived
                    } else {
                        // a row-step with more nonzeros than slots: send this
                        // batch's dense masks too (rare: the slots are sized
                        // well above the supports sparsemax produces)
                        const uint8_t* cnt = mc.host + b->off + b->out_cnt;
                        const size_t rs = (size_t)b->rows * mc.d.n_steps;
                        bool over = false;
                        for (size_t i = 0; i < rs && !over; ++i) over = cnt[i] > mc.slots;
                        if (over) {
                            const size_t mk_bytes = rs * mc.d.d_emb * 4;
                            cudaStream_t st = mc.streams[b->stream_idx];
                            cudaMemcpyAsync(mc.host + b->off + b->out_mk, mc.dev + b->off + b->out_mk, mk_bytes,
                                            cudaMemcpyDeviceToHost, st);
                            cudaEventRecord(b->done, st);
                            b->dense_pending = true;
                            b->next_query = t_now + std::chrono::microseconds(10);
                            blocked |= bit;
                            continue;
                        }
                    }
                }
                const auto now = Clock::now();
                std::lock_guard<ServerMutex> lk(S->mu);
                b->complete = true;
                --mc.running;
                for (uint64_t t : b->tickets) {
                    auto it = S->reqs.find(t);
                    if (it == S->reqs.end()) continue;
                    if (it->second->measured) {
                        S->lat_ms.push(std::chrono::duration<double, std::milli>(now - it->second->t_arrival).count());
                        S->sub_ms.push(std::chrono::duration<double, std::milli>(now - it->second->t_submit).count());
                        S->queue_ms.push(
                            std::chrono::duration<double, std::milli>(b->t_launch - it->second->t_arrival).count());
                    }
                    S->completed.push_back(t);
                    S->rows_done += it->second->rows;
                    ++S->n_completed;
                }
                if (q != cudaSuccess && S->error == TABNET_OK) S->error = TABNET_ERR_CUDA;
                did = true;
            }
            std::lock_guard<ServerMutex> lk(S->mu);
            // input rows of finished batches go back at once, in ring order
            while (!mc.in_order.empty() && mc.in_order.front()->complete) {
                Batch* b = mc.in_order.front();
                ring_free_front(mc.in, (size_t)b->in_row0, (size_t)b->rows);
                mc.in_order.pop_front();
                did = true;
            }
            // output regions once every request of the batch is released
            while (!mc.inflight.empty() && mc.inflight.front()->complete &&
                   mc.inflight.front()->released == (int)mc.inflight.front()->tickets.size()) {
                Batch* b = mc.inflight.front();
                ring_free_front(mc.out, b->off, b->bytes);
                mc.inflight.pop_front();
                S->free_events.push_back(b->done);
                delete b;
                did = true;
            }
        }
        if (did) S->cv.notify_all();
        // 2. form and launch batches: consecutive staged requests, as many as fit
        for (int mi = 0; mi < (int)S->models.size(); ++mi) {
            ModelCtx& mc = S->models[mi];
            const tabnet_dims& d = mc.d;
            take.clear();
            stage_now.clear();
            int64_t rows = 0;
            size_t off = 0, bytes = 0;
            {
                std::lock_guard<ServerMutex> lk(S->mu);
                // only batches still on the GPU count; finished results hold ring memory instead
                if (mc.pending.empty() || mc.running >= S->cfg.max_inflight_batches) continue;
                // Under load (batch_busy of the model's batches running) a small
                // batch waits for more requests -- up to batch_wait_us for its
                // oldest -- so that the engine's fixed cost per launch is shared
                // by more rows.
                if (S->cfg.batch_min_rows > 0 && mc.running >= S->cfg.batch_busy &&
                    mc.pending_rows < S->cfg.batch_min_rows &&
                    Clock::now() - mc.pending.front()->t_arrival < std::chrono::microseconds(S->cfg.batch_wait_us))
                    continue;
                int64_t next_row = -1;  // the input row the batch continues at
                while (!mc.pending.empty()) {
                    Request* r = mc.pending.front();
                    if (r->in_row0 < 0) {
                        // not staged at submission (the input ring was full then)
                        if (r->rows > mc.stage_max) {
                            if (!take.empty()) break;
                            // could never fit: reject
                            mc.pending.pop_front();
                            mc.pending_rows -= r->rows;
                            mc.unstaged.pop_front();  // r: the oldest unstaged request
                            S->reqs.erase(r->ticket);
                            ++S->rejected;
                            delete r;
                            continue;
                        }
                        size_t row0 = 0;
                        if (!ring_alloc(mc.in, (size_t)r->rows, &row0)) break;  // admission waits for memory
                        r->in_row0 = (int64_t)row0;
                        mc.unstaged.pop_front();
                        ++S->engine_staged;
                        stage_now.push_back(r);  // copied below, outside the lock
                    } else if (!r->ready.load(std::memory_order_acquire)) {
                        break;  // its submitter is still copying the inputs
                    }
                    if (next_row >= 0 && r->in_row0 != next_row) break;  // the input ring wrapped
                    const int64_t nr = rows + r->rows;
                    if (!take.empty() && nr > S->cfg.max_batch_rows) break;
                    if (align256(kRegionSlack + (size_t)nr * mc.out_row) > mc.out.cap) break;
                    take.push_back(r);
                    rows = nr;
                    next_row = r->in_row0 + r->rows;
                    mc.pending.pop_front();
                    mc.pending_rows -= r->rows;
                }
                if (!take.empty()) {
                    // whole 256-byte units, so that every region starts aligned
                    bytes = align256(kRegionSlack + (size_t)rows * mc.out_row);
                    if (!ring_alloc(mc.out, bytes, &off)) {  // no room now: admission waits for memory
                        for (auto it = take.rbegin(); it != take.rend(); ++it) {
                            mc.pending.push_front(*it);
                            mc.pending_rows += (*it)->rows;
                        }
                        take.clear();
                    }
                }
            }
            // requests staged by the engine (every one of them is in `take`
            // or at the front of the queue): copy, then mark ready
            for (Request* r : stage_now) stage_inputs(mc, r);
            if (!stage_now.empty()) did = true;
            if (take.empty()) continue;
            Batch* b = new Batch();
            b->model = mi;
            b->off = off;
            b->bytes = bytes;
            b->rows = rows;
            b->in_row0 = take.front()->in_row0;
            layout_region(mc, b);
            int64_t r0 = 0;
            for (Request* r : take) {
                r->row0 = r0;
                r->batch = b;
                b->tickets.push_back(r->ticket);
                r0 += r->rows;
            }
            b->stream_idx = mc.next_stream;
            mc.next_stream = (mc.next_stream + 1) % (int)mc.streams.size();
            cudaStream_t st = mc.streams[b->stream_idx];
            if (!S->free_events.empty()) {
                b->done = S->free_events.back();
                S->free_events.pop_back();
            } else {
                cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
            }
            const size_t in0 = (size_t)b->in_row0 * mc.in_row;
            cudaMemcpyAsync(mc.in_dev + in0, mc.in_host + in0, (size_t)rows * mc.in_row, cudaMemcpyHostToDevice, st);
            uint8_t* dv = mc.dev + off;
            int rc = tabnet::forward_interleaved(mc.model, mc.in_dev + in0, rows, (float*)(dv + b->out_lg),
                                                 (float*)(dv + b->out_mk), (float*)(dv + b->out_ag), st);
            if (mc.slots && rc == TABNET_OK &&
                tabnet::mask_compact_launch((const float*)(dv + b->out_mk), rows * d.n_steps, d.d_emb, mc.slots,
                                            dv + b->out_cnt, (uint16_t*)(dv + b->out_col), (float*)(dv + b->out_val),
                                            st) != cudaSuccess)
                rc = TABNET_ERR_CUDA;
            cudaMemcpyAsync(mc.host + off, dv, b->copy_bytes, cudaMemcpyDeviceToHost, st);
            cudaEventRecord(b->done, st);
            b->t_launch = Clock::now();
            b->next_query = b->t_launch + std::chrono::microseconds(std::max<int64_t>(20, (int64_t)(0.75 * mc.est_us)));
            {
                std::lock_guard<ServerMutex> lk(S->mu);
                if (rc != TABNET_OK && S->error == TABNET_OK) S->error = rc;
                mc.inflight.push_back(b);
                mc.in_order.push_back(b);
                ++mc.running;
                ++S->batches;
                S->batch_rows += rows;
            }
            did = true;
        }
        {
            const double pass_ms = std::chrono::duration<double, std::milli>(Clock::now() - t_pass).count();
            std::lock_guard<ServerMutex> lk(S->mu);
            S->engine_max_pass_ms = std::max(S->engine_max_pass_ms, pass_ms);
        }
        if (!did) {
            std::unique_lock<ServerMutex> lk(S->mu);
            S->engine_idle.store(true, std::memory_order_relaxed);
            const auto t_sleep = Clock::now();
            S->cv.wait_for(lk, std::chrono::microseconds(50));
            S->engine_sleep_s += std::chrono::duration<double>(Clock::now() - t_sleep).count();
            S->engine_idle.store(false, std::memory_order_relaxed);
        }
    }
}

}  // namespace

extern "C" {

int tabnet_server_create(tabnet_model* const* models, int n_models, const tabnet_server_config* cfg,
                         tabnet_server** out) {
    if (!models || n_models <= 0 || !out) return tabnet::set_last_error(TABNET_ERR_ARG, "no models or null output");
    *out = nullptr;
    tabnet_server* S = new (std::nothrow) tabnet_server();
    if (!S) return tabnet::set_last_error(TABNET_ERR_OOM, "host allocation failed");
    // buckets for the requests a loaded server holds, so that the ticket map
    // is not rehashed (all of it, under the server lock) as a backlog grows
    S->reqs.reserve(1 << 16);
    S->cfg.device_bytes = cfg && cfg->device_bytes ? cfg->device_bytes : ((size_t)1 << 30);
    S->cfg.max_batch_rows = cfg && cfg->max_batch_rows > 0 ? cfg->max_batch_rows : 65536;
    S->cfg.max_inflight_batches = cfg && cfg->max_inflight_batches > 0 ? cfg->max_inflight_batches : 32;
    S->cfg.streams_per_model = cfg && cfg->streams_per_model > 0 ? std::min(cfg->streams_per_model, 64) : 8;
    S->cfg.batch_min_rows = cfg && cfg->batch_min_rows != 0 ? cfg->batch_min_rows : 2048;
    S->cfg.batch_wait_us = cfg && cfg->batch_wait_us > 0 ? cfg->batch_wait_us : 200;
    S->cfg.batch_busy = cfg && cfg->batch_busy > 0 ? cfg->batch_busy : 2;
    S->cfg.mask_slots = cfg ? cfg->mask_slots : 0;
    S->device = models[0]->device;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(S->device);
    // ring shares proportional to each model's bytes per row
    double wsum = 0;
    std::vector<double> w(n_models);
    for (int i = 0; i < n_models; ++i) {
        if (!models[i] || models[i]->device != S->device) {
            cudaSetDevice(prev);
            delete S;
            return tabnet::set_last_error(TABNET_ERR_ARG, "null model or models on different devices");
        }
        tabnet_dims d;
        tabnet_dims_of(models[i], &d);
        w[i] = 4.0 * (d.n_num + d.n_cat + d.n_classes + (double)d.n_steps * d.d_emb + d.n_feat);
        wsum += w[i];
    }
    S->models.resize(n_models);
    for (int i = 0; i < n_models; ++i) {
        ModelCtx& mc = S->models[i];
        mc.model = models[i];
        // the models' kernels will share SMs: size their launches so that
        // co-located CTAs always fit in tensor memory (keeping each launch
        // shape)
        if (models[i]->precision != TABNET_FP32 && !models[i]->tmem_shared) {
            const tabnet::TcLaunch keep = models[i]->tc_launch_cfg;
            models[i]->tmem_shared = true;
            std::string why;
            if (tabnet::tc_choose_launch(models[i], keep.nwg, keep.n_slots, keep.ctas_per_sm, &why) != TABNET_OK)
                models[i]->tc_launch_cfg = keep;  // the shape no longer fits: keep the old one
        }
        tabnet_dims_of(models[i], &mc.d);
        mc.in_row = 4 * (size_t)(mc.d.n_num + mc.d.n_cat);
        // compact mask transfer: `slots` (column, value) pairs per row-step;
        // by default max(16, de / 5) rounded up to 8 -- well above the
        // supports sparsemax gives (at most 25 of 160 columns, 13 of 35 on
        // the synthetic workloads) -- where that is at most 3/4 of the dense
        // bytes; a row-step with more sends its batch densely
        const int de = mc.d.d_emb;
        int slots = S->cfg.mask_slots;
        if (slots == 0) {
            slots = (std::max(16, (de + 4) / 5) + 7) / 8 * 8;
            if (1 + 6 * slots > 3 * de) slots = 0;
        }
        // (a count saturates at 255, so 255 itself always reads as overflow)
        mc.slots = slots < 0 ? 0 : std::min(slots, 254);
        mc.out_row = 4 * (size_t)(mc.d.n_classes + mc.d.n_steps * de + mc.d.n_feat) +
                     (mc.slots ? (size_t)mc.d.n_steps * (1 + 6 * (size_t)mc.slots) : 0);
        // the model's share, split so that both rings hold about as many rows
        const size_t share = (size_t)(S->cfg.device_bytes * (w[i] / wsum));
        const size_t ring_rows = share / (mc.in_row + mc.out_row);
        mc.out.cap = (ring_rows * mc.out_row + kRegionSlack) / 256 * 256;
        // the input ring holds four times the output ring's rows (inputs are
        // at most 400 bytes a row here, outputs up to 8.7 KB): a backlog
        // waiting for output space must not fill it, or staging falls back
        // onto the engine thread, whose time per request bounds the rate
        mc.in.cap = 4 * ring_rows;
        const size_t in_bytes = align256(mc.in.cap * mc.in_row);
        mc.stage_max = (int64_t)std::min(ring_rows, (mc.out.cap - kRegionSlack - 256) / mc.out_row);
        cudaError_t e1 = cudaMalloc(&mc.dev, mc.out.cap);
        cudaError_t e2 = cudaHostAlloc(&mc.host, mc.out.cap, cudaHostAllocDefault);
        cudaError_t e3 = cudaMalloc(&mc.in_dev, in_bytes);
        cudaError_t e4 = cudaHostAlloc(&mc.in_host, in_bytes, cudaHostAllocDefault);
        if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess || e4 != cudaSuccess || ring_rows == 0) {
            tabnet_server_destroy(S);
            cudaSetDevice(prev);
            return tabnet::set_last_error(TABNET_ERR_OOM, "server ring allocation failed");
        }
        mc.streams.resize(S->cfg.streams_per_model);
        for (auto& st : mc.streams) cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    }
    cudaSetDevice(prev);
    S->engine = std::thread(engine_loop, S);
    *out = S;
    return TABNET_OK;
}

namespace {
int submit_at(tabnet_server* S, int model, const float* x_num, const int32_t* x_cat, int64_t rows,
              Clock::time_point t_arrival, bool measured, uint64_t* ticket) {
    if (!S || !ticket || model < 0 || model >= (int)S->models.size() || rows <= 0)
        return tabnet::set_last_error(TABNET_ERR_ARG, "bad server, model index, rows or ticket pointer");
    const tabnet_dims& d = S->models[model].d;
    if ((d.n_num && !x_num) || (d.n_cat && !x_cat)) return tabnet::set_last_error(TABNET_ERR_ARG, "null input");
    Request* r = new (std::nothrow) Request();
    if (!r) return tabnet::set_last_error(TABNET_ERR_OOM, "host allocation failed");
    r->model = model;
    r->x_num = x_num;
    r->x_cat = x_cat;
    r->rows = rows;
    r->t_arrival = t_arrival;
    r->measured = measured;
    r->t_submit = Clock::now();
    r->ticket = S->next_ticket.fetch_add(1);
    ModelCtx& mc = S->models[model];
    // requests this call copies in: older ones still waiting for room in the
    // input ring first (in order), then this one
    Request* to_stage[8];
    int n_stage = 0;
    {
        std::lock_guard<ServerMutex> lk(S->mu);
        S->reqs.emplace(r->ticket, r);
        mc.unstaged.push_back(r);
        // The inputs go to the input ring in submission order.  A request
        // that finds it full waits, unstaged; later submissions take over
        // the oldest waiting ones as room frees (a few per call), so that a
        // backlog's copies do not fall to the engine thread, whose time per
        // request bounds the rate (the engine copies one only when it comes
        // to the front of a batch with nobody having taken it).
        while (!mc.unstaged.empty() && n_stage < 8) {
            Request* u = mc.unstaged.front();
            size_t row0 = 0;
            if (u->rows > mc.stage_max || !ring_alloc(mc.in, (size_t)u->rows, &row0)) break;
            u->in_row0 = (int64_t)row0;
            mc.unstaged.pop_front();
            to_stage[n_stage++] = u;
        }
        mc.pending.push_back(r);
        mc.pending_rows += rows;
        ++S->submitted;
    }
    // the copies run on the submitting thread, outside the lock; the engine
    // takes a request into a batch once it is marked ready
    for (int i = 0; i < n_stage; ++i) stage_inputs(mc, to_stage[i]);
    // a wake-up only when the engine sleeps, and by one caller per nap (a
    // missed one costs at most its 50 us nap): a notify takes the condition
    // variable's own lock and makes a system call, and submit runs per request
    if (S->engine_idle.exchange(false, std::memory_order_relaxed)) S->cv.notify_all();
    *ticket = r->ticket;
    return TABNET_OK;
}
}  // namespace

int tabnet_server_submit(tabnet_server* S, int model, const float* x_num, const int32_t* x_cat, int64_t rows,
                         uint64_t* ticket) {
    return submit_at(S, model, x_num, x_cat, rows, Clock::now(), true, ticket);
}

int tabnet_server_poll(tabnet_server* S, uint64_t* tickets, int max_tickets, int* n_done) {
    if (!S || !n_done || (max_tickets > 0 && !tickets)) return tabnet::set_last_error(TABNET_ERR_ARG, "null pointer");
    std::lock_guard<ServerMutex> lk(S->mu);
    int n = 0;
    while (n < max_tickets && !S->completed.empty()) {
        tickets[n++] = S->completed.front();
        S->completed.pop_front();
    }
    *n_done = n;
    return S->error;
}

int tabnet_server_result(tabnet_server* S, uint64_t ticket, const float** logits, const float** step_masks,
                         const float** agg_mask, int64_t* rows) {
    if (!S) return tabnet::set_last_error(TABNET_ERR_ARG, "null server");
    Request* r = nullptr;
    const uint8_t* h = nullptr;
    Batch* b = nullptr;
    int slots = 0;
    {
        std::lock_guard<ServerMutex> lk(S->mu);
        auto it = S->reqs.find(ticket);
        if (it == S->reqs.end() || !it->second->batch || !it->second->batch->complete)
            return tabnet::set_last_error(TABNET_ERR_ARG, "ticket unknown, released or not complete");
        r = it->second;
        b = r->batch;
        h = S->models[r->model].host + b->off;
        slots = S->models[r->model].slots;
    }
    // the request's result memory stays put until the ticket is released
    const tabnet_dims& d = S->models[r->model].d;
    const int64_t S_de = (int64_t)d.n_steps * d.d_emb;
    if (logits) *logits = (const float*)(h + b->out_lg) + r->row0 * d.n_classes;
    if (agg_mask) *agg_mask = (const float*)(h + b->out_ag) + r->row0 * d.n_feat;
    if (step_masks) {
        if (b->dense) {
            *step_masks = (const float*)(h + b->out_mk) + r->row0 * S_de;
        } else {
            if (r->dense_masks.empty()) {  // expand the compact form once
                r->dense_masks.assign((size_t)(r->rows * S_de), 0.f);
                const int64_t rs0 = r->row0 * d.n_steps, nrs = r->rows * d.n_steps;
                const uint8_t* cnt = h + b->out_cnt + rs0;
                const uint16_t* col = (const uint16_t*)(h + b->out_col) + rs0 * slots;
                const float* val = (const float*)(h + b->out_val) + rs0 * slots;
                for (int64_t i = 0; i < nrs; ++i) {
                    float* dst = r->dense_masks.data() + i * d.d_emb;
                    for (int j = 0; j < cnt[i]; ++j) dst[col[i * slots + j]] = val[i * slots + j];
                }
            }
            *step_masks = r->dense_masks.data();
        }
    }
    if (rows) *rows = r->rows;
    return TABNET_OK;
}

int tabnet_server_result_compact(tabnet_server* S, uint64_t ticket, const uint8_t** counts, const uint16_t** cols,
                                 const float** vals, int* slots, int64_t* rows) {
    if (!S || !counts || !cols || !vals || !slots) return tabnet::set_last_error(TABNET_ERR_ARG, "null pointer");
    std::lock_guard<ServerMutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end() || !it->second->batch || !it->second->batch->complete)
        return tabnet::set_last_error(TABNET_ERR_ARG, "ticket unknown, released or not complete");
    const Request* r = it->second;
    const Batch* b = r->batch;
    const ModelCtx& mc = S->models[r->model];
    if (rows) *rows = r->rows;
    if (b->dense) {  // sent densely: read the masks through tabnet_server_result
        *counts = nullptr;
        *cols = nullptr;
        *vals = nullptr;
        *slots = 0;
        return TABNET_OK;
    }
    const uint8_t* h = mc.host + b->off;
    const int64_t rs0 = r->row0 * mc.d.n_steps;
    *counts = h + b->out_cnt + rs0;
    *cols = (const uint16_t*)(h + b->out_col) + rs0 * mc.slots;
    *vals = (const float*)(h + b->out_val) + rs0 * mc.slots;
    *slots = mc.slots;
    return TABNET_OK;
}

namespace {
// Release one ticket (the server lock held).
int release_locked(tabnet_server* S, uint64_t ticket, Request** freed = nullptr) {
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end() || !it->second->batch || !it->second->batch->complete)
        return tabnet::set_last_error(TABNET_ERR_ARG, "ticket unknown, released or not complete");
    it->second->batch->released++;
    if (freed) *freed = it->second;  // the caller deletes it outside the lock
    else delete it->second;
    S->reqs.erase(it);
    return TABNET_OK;
}

// Release k tickets, at most 32 under one acquisition of the lock (the load
// driver's path: one lock per ticket would contend with the engine at high
// rates, and a whole poll's worth -- up to a thousand after a burst -- would
// hold the clients' submissions for most of a millisecond); the requests'
// memory is freed outside the lock.
void release_group(tabnet_server* S, const uint64_t* tickets, int k) {
    if (k <= 0) return;
    constexpr int kGroup = 32;
    Request* freed[kGroup];
    for (int j0 = 0; j0 < k; j0 += kGroup) {
        const int n = std::min(kGroup, k - j0);
        int nf = 0;
        {
            std::lock_guard<ServerMutex> lk(S->mu);
            for (int j = 0; j < n; ++j) {
                Request* r = nullptr;
                if (release_locked(S, tickets[j0 + j], &r) == TABNET_OK) freed[nf++] = r;
            }
        }
        for (int j = 0; j < nf; ++j) delete freed[j];
    }
    if (S->engine_idle.exchange(false, std::memory_order_relaxed)) S->cv.notify_all();
}
}  // namespace

int tabnet_server_release(tabnet_server* S, uint64_t ticket) {
    if (!S) return tabnet::set_last_error(TABNET_ERR_ARG, "null server");
    int rc;
    {
        std::lock_guard<ServerMutex> lk(S->mu);
        rc = release_locked(S, ticket);
    }
    if (rc == TABNET_OK && S->engine_idle.exchange(false, std::memory_order_relaxed)) S->cv.notify_all();
    return rc;
}

int tabnet_server_wait(tabnet_server* S, uint64_t ticket, double timeout_s) {
    if (!S) return tabnet::set_last_error(TABNET_ERR_ARG, "null server");
    std::unique_lock<ServerMutex> lk(S->mu);
    const auto deadline = Clock::now() + std::chrono::duration<double>(timeout_s);
    while (true) {
        auto it = S->reqs.find(ticket);
        if (it == S->reqs.end()) return tabnet::set_last_error(TABNET_ERR_ARG, "ticket unknown or released");
        if (it->second->batch && it->second->batch->complete) return TABNET_OK;
        if (S->error != TABNET_OK) return S->error;
        if (S->cv.wait_until(lk, deadline) == std::cv_status::timeout && Clock::now() >= deadline)
            return tabnet::set_last_error(TABNET_ERR_TIMEOUT, "request not complete before the timeout");
    }
}

int tabnet_server_get_stats(tabnet_server* S, tabnet_server_stats* st) {
    if (!S || !st) return tabnet::set_last_error(TABNET_ERR_ARG, "null pointer");
    std::vector<double> lat, qms, sms;
    {
        std::lock_guard<ServerMutex> lk(S->mu);
        lat = S->lat_ms.v;
        qms = S->queue_ms.v;
        sms = S->sub_ms.v;
        st->submitted = S->submitted;
        st->completed = S->n_completed;
        st->rejected = S->rejected;
        st->rows_completed = S->rows_done;
        st->batches = S->batches;
        st->mean_batch_rows = S->batches ? (double)S->batch_rows / S->batches : 0.0;
        int64_t q = 0, inflight = 0;
        size_t used = 0;
        for (auto& mc : S->models) {
            q += (int64_t)mc.pending.size();
            inflight += (int64_t)mc.running;
            used += mc.out.used + mc.in.used * mc.in_row;
        }
        st->queue_depth = q;
        st->inflight_batches = inflight;
        st->device_bytes_in_use = used;
        st->engine_staged = S->engine_staged;
        const double secs = std::chrono::duration<double>(Clock::now() - S->t_reset).count();
        st->rows_per_s = secs > 0 ? S->rows_done / secs : 0.0;
        st->engine_busy = secs > 0 ? std::max(0.0, 1.0 - S->engine_sleep_s / secs) : 0.0;
        st->engine_max_pass_ms = S->engine_max_pass_ms;
        st->replay_max_late_ms = S->replay_max_late_ns.load() * 1e-6;
    }
    std::sort(lat.begin(), lat.end());
    auto pct = [&](double q) { return lat.empty() ? 0.0 : lat[std::min(lat.size() - 1, (size_t)(q * (lat.size() - 1) + 0.5))]; };
    st->p50_ms = pct(0.50);
    st->p95_ms = pct(0.95);
    st->p99_ms = pct(0.99);
    st->max_ms = lat.empty() ? 0.0 : lat.back();
    double sum = 0;
    for (double v : lat) sum += v;
    st->mean_ms = lat.empty() ? 0.0 : sum / lat.size();
    std::sort(qms.begin(), qms.end());
    auto qpct = [&](double q) { return qms.empty() ? 0.0 : qms[std::min(qms.size() - 1, (size_t)(q * (qms.size() - 1) + 0.5))]; };
    st->p50_queue_ms = qpct(0.50);
    st->p99_queue_ms = qpct(0.99);
    std::sort(sms.begin(), sms.end());
    auto spct = [&](double q) { return sms.empty() ? 0.0 : sms[std::min(sms.size() - 1, (size_t)(q * (sms.size() - 1) + 0.5))]; };
    st->p50_submit_ms = spct(0.50);
    st->p99_submit_ms = spct(0.99);
    return S->error;
}

int tabnet_server_reset_stats(tabnet_server* S) {
    if (!S) return tabnet::set_last_error(TABNET_ERR_ARG, "null server");
    std::lock_guard<ServerMutex> lk(S->mu);
    S->lat_ms.clear();
    S->queue_ms.clear();
    S->sub_ms.clear();
    S->engine_sleep_s = 0;
    S->engine_max_pass_ms = 0;
    S->replay_max_late_ns = 0;
    S->submitted = S->n_completed = S->rejected = S->rows_done = S->batches = S->batch_rows = S->engine_staged = 0;
    S->t_reset = Clock::now();
    return TABNET_OK;
}

int tabnet_server_replay(tabnet_server* S, const tabnet_server_request* reqs, int n, int release, int threads,
                         int warmup) {
    if (!S || (n > 0 && !reqs) || n < 0) return tabnet::set_last_error(TABNET_ERR_ARG, "bad arguments");
    if (threads <= 0) threads = 1;
    threads = std::min(threads, 64);
    const auto t0 = Clock::now();
    // Release finished requests every 20 us (one thread at a time) -- while
    // waiting for the next arrival and also between submissions when behind
    // schedule: a client that only releases when it has time to spare stops
    // freeing output memory exactly when a burst has put it behind, and the
    // batches that would clear the burst then wait for that memory.
    // (Polling on every spin would contend for the engine's lock.)
    std::atomic<int64_t> last_poll{0};  // ns since t0
    std::atomic<int> first_error{TABNET_OK};
    auto poll_release = [&](std::vector<uint64_t>& done, Clock::time_point now) {
        const int64_t t = std::chrono::duration_cast<std::chrono::nanoseconds>(now - t0).count();
        int64_t last = last_poll.load(std::memory_order_relaxed);
        if (t - last < 20000 || !last_poll.compare_exchange_strong(last, t)) return;
        int k = 0;
        tabnet_server_poll(S, done.data(), (int)done.size(), &k);
        release_group(S, done.data(), k);
    };
    // Submitting thread j takes requests j, j + T, j + 2T, ... in order; each
    // is submitted at its arrival offset and its latency counts from there.
    auto drive = [&](int j) {
        std::vector<uint64_t> done(1024);
        for (int i = j; i < n && first_error.load(std::memory_order_relaxed) == TABNET_OK; i += threads) {
            const auto due =
                t0 + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(reqs[i].arrival_s));
            for (auto now = Clock::now();; now = Clock::now()) {
                if (release) poll_release(done, now);
                if (now >= due) break;
            }
            const int64_t late = std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now() - due).count();
            for (int64_t m = S->replay_max_late_ns.load(std::memory_order_relaxed);
                 late > m && !S->replay_max_late_ns.compare_exchange_weak(m, late);) {
            }
            uint64_t t;
            const int rc = submit_at(S, reqs[i].model, reqs[i].x_num, reqs[i].x_cat, reqs[i].rows, due, i >= warmup, &t);
            if (rc != TABNET_OK) {
                int ok = TABNET_OK;
                first_error.compare_exchange_strong(ok, rc);
            }
        }
    };
    if (threads == 1) {
        drive(0);
    } else {
        std::vector<std::thread> pool;
        for (int j = 0; j < threads; ++j) pool.emplace_back(drive, j);
        for (auto& th : pool) th.join();
    }
    if (first_error.load() != TABNET_OK) return first_error.load();
    if (release) {  // drain
        std::vector<uint64_t> done(1024);
        while (true) {
            int k = 0;
            const int rc = tabnet_server_poll(S, done.data(), (int)done.size(), &k);
            release_group(S, done.data(), k);
            if (rc != TABNET_OK) return rc;
            bool all_done;
            {
                std::lock_guard<ServerMutex> lk(S->mu);
                all_done = S->n_completed + S->rejected >= S->submitted;
            }
            if (all_done && k == 0) break;
            std::this_thread::sleep_for(std::chrono::microseconds(20));
        }
    }
    return TABNET_OK;
}

void tabnet_server_destroy(tabnet_server* S) {
    if (!S) return;
    S->stop = true;
    S->cv.notify_all();
    if (S->engine.joinable()) S->engine.join();
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(S->device);
    for (auto& mc : S->models) {
        for (auto st : mc.streams) {
            cudaStreamSynchronize(st);
            cudaStreamDestroy(st);
        }
        for (Batch* b : mc.inflight) {
            if (b->done) cudaEventDestroy(b->done);
            delete b;
        }
        for (Request* r : mc.pending) delete r;
        if (mc.dev) cudaFree(mc.dev);
        if (mc.host) cudaFreeHost(mc.host);
        if (mc.in_dev) cudaFree(mc.in_dev);
        if (mc.in_host) cudaFreeHost(mc.in_host);
    }
    for (cudaEvent_t e : S->free_events) cudaEventDestroy(e);
    for (auto& kv : S->reqs) {
        bool pending = false;
        for (auto& mc : S->models)
            for (Request* r : mc.pending) pending |= (r == kv.second);
        if (!pending) delete kv.second;
    }
    cudaSetDevice(prev);
    delete S;
}

}  // extern "C"
