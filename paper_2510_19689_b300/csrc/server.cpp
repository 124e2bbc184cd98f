// Continuous-batching request server over resident models.
//
// The paper serves TabNet from GPU functions that keep the model in GPU
// memory after a cold start and take a batch of records per invocation
// (Sec. III-B), reporting p50/p95/p99 latency beside throughput (Sec. IV-C).
// This engine does that for many concurrent requests on one GPU:
//
//   * every model has a device ring buffer and a pinned host mirror of the
//     same size (its share of the memory budget); a batch occupies one
//     contiguous region of the ring: all inputs, then all outputs;
//   * an engine thread takes, per model, every request that has arrived
//     (up to max_batch_rows) and packs it into the next region the ring can
//     hold -- admission is by device memory: a request waits while its
//     model's ring is full and is rejected only if it could never fit;
//   * the batch is copied in with one host-to-device copy, run as ONE
//     forward launch over its packed rows, and copied out with one
//     device-to-host copy, on one of the model's streams; the engine never
//     waits for a batch before forming the next one, so requests that arrive
//     while others are on the GPU are admitted as soon as ring space frees
//     and their batches overlap on the device (streams of other batches and
//     of the other models);
//   * completion is observed by polling the batch's event; the request's
//     results stay in the pinned mirror until the caller releases it, and a
//     region is reused once its batch and every older batch of the ring are
//     released.
// Latency of a request = completion observed on the host - submission time.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
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
}

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket;
    int model;
    const float* x_num;
    const int32_t* x_cat;
    int64_t rows;
    Clock::time_point t_submit;
    // filled when batched
    int64_t row0 = 0;       // first row inside its batch
    struct Batch* batch = nullptr;
};

struct Batch {
    int model;
    int stream_idx;
    size_t off = 0, bytes = 0;  // ring region
    int64_t rows = 0;
    size_t in_num = 0, in_cat = 0, out_lg = 0, out_mk = 0, out_ag = 0;  // offsets inside the region
    std::vector<uint64_t> tickets;
    cudaEvent_t done = nullptr;
    Clock::time_point t_launch;
    bool complete = false;
    int released = 0;
};

struct ModelCtx {
    tabnet_model* model;
    tabnet_dims d;
    size_t in_row, out_row;        // bytes per row (inputs, outputs)
    uint8_t* dev = nullptr;        // device ring
    uint8_t* host = nullptr;       // pinned mirror
    size_t cap = 0, head = 0, tail = 0, used = 0;  // ring: allocate at head, free at tail
    std::deque<Batch*> inflight;   // in ring order
    std::deque<Request*> pending;
    std::vector<cudaStream_t> streams;
    int next_stream = 0;
    int running = 0;               // batches launched and not yet complete
    int64_t pending_rows = 0;      // rows of the pending requests
};

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

struct tabnet_server {
    std::vector<ModelCtx> models;
    tabnet_server_config cfg{};
    std::mutex mu;                       // guards pending queues, requests, stats
    std::condition_variable cv;
    std::unordered_map<uint64_t, Request*> reqs;
    std::atomic<uint64_t> next_ticket{1};
    std::deque<uint64_t> completed;      // tickets completed, not yet returned by poll
    std::vector<double> lat_ms;          // completed requests' latencies since the last reset
    uint64_t submitted = 0, n_completed = 0, rejected = 0, rows_done = 0, batches = 0, batch_rows = 0;
    Clock::time_point t_reset = Clock::now();
    std::thread engine;
    std::atomic<bool> stop{false};
    int device = 0;
    int error = TABNET_OK;
    std::vector<cudaEvent_t> free_events;  // completion events of freed batches, reused (engine thread only)
};

namespace {

// Reserve `bytes` contiguous bytes at the ring head (wrapping to 0 when the
// tail leaves room there).  Returns false when the ring cannot hold them now.
bool ring_alloc(ModelCtx& mc, size_t bytes, size_t* off) {
    if (bytes > mc.cap) return false;
    if (mc.used == 0) mc.head = mc.tail = 0;
    if (mc.head >= mc.tail && mc.used < mc.cap) {
        if (mc.cap - mc.head >= bytes) { *off = mc.head; mc.head += bytes; mc.used += bytes; return true; }
        if (mc.tail >= bytes) {  // wrap: waste the end of the ring
            mc.used += (mc.cap - mc.head) + bytes;
            *off = 0;
            mc.head = bytes;
            return true;
        }
        return false;
    }
    if (mc.head < mc.tail && mc.tail - mc.head >= bytes) { *off = mc.head; mc.head += bytes; mc.used += bytes; return true; }
    return false;
}

// Free the oldest batch's region (regions are released in ring order).
void ring_free_front(ModelCtx& mc) {
    Batch* b = mc.inflight.front();
    const size_t end = b->off + b->bytes;
    if (b->off < mc.tail) {  // this batch wrapped: the waste before it goes too
        mc.used -= (mc.cap - mc.tail);
        mc.tail = 0;
    }
    mc.used -= b->bytes;
    mc.tail = end;
    if (mc.used == 0) mc.head = mc.tail = 0;
    mc.inflight.pop_front();
}

void engine_loop(tabnet_server* S) {
    cudaSetDevice(S->device);
    std::vector<Request*> take;
    while (!S->stop.load(std::memory_order_relaxed)) {
        bool did = false;
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
                // no batch completes within 20 us of its launch (copies and
                // one kernel): do not spend a query on it
                if (t_now - b->t_launch < std::chrono::microseconds(20)) {
                    blocked |= bit;
                    continue;
                }
                const cudaError_t q = cudaEventQuery(b->done);
                if (q == cudaErrorNotReady) {
                    blocked |= bit;
                    continue;
                }
                const auto now = Clock::now();
                std::lock_guard<std::mutex> lk(S->mu);
                b->complete = true;
                --mc.running;
                for (uint64_t t : b->tickets) {
                    auto it = S->reqs.find(t);
                    if (it == S->reqs.end()) continue;
                    S->lat_ms.push_back(std::chrono::duration<double, std::milli>(now - it->second->t_submit).count());
                    S->completed.push_back(t);
                    S->rows_done += it->second->rows;
                    ++S->n_completed;
                }
                if (q != cudaSuccess && S->error == TABNET_OK) S->error = TABNET_ERR_CUDA;
                did = true;
            }
            // free released batches at the front of the ring
            std::lock_guard<std::mutex> lk(S->mu);
            while (!mc.inflight.empty() && mc.inflight.front()->complete &&
                   mc.inflight.front()->released == (int)mc.inflight.front()->tickets.size()) {
                Batch* b = mc.inflight.front();
                ring_free_front(mc);
                S->free_events.push_back(b->done);
                delete b;
                did = true;
            }
        }
        if (did) S->cv.notify_all();
        // 2. form and launch batches: everything pending that fits
        for (int mi = 0; mi < (int)S->models.size(); ++mi) {
            ModelCtx& mc = S->models[mi];
            take.clear();
            int64_t rows = 0;
            size_t off = 0, bytes = 0;
            {
                std::lock_guard<std::mutex> lk(S->mu);
                // only batches still on the GPU count; finished results hold ring memory instead
                if (mc.pending.empty() || mc.running >= S->cfg.max_inflight_batches) continue;
                // Under load (half the model's streams busy) a small batch waits
                // for more requests -- up to batch_wait_us for its oldest -- so
                // that the engine's fixed cost per launch is shared by more rows.
                if (S->cfg.batch_min_rows > 0 && mc.running >= std::max(2, S->cfg.streams_per_model / 2) &&
                    mc.pending_rows < S->cfg.batch_min_rows &&
                    Clock::now() - mc.pending.front()->t_submit < std::chrono::microseconds(S->cfg.batch_wait_us))
                    continue;
                while (!mc.pending.empty()) {
                    Request* r = mc.pending.front();
                    const int64_t nr = rows + r->rows;
                    if (!take.empty() && nr > S->cfg.max_batch_rows) break;
                    const size_t need = 5 * 256 + (size_t)nr * (mc.in_row + mc.out_row);
                    if (need > mc.cap) {
                        if (take.empty()) {  // could never fit: reject
                            mc.pending.pop_front();
                            mc.pending_rows -= r->rows;
                            S->reqs.erase(r->ticket);
                            ++S->rejected;
                            delete r;
                            continue;
                        }
                        break;
                    }
                    take.push_back(r);
                    rows = nr;
                    mc.pending.pop_front();
                    mc.pending_rows -= r->rows;
                }
                if (take.empty()) continue;
                bytes = 5 * 256 + (size_t)rows * (mc.in_row + mc.out_row);
                if (!ring_alloc(mc, bytes, &off)) {  // no room now: admission waits for memory
                    for (auto it = take.rbegin(); it != take.rend(); ++it) {
                        mc.pending.push_front(*it);
                        mc.pending_rows += (*it)->rows;
                    }
                    continue;
                }
            }
            const tabnet_dims& d = mc.d;
            Batch* b = new Batch();
            b->model = mi;
            b->off = off;
            b->bytes = bytes;
            b->rows = rows;
            b->in_num = 0;
            b->in_cat = align256((size_t)rows * d.n_num * 4);
            b->out_lg = b->in_cat + align256((size_t)rows * d.n_cat * 4);
            b->out_mk = b->out_lg + align256((size_t)rows * d.n_classes * 4);
            b->out_ag = b->out_mk + align256((size_t)rows * d.n_steps * d.d_emb * 4);
            const size_t in_bytes = b->out_lg;
            uint8_t* h = mc.host + off;
            int64_t r0 = 0;
            for (Request* r : take) {
                if (d.n_num) std::memcpy(h + b->in_num + (size_t)r0 * d.n_num * 4, r->x_num, (size_t)r->rows * d.n_num * 4);
                if (d.n_cat) std::memcpy(h + b->in_cat + (size_t)r0 * d.n_cat * 4, r->x_cat, (size_t)r->rows * d.n_cat * 4);
                r->row0 = r0;
                r->batch = b;
                b->tickets.push_back(r->ticket);
                r0 += r->rows;
            }
            b->stream_idx = mc.next_stream;
            mc.next_stream = (mc.next_stream + 1) % (int)mc.streams.size();
            cudaStream_t st = mc.streams[b->stream_idx];
            uint8_t* dv = mc.dev + off;
            if (!S->free_events.empty()) {
                b->done = S->free_events.back();
                S->free_events.pop_back();
            } else {
                cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
            }
            cudaMemcpyAsync(dv, h, in_bytes, cudaMemcpyHostToDevice, st);
            int rc = tabnet_forward(mc.model, d.n_num ? (const float*)(dv + b->in_num) : nullptr,
                                    d.n_cat ? (const int32_t*)(dv + b->in_cat) : nullptr, rows,
                                    (float*)(dv + b->out_lg), (float*)(dv + b->out_mk), (float*)(dv + b->out_ag), st);
            cudaMemcpyAsync(h + b->out_lg, dv + b->out_lg, b->bytes - b->out_lg - 0, cudaMemcpyDeviceToHost, st);
            cudaEventRecord(b->done, st);
            b->t_launch = Clock::now();
            {
                std::lock_guard<std::mutex> lk(S->mu);
                if (rc != TABNET_OK && S->error == TABNET_OK) S->error = rc;
                mc.inflight.push_back(b);
                ++mc.running;
                ++S->batches;
                S->batch_rows += rows;
            }
            did = true;
        }
        if (!did) {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv.wait_for(lk, std::chrono::microseconds(50));
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
    S->cfg.device_bytes = cfg && cfg->device_bytes ? cfg->device_bytes : ((size_t)1 << 30);
    S->cfg.max_batch_rows = cfg && cfg->max_batch_rows > 0 ? cfg->max_batch_rows : 65536;
    S->cfg.max_inflight_batches = cfg && cfg->max_inflight_batches > 0 ? cfg->max_inflight_batches : 32;
    S->cfg.streams_per_model = cfg && cfg->streams_per_model > 0 ? std::min(cfg->streams_per_model, 64) : 8;
    S->cfg.batch_min_rows = cfg && cfg->batch_min_rows != 0 ? cfg->batch_min_rows : 512;
    S->cfg.batch_wait_us = cfg && cfg->batch_wait_us > 0 ? cfg->batch_wait_us : 200;
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
        mc.out_row = 4 * (size_t)(mc.d.n_classes + mc.d.n_steps * mc.d.d_emb + mc.d.n_feat);
        mc.cap = (size_t)(S->cfg.device_bytes * (w[i] / wsum)) / 256 * 256;
        cudaError_t e1 = cudaMalloc(&mc.dev, mc.cap);
        cudaError_t e2 = cudaHostAlloc(&mc.host, mc.cap, cudaHostAllocDefault);
        if (e1 != cudaSuccess || e2 != cudaSuccess) {
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

int tabnet_server_submit(tabnet_server* S, int model, const float* x_num, const int32_t* x_cat, int64_t rows,
                         uint64_t* ticket) {
    if (!S || !ticket || model < 0 || model >= (int)S->models.size() || rows <= 0)
        return tabnet::set_last_error(TABNET_ERR_ARG, "bad server, model index, rows or ticket pointer");
    const tabnet_dims& d = S->models[model].d;
    if ((d.n_num && !x_num) || (d.n_cat && !x_cat)) return tabnet::set_last_error(TABNET_ERR_ARG, "null input");
    Request* r = new (std::nothrow) Request{0, model, x_num, x_cat, rows, Clock::now()};
    if (!r) return tabnet::set_last_error(TABNET_ERR_OOM, "host allocation failed");
    r->ticket = S->next_ticket.fetch_add(1);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->reqs.emplace(r->ticket, r);
        S->models[model].pending.push_back(r);
        S->models[model].pending_rows += rows;
        ++S->submitted;
    }
    S->cv.notify_all();
    *ticket = r->ticket;
    return TABNET_OK;
}

int tabnet_server_poll(tabnet_server* S, uint64_t* tickets, int max_tickets, int* n_done) {
    if (!S || !n_done || (max_tickets > 0 && !tickets)) return tabnet::set_last_error(TABNET_ERR_ARG, "null pointer");
    std::lock_guard<std::mutex> lk(S->mu);
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
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end() || !it->second->batch || !it->second->batch->complete)
        return tabnet::set_last_error(TABNET_ERR_ARG, "ticket unknown, released or not complete");
    Request* r = it->second;
    Batch* b = r->batch;
    const ModelCtx& mc = S->models[r->model];
    const tabnet_dims& d = mc.d;
    const uint8_t* h = mc.host + b->off;
    if (logits) *logits = (const float*)(h + b->out_lg) + r->row0 * d.n_classes;
    if (step_masks) *step_masks = (const float*)(h + b->out_mk) + r->row0 * (int64_t)d.n_steps * d.d_emb;
    if (agg_mask) *agg_mask = (const float*)(h + b->out_ag) + r->row0 * d.n_feat;
    if (rows) *rows = r->rows;
    return TABNET_OK;
}

int tabnet_server_release(tabnet_server* S, uint64_t ticket) {
    if (!S) return tabnet::set_last_error(TABNET_ERR_ARG, "null server");
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->reqs.find(ticket);
        if (it == S->reqs.end() || !it->second->batch || !it->second->batch->complete)
            return tabnet::set_last_error(TABNET_ERR_ARG, "ticket unknown, released or not complete");
        it->second->batch->released++;
        delete it->second;
        S->reqs.erase(it);
    }
    S->cv.notify_all();
    return TABNET_OK;
}

int tabnet_server_wait(tabnet_server* S, uint64_t ticket, double timeout_s) {
    if (!S) return tabnet::set_last_error(TABNET_ERR_ARG, "null server");
    std::unique_lock<std::mutex> lk(S->mu);
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
    std::vector<double> lat;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        lat = S->lat_ms;
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
            used += mc.used;
        }
        st->queue_depth = q;
        st->inflight_batches = inflight;
        st->device_bytes_in_use = used;
        const double secs = std::chrono::duration<double>(Clock::now() - S->t_reset).count();
        st->rows_per_s = secs > 0 ? S->rows_done / secs : 0.0;
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
    return S->error;
}

int tabnet_server_reset_stats(tabnet_server* S) {
    if (!S) return tabnet::set_last_error(TABNET_ERR_ARG, "null server");
    std::lock_guard<std::mutex> lk(S->mu);
    S->lat_ms.clear();
    S->submitted = S->n_completed = S->rejected = S->rows_done = S->batches = S->batch_rows = 0;
    S->t_reset = Clock::now();
    return TABNET_OK;
}

int tabnet_server_replay(tabnet_server* S, const tabnet_server_request* reqs, int n, int release) {
    if (!S || (n > 0 && !reqs) || n < 0) return tabnet::set_last_error(TABNET_ERR_ARG, "bad arguments");
    const auto t0 = Clock::now();
    std::vector<uint64_t> done(1024);
    // Release finished requests while waiting for the next arrival, at most
    // every 20 us: polling on every spin would contend for the engine's lock.
    auto last_poll = t0;
    for (int i = 0; i < n; ++i) {
        const auto due = t0 + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(reqs[i].arrival_s));
        for (auto now = Clock::now(); now < due; now = Clock::now()) {
            if (release && now - last_poll >= std::chrono::microseconds(20)) {
                last_poll = now;
                int k = 0;
                tabnet_server_poll(S, done.data(), (int)done.size(), &k);
                for (int j = 0; j < k; ++j) tabnet_server_release(S, done[j]);
            }
        }
        uint64_t t;
        int rc = tabnet_server_submit(S, reqs[i].model, reqs[i].x_num, reqs[i].x_cat, reqs[i].rows, &t);
        if (rc != TABNET_OK) return rc;
    }
    if (release) {  // drain
        while (true) {
            int k = 0;
            const int rc = tabnet_server_poll(S, done.data(), (int)done.size(), &k);
            for (int j = 0; j < k; ++j) tabnet_server_release(S, done[j]);
            if (rc != TABNET_OK) return rc;
            tabnet_server_stats st;
            tabnet_server_get_stats(S, &st);
            if (st.completed + st.rejected >= st.submitted && k == 0) break;
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
