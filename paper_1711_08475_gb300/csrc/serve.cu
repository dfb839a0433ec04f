// Serving loop: continuous batching of query requests over a resident
// dictionary.
//
// Requests (a pattern batch with its own k and metric) are copied into host
// memory by fp_server_submit and queued.  One scheduler thread owns the GPU
// side.  It keeps up to `lanes` launches in flight, each on its own CUDA
// stream; whenever a lane is idle and the queue is not empty, it takes the
// oldest queued requests that fit one launch (patterns, bytes, requests,
// distinct (k, metric) groups) and whose device footprint fits what is left
// of the memory budget, packs them into the lane's pinned staging buffers and
// enqueues the batched pipeline (pipe.cuh) on the lane's stream, with the
// run's buffers in one stream-ordered allocation of exactly its size.
// Requests that arrive while other launches are on the GPU are admitted as
// lanes and memory free up, and their launches overlap on the device with
// the ones already running.
//
// A host function queued behind each launch wakes the scheduler (no polling).
// A finished launch goes through two stages on its stream: counters back ->
// (match buffer too small: re-run with the exact size) -> CSR copy to pinned
// memory -> the launch's rows are split into one host-side fp_result per
// request.  Latency is measured from submit to the moment its result is
// ready.  Every wait the caller makes is bounded (FP_E_TIMEOUT).
#include <string.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "pipe.cuh"

using namespace fpk;
using Clock = std::chrono::steady_clock;

namespace {

struct Request {
    int64_t id = 0;
    std::vector<uint8_t> chars;
    std::vector<int64_t> off;
    int64_t n = 0;
    int k = 0, metric = 0;
    Clock::time_point t_submit, t_admit, t_done;
    bool done = false;
    int rc = FP_OK;
    std::string err;
    fp_result *res = nullptr;
};

enum LaneState { IDLE = 0, RUNNING = 1, COPYING = 2 };

struct Lane {
    fp_server *srv = nullptr;
    cudaStream_t st = nullptr;
    int state = IDLE;
    bool signal = false;  // set by the host function behind the lane's last stage (under the server mutex)
    std::vector<Request *> reqs;
    int64_t n = 0, total = 0;
    int nb = 0, ng = 0;
    PipeShape shape;
    size_t bytes = 0;  // admitted device bytes
    uint8_t *arena = nullptr;
    Pipe pipe;
    int attempts = 0;
    // pinned staging
    uint8_t *h_chars = nullptr;
    int64_t *h_off = nullptr, *h_bs = nullptr;
    int32_t *h_bg = nullptr, *h_km = nullptr;
    uint64_t *h_scal = nullptr;
    int64_t *h_row = nullptr;
    int32_t *h_idx = nullptr;
    int64_t h_idx_cap = 0;
    std::vector<fp_batch> batches;
};

void CUDART_CB lane_done(void *arg);

}  // namespace

struct fp_server {
    fp_index *ix = nullptr;
    fp_server_opts o{};
    FilterCfg cfg{};
    int device = 0;
    int64_t budget = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> queue;
    std::unordered_map<int64_t, Request *> reqs;
    std::vector<Lane> lanes;
    std::thread worker;
    bool stop = false;
    int64_t next_id = 1;
    int64_t used = 0;
    // statistics
    fp_server_stats s{};
    std::vector<double> lat_ms;
    double queue_ms_sum = 0;
    int busy = 0;
    Clock::time_point busy_since;
    double busy_s = 0;
};

namespace {

void CUDART_CB lane_done(void *arg) {
    Lane *L = (Lane *)arg;
    fp_server *S = L->srv;
    {
        std::lock_guard<std::mutex> g(S->mu);
        L->signal = true;
    }
    S->cv_work.notify_one();
}

// Device bytes a launch of this shape holds.
size_t footprint(const PipeShape &sh) { return pipe_layout(sh, nullptr, nullptr); }

int64_t estimate_matches(int64_t n) { return std::max<int64_t>(4096, 4 * n); }

// Finishes every request of the lane with `rc` (under the server mutex).
void finish_lane_locked(fp_server *S, Lane &L, int rc, const std::string &err) {
    const Clock::time_point now = Clock::now();
    for (Request *r : L.reqs) {
        r->t_done = now;
        r->done = true;
        if (rc != FP_OK) {
            r->rc = rc;
            r->err = err;
        } else {
            const double ms = std::chrono::duration<double, std::milli>(now - r->t_submit).count();
            S->lat_ms.push_back(ms);
            S->s.completed++;
            S->s.queries += r->n;
            if (r->res) r->res->stats.ms_total = (float)ms;
        }
    }
    L.reqs.clear();
    S->used -= (int64_t)L.bytes;
    L.bytes = 0;
    L.state = IDLE;
    if (--S->busy == 0) S->busy_s += std::chrono::duration<double>(now - S->busy_since).count();
}

// Copies the lane's inputs from its pinned staging into the arena and
// enqueues the pipeline and the wake-up.  No lock held.
int enqueue_run(fp_server *S, Lane &L) {
    Pipe &P = L.pipe;
    FP_CUDA(cudaMemcpyAsync(P.d_off, L.h_off, 8 * (size_t)(L.n + 1), cudaMemcpyHostToDevice, L.st));
    if (L.total > 0) FP_CUDA(cudaMemcpyAsync(P.d_chars, L.h_chars, (size_t)L.total, cudaMemcpyHostToDevice, L.st));
    FP_CUDA(cudaMemcpyAsync(P.d_batch_start, L.h_bs, 8 * (size_t)(L.nb + 1), cudaMemcpyHostToDevice, L.st));
    FP_CUDA(cudaMemcpyAsync(P.d_batch_group, L.h_bg, 4 * (size_t)L.nb, cudaMemcpyHostToDevice, L.st));
    FP_CUDA(cudaMemcpyAsync(P.d_group_km, L.h_km, 4 * 2 * MAX_GROUPS, cudaMemcpyHostToDevice, L.st));
    FP_TRY(pipe_enqueue(S->ix, S->cfg, P, L.n, L.total, L.nb, L.ng, L.st, L.h_scal, nullptr));
    FP_CUDA(cudaLaunchHostFunc(L.st, lane_done, &L));
    return FP_OK;
}

int place_arena(Lane &L) {
    L.arena = nullptr;
    FP_CUDA(cudaMallocAsync((void **)&L.arena, L.bytes, L.st));
    pipe_layout(L.shape, L.arena, &L.pipe);
    return FP_OK;
}

// Starts a launch for the lane's requests (packed already).  No lock held.
int start_launch(fp_server *S, Lane &L) {
    FP_TRY(place_arena(L));
    L.attempts = 0;
    return enqueue_run(S, L);
}

// Next stage of a lane whose last stage finished.  No lock held; returns
// FP_OK, or an error that fails the lane's requests.
int advance(fp_server *S, Lane &L, bool *finished) {
    *finished = false;
    const uint64_t *sc = L.h_scal;
    if (L.state == RUNNING) {
        if (((const int32_t *)(sc + 8))[0]) return fail(FP_E_INVAL, "string longer than 255 bytes");
        if (sc[6]) return fail(FP_E_NOMEM, "tile plan overflow");
        const int64_t nm = (int64_t)sc[5];
        if (nm > L.pipe.match_cap) {
            // more matches than estimated: the same run once more with the exact size
            if (++L.attempts > 1) return fail(FP_E_NOMEM, "match buffer sizing failed");
            FP_CUDA(cudaFreeAsync(L.arena, L.st));
            L.arena = nullptr;
            const size_t old = L.bytes;
            L.shape.match_cap = nm;
            L.bytes = footprint(L.shape);
            {
                std::lock_guard<std::mutex> g(S->mu);
                S->used += (int64_t)L.bytes - (int64_t)old;
                S->s.peak_bytes = std::max(S->s.peak_bytes, S->used);
                S->s.reruns++;
            }
            FP_TRY(place_arena(L));
            return enqueue_run(S, L);
        }
        if (nm > L.h_idx_cap) {
            const int64_t cap = std::max<int64_t>(nm, 2 * L.h_idx_cap);
            if (L.h_idx) cudaFreeHost(L.h_idx);
            L.h_idx = nullptr;
            L.h_idx_cap = 0;
            FP_CUDA(cudaMallocHost((void **)&L.h_idx, 4 * (size_t)cap));
            L.h_idx_cap = cap;
        }
        {
            std::lock_guard<std::mutex> g(S->mu);
            S->s.pairs += (int64_t)sc[2];
            S->s.survivors += (int64_t)sc[4];
            S->s.matches += nm;
        }
        FP_CUDA(cudaMemcpyAsync(L.h_row, L.pipe.row_ptr, 8 * (size_t)(L.n + 1), cudaMemcpyDeviceToHost, L.st));
        if (nm > 0) FP_CUDA(cudaMemcpyAsync(L.h_idx, L.pipe.idx, 4 * (size_t)nm, cudaMemcpyDeviceToHost, L.st));
        FP_CUDA(cudaFreeAsync(L.arena, L.st));
        L.arena = nullptr;
        FP_CUDA(cudaLaunchHostFunc(L.st, lane_done, &L));
        L.state = COPYING;
        return FP_OK;
    }
    // COPYING done: one host-side result per request
    int64_t q0 = 0;
    for (Request *r : L.reqs) {
        fp_result *res = new fp_result();
        res->n_queries = r->n;
        const int64_t base = L.h_row[q0], end = L.h_row[q0 + r->n];
        res->n_matches = end - base;
        res->h_row_ptr.resize((size_t)r->n + 1);
        for (int64_t i = 0; i <= r->n; i++) res->h_row_ptr[(size_t)i] = L.h_row[q0 + i] - base;
        res->h_idx.assign(L.h_idx + base, L.h_idx + end);
        if (res->h_idx.empty()) res->h_idx.resize(1);
        res->host_ready = true;
        res->stats.n_queries = r->n;
        res->stats.matches = res->n_matches;
        r->res = res;
        q0 += r->n;
    }
    *finished = true;
    return FP_OK;
}

// Takes the oldest queued requests that fit one launch and the memory left
// (under the server mutex).  Returns false when nothing can be admitted now.
bool admit_locked(fp_server *S, Lane &L) {
    L.reqs.clear();
    L.batches.clear();
    int64_t n = 0, total = 0;
    int32_t km[2 * MAX_GROUPS];
    int ng = 0;
    size_t bytes = 0;
    PipeShape sh;
    for (Request *r : S->queue) {
        if ((int)L.reqs.size() >= S->o.max_requests) break;
        if (n + r->n > S->o.max_queries || total + (int64_t)r->chars.size() > S->o.max_chars) break;
        int g = 0;
        while (g < ng && !(km[g] == r->k && km[MAX_GROUPS + g] == r->metric)) g++;
        const int ng2 = g == ng ? ng + 1 : ng;
        if (ng2 > MAX_GROUPS) break;
        PipeShape t;
        t.queries = n + r->n;
        t.chars = total + (int64_t)r->chars.size();
        t.batches = (int32_t)L.reqs.size() + 1;
        t.groups = ng2;
        t.match_cap = estimate_matches(t.queries);
        const size_t b = footprint(t);
        if (S->used + (int64_t)b > S->budget) break;  // wait for memory (oldest first)
        if (g == ng) {
            km[g] = r->k;
            km[MAX_GROUPS + g] = r->metric;
        }
        ng = ng2;
        n = t.queries;
        total = t.chars;
        sh = t;
        bytes = b;
        L.reqs.push_back(r);
        L.batches.push_back(fp_batch{r->n, r->k, r->metric});
    }
    if (L.reqs.empty()) return false;
    S->queue.erase(S->queue.begin(), S->queue.begin() + (long)L.reqs.size());
    const Clock::time_point now = Clock::now();
    for (Request *r : L.reqs) {
        r->t_admit = now;
        S->queue_ms_sum += std::chrono::duration<double, std::milli>(now - r->t_submit).count();
    }
    L.n = n;
    L.total = total;
    L.nb = (int)L.reqs.size();
    L.shape = sh;
    L.bytes = bytes;
    L.state = RUNNING;
    L.signal = false;
    S->used += (int64_t)bytes;
    S->s.peak_bytes = std::max(S->s.peak_bytes, S->used);
    S->s.launches++;
    S->s.max_requests_per_launch = std::max(S->s.max_requests_per_launch, (int32_t)L.reqs.size());
    if (S->busy++ == 0) S->busy_since = now;
    S->s.max_lanes_busy = std::max(S->s.max_lanes_busy, (int32_t)S->busy);
    return true;
}

// Packs the admitted requests into the lane's pinned staging.  No lock held
// (the lane's requests are not touched by other threads until they are done).
int pack(fp_server *S, Lane &L) {
    int64_t q = 0, c = 0;
    L.h_off[0] = 0;
    for (Request *r : L.reqs) {
        if (!r->chars.empty()) memcpy(L.h_chars + c, r->chars.data(), r->chars.size());
        for (int64_t i = 1; i <= r->n; i++) L.h_off[q + i] = c + r->off[(size_t)i];
        q += r->n;
        c += (int64_t)r->chars.size();
    }
    return group_batches(S->ix, L.batches.data(), L.nb, L.n, L.h_bs, L.h_bg, L.h_km, &L.ng);
}

void scheduler(fp_server *S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        bool progressed = false;
        for (Lane &L : S->lanes) {
            if (L.state == IDLE || !L.signal) continue;
            L.signal = false;
            progressed = true;
            lk.unlock();
            bool finished = false;
            int rc = advance(S, L, &finished);
            std::string err = rc != FP_OK ? fp_last_error() : std::string();
            if (rc != FP_OK && L.arena) {
                cudaFreeAsync(L.arena, L.st);
                L.arena = nullptr;
            }
            if (rc != FP_OK) cudaStreamSynchronize(L.st);  // nothing of the lane may still be queued
            lk.lock();
            if (rc != FP_OK || finished) {
                finish_lane_locked(S, L, rc, err);
                S->cv_done.notify_all();
            }
        }
        for (Lane &L : S->lanes) {
            if (L.state != IDLE || S->queue.empty()) continue;
            if (!admit_locked(S, L)) break;
            progressed = true;
            lk.unlock();
            int rc = pack(S, L);
            if (rc == FP_OK) rc = start_launch(S, L);
            std::string err = rc != FP_OK ? fp_last_error() : std::string();
            if (rc != FP_OK) {
                if (L.arena) cudaFreeAsync(L.arena, L.st);
                L.arena = nullptr;
                cudaStreamSynchronize(L.st);
            }
            lk.lock();
            if (rc != FP_OK) {
                finish_lane_locked(S, L, rc, err);
                S->cv_done.notify_all();
            }
        }
        bool idle = true;
        for (Lane &L : S->lanes) idle = idle && L.state == IDLE;
        if (S->stop && idle && S->queue.empty()) break;
        if (!progressed) S->cv_work.wait_for(lk, std::chrono::milliseconds(100));
    }
}

void free_lane(Lane &L) {
    if (L.st) cudaStreamSynchronize(L.st);
    if (L.arena) cudaFree(L.arena);
    if (L.h_chars) cudaFreeHost(L.h_chars);
    if (L.h_off) cudaFreeHost(L.h_off);
    if (L.h_bs) cudaFreeHost(L.h_bs);
    if (L.h_bg) cudaFreeHost(L.h_bg);
    if (L.h_km) cudaFreeHost(L.h_km);
    if (L.h_scal) cudaFreeHost(L.h_scal);
    if (L.h_row) cudaFreeHost(L.h_row);
    if (L.h_idx) cudaFreeHost(L.h_idx);
    if (L.st) cudaStreamDestroy(L.st);
    L = Lane{};
}

}  // namespace

extern "C" {

int fp_server_create(fp_index *ix, const fp_server_opts *opts, fp_server **out) {
    if (!ix || !out) return fail(FP_E_INVAL, "fp_server_create: null argument");
    *out = nullptr;
    fp_server_opts o{};
    if (opts) o = *opts;
    if (o.lanes < 0 || o.lanes > 64 || o.max_requests < 0 || o.max_queries < 0 || o.max_chars < 0 ||
        o.memory_budget < 0 || o.max_queries > 0x7FFFFFFFLL)
        return fail(FP_E_INVAL, "fp_server_create: bad option");
    if (o.lanes == 0) o.lanes = 4;
    if (o.max_requests == 0) o.max_requests = 64;
    if (o.max_queries == 0) o.max_queries = 16384;
    if (o.max_chars == 0) o.max_chars = 128 * o.max_queries;
    init_pool();
    fp_server *S = new fp_server();
    S->ix = ix;
    S->cfg.mode = FP_MODE_FUSED;
    S->cfg.v = 4;
    S->cfg.tq = o.tile_queries > 0 ? std::min(o.tile_queries, 256) : 256;
    S->cfg.k1mix = o.variant == 0;
    S->cfg.mma = o.variant == 2;
    cudaGetDevice(&S->device);
    if (o.memory_budget == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            delete S;
            return cuda_fail(cudaGetLastError(), "cudaMemGetInfo");
        }
        o.memory_budget = (int64_t)(fr / 4);
    }
    S->o = o;
    S->budget = o.memory_budget;
    S->s.budget_bytes = o.memory_budget;
    S->lanes.resize((size_t)o.lanes);
    int rc = FP_OK;
    for (Lane &L : S->lanes) {
        L.srv = S;
        if (cudaStreamCreateWithFlags(&L.st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaMallocHost((void **)&L.h_chars, (size_t)o.max_chars + 16) != cudaSuccess ||
            cudaMallocHost((void **)&L.h_off, 8 * (size_t)(o.max_queries + 1)) != cudaSuccess ||
            cudaMallocHost((void **)&L.h_bs, 8 * (size_t)(o.max_requests + 1)) != cudaSuccess ||
            cudaMallocHost((void **)&L.h_bg, 4 * (size_t)o.max_requests) != cudaSuccess ||
            cudaMallocHost((void **)&L.h_km, 4 * 2 * MAX_GROUPS) != cudaSuccess ||
            cudaMallocHost((void **)&L.h_scal, 8 * 16) != cudaSuccess ||
            cudaMallocHost((void **)&L.h_row, 8 * (size_t)(o.max_queries + 1)) != cudaSuccess ||
            cudaMallocHost((void **)&L.h_idx, 4 * (size_t)estimate_matches(o.max_queries)) != cudaSuccess) {
            rc = cuda_fail(cudaGetLastError(), "fp_server_create: stream / pinned staging");
            break;
        }
        L.h_idx_cap = estimate_matches(o.max_queries);
    }
    if (rc == FP_OK) {
        // the smallest launch must fit the budget, or nothing could ever run
        PipeShape one;
        one.queries = 1;
        one.chars = MAX_LEN;
        one.match_cap = estimate_matches(1);
        if ((int64_t)footprint(one) > S->budget) rc = fail(FP_E_NOMEM, "memory budget below one launch");
    }
    if (rc != FP_OK) {
        for (Lane &L : S->lanes) free_lane(L);
        delete S;
        return rc;
    }
    S->worker = std::thread(scheduler, S);
    *out = S;
    return FP_OK;
}

int fp_server_submit(fp_server *S, const uint8_t *chars, const int64_t *offsets, int64_t n_queries, int k, int metric,
                     int64_t *request_id) {
    if (!S || !offsets || !request_id || n_queries < 1) return fail(FP_E_INVAL, "fp_server_submit: bad argument");
    if (k < 0 || k > 15 || (metric != FP_HAM && metric != FP_LEV)) return fail(FP_E_INVAL, "k in 0..15, metric");
    if (metric == FP_LEV && (S->ix->P.type == FP_OCC_HALVED || S->ix->P.type == FP_POS))
        return fail(FP_E_UNSUPPORTED, "occurrence-halved and position fingerprints bound only the Hamming distance");
    if (is_device_ptr(offsets) || (chars && is_device_ptr(chars)))
        return fail(FP_E_INVAL, "fp_server_submit takes host buffers");
    FP_TRY(check_host_offsets(offsets, n_queries));
    const int64_t total = offsets[n_queries];
    if (total > 0 && !chars) return fail(FP_E_INVAL, "chars is null");
    for (int64_t i = 0; i < n_queries; i++)
        if (offsets[i + 1] - offsets[i] > MAX_LEN) return fail(FP_E_INVAL, "pattern longer than 255 bytes");
    if (n_queries > S->o.max_queries || total > S->o.max_chars)
        return fail(FP_E_INVAL, "request larger than one launch (max_queries / max_chars)");
    PipeShape alone;
    alone.queries = n_queries;
    alone.chars = total;
    alone.match_cap = estimate_matches(n_queries);
    if ((int64_t)footprint(alone) > S->budget) return fail(FP_E_NOMEM, "request alone exceeds the memory budget");
    Request *r = new Request();
    r->chars.assign(chars ? chars : (const uint8_t *)"", chars ? chars + total : (const uint8_t *)"");
    r->off.assign(offsets, offsets + n_queries + 1);
    r->n = n_queries;
    r->k = k;
    r->metric = metric;
    {
        std::lock_guard<std::mutex> g(S->mu);
        if (S->stop) {
            delete r;
            return fail(FP_E_INVAL, "server is shutting down");
        }
        r->id = S->next_id++;
        r->t_submit = Clock::now();
        S->reqs[r->id] = r;
        S->queue.push_back(r);
        S->s.submitted++;
    }
    S->cv_work.notify_one();
    *request_id = r->id;
    return FP_OK;
}

int fp_server_wait(fp_server *S, int64_t request_id, int64_t timeout_us, fp_result **out) {
    if (!S || !out || timeout_us < 0) return fail(FP_E_INVAL, "fp_server_wait: bad argument");
    *out = nullptr;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(request_id);
    if (it == S->reqs.end()) return fail(FP_E_INVAL, "unknown request id (or its result was taken)");
    Request *r = it->second;
    const Clock::time_point until = Clock::now() + std::chrono::microseconds(timeout_us);
    while (!r->done)
        if (S->cv_done.wait_until(lk, until) == std::cv_status::timeout && !r->done)
            return fail(FP_E_TIMEOUT, "request not finished within the timeout");
    S->reqs.erase(it);
    lk.unlock();
    const int rc = r->rc;
    if (rc != FP_OK) {
        fail(rc, r->err);
        delete r;
        return rc;
    }
    *out = r->res;
    delete r;
    return FP_OK;
}

int fp_server_stats_get(fp_server *S, fp_server_stats *out) {
    if (!S || !out) return fail(FP_E_INVAL, "null argument");
    std::lock_guard<std::mutex> g(S->mu);
    fp_server_stats s = S->s;
    std::vector<double> v = S->lat_ms;
    if (!v.empty()) {
        std::sort(v.begin(), v.end());
        auto pct = [&](double q) {  // nearest rank
            size_t i = (size_t)std::ceil(q * (double)v.size());
            return v[std::min(v.size(), std::max<size_t>(i, 1)) - 1];
        };
        s.p50_ms = pct(0.50);
        s.p99_ms = pct(0.99);
        s.max_ms = v.back();
        double sum = 0;
        for (double x : v) sum += x;
        s.mean_ms = sum / (double)v.size();
    }
    const int64_t admitted = s.submitted - (int64_t)S->queue.size();
    s.mean_queue_ms = admitted > 0 ? S->queue_ms_sum / (double)admitted : 0.0;
    s.busy_seconds = S->busy_s + (S->busy > 0 ? std::chrono::duration<double>(Clock::now() - S->busy_since).count() : 0);
    s.in_use_bytes = S->used;
    *out = s;
    return FP_OK;
}

int fp_server_replay(fp_server *S, const uint8_t *chars, const int64_t *offsets, const int64_t *request_sizes,
                     const int64_t *arrival_us, int64_t n_requests, int k, int metric, int64_t timeout_us,
                     double *latency_ms, fp_result **out) {
    if (!S || !offsets || !request_sizes || !arrival_us || n_requests < 1 || timeout_us < 0 || !out)
        return fail(FP_E_INVAL, "fp_server_replay: bad argument");
    *out = nullptr;
    int64_t nq = 0;
    for (int64_t r = 0; r < n_requests; r++) {
        if (request_sizes[r] < 1 || arrival_us[r] < 0 || (r > 0 && arrival_us[r] < arrival_us[r - 1]))
            return fail(FP_E_INVAL, "request sizes >= 1 and arrival times non-decreasing");
        nq += request_sizes[r];
    }
    FP_TRY(check_host_offsets(offsets, nq));
    std::vector<int64_t> ids((size_t)n_requests, 0);
    std::vector<int64_t> off;
    const Clock::time_point t0 = Clock::now();
    int rc = FP_OK;
    int64_t q = 0, submitted = 0;
    for (int64_t r = 0; r < n_requests && rc == FP_OK; r++) {
        std::this_thread::sleep_until(t0 + std::chrono::microseconds(arrival_us[r]));
        const int64_t n = request_sizes[r];
        off.resize((size_t)n + 1);
        for (int64_t i = 0; i <= n; i++) off[(size_t)i] = offsets[q + i] - offsets[q];
        rc = fp_server_submit(S, chars ? chars + offsets[q] : nullptr, off.data(), n, k, metric, &ids[(size_t)r]);
        if (rc == FP_OK) submitted++;
        q += n;
    }
    // collect every submitted request (also after a failure, so none is left behind)
    fp_result *all = rc == FP_OK ? new fp_result() : nullptr;
    if (all) {
        all->n_queries = nq;
        all->h_row_ptr.assign(1, 0);
        all->stats.n_queries = nq;
    }
    const Clock::time_point until = Clock::now() + std::chrono::microseconds(timeout_us);
    for (int64_t r = 0; r < submitted; r++) {
        const int64_t left = std::max<int64_t>(
            0, std::chrono::duration_cast<std::chrono::microseconds>(until - Clock::now()).count());
        fp_result *res = nullptr;
        const int rr = fp_server_wait(S, ids[(size_t)r], left, &res);
        if (rr != FP_OK) {
            if (rc == FP_OK) rc = rr;
            if (rr == FP_E_TIMEOUT) break;  // the server keeps the rest; fp_server_free drains them
            continue;
        }
        if (latency_ms) latency_ms[r] = res->stats.ms_total;
        if (all) {
            const int64_t base = all->h_row_ptr.back();
            for (int64_t i = 1; i <= res->n_queries; i++) all->h_row_ptr.push_back(base + res->h_row_ptr[(size_t)i]);
            all->h_idx.insert(all->h_idx.end(), res->h_idx.begin(), res->h_idx.begin() + res->n_matches);
        }
        fp_result_free(res);
    }
    if (rc != FP_OK) {
        fp_result_free(all);
        return rc;
    }
    all->n_matches = (int64_t)all->h_idx.size();
    all->stats.matches = all->n_matches;
    if (all->h_idx.empty()) all->h_idx.resize(1);
    all->host_ready = true;
    *out = all;
    return FP_OK;
}

void fp_server_free(fp_server *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_one();
    if (S->worker.joinable()) S->worker.join();  // drains the queue and every launch in flight
    for (Lane &L : S->lanes) free_lane(L);
    for (auto &kv : S->reqs) {
        fp_result_free(kv.second->res);
        delete kv.second;
    }
    delete S;
}

}  // extern "C"
