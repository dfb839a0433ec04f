// Query plans: the whole query pipeline on plan-owned device buffers,
// captured once into a CUDA graph and replayed (a8 of the build plan).
//
// A plan holds every buffer a batch of up to max_queries patterns
// (max_chars bytes, max_batches batches) needs.  fp_plan_run copies the
// inputs into the plan's buffers, then launches the pipeline:
//   per-pattern group ids -> bucketing by (group, length) + fingerprints ->
//   tile plan -> fused filter + verify (one persistent kernel over every
//   batch and length bucket) -> sorted CSR -> counters to pinned memory.
// The first run of a given shape (patterns, bytes, batches, groups) records
// that sequence into a CUDA graph on the plan's stream; later runs of the
// same shape replay it with one cudaGraphLaunch.  Batches that share
// (k, metric) form one group; a tile never mixes groups, so every tile has
// one threshold 2k (Eq. 1) and one verification routine (Sec. 4).
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"

using namespace fpk;

struct fp_plan {
    fp_index *ix = nullptr;
    int64_t max_queries = 0, max_chars = 0;
    int32_t max_batches = 0;
    FilterCfg cfg{};
    bool use_graph = true;
    cudaStream_t st = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_f0 = nullptr, ev_f1 = nullptr, ev_t0 = nullptr,
                ev_t1 = nullptr;
    // inputs
    uint8_t *d_chars = nullptr;
    int64_t *d_off = nullptr;
    int64_t *d_batch_start = nullptr;  // [max_batches + 1]
    int32_t *d_batch_group = nullptr;  // [max_batches]
    int32_t *d_group_km = nullptr;     // [2 * 32]: k then metric per group
    int32_t *d_group = nullptr;        // [max_queries]
    int64_t *h_batch_start = nullptr;  // pinned staging
    int32_t *h_batch_group = nullptr;
    int32_t *h_group_km = nullptr;
    // bucketed patterns and scratch
    Bucketed Q;
    BucketScratch S{};
    QueryPlan qp;
    int32_t *d_err = nullptr;
    // matches and output
    int64_t match_cap = 0;
    uint64_t *matches = nullptr, *tmp = nullptr;
    uint32_t *radix_hist = nullptr;
    int64_t *row_ptr = nullptr;
    int32_t *idx = nullptr;
    uint64_t *h_scal = nullptr;  // pinned: counters + error flag
    // captured graph and its shape
    cudaGraphExec_t exec = nullptr;
    int64_t shape[4] = {-1, -1, -1, -1};
    int64_t kernels_per_run = 0;
    std::vector<void *> dev_allocs;
};

namespace {

constexpr int MAX_GROUPS = 32;

int palloc(fp_plan *p, void **ptr, size_t bytes) {
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "fp_plan allocation");
    p->dev_allocs.push_back(*ptr);
    return FP_OK;
}

int alloc_matches(fp_plan *p, int64_t cap) {
    if (p->matches) cudaFree(p->matches);
    if (p->tmp) cudaFree(p->tmp);
    if (p->idx) cudaFree(p->idx);
    if (p->radix_hist) cudaFree(p->radix_hist);
    p->matches = nullptr;
    p->tmp = nullptr;
    p->idx = nullptr;
    p->radix_hist = nullptr;
    p->match_cap = cap;
    const int64_t rh = 256 * (int64_t)std::max(radix_blocks(cap), radix_blocks(p->max_queries));
    FP_CUDA(cudaMalloc((void **)&p->matches, sizeof(uint64_t) * (size_t)cap));
    FP_CUDA(cudaMalloc((void **)&p->tmp, sizeof(uint64_t) * (size_t)cap));
    FP_CUDA(cudaMalloc((void **)&p->idx, sizeof(int32_t) * (size_t)cap));
    FP_CUDA(cudaMalloc((void **)&p->radix_hist, sizeof(uint32_t) * (size_t)rh));
    p->S.radix_hist = p->radix_hist;
    return FP_OK;
}

// Enqueues the device pipeline on p->st (recorded into a graph when capturing).
int enqueue(fp_plan *p, int64_t n, int64_t total, int n_batches, int n_groups) {
    fp_index *ix = p->ix;
    const int nbins = 256 * n_groups;
    cudaGetLastError();  // launch checks below must not see an unrelated earlier error
    FP_CUDA(cudaEventRecord(p->ev_t0, p->st));
    FP_CUDA(cudaMemsetAsync(p->d_err, 0, sizeof(int32_t), p->st));
    FP_TRY(fill_groups(p->d_batch_start, p->d_batch_group, n_batches, p->d_group, p->st));
    FP_TRY(bucketize_into(p->d_chars, p->d_off, n, total, p->d_group, n_groups, ix->d_map, ix->P, p->st, &p->Q, p->S,
                          p->d_err));
    p->qp.max_segments = nbins * 31;
    FP_TRY(plan_segments(p->Q, ix->D, p->d_group_km, p->d_group_km + MAX_GROUPS, p->cfg.tq,
                         tile_words(ix->P.width, p->cfg.v), &p->qp, p->st));
    FP_CUDA(cudaEventRecord(p->ev_f0, p->st));
    FP_TRY(launch_fused(p->Q, ix->D, p->qp, ix->P, p->cfg, ix->idx_bits, p->matches, p->match_cap, p->st, nullptr));
    FP_CUDA(cudaEventRecord(p->ev_f1, p->st));
    FP_TRY(build_csr_into(p->matches, p->tmp, p->radix_hist, p->qp.scal + 5, p->match_cap, bits_for(n),
                          ix->idx_bits, n, p->row_ptr, p->idx, p->st));
    FP_CUDA(cudaMemcpyAsync(p->h_scal, p->qp.scal, 8 * sizeof(uint64_t), cudaMemcpyDeviceToHost, p->st));
    FP_CUDA(cudaMemcpyAsync(p->h_scal + 8, p->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, p->st));
    FP_CUDA(cudaEventRecord(p->ev_t1, p->st));
    return FP_OK;
}

}  // namespace

extern "C" {

int fp_plan_create(fp_index *ix, int64_t max_queries, int64_t max_chars, int32_t max_batches,
                   const fp_query_opts *opts, fp_plan **out) {
    if (!ix || !out || max_queries < 1 || max_queries > 0x7FFFFFFFLL || max_chars < 0 || max_batches < 1)
        return fail(FP_E_INVAL, "fp_plan_create: bad argument");
    *out = nullptr;
    init_pool();
    fp_query_opts o{};
    if (opts) o = *opts;
    fp_plan *p = new fp_plan();
    p->ix = ix;
    p->max_queries = max_queries;
    p->max_chars = max_chars;
    p->max_batches = max_batches;
    p->cfg.mode = FP_MODE_FUSED;
    p->cfg.v = 4;
    p->cfg.tq = o.tile_queries > 0 ? std::min(o.tile_queries, 256) : 256;
    p->cfg.k1mix = o.variant == 0;  // the kernel takes the mixed test only in k = 1 tiles
    p->use_graph = o.mode != FP_MODE_PLAIN;  // FP_MODE_PLAIN here means: run the pipeline without a graph
    const int64_t nbins = 256 * MAX_GROUPS;
    const int64_t slots = max_queries + (int64_t)(SLOT_ALIGN - 1) * nbins;
    const int64_t strb = max_chars + 15 * max_queries + STR_SLACK;
    int rc = FP_OK;
#define P_ALLOC(ptr, bytes)                                       \
    do {                                                          \
        if ((rc = palloc(p, (void **)&(ptr), (size_t)(bytes))) != FP_OK) goto fail_out; \
    } while (0)
    if (cudaStreamCreateWithFlags(&p->st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_out, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreate(&p->ev_f0) != cudaSuccess || cudaEventCreate(&p->ev_f1) != cudaSuccess ||
        cudaEventCreate(&p->ev_t0) != cudaSuccess || cudaEventCreate(&p->ev_t1) != cudaSuccess) {
        rc = cuda_fail(cudaGetLastError(), "fp_plan_create: stream / events");
        goto fail_out;
    }
    P_ALLOC(p->d_chars, max_chars + 16);
    P_ALLOC(p->d_off, 8 * (max_queries + 1));
    P_ALLOC(p->d_batch_start, 8 * (max_batches + 1));
    P_ALLOC(p->d_batch_group, 4 * max_batches);
    P_ALLOC(p->d_group_km, 4 * 2 * MAX_GROUPS);
    P_ALLOC(p->d_group, 4 * max_queries);
    P_ALLOC(p->Q.fp, 4 * (slots + FP_SLACK_SLOTS));
    P_ALLOC(p->Q.idx, 4 * slots);
    P_ALLOC(p->Q.len, slots);
    P_ALLOC(p->Q.row16, 4 * slots);
    P_ALLOC(p->Q.str, strb);
    P_ALLOC(p->Q.b_start, 4 * nbins);
    P_ALLOC(p->Q.b_count, 4 * nbins);
    P_ALLOC(p->S.keys, 8 * max_queries);
    P_ALLOC(p->S.keys2, 8 * max_queries);
    P_ALLOC(p->S.hist, 4 * nbins);
    P_ALLOC(p->S.ustart, 4 * nbins);
    P_ALLOC(p->S.str16, 8 * nbins);
    P_ALLOC(p->S.tot, 16);
    P_ALLOC(p->qp.seg, sizeof(Segment) * nbins * 31);
    P_ALLOC(p->qp.scal, 8 * 8);
    P_ALLOC(p->d_err, 4);
    P_ALLOC(p->row_ptr, 8 * (max_queries + 1));
#undef P_ALLOC
    if (cudaMallocHost((void **)&p->h_batch_start, 8 * (size_t)(max_batches + 1)) != cudaSuccess ||
        cudaMallocHost((void **)&p->h_batch_group, 4 * (size_t)max_batches) != cudaSuccess ||
        cudaMallocHost((void **)&p->h_group_km, 4 * 2 * MAX_GROUPS) != cudaSuccess ||
        cudaMallocHost((void **)&p->h_scal, 16 * sizeof(uint64_t)) != cudaSuccess) {
        rc = cuda_fail(cudaErrorMemoryAllocation, "fp_plan_create: pinned staging");
        goto fail_out;
    }
    if ((rc = alloc_matches(p, std::max<int64_t>(1 << 20, std::min<int64_t>(max_queries * 64, 1LL << 28)))) != FP_OK)
        goto fail_out;
    *out = p;
    return FP_OK;
fail_out:
    fp_plan_free(p);
    return rc;
}

void fp_plan_free(fp_plan *p) {
    if (!p) return;
    if (p->st) cudaStreamSynchronize(p->st);
    if (p->exec) cudaGraphExecDestroy(p->exec);
    for (void *q : p->dev_allocs) cudaFree(q);
    if (p->matches) cudaFree(p->matches);
    if (p->tmp) cudaFree(p->tmp);
    if (p->idx) cudaFree(p->idx);
    if (p->radix_hist) cudaFree(p->radix_hist);
    if (p->h_batch_start) cudaFreeHost(p->h_batch_start);
    if (p->h_batch_group) cudaFreeHost(p->h_batch_group);
    if (p->h_group_km) cudaFreeHost(p->h_group_km);
    if (p->h_scal) cudaFreeHost(p->h_scal);
    cudaEvent_t evs[] = {p->ev_in, p->ev_out, p->ev_f0, p->ev_f1, p->ev_t0, p->ev_t1};
    for (cudaEvent_t e : evs)
        if (e) cudaEventDestroy(e);
    if (p->st) cudaStreamDestroy(p->st);
    delete p;
}

int fp_plan_run(fp_plan *p, const uint8_t *chars, const int64_t *offsets, int64_t n_queries, const fp_batch *batches,
                int32_t n_batches, void *cuda_stream, fp_result **out) {
    if (!p || !offsets || !batches || !out || n_queries < 0 || n_batches < 1) return fail(FP_E_INVAL, "fp_plan_run: bad argument");
    *out = nullptr;
    if (n_queries > p->max_queries || n_batches > p->max_batches)
        return fail(FP_E_INVAL, "fp_plan_run: more patterns or batches than the plan was made for");
    fp_index *ix = p->ix;
    // batches -> groups of equal (k, metric)
    int n_groups = 0;
    int64_t start = 0;
    for (int b = 0; b < n_batches; b++) {
        const fp_batch &B = batches[b];
        if (B.n_queries < 0 || B.k < 0 || B.k > 15 || (B.metric != FP_HAM && B.metric != FP_LEV))
            return fail(FP_E_INVAL, "fp_plan_run: bad batch (n_queries, k in 0..15, metric)");
        if (B.metric == FP_LEV && (ix->P.type == FP_OCC_HALVED || ix->P.type == FP_POS))
            return fail(FP_E_UNSUPPORTED, "occurrence-halved and position fingerprints bound only the Hamming distance");
        int g = 0;
        while (g < n_groups && !(p->h_group_km[g] == B.k && p->h_group_km[MAX_GROUPS + g] == B.metric)) g++;
        if (g == n_groups) {
            p->h_group_km[g] = B.k;
            p->h_group_km[MAX_GROUPS + g] = B.metric;
            n_groups++;
        }
        p->h_batch_start[b] = start;
        p->h_batch_group[b] = g;
        start += B.n_queries;
    }
    p->h_batch_start[n_batches] = start;
    if (start != n_queries) return fail(FP_E_INVAL, "fp_plan_run: batch sizes do not add up to n_queries");
    cudaStream_t cs = (cudaStream_t)cuda_stream;
    // inputs into the plan's buffers, ordered after the caller's stream
    int64_t total = 0;
    if (is_device_ptr(offsets)) {
        int64_t ends[2];
        FP_CUDA(cudaMemcpyAsync(&ends[0], offsets, 8, cudaMemcpyDeviceToHost, cs));
        FP_CUDA(cudaMemcpyAsync(&ends[1], offsets + n_queries, 8, cudaMemcpyDeviceToHost, cs));
        FP_CUDA(cudaStreamSynchronize(cs));
        if (ends[0] != 0 || ends[1] < 0) return fail(FP_E_INVAL, "offsets[0] must be 0 and offsets non-decreasing");
        total = ends[1];
    } else {
        FP_TRY(check_host_offsets(offsets, n_queries));
        total = offsets[n_queries];
    }
    if (total > p->max_chars) return fail(FP_E_INVAL, "fp_plan_run: more pattern bytes than the plan was made for");
    if (total > 0 && !chars) return fail(FP_E_INVAL, "chars is null");
    FP_CUDA(cudaEventRecord(p->ev_in, cs));
    FP_CUDA(cudaStreamWaitEvent(p->st, p->ev_in, 0));
    FP_CUDA(cudaMemcpyAsync(p->d_off, offsets, 8 * (size_t)(n_queries + 1), cudaMemcpyDefault, p->st));
    if (total > 0) FP_CUDA(cudaMemcpyAsync(p->d_chars, chars, (size_t)total, cudaMemcpyDefault, p->st));
    FP_CUDA(cudaMemcpyAsync(p->d_batch_start, p->h_batch_start, 8 * (size_t)(n_batches + 1), cudaMemcpyHostToDevice,
                            p->st));
    FP_CUDA(cudaMemcpyAsync(p->d_batch_group, p->h_batch_group, 4 * (size_t)n_batches, cudaMemcpyHostToDevice, p->st));
    FP_CUDA(cudaMemcpyAsync(p->d_group_km, p->h_group_km, 4 * 2 * MAX_GROUPS, cudaMemcpyHostToDevice, p->st));

    fp_result *res = new fp_result();
    res->n_queries = n_queries;
    res->stats.n_queries = n_queries;
    int rc = FP_OK;
    for (int attempt = 0; attempt < 2; attempt++) {
        const int64_t shape[4] = {n_queries, total, n_batches, n_groups};
        const bool graph = p->use_graph && attempt == 0;
        if (graph && !(p->exec && memcmp(shape, p->shape, sizeof shape) == 0)) {
            if (p->exec) {
                cudaGraphExecDestroy(p->exec);
                p->exec = nullptr;
            }
            cudaGraph_t g = nullptr;
            const int64_t before = g_launches.load();
            if (cudaStreamBeginCapture(p->st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
                rc = cuda_fail(cudaGetLastError(), "cudaStreamBeginCapture");
                break;
            }
            rc = enqueue(p, n_queries, total, n_batches, n_groups);
            cudaError_t e = cudaStreamEndCapture(p->st, &g);
            if (rc == FP_OK && e != cudaSuccess) rc = cuda_fail(e, "cudaStreamEndCapture");
            if (rc == FP_OK && (e = cudaGraphInstantiate(&p->exec, g, 0)) != cudaSuccess)
                rc = cuda_fail(e, "cudaGraphInstantiate");
            if (g) cudaGraphDestroy(g);
            if (rc != FP_OK) break;
            p->kernels_per_run = g_launches.load() - before;
            g_launches.fetch_sub(p->kernels_per_run);  // counted when the graph runs
            memcpy(p->shape, shape, sizeof shape);
        }
        if (graph) {
            cudaError_t e = cudaGraphLaunch(p->exec, p->st);
            if (e != cudaSuccess) {
                rc = cuda_fail(e, "cudaGraphLaunch");
                break;
            }
            g_launches.fetch_add(p->kernels_per_run);
        } else {
            if ((rc = enqueue(p, n_queries, total, n_batches, n_groups)) != FP_OK) break;
        }
        cudaError_t e = cudaStreamSynchronize(p->st);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "fp_plan_run");
            break;
        }
        const uint64_t *sc = p->h_scal;
        if (((const int32_t *)(sc + 8))[0]) {
            rc = fail(FP_E_INVAL, "string longer than 255 bytes or offsets not monotone");
            break;
        }
        if (sc[6]) {
            rc = fail(FP_E_NOMEM, "tile plan overflow");
            break;
        }
        if ((int64_t)sc[5] <= p->match_cap) {
            res->n_matches = (int64_t)sc[5];
            res->stats.pairs = (int64_t)sc[2];
            res->stats.survivors = (int64_t)sc[4];
            res->stats.matches = (int64_t)sc[5];
            res->stats.filter_launches = 1;
            // stage times from the events the pipeline records (left at 0 if the
            // runtime cannot time them); a failure here must not linger as the
            // thread's last error
            if (cudaEventElapsedTime(&res->stats.ms_filter, p->ev_f0, p->ev_f1) != cudaSuccess ||
                cudaEventElapsedTime(&res->stats.ms_prepare, p->ev_t0, p->ev_f0) != cudaSuccess ||
                cudaEventElapsedTime(&res->stats.ms_emit, p->ev_f1, p->ev_t1) != cudaSuccess ||
                cudaEventElapsedTime(&res->stats.ms_total, p->ev_t0, p->ev_t1) != cudaSuccess)
                cudaGetLastError();
            break;
        }
        // more matches than the buffer holds: grow it to the exact count (the graph
        // refers to the old buffers, so it is dropped) and run once more
        if (attempt == 1) {
            rc = fail(FP_E_NOMEM, "match buffer sizing failed");
            break;
        }
        if (p->exec) {
            cudaGraphExecDestroy(p->exec);
            p->exec = nullptr;
            p->shape[0] = -1;
        }
        if ((rc = alloc_matches(p, (int64_t)sc[5])) != FP_OK) break;
    }
    if (rc == FP_OK) {
        // the result owns copies of the plan's output (ordered on the caller's stream)
        cudaError_t e;
        if ((e = cudaEventRecord(p->ev_out, p->st)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(cs, p->ev_out, 0)) != cudaSuccess ||
            (e = cudaMallocAsync((void **)&res->d_row_ptr, 8 * (size_t)(n_queries + 1), cs)) != cudaSuccess ||
            (e = cudaMallocAsync((void **)&res->d_idx, 4 * (size_t)std::max<int64_t>(res->n_matches, 1), cs)) !=
                cudaSuccess ||
            (e = cudaMemcpyAsync(res->d_row_ptr, p->row_ptr, 8 * (size_t)(n_queries + 1), cudaMemcpyDeviceToDevice,
                                 cs)) != cudaSuccess ||
            (res->n_matches > 0 && (e = cudaMemcpyAsync(res->d_idx, p->idx, 4 * (size_t)res->n_matches,
                                                         cudaMemcpyDeviceToDevice, cs)) != cudaSuccess) ||
            (e = cudaStreamSynchronize(cs)) != cudaSuccess)
            rc = cuda_fail(e, "fp_plan_run: result copy");
    }
    if (rc != FP_OK) {
        fp_result_free(res);
        return rc;
    }
    *out = res;
    return FP_OK;
}

int fp_query_batched(fp_index *ix, const uint8_t *chars, const int64_t *offsets, int64_t n_queries,
                     const fp_batch *batches, int32_t n_batches, const fp_query_opts *opts, void *cuda_stream,
                     fp_result **out) {
    if (!ix || !offsets || !batches || !out || n_queries < 0 || n_batches < 1)
        return fail(FP_E_INVAL, "fp_query_batched: bad argument");
    int64_t total = 0;
    if (is_device_ptr(offsets)) {
        FP_CUDA(cudaMemcpy(&total, offsets + n_queries, 8, cudaMemcpyDeviceToHost));
    } else {
        FP_TRY(check_host_offsets(offsets, n_queries));
        total = offsets[n_queries];
    }
    fp_query_opts o{};
    if (opts) o = *opts;
    o.mode = FP_MODE_PLAIN;  // one-off: no graph
    fp_plan *p = nullptr;
    FP_TRY(fp_plan_create(ix, std::max<int64_t>(n_queries, 1), total, n_batches, &o, &p));
    int rc = fp_plan_run(p, chars, offsets, n_queries, batches, n_batches, cuda_stream, out);
    fp_plan_free(p);
    return rc;
}

}  // extern "C"
