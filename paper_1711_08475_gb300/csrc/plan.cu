// Query plans: the batched pipeline of pipe.cuh on plan-owned device
// buffers, captured once into a CUDA graph and replayed.
//
// A plan holds one arena sized for its largest run (max_queries patterns,
// max_chars bytes, max_batches batches, 32 distinct (k, metric) groups).
// fp_plan_run copies the inputs into it, then launches the pipeline:
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

#include "pipe.cuh"

using namespace fpk;

struct fp_plan {
    fp_index *ix = nullptr;
    PipeShape cap;  // largest run the arena holds (groups = MAX_GROUPS)
    FilterCfg cfg{};
    bool use_graph = true;
    cudaStream_t st = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};  // start, filter start, filter end, end
    uint8_t *arena = nullptr;
    Pipe pipe;
    int64_t *h_batch_start = nullptr;  // pinned staging
    int32_t *h_batch_group = nullptr;
    int32_t *h_group_km = nullptr;
    uint64_t *h_scal = nullptr;  // pinned: counters + error flag
    // captured graph and its shape
    cudaGraphExec_t exec = nullptr;
    int64_t shape[4] = {-1, -1, -1, -1};
    int64_t kernels_per_run = 0;
};

namespace fpk {

namespace {
size_t carve(size_t &off, size_t bytes) {
    const size_t at = off;
    off += (bytes + 255) & ~(size_t)255;
    return at;
}
}  // namespace

size_t pipe_layout(const PipeShape &s, uint8_t *base, Pipe *p) {
    const int64_t nbins = 256 * (int64_t)s.groups;
    const int64_t n = std::max<int64_t>(s.queries, 1);
    const int64_t slots = n + (int64_t)(SLOT_ALIGN - 1) * nbins;
    const int64_t strb = s.chars + 15 * n + STR_SLACK;
    const int64_t cap = std::max<int64_t>(s.match_cap, 1);
    const int64_t rh = 256 * (int64_t)std::max(radix_blocks(cap), radix_blocks(n));
    // segments: whole buckets need bins x 31 at most; weight bands about 40 per
    // tile of 64 patterns (three lengths, several runs of cells each) -- a
    // plan that needs more falls back to whole buckets on the device
    const int64_t seg_cap = std::min<int64_t>(0x7FFFFFFF, std::max<int64_t>(nbins * 31, (n / 64 + nbins) * 40));
    // the banded planner's scratch, for tiles of 32 patterns or more (smaller
    // tiles plan whole buckets)
    const int64_t units_cap = std::min<int64_t>(0x7FFFFFFF, n / 32 + nbins);
    size_t off = 0;
    const size_t o_chars = carve(off, (size_t)s.chars + 16), o_off = carve(off, 8 * (size_t)(n + 1)),
                 o_bs = carve(off, 8 * (size_t)(s.batches + 1)), o_bg = carve(off, 4 * (size_t)s.batches),
                 o_km = carve(off, 4 * 2 * MAX_GROUPS), o_grp = carve(off, 4 * (size_t)n),
                 o_qfp = carve(off, 4 * (size_t)(slots + FP_SLACK_SLOTS)), o_qfp2 = carve(off, 4 * (size_t)slots),
                 o_qidx = carve(off, 4 * (size_t)slots),
                 o_qlen = carve(off, (size_t)slots), o_qrow = carve(off, 4 * (size_t)slots),
                 o_qstr = carve(off, (size_t)strb), o_bst = carve(off, 4 * (size_t)nbins),
                 o_bct = carve(off, 4 * (size_t)nbins), o_k1 = carve(off, 8 * (size_t)n),
                 o_k2 = carve(off, 8 * (size_t)n), o_hist = carve(off, 4 * (size_t)nbins),
                 o_ust = carve(off, 4 * (size_t)nbins), o_s16 = carve(off, 8 * (size_t)nbins),
                 o_tot = carve(off, 16), o_seg = carve(off, sizeof(Segment) * (size_t)seg_cap),
                 o_pls = carve(off, plan_scratch_bytes(units_cap, (int)nbins)),
                 o_scal = carve(off, 8 * 8), o_err = carve(off, 4), o_row = carve(off, 8 * (size_t)(n + 1)),
                 o_m = carve(off, 8 * (size_t)cap), o_t = carve(off, 8 * (size_t)cap),
                 o_idx = carve(off, 4 * (size_t)cap), o_rh = carve(off, 4 * (size_t)rh);
    if (base && p) {
        p->d_chars = base + o_chars;
        p->d_off = (int64_t *)(base + o_off);
        p->d_batch_start = (int64_t *)(base + o_bs);
        p->d_batch_group = (int32_t *)(base + o_bg);
        p->d_group_km = (int32_t *)(base + o_km);
        p->d_group = (int32_t *)(base + o_grp);
        p->Q = Bucketed{};
        p->Q.fp = base + o_qfp;
        p->q_fp2 = (uint32_t *)(base + o_qfp2);
        p->Q.idx = (int32_t *)(base + o_qidx);
        p->Q.len = base + o_qlen;
        p->Q.row16 = (uint32_t *)(base + o_qrow);
        p->Q.str = base + o_qstr;
        p->Q.b_start = (int32_t *)(base + o_bst);
        p->Q.b_count = (int32_t *)(base + o_bct);
        p->S.keys = (uint64_t *)(base + o_k1);
        p->S.keys2 = (uint64_t *)(base + o_k2);
        p->S.hist = (int32_t *)(base + o_hist);
        p->S.ustart = (int32_t *)(base + o_ust);
        p->S.str16 = (int64_t *)(base + o_s16);
        p->S.tot = (int64_t *)(base + o_tot);
        p->S.radix_hist = (uint32_t *)(base + o_rh);
        p->qp.seg = (Segment *)(base + o_seg);
        p->seg_cap = (int32_t)seg_cap;
        plan_scratch_place(&p->qp, base + o_pls, units_cap, (int)nbins);
        p->qp.scal = (uint64_t *)(base + o_scal);
        p->d_err = (int32_t *)(base + o_err);
        p->row_ptr = (int64_t *)(base + o_row);
        p->match_cap = cap;
        p->matches = (uint64_t *)(base + o_m);
        p->tmp = (uint64_t *)(base + o_t);
        p->idx = (int32_t *)(base + o_idx);
    }
    return off;
}

int group_batches(const fp_index *ix, const fp_batch *batches, int n_batches, int64_t n_queries,
                  int64_t *batch_start, int32_t *batch_group, int32_t *group_km, int *n_groups) {
    int ng = 0;
    int64_t start = 0;
    for (int b = 0; b < n_batches; b++) {
        const fp_batch &B = batches[b];
        if (B.n_queries < 0 || B.k < 0 || B.k > 15 || (B.metric != FP_HAM && B.metric != FP_LEV))
            return fail(FP_E_INVAL, "bad batch (n_queries, k in 0..15, metric)");
        if (B.metric == FP_LEV && (ix->P.type == FP_OCC_HALVED || ix->P.type == FP_POS))
            return fail(FP_E_UNSUPPORTED, "occurrence-halved and position fingerprints bound only the Hamming distance");
        int g = 0;
        while (g < ng && !(group_km[g] == B.k && group_km[MAX_GROUPS + g] == B.metric)) g++;
        if (g == ng) {
            if (ng == MAX_GROUPS) return fail(FP_E_INVAL, "more than 32 distinct (k, metric) pairs in one run");
            group_km[g] = B.k;
            group_km[MAX_GROUPS + g] = B.metric;
            ng++;
        }
        batch_start[b] = start;
        batch_group[b] = g;
        start += B.n_queries;
    }
    batch_start[n_batches] = start;
    if (start != n_queries) return fail(FP_E_INVAL, "batch sizes do not add up to n_queries");
    *n_groups = ng;
    return FP_OK;
}

int pipe_enqueue(fp_index *ix, const FilterCfg &cfg, Pipe &p, int64_t n, int64_t total, int n_batches, int n_groups,
                 cudaStream_t st, uint64_t *h_scal, cudaEvent_t *ev) {
    const int nbins = 256 * n_groups;
    cudaGetLastError();  // launch checks below must not see an unrelated earlier error
    if (ev) FP_CUDA(cudaEventRecord(ev[0], st));
    FP_CUDA(cudaMemsetAsync(p.d_err, 0, sizeof(int32_t), st));
    FP_TRY(fill_groups(p.d_batch_start, p.d_batch_group, n_batches, p.d_group, st));
    // weight bands whenever the index has its cell table (not for position
    // fingerprints): patterns in cell order, tiles restricted to runs of cells
    const bool band = ix->d_wstart != nullptr;
    FP_TRY(bucketize_into(p.d_chars, p.d_off, n, total, p.d_group, n_groups, ix->d_map, ix->P, st, &p.Q, p.S,
                          p.d_err, band));
    // combined types (f3): the patterns' second fingerprints, so that the fused
    // kernel keeps a pair only if both fingerprints pass
    p.Q.fp2 = ix->d_map2 ? p.q_fp2 : nullptr;
    if (ix->d_map2) FP_TRY(second_fingerprints(&p.Q, ix->d_map2, ix->P2, st));
    p.qp.max_segments = p.seg_cap;
    int tq = 0, tw = 0;
    tile_shape(cfg, ix->P, &tq, &tw);
    FP_TRY(plan_segments(p.Q, ix->D, p.d_group_km, p.d_group_km + MAX_GROUPS, tq, tw, &p.qp, st,
                         band ? ix->d_wstart : nullptr, ix->P.width, ix->P.q));
    if (ev) FP_CUDA(cudaEventRecord(ev[1], st));
    FP_TRY(launch_fused(p.Q, ix->D, p.qp, ix->P, cfg, ix->idx_bits, p.matches, p.match_cap, st, nullptr));
    if (ev) FP_CUDA(cudaEventRecord(ev[2], st));
    FP_TRY(build_csr_into(p.matches, p.tmp, p.S.radix_hist, p.qp.scal + 5, p.match_cap, bits_for(n), ix->idx_bits,
                          n, p.row_ptr, p.idx, st));
    FP_CUDA(cudaMemcpyAsync(h_scal, p.qp.scal, 8 * sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    FP_CUDA(cudaMemcpyAsync(h_scal + 8, p.d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    if (ev) FP_CUDA(cudaEventRecord(ev[3], st));
    return FP_OK;
}

}  // namespace fpk

namespace {

// (Re)places the plan's arena for its capacity with `match_cap` matches.
int plan_arena(fp_plan *p, int64_t match_cap) {
    if (p->arena) cudaFree(p->arena);
    p->arena = nullptr;
    p->cap.match_cap = match_cap;
    const size_t bytes = pipe_layout(p->cap, nullptr, nullptr);
    FP_CUDA(cudaMalloc((void **)&p->arena, bytes));
    pipe_layout(p->cap, p->arena, &p->pipe);
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
    if (o.mode != FP_MODE_TILED && o.mode != FP_MODE_FUSED)
        return fail(FP_E_UNSUPPORTED, "fp_plan_create: plans run the fused pipeline (mode TILED or FUSED)");
    if (o.flags & ~FP_OPT_NO_GRAPH) return fail(FP_E_INVAL, "fp_plan_create: unknown flags");
    fp_plan *p = new fp_plan();
    p->ix = ix;
    p->cap.queries = max_queries;
    p->cap.chars = max_chars;
    p->cap.batches = max_batches;
    p->cap.groups = MAX_GROUPS;
    p->cfg.mode = FP_MODE_FUSED;
    p->cfg.v = 4;
    p->cfg.tq = o.tile_queries > 0 ? std::min(o.tile_queries, 256) : 256;
    p->cfg.k1mix = o.variant == 0;  // the kernel takes the mixed test only in k = 1 tiles
    p->cfg.mma = o.variant == 2;
    p->use_graph = !(o.flags & FP_OPT_NO_GRAPH);
    int rc = FP_OK;
    if (cudaStreamCreateWithFlags(&p->st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_out, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreate(&p->ev[0]) != cudaSuccess || cudaEventCreate(&p->ev[1]) != cudaSuccess ||
        cudaEventCreate(&p->ev[2]) != cudaSuccess || cudaEventCreate(&p->ev[3]) != cudaSuccess) {
        rc = cuda_fail(cudaGetLastError(), "fp_plan_create: stream / events");
    } else if (cudaMallocHost((void **)&p->h_batch_start, 8 * (size_t)(max_batches + 1)) != cudaSuccess ||
               cudaMallocHost((void **)&p->h_batch_group, 4 * (size_t)max_batches) != cudaSuccess ||
               cudaMallocHost((void **)&p->h_group_km, 4 * 2 * MAX_GROUPS) != cudaSuccess ||
               cudaMallocHost((void **)&p->h_scal, 16 * sizeof(uint64_t)) != cudaSuccess) {
        rc = cuda_fail(cudaErrorMemoryAllocation, "fp_plan_create: pinned staging");
    } else {
        rc = plan_arena(p, std::max<int64_t>(1 << 20, std::min<int64_t>(max_queries * 64, 1LL << 28)));
    }
    if (rc != FP_OK) {
        fp_plan_free(p);
        return rc;
    }
    *out = p;
    return FP_OK;
}

void fp_plan_free(fp_plan *p) {
    if (!p) return;
    if (p->st) cudaStreamSynchronize(p->st);
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->arena) cudaFree(p->arena);
    if (p->h_batch_start) cudaFreeHost(p->h_batch_start);
    if (p->h_batch_group) cudaFreeHost(p->h_batch_group);
    if (p->h_group_km) cudaFreeHost(p->h_group_km);
    if (p->h_scal) cudaFreeHost(p->h_scal);
    cudaEvent_t evs[] = {p->ev_in, p->ev_out, p->ev[0], p->ev[1], p->ev[2], p->ev[3]};
    for (cudaEvent_t e : evs)
        if (e) cudaEventDestroy(e);
    if (p->st) cudaStreamDestroy(p->st);
    delete p;
}

int fp_plan_run(fp_plan *p, const uint8_t *chars, const int64_t *offsets, int64_t n_queries, const fp_batch *batches,
                int32_t n_batches, void *cuda_stream, fp_result **out) {
    if (!p || !offsets || !batches || !out || n_queries < 0 || n_batches < 1) return fail(FP_E_INVAL, "fp_plan_run: bad argument");
    *out = nullptr;
    if (n_queries > p->cap.queries || n_batches > p->cap.batches)
        return fail(FP_E_INVAL, "fp_plan_run: more patterns or batches than the plan was made for");
    int n_groups = 0;
    FP_TRY(group_batches(p->ix, batches, n_batches, n_queries, p->h_batch_start, p->h_batch_group, p->h_group_km,
                         &n_groups));
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
    if (total > p->cap.chars) return fail(FP_E_INVAL, "fp_plan_run: more pattern bytes than the plan was made for");
    if (total > 0 && !chars) return fail(FP_E_INVAL, "chars is null");
    Pipe &P = p->pipe;
    FP_CUDA(cudaEventRecord(p->ev_in, cs));
    FP_CUDA(cudaStreamWaitEvent(p->st, p->ev_in, 0));
    FP_CUDA(cudaMemcpyAsync(P.d_off, offsets, 8 * (size_t)(n_queries + 1), cudaMemcpyDefault, p->st));
    if (total > 0) FP_CUDA(cudaMemcpyAsync(P.d_chars, chars, (size_t)total, cudaMemcpyDefault, p->st));
    FP_CUDA(cudaMemcpyAsync(P.d_batch_start, p->h_batch_start, 8 * (size_t)(n_batches + 1), cudaMemcpyHostToDevice,
                            p->st));
    FP_CUDA(cudaMemcpyAsync(P.d_batch_group, p->h_batch_group, 4 * (size_t)n_batches, cudaMemcpyHostToDevice, p->st));
    FP_CUDA(cudaMemcpyAsync(P.d_group_km, p->h_group_km, 4 * 2 * MAX_GROUPS, cudaMemcpyHostToDevice, p->st));

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
            rc = pipe_enqueue(p->ix, p->cfg, P, n_queries, total, n_batches, n_groups, p->st, p->h_scal, p->ev);
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
            if ((rc = pipe_enqueue(p->ix, p->cfg, P, n_queries, total, n_batches, n_groups, p->st, p->h_scal,
                                   p->ev)) != FP_OK)
                break;
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
        if ((int64_t)sc[5] <= P.match_cap) {
            res->n_matches = (int64_t)sc[5];
            res->stats.pairs = (int64_t)sc[2];
            res->stats.pairs_tested = (int64_t)sc[7];
            res->stats.survivors = (int64_t)sc[4];
            res->stats.matches = (int64_t)sc[5];
            res->stats.filter_launches = 1;
            // stage times from the events the pipeline records (left at 0 if the
            // runtime cannot time them); a failure here must not linger as the
            // thread's last error
            if (cudaEventElapsedTime(&res->stats.ms_filter, p->ev[1], p->ev[2]) != cudaSuccess ||
                cudaEventElapsedTime(&res->stats.ms_prepare, p->ev[0], p->ev[1]) != cudaSuccess ||
                cudaEventElapsedTime(&res->stats.ms_emit, p->ev[2], p->ev[3]) != cudaSuccess ||
                cudaEventElapsedTime(&res->stats.ms_total, p->ev[0], p->ev[3]) != cudaSuccess)
                cudaGetLastError();
            break;
        }
        // more matches than the buffer holds: re-place the arena for the exact
        // count (the graph refers to the old buffers, so it is dropped), copy the
        // inputs again and run once more
        if (attempt == 1) {
            rc = fail(FP_E_NOMEM, "match buffer sizing failed");
            break;
        }
        if (p->exec) {
            cudaGraphExecDestroy(p->exec);
            p->exec = nullptr;
            p->shape[0] = -1;
        }
        if ((rc = plan_arena(p, (int64_t)sc[5])) != FP_OK) break;
        cudaError_t ce;
        if ((ce = cudaMemcpyAsync(P.d_off, offsets, 8 * (size_t)(n_queries + 1), cudaMemcpyDefault, p->st)) !=
                cudaSuccess ||
            (total > 0 && (ce = cudaMemcpyAsync(P.d_chars, chars, (size_t)total, cudaMemcpyDefault, p->st)) !=
                              cudaSuccess) ||
            (ce = cudaMemcpyAsync(P.d_batch_start, p->h_batch_start, 8 * (size_t)(n_batches + 1),
                                  cudaMemcpyHostToDevice, p->st)) != cudaSuccess ||
            (ce = cudaMemcpyAsync(P.d_batch_group, p->h_batch_group, 4 * (size_t)n_batches, cudaMemcpyHostToDevice,
                                  p->st)) != cudaSuccess ||
            (ce = cudaMemcpyAsync(P.d_group_km, p->h_group_km, 4 * 2 * MAX_GROUPS, cudaMemcpyHostToDevice, p->st)) !=
                cudaSuccess) {
            rc = cuda_fail(ce, "fp_plan_run: input copy");
            break;
        }
    }
    if (rc == FP_OK) {
        // the result owns copies of the plan's output (ordered on the caller's stream)
        cudaError_t e;
        if ((e = cudaEventRecord(p->ev_out, p->st)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(cs, p->ev_out, 0)) != cudaSuccess ||
            (e = cudaMallocAsync((void **)&res->d_row_ptr, 8 * (size_t)(n_queries + 1), cs)) != cudaSuccess ||
            (e = cudaMallocAsync((void **)&res->d_idx, 4 * (size_t)std::max<int64_t>(res->n_matches, 1), cs)) !=
                cudaSuccess ||
            (e = cudaMemcpyAsync(res->d_row_ptr, P.row_ptr, 8 * (size_t)(n_queries + 1), cudaMemcpyDeviceToDevice,
                                 cs)) != cudaSuccess ||
            (res->n_matches > 0 && (e = cudaMemcpyAsync(res->d_idx, P.idx, 4 * (size_t)res->n_matches,
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
    o.mode = FP_MODE_FUSED;
    o.flags |= FP_OPT_NO_GRAPH;  // one-off: no graph
    fp_plan *p = nullptr;
    FP_TRY(fp_plan_create(ix, std::max<int64_t>(n_queries, 1), total, n_batches, &o, &p));
    int rc = fp_plan_run(p, chars, offsets, n_queries, batches, n_batches, cuda_stream, out);
    fp_plan_free(p);
    return rc;
}

}  // extern "C"
