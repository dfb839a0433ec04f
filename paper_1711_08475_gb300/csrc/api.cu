// C ABI: index construction, query pipeline, results and diagnostics.
//
// fp_query runs, in stream order and without host round trips until the end:
//   copy-in -> bucket the patterns by length and build their fingerprints
//   (Sec. 4: the query fingerprint is computed once) -> plan the tiles of
//   (query bucket, dictionary bucket) pairs -> filter by Eq. 1 -> verify the
//   survivors (Sec. 4) -> sort the matches into per-query ascending lists.
// One synchronisation at the end reads the counters; if a survivor or match
// buffer turned out too small, the filter, verify and emit stages run once
// more with exact sizes.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"

namespace fpk {

std::atomic<int64_t> g_launches{0};
static thread_local std::string t_err;

void set_error(const std::string &msg) { t_err = msg; }

int cuda_fail(cudaError_t e, const char *what) {
    cudaGetLastError();
    t_err = std::string(what) + ": " + cudaGetErrorName(e) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? FP_E_NOMEM : FP_E_CUDA;
}

// Keeps freed stream-ordered memory in the device pool instead of returning it
// at every synchronisation, so repeated queries reuse their buffers.
void init_pool() {
    static bool done = false;
    if (done) return;
    done = true;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
}

int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

int fail(int code, const std::string &msg) {
    t_err = msg;
    return code;
}

bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int bits_for(int64_t n) {  // bits to hold values 0 .. n-1 (at least 1)
    int b = 1;
    while (b < 63 && ((int64_t)1 << b) < n) b++;
    return b;
}

// Validates host offsets: offsets[0] == 0, non-decreasing, lengths <= 255.
int check_host_offsets(const int64_t *off, int64_t n) {
    if (off[0] != 0) return fail(FP_E_INVAL, "offsets[0] must be 0");
    for (int64_t i = 0; i < n; i++) {
        int64_t L = off[i + 1] - off[i];
        if (L < 0) return fail(FP_E_INVAL, "offsets must be non-decreasing");
        if (L > MAX_LEN) return fail(FP_E_INVAL, "string longer than 255 bytes");
    }
    return FP_OK;
}

// Device copies of a (chars, offsets) list given from either side.
struct DevStrings {
    const uint8_t *chars = nullptr;
    const int64_t *off = nullptr;
    uint8_t *own_chars = nullptr;
    int64_t *own_off = nullptr;
    int64_t total = 0;
    std::vector<int64_t> host_len_hist;  // lengths histogram when the host saw the offsets
    bool host_checked = false;
    void release(cudaStream_t st) {
        if (own_chars) cudaFreeAsync(own_chars, st);
        if (own_off) cudaFreeAsync(own_off, st);
        own_chars = nullptr;
        own_off = nullptr;
    }
};

static int stage_strings(const uint8_t *chars, const int64_t *off, int64_t n, cudaStream_t st, DevStrings *S) {
    const bool dev_off = is_device_ptr(off);
    if (!dev_off) {
        FP_TRY(check_host_offsets(off, n));
        S->total = off[n];
        S->host_checked = true;
        S->host_len_hist.assign(256, 0);
        for (int64_t i = 0; i < n; i++) S->host_len_hist[off[i + 1] - off[i]]++;
        FP_CUDA(cudaMallocAsync((void **)&S->own_off, sizeof(int64_t) * (size_t)(n + 1), st));
        FP_CUDA(cudaMemcpyAsync(S->own_off, off, sizeof(int64_t) * (size_t)(n + 1), cudaMemcpyHostToDevice, st));
        S->off = S->own_off;
    } else {
        int64_t ends[2];
        FP_CUDA(cudaMemcpyAsync(&ends[0], off, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        FP_CUDA(cudaMemcpyAsync(&ends[1], off + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        FP_CUDA(cudaStreamSynchronize(st));
        if (ends[0] < 0 || ends[1] < ends[0]) return fail(FP_E_INVAL, "offsets must be non-decreasing");
        S->total = ends[1];
        S->off = off;
    }
    if (S->total > 0 && !chars) return fail(FP_E_INVAL, "chars is null");
    if (S->total > 0 && !is_device_ptr(chars)) {
        FP_CUDA(cudaMallocAsync((void **)&S->own_chars, (size_t)S->total + 16, st));
        FP_CUDA(cudaMemcpyAsync(S->own_chars, chars, (size_t)S->total, cudaMemcpyHostToDevice, st));
        S->chars = S->own_chars;
    } else if (S->total == 0) {
        FP_CUDA(cudaMallocAsync((void **)&S->own_chars, 16, st));
        S->chars = S->own_chars;
    } else {
        S->chars = chars;
    }
    return FP_OK;
}

}  // namespace fpk

using namespace fpk;


namespace fpk {

// Pinned host memory for copying match lists back: blocks are sized in powers
// of two from 64 KB, and freed blocks are kept (up to 1 GB in total) for the
// next result, so a result is copied at pinned-memory speed without a
// cudaMallocHost per result.
namespace {
std::mutex g_pin_mu;
std::vector<std::pair<size_t, void *>> g_pin_free;
size_t g_pin_kept = 0;
constexpr size_t PIN_KEEP = size_t(1) << 30;
}  // namespace

void *pinned_get(size_t bytes, size_t *cap) {
    size_t c = size_t(1) << 16;
    while (c < bytes) c <<= 1;
    {
        std::lock_guard<std::mutex> g(g_pin_mu);
        for (size_t i = 0; i < g_pin_free.size(); i++)
            if (g_pin_free[i].first == c) {
                void *p = g_pin_free[i].second;
                g_pin_free.erase(g_pin_free.begin() + (long)i);
                g_pin_kept -= c;
                *cap = c;
                return p;
            }
    }
    void *p = nullptr;
    if (cudaMallocHost(&p, c) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    *cap = c;
    return p;
}

void pinned_put(void *p, size_t cap) {
    if (!p) return;
    {
        std::lock_guard<std::mutex> g(g_pin_mu);
        if (g_pin_kept + cap <= PIN_KEEP) {
            g_pin_free.emplace_back(cap, p);
            g_pin_kept += cap;
            return;
        }
    }
    cudaFreeHost(p);
}

}  // namespace fpk

extern "C" {

const char *fp_version(void) { return "fpmatch-gb300 1.0 (sm_103a)"; }

const char *fp_strerror(int code) {
    switch (code) {
        case FP_OK: return "ok";
        case FP_E_INVAL: return "invalid argument";
        case FP_E_UNSUPPORTED: return "unsupported fingerprint type / metric / layout";
        case FP_E_NOMEM: return "out of memory";
        case FP_E_CUDA: return "CUDA error";
        case FP_E_TIMEOUT: return "timed out";
        case FP_E_OVERFLOW: return "fixed-capacity buffer overflow";
    }
    return "unknown error";
}

const char *fp_last_error(void) { return t_err.c_str(); }

int64_t fp_launch_count(void) { return g_launches.load(); }

int fp_build(const uint8_t *chars, const int64_t *offsets, int64_t n_words, int type, int width_bits,
             const fp_build_opts *opts, void *cuda_stream, fp_index **out) {
    if (!out || !offsets || n_words < 0 || n_words > 0x7FFFFFFFLL) return fail(FP_E_INVAL, "bad argument");
    *out = nullptr;
    init_pool();
    cudaStream_t st = (cudaStream_t)cuda_stream;
    fp_build_opts o{};
    if (opts) o = *opts;
    FpParams P;
    if (type == FP_QGRAM && (o.qgram < 0 || o.qgram > 3)) return fail(FP_E_UNSUPPORTED, "q-grams: q must be 1..3");
    int rc = make_params(type, width_bits, o.count_bits, o.pos_bits, &P, o.qgram);
    if (rc != FP_OK) return fail(rc, "fingerprint type / width / b / p not supported");
    if (o.set < FP_SET_COMMON || o.set > FP_SET_CUSTOM) return fail(FP_E_INVAL, "bad symbol set");
    if (type == FP_QGRAM && o.set != FP_SET_COMMON)
        return fail(FP_E_UNSUPPORTED, "q-gram fingerprints take the most frequent q-grams only");
    if (o.combined != 0 && o.combined != 1) return fail(FP_E_INVAL, "combined must be 0 or 1");
    if (o.combined && (type != FP_COUNT || width_bits != 32))
        return fail(FP_E_UNSUPPORTED, "combined types: count fingerprints of 32 bits only");
    if (o.set == FP_SET_CUSTOM) {
        if (!o.custom_map) return fail(FP_E_INVAL, "custom map is null");
        for (int c = 0; c < 256; c++)
            if (o.custom_map[c] < -1 || o.custom_map[c] >= P.sigma)
                return fail(FP_E_INVAL, "custom map field out of range");
    }
    fp_index *ix = new fp_index();
    ix->P = P;
    ix->set = o.set;
    ix->n_words = n_words;
    ix->idx_bits = bits_for(n_words);
    DevStrings S;
    int32_t *d_err = nullptr;
    int32_t h_err = 0;
    rc = stage_strings(chars, offsets, n_words, st, &S);
    if (rc != FP_OK) goto fail_out;
    if (cudaMalloc((void **)&ix->d_map, 256) != cudaSuccess ||
        cudaMalloc((void **)&ix->d_counts, 256 * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMallocAsync((void **)&d_err, sizeof(int32_t), st) != cudaSuccess) {
        rc = cuda_fail(cudaErrorMemoryAllocation, "index allocation");
        goto fail_out;
    }
    if (cudaMemsetAsync(d_err, 0, sizeof(int32_t), st) != cudaSuccess) {
        rc = cuda_fail(cudaGetLastError(), "cudaMemsetAsync");
        goto fail_out;
    }
    if (type == FP_QGRAM) {  // fields are q-grams: no symbol map, a q-gram table instead
        if (S.total > (int64_t)0xFFFFFFFFLL) {
            rc = fail(FP_E_UNSUPPORTED, "q-gram fingerprints: at most 2^32 - 1 dictionary bytes");
            goto fail_out;
        }
        memset(ix->h_map, 0xFF, 256);
        if (cudaMemsetAsync(ix->d_map, 0xFF, 256, st) != cudaSuccess ||
            cudaMemsetAsync(ix->d_counts, 0, 256 * sizeof(unsigned long long), st) != cudaSuccess ||
            cudaMalloc((void **)&ix->d_gmap, (size_t)1 << (8 * P.q)) != cudaSuccess) {
            rc = cuda_fail(cudaErrorMemoryAllocation, "q-gram table");
            goto fail_out;
        }
        rc = qgram_map(S.chars, S.off, n_words, P.q, P.sigma, ix->d_gmap, ix->h_gram, &ix->n_grams, st);
        if (rc != FP_OK) goto fail_out;
        P.gmap = ix->d_gmap;
        ix->P = P;
    } else if (o.set == FP_SET_CUSTOM) {
        memcpy(ix->h_map, o.custom_map, 256);
        if (cudaMemcpy(ix->d_map, ix->h_map, 256, cudaMemcpyHostToDevice) != cudaSuccess) {
            rc = cuda_fail(cudaGetLastError(), "map copy");
            goto fail_out;
        }
        cudaMemsetAsync(ix->d_counts, 0, 256 * sizeof(unsigned long long), st);
    } else {
        rc = symbol_map(S.chars, S.total, o.set, P.sigma, ix->d_map, ix->d_counts, st);
        if (rc != FP_OK) goto fail_out;
    }
    rc = bucketize(S.chars, S.off, n_words, S.total, nullptr, 1, ix->d_map, P, false, st, &ix->D, d_err);
    if (rc != FP_OK) goto fail_out;
    if (banded_type(P.type)) {  // weight order of every bucket (population-count fingerprints)
        if (cudaMalloc((void **)&ix->d_wstart, sizeof(int32_t) * 256 * (size_t)(cell_count(P.width) + 1)) !=
            cudaSuccess) {
            rc = cuda_fail(cudaGetLastError(), "weight table");
            goto fail_out;
        }
        rc = weight_order(&ix->D, P, ix->d_wstart, st);
        if (rc != FP_OK) goto fail_out;
    }
    if (o.combined) {  // the second fingerprint: occurrence over the 32 most frequent symbols
        if (cudaMalloc((void **)&ix->d_map2, 256) != cudaSuccess) {
            rc = cuda_fail(cudaGetLastError(), "second map");
            goto fail_out;
        }
        if ((rc = make_params(FP_OCC, 32, 0, 0, &ix->P2)) != FP_OK ||
            (rc = symbol_map(S.chars, S.total, FP_SET_COMMON, ix->P2.sigma, ix->d_map2, ix->d_counts, st)) != FP_OK ||
            (rc = second_fingerprints(&ix->D, ix->d_map2, ix->P2, st)) != FP_OK)
            goto fail_out;
        if (cudaMemcpyAsync(ix->h_map2, ix->d_map2, 256, cudaMemcpyDeviceToHost, st) != cudaSuccess) {
            rc = cuda_fail(cudaGetLastError(), "second map copy");
            goto fail_out;
        }
    }
    {
        cudaError_t e;
        if ((e = cudaMemcpyAsync(ix->h_count, ix->D.b_count, sizeof(ix->h_count), cudaMemcpyDeviceToHost, st)) !=
                cudaSuccess ||
            (e = cudaMemcpyAsync(ix->h_start, ix->D.b_start, sizeof(ix->h_start), cudaMemcpyDeviceToHost, st)) !=
                cudaSuccess ||
            (e = cudaMemcpyAsync(&h_err, d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess) {
            rc = cuda_fail(e, "fp_build");
            goto fail_out;
        }
        if (o.set != FP_SET_CUSTOM && type != FP_QGRAM &&
            cudaMemcpy(ix->h_map, ix->d_map, 256, cudaMemcpyDeviceToHost) != cudaSuccess) {
            rc = cuda_fail(cudaGetLastError(), "map copy");
            goto fail_out;
        }
    }
    if (h_err) {
        rc = fail(FP_E_INVAL, "string longer than 255 bytes or offsets not monotone");
        goto fail_out;
    }
    ix->device_bytes = ix->D.n_slots * (4 + 1 + 4) + (ix->D.n_slots + FP_SLACK_SLOTS) * (P.width / 8) +
                       ix->D.str_bytes + STR_SLACK + 256 * 9 + (ix->D.fp2 ? (ix->D.n_slots + FP_SLACK_SLOTS) * 4 + 256 : 0) +
                       (ix->d_wstart ? 256 * 4 * (int64_t)(cell_count(P.width) + 1) : 0) +
                       (ix->d_gmap ? (int64_t)1 << (8 * P.q) : 0);
    S.release(st);
    cudaFreeAsync(d_err, st);
    cudaStreamSynchronize(st);
    *out = ix;
    return FP_OK;
fail_out:
    S.release(st);
    if (d_err) cudaFreeAsync(d_err, st);
    cudaStreamSynchronize(st);
    fp_free(ix);
    return rc;
}

void fp_free(fp_index *ix) {
    if (!ix) return;
    free_bucketed(&ix->D, 0);
    if (ix->d_map) cudaFree(ix->d_map);
    if (ix->d_counts) cudaFree(ix->d_counts);
    if (ix->d_wstart) cudaFree(ix->d_wstart);
    if (ix->d_map2) cudaFree(ix->d_map2);
    if (ix->d_gmap) cudaFree(ix->d_gmap);
    delete ix;
}

int fp_index_info_get(const fp_index *ix, fp_index_info *info) {
    if (!ix || !info) return fail(FP_E_INVAL, "null argument");
    memset(info, 0, sizeof(*info));
    info->n_words = ix->n_words;
    info->type = ix->P.type;
    info->width_bits = ix->P.width;
    info->count_bits = ix->P.b;
    info->pos_bits = ix->P.p;
    info->n_pos = ix->P.n_pos;
    info->sigma = ix->P.sigma;
    for (int L = 0; L < 256; L++) info->bucket_count[L] = ix->h_count[L];
    info->device_bytes = ix->device_bytes;
    info->qgram = ix->P.q;
    info->combined = ix->d_map2 != nullptr;
    return FP_OK;
}

int fp_index_qgrams(const fp_index *ix, uint8_t *grams_out, int32_t *n_grams, int32_t *q) {
    if (!ix || !grams_out || !n_grams || !q) return fail(FP_E_INVAL, "null argument");
    if (ix->P.type != FP_QGRAM) return fail(FP_E_UNSUPPORTED, "not a q-gram index");
    *q = ix->P.q;
    *n_grams = ix->n_grams;
    for (int f = 0; f < ix->n_grams; f++)
        for (int j = 0; j < ix->P.q; j++) grams_out[f * ix->P.q + j] = (uint8_t)(ix->h_gram[f] >> (8 * (ix->P.q - 1 - j)));
    return FP_OK;
}

int fp_index_map(const fp_index *ix, int8_t *map_out) {
    if (!ix || !map_out) return fail(FP_E_INVAL, "null argument");
    memcpy(map_out, ix->h_map, 256);
    return FP_OK;
}

int fp_set_symbol_map(fp_index *ix, const int8_t *map) {
    if (!ix || !map) return fail(FP_E_INVAL, "null argument");
    if (ix->P.type == FP_QGRAM) return fail(FP_E_UNSUPPORTED, "the fields of a q-gram index are q-grams");
    for (int c = 0; c < 256; c++)
        if (map[c] < -1 || map[c] >= ix->P.sigma) return fail(FP_E_INVAL, "map field out of range");
    memcpy(ix->h_map, map, 256);
    FP_CUDA(cudaMemcpy(ix->d_map, ix->h_map, 256, cudaMemcpyHostToDevice));
    ix->set = FP_SET_CUSTOM;
    FP_TRY(refingerprint(&ix->D, ix->d_map, ix->P, 0));
    if (ix->d_wstart) FP_TRY(weight_order(&ix->D, ix->P, ix->d_wstart, 0));  // the weights changed with the map
    if (ix->d_map2) FP_TRY(second_fingerprints(&ix->D, ix->d_map2, ix->P2, 0));  // the slots moved
    FP_CUDA(cudaDeviceSynchronize());
    return FP_OK;
}

int fp_fingerprint(const fp_index *ix, const uint8_t *chars, const int64_t *offsets, int64_t n_strings,
                   uint32_t *out_fp, void *cuda_stream) {
    if (!ix || !offsets || !out_fp || n_strings < 0) return fail(FP_E_INVAL, "bad argument");
    if (n_strings == 0) return FP_OK;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    DevStrings S;
    FP_TRY(stage_strings(chars, offsets, n_strings, st, &S));
    const bool dev_out = is_device_ptr(out_fp);
    uint32_t *d_out = out_fp;
    if (!dev_out) FP_CUDA(cudaMallocAsync((void **)&d_out, sizeof(uint32_t) * (size_t)n_strings, st));
    int rc = fingerprint_list(S.chars, S.off, n_strings, ix->d_map, ix->P, d_out, st);
    if (rc == FP_OK && !dev_out) {
        cudaError_t e = cudaMemcpyAsync(out_fp, d_out, sizeof(uint32_t) * (size_t)n_strings,
                                        cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) rc = cuda_fail(e, "copy-out");
    }
    if (!dev_out) cudaFreeAsync(d_out, st);
    S.release(st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (rc == FP_OK && e != cudaSuccess) rc = cuda_fail(e, "fp_fingerprint");
    return rc;
}

// ---------------------------------------------------------------------------
// query
// ---------------------------------------------------------------------------

struct QueryRun {
    cudaEvent_t ev[6] = {};
    Bucketed Q;
    QueryPlan plan;
    int32_t *d_group = nullptr;  // [0] k  [1] metric
    int32_t *d_err = nullptr;
    uint64_t *surv = nullptr, *matches = nullptr;
    int64_t surv_cap = 0, match_cap = 0;
    uint8_t *plan_scratch = nullptr;
};

static void release_run(QueryRun &R, cudaStream_t st) {
    free_bucketed(&R.Q, st);
    if (R.plan.seg) cudaFreeAsync(R.plan.seg, st);
    if (R.plan.scal) cudaFreeAsync(R.plan.scal, st);
    if (R.plan_scratch) cudaFreeAsync(R.plan_scratch, st);
    if (R.d_group) cudaFreeAsync(R.d_group, st);
    if (R.d_err) cudaFreeAsync(R.d_err, st);
    if (R.surv) cudaFreeAsync(R.surv, st);
    if (R.matches) cudaFreeAsync(R.matches, st);
    for (auto &e : R.ev)
        if (e) cudaEventDestroy(e);
    R = QueryRun{};
}

static int64_t host_pairs(const fp_index *ix, const std::vector<int64_t> &qhist, int k, int metric) {
    int64_t pairs = 0;
    for (int n = 0; n < 256; n++) {
        if (!qhist[n]) continue;
        int lo = metric == FP_HAM ? n : std::max(0, n - k), hi = metric == FP_HAM ? n : std::min(255, n + k);
        for (int L = lo; L <= hi; L++) pairs += qhist[n] * (int64_t)ix->h_count[L];
    }
    return pairs;
}

int fp_query_ex(fp_index *ix, const uint8_t *chars, const int64_t *offsets, int64_t n_queries, int k, int metric,
                const fp_query_opts *opts, void *cuda_stream, fp_result **out) {
    if (!ix || !out || !offsets || n_queries < 0 || n_queries > 0x7FFFFFFFLL) return fail(FP_E_INVAL, "bad argument");
    *out = nullptr;
    if (k < 0 || k > 15) return fail(FP_E_INVAL, "k must be in 0..15");
    if (metric != FP_HAM && metric != FP_LEV) return fail(FP_E_INVAL, "bad metric");
    if (metric == FP_LEV && (ix->P.type == FP_OCC_HALVED || ix->P.type == FP_POS))
        return fail(FP_E_UNSUPPORTED, "occurrence-halved and position fingerprints bound only the Hamming distance");
    fp_query_opts o{};
    if (opts) o = *opts;
    if (o.mode != FP_MODE_TILED && o.mode != FP_MODE_PLAIN && o.mode != FP_MODE_FUSED)
        return fail(FP_E_UNSUPPORTED, "query mode not available");
    FilterCfg cfg{};
    cfg.mode = o.mode;
    // defaults from a sweep on the 1M-word English-like workload: 4 words per
    // thread; 64 queries per tile with weight bands (narrower cell ranges per
    // tile; measured against 96 .. 256), 256 without
    cfg.v = o.words_per_thread == 8 ? 8 : 4;
    cfg.tq = o.mode == FP_MODE_PLAIN
                 ? 1
                 : (o.tile_queries > 0 ? std::min(o.tile_queries, 256) : (ix->d_wstart != nullptr ? 64 : 256));
    cfg.k1mix = o.variant == 0 && k == 1;
    cfg.mma = o.variant == 2 && o.mode != FP_MODE_PLAIN;
    const bool fused = o.mode == FP_MODE_FUSED;
    if (fused) cfg.v = 4;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    init_pool();
    cudaGetLastError();  // launch checks below must not see an unrelated earlier error

    fp_result *res = new fp_result();
    res->n_queries = n_queries;
    res->stats.n_queries = n_queries;
    if (n_queries == 0) {
        res->h_row_ptr.assign(1, 0);
        res->host_ready = true;
        if (cudaMallocAsync((void **)&res->d_row_ptr, sizeof(int64_t), st) != cudaSuccess ||
            cudaMemsetAsync(res->d_row_ptr, 0, sizeof(int64_t), st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            fp_result_free(res);
            return cuda_fail(cudaErrorMemoryAllocation, "result");
        }
        *out = res;
        return FP_OK;
    }
    DevStrings S;
    QueryRun R;
    int rc = FP_OK;
    uint64_t scal[8] = {0};
    int32_t h_err = 0;
    const int q_bits = bits_for(n_queries), idx_bits = ix->idx_bits;
    int tq = 0, tw = 0;
    tile_shape(cfg, ix->P, &tq, &tw);
    const bool band = ix->d_wstart != nullptr && o.mode != FP_MODE_PLAIN;
    int64_t pairs_bound;
    cudaError_t e;
#define CK(call)                                 \
    do {                                         \
        if ((e = (call)) != cudaSuccess) {       \
            rc = cuda_fail(e, #call);            \
            goto done;                           \
        }                                        \
    } while (0)
#define TRY(call)                  \
    do {                           \
        if ((rc = (call)) != FP_OK) goto done; \
    } while (0)
    for (auto &ev : R.ev) CK(cudaEventCreate(&ev));
    CK(cudaEventRecord(R.ev[0], st));
    TRY(stage_strings(chars, offsets, n_queries, st, &S));
    CK(cudaMallocAsync((void **)&R.d_group, 2 * sizeof(int32_t), st));
    CK(cudaMallocAsync((void **)&R.d_err, sizeof(int32_t), st));
    {
        static thread_local int32_t hg[2];  // pageable; copied before the call returns
        hg[0] = k;
        hg[1] = metric;
        CK(cudaMemcpyAsync(R.d_group, hg, 2 * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    }
    CK(cudaMemsetAsync(R.d_err, 0, sizeof(int32_t), st));
    TRY(bucketize(S.chars, S.off, n_queries, S.total, nullptr, 1, ix->d_map, ix->P, true, st, &R.Q, R.d_err, band));
    if (ix->d_map2) TRY(second_fingerprints(&R.Q, ix->d_map2, ix->P2, st));  // combined types
    // weight bands: patterns in cell order; per tile of tq patterns and
    // dictionary bucket a few runs of cells (at most one per admissible
    // (x, y)); a plan that needs more than 32 per (tile, bucket) on average
    // falls back to whole buckets on the device (the plain scan tests every
    // pair)
    if (band) {
        R.plan.max_segments = (int)std::min<int64_t>(
            0x7FFFFFFF, ((n_queries + tq - 1) / tq + 256) * (metric == FP_HAM ? 1 : 2 * k + 1) * 32);
    } else {
        R.plan.max_segments = 256 * (2 * k + 1);
    }
    CK(cudaMallocAsync((void **)&R.plan.seg, sizeof(Segment) * (size_t)R.plan.max_segments, st));
    CK(cudaMallocAsync((void **)&R.plan.scal, 8 * sizeof(uint64_t), st));
    if (band) {  // the planner's scratch: one thread per tile of patterns
        const int64_t ucap = (n_queries + tq - 1) / tq + R.Q.nbins;
        CK(cudaMallocAsync((void **)&R.plan_scratch, plan_scratch_bytes(ucap, R.Q.nbins), st));
        plan_scratch_place(&R.plan, R.plan_scratch, ucap, R.Q.nbins);
    }
    TRY(plan_segments(R.Q, ix->D, R.d_group, R.d_group + 1, tq, tw, &R.plan, st, band ? ix->d_wstart : nullptr,
                      ix->P.width, ix->P.q));
    // survivor capacity: exact pair count when the host saw the lengths, else a bound
    if (S.host_checked) {
        pairs_bound = host_pairs(ix, S.host_len_hist, k, metric);
    } else {
        int64_t widest = 0;
        for (int n = 0; n < 256; n++) {
            std::vector<int64_t> h(256, 0);
            h[n] = 1;
            widest = std::max(widest, host_pairs(ix, h, k, metric));
        }
        pairs_bound = widest * n_queries;
    }
    // survivors are sized from the pass ratio seen on this index before (x1.5),
    // 1/64 of the pairs at first; a larger count reruns the pass with exact sizes
    R.surv_cap = std::max<int64_t>(
        1, std::min<int64_t>(pairs_bound, std::max<int64_t>(1 << 20, (int64_t)(pairs_bound * ix->surv_ratio * 1.5))));
    R.match_cap = std::max<int64_t>(1, std::min<int64_t>(R.surv_cap, std::max<int64_t>(1 << 20, n_queries * 64)));
    CK(cudaEventRecord(R.ev[1], st));
    if (fused) R.surv_cap = 1;  // the fused form keeps survivors on chip
    for (int attempt = 0; attempt < 2; attempt++) {
        CK(cudaMallocAsync((void **)&R.surv, sizeof(uint64_t) * (size_t)R.surv_cap, st));
        CK(cudaMallocAsync((void **)&R.matches, sizeof(uint64_t) * (size_t)R.match_cap, st));
        if (attempt > 0) {  // reset the tile counter and the survivor / match counters
            CK(cudaMemsetAsync(R.plan.scal + 3, 0, 3 * sizeof(uint64_t), st));
            CK(cudaEventRecord(R.ev[1], st));
        }
        if (fused) {
            TRY(launch_fused(R.Q, ix->D, R.plan, ix->P, cfg, idx_bits, R.matches, R.match_cap, st,
                             &res->stats.filter_launches));
            CK(cudaEventRecord(R.ev[2], st));
        } else {
            TRY(launch_filter(R.Q, ix->D, R.plan, ix->P, cfg, R.surv, R.surv_cap, st, &res->stats.filter_launches));
            CK(cudaEventRecord(R.ev[2], st));
            TRY(launch_verify(R.Q, ix->D, R.surv, R.plan.scal + 4, R.surv_cap, k, metric, idx_bits, R.matches,
                              R.plan.scal + 5, R.match_cap, st));
        }
        CK(cudaEventRecord(R.ev[3], st));
        // result buffers sized by the match capacity; the sort borrows the survivor buffer
        if (!res->d_row_ptr)
            CK(cudaMallocAsync((void **)&res->d_row_ptr, sizeof(int64_t) * (size_t)(n_queries + 1), st));
        if (res->d_idx) {
            cudaFreeAsync(res->d_idx, st);
            res->d_idx = nullptr;
        }
        CK(cudaMallocAsync((void **)&res->d_idx, sizeof(int32_t) * (size_t)R.match_cap, st));
        {
            uint64_t *tmp = R.surv;
            uint64_t *own_tmp = nullptr;
            if (R.surv_cap < R.match_cap) {
                CK(cudaMallocAsync((void **)&own_tmp, sizeof(uint64_t) * (size_t)R.match_cap, st));
                tmp = own_tmp;
            }
            // the sort reads min(match counter, capacity); a counter above the capacity
            // makes the whole pass run again with exact sizes
            TRY(build_csr(R.matches, tmp, R.plan.scal + 5, R.match_cap, q_bits, idx_bits, n_queries,
                          res->d_row_ptr, res->d_idx, st));
            if (own_tmp) cudaFreeAsync(own_tmp, st);
        }
        CK(cudaEventRecord(R.ev[4], st));
        CK(cudaMemcpyAsync(scal, R.plan.scal, sizeof(scal), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(&h_err, R.d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        CK(cudaEventRecord(R.ev[5], st));
        CK(cudaStreamSynchronize(st));
        if (h_err) {
            rc = fail(FP_E_INVAL, "string longer than 255 bytes or offsets not monotone");
            goto done;
        }
        if (scal[6]) {
            rc = fail(FP_E_NOMEM, "tile plan overflow");
            goto done;
        }
        if ((fused || (int64_t)scal[4] <= R.surv_cap) && (int64_t)scal[5] <= R.match_cap) break;
        // too small: redo filter, verify and emit with exact sizes.  After a
        // survivor overflow only part of the survivors were verified, so the
        // match count is a lower bound and the survivor count bounds it.
        cudaFreeAsync(R.surv, st);
        cudaFreeAsync(R.matches, st);
        R.surv = R.matches = nullptr;
        if (!fused && (int64_t)scal[4] > R.surv_cap) {
            R.surv_cap = std::max<int64_t>(1, (int64_t)scal[4]);
            R.match_cap = R.surv_cap;
        } else {
            R.match_cap = std::max<int64_t>(1, (int64_t)scal[5]);
        }
        if (attempt == 1) {
            rc = fail(FP_E_NOMEM, "survivor buffer sizing failed");
            goto done;
        }
    }
    res->n_matches = (int64_t)scal[5];
    res->stats.pairs = (int64_t)scal[2];
    res->stats.pairs_tested = (int64_t)scal[7];
    res->stats.survivors = (int64_t)scal[4];
    if (scal[2] > 0) ix->surv_ratio = std::max(1.0 / 4096.0, (double)scal[4] / (double)scal[2]);
    res->stats.matches = (int64_t)scal[5];
    if (cudaEventElapsedTime(&res->stats.ms_prepare, R.ev[0], R.ev[1]) != cudaSuccess ||
        cudaEventElapsedTime(&res->stats.ms_filter, R.ev[1], R.ev[2]) != cudaSuccess ||
        cudaEventElapsedTime(&res->stats.ms_verify, R.ev[2], R.ev[3]) != cudaSuccess ||
        cudaEventElapsedTime(&res->stats.ms_emit, R.ev[3], R.ev[4]) != cudaSuccess ||
        cudaEventElapsedTime(&res->stats.ms_total, R.ev[0], R.ev[5]) != cudaSuccess)
        cudaGetLastError();
done:
#undef CK
#undef TRY
    S.release(st);
    release_run(R, st);
    if (rc != FP_OK) {
        cudaStreamSynchronize(st);
        fp_result_free(res);
        return rc;
    }
    *out = res;
    return FP_OK;
}

int fp_query(fp_index *ix, const uint8_t *chars, const int64_t *offsets, int64_t n_queries, int k, int metric,
             void *cuda_stream, fp_result **out) {
    return fp_query_ex(ix, chars, offsets, n_queries, k, metric, nullptr, cuda_stream, out);
}

int fp_result_csr(fp_result *r, const int64_t **row_ptr, const int32_t **idx, int on_device) {
    if (!r || !row_ptr || !idx) return fail(FP_E_INVAL, "null argument");
    if (on_device) {
        if (!r->d_row_ptr) return fail(FP_E_INVAL, "this result is held in host memory only");
        *row_ptr = r->d_row_ptr;
        *idx = r->d_idx;
        return FP_OK;
    }
    if (!r->host_ready && !r->pin) {
        const size_t rb = sizeof(int64_t) * (size_t)(r->n_queries + 1);
        const size_t ib = sizeof(int32_t) * (size_t)std::max<int64_t>(r->n_matches, 1);
        size_t cap = 0;
        void *p = pinned_get(rb + ib, &cap);
        if (p) {  // one pinned block: row_ptr, then idx
            cudaError_t e = cudaMemcpy(p, r->d_row_ptr, rb, cudaMemcpyDeviceToHost);
            if (e == cudaSuccess && r->n_matches > 0)
                e = cudaMemcpy((uint8_t *)p + rb, r->d_idx, sizeof(int32_t) * (size_t)r->n_matches,
                               cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) {
                pinned_put(p, cap);
                return cuda_fail(e, "fp_result_csr");
            }
            r->pin = p;
            r->pin_cap = cap;
        } else {  // no pinned memory to be had: ordinary host memory
            r->h_row_ptr.resize((size_t)r->n_queries + 1);
            r->h_idx.resize((size_t)std::max<int64_t>(r->n_matches, 1));
            FP_CUDA(cudaMemcpy(r->h_row_ptr.data(), r->d_row_ptr, rb, cudaMemcpyDeviceToHost));
            if (r->n_matches > 0)
                FP_CUDA(cudaMemcpy(r->h_idx.data(), r->d_idx, sizeof(int32_t) * (size_t)r->n_matches,
                                   cudaMemcpyDeviceToHost));
            r->host_ready = true;
        }
    }
    if (r->pin) {
        *row_ptr = (const int64_t *)r->pin;
        *idx = (const int32_t *)((const uint8_t *)r->pin + sizeof(int64_t) * (size_t)(r->n_queries + 1));
    } else {
        *row_ptr = r->h_row_ptr.data();
        *idx = r->h_idx.data();
    }
    return FP_OK;
}

int fp_result_stats(const fp_result *r, fp_stats *s) {
    if (!r || !s) return fail(FP_E_INVAL, "null argument");
    *s = r->stats;
    return FP_OK;
}

void fp_result_free(fp_result *r) {
    if (!r) return;
    // result buffers come from the stream-ordered pool; the legacy stream orders
    // the release after all work on blocking streams
    if (r->d_row_ptr) cudaFreeAsync(r->d_row_ptr, 0);
    if (r->d_idx) cudaFreeAsync(r->d_idx, 0);
    pinned_put(r->pin, r->pin_cap);
    delete r;
}

}  // extern "C"
