// Autotuner for the tile shape of the filter (queries per block, dictionary
// fingerprints per thread) and the k = 1 test variant.  It times every
// candidate on a sample of the caller's patterns with the library's own
// stage events and returns the fastest; the results of a candidate are
// checked against the first candidate's so a shape can never change the
// answer.  No paper counterpart (the paper scans one pattern at a time).
#include <string.h>

#include <vector>

#include "common.cuh"

extern "C" int fp_autotune(fp_index *ix, const uint8_t *chars, const int64_t *offsets, int64_t n_queries, int k,
                           int metric, int mode, int reps, void *cuda_stream, fp_tune_result *best,
                           fp_tune_result *all, int32_t max_all, int32_t *n_all) {
    if (!ix || !offsets || !best || n_queries < 1 || reps < 1 || (mode != FP_MODE_TILED && mode != FP_MODE_FUSED))
        return fpk::fail(FP_E_INVAL, "fp_autotune: bad argument");
    struct Cand {
        int tq, v, variant;
    };
    std::vector<Cand> cands;
    const int tqs[] = {32, 64, 128, 256};
    const int vs[] = {4, 8};
    for (int variant = 0; variant < (k == 1 ? 2 : 1); variant++)
        for (int tq : tqs)
            for (int v : vs) {
                if (mode == FP_MODE_FUSED && v != 4) continue;
                cands.push_back({tq, v, variant});
            }
    int count = 0;
    std::vector<int64_t> ref_rp;
    std::vector<int32_t> ref_idx;
    best->ms = 1e30f;
    for (const Cand &c : cands) {
        fp_query_opts o{};
        o.mode = mode;
        o.tile_queries = c.tq;
        o.words_per_thread = c.v;
        o.variant = c.variant;
        float t = 1e30f;
        for (int r = 0; r < reps + 1; r++) {  // the first run warms the caches and is not counted
            fp_result *res = nullptr;
            int rc = fp_query_ex(ix, chars, offsets, n_queries, k, metric, &o, cuda_stream, &res);
            if (rc != FP_OK) return rc;
            fp_stats s;
            fp_result_stats(res, &s);
            const float ms = s.ms_filter + s.ms_verify;
            if (r > 0 && ms < t) t = ms;
            if (r == 0) {
                const int64_t *rp;
                const int32_t *ix_;
                rc = fp_result_csr(res, &rp, &ix_, 0);
                if (rc != FP_OK) {
                    fp_result_free(res);
                    return rc;
                }
                if (ref_rp.empty()) {
                    ref_rp.assign(rp, rp + n_queries + 1);
                    ref_idx.assign(ix_, ix_ + rp[n_queries]);
                } else if (memcmp(ref_rp.data(), rp, sizeof(int64_t) * (n_queries + 1)) != 0 ||
                           (rp[n_queries] > 0 &&
                            memcmp(ref_idx.data(), ix_, sizeof(int32_t) * (size_t)rp[n_queries]) != 0)) {
                    fp_result_free(res);
                    return fpk::fail(FP_E_CUDA, "fp_autotune: a tile shape changed the match lists");
                }
            }
            fp_result_free(res);
        }
        fp_tune_result tr{c.tq, c.v, c.variant, mode, t};
        if (all && count < max_all) all[count] = tr;
        count++;
        if (t < best->ms) *best = tr;
    }
    if (n_all) *n_all = count;
    return FP_OK;
}
