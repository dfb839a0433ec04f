// The batched query pipeline on caller-placed device buffers, shared by the
// captured query plans and the serving loop.
//
// One pipeline run takes a batch of patterns split into batches of equal
// (k, metric), and leaves the sorted CSR of original dictionary indices per
// pattern:
//   per-pattern group ids -> bucketing by (group, length) + fingerprints
//   (Sec. 3.2) -> tile plan -> fused filter (Eq. 1) + verification (Sec. 4)
//   -> sorted CSR -> counters to pinned host memory.
// Every buffer of a run sits in one arena whose layout pipe_layout computes
// from the run's shape, so a run can be placed in a plan's long-lived
// allocation or in a stream-ordered allocation of exactly its size.
#pragma once

#include "common.cuh"

namespace fpk {

constexpr int MAX_GROUPS = 32;  // distinct (k, metric) pairs in one run

struct PipeShape {
    int64_t queries = 0;    // patterns (upper bound)
    int64_t chars = 0;      // pattern bytes (upper bound)
    int32_t batches = 1;    // batches (upper bound)
    int32_t groups = 1;     // distinct (k, metric) (upper bound, <= MAX_GROUPS)
    int64_t match_cap = 0;  // matches the output buffers hold
};

struct Pipe {
    uint8_t *d_chars = nullptr;
    int64_t *d_off = nullptr;
    int64_t *d_batch_start = nullptr;  // [batches + 1]
    int32_t *d_batch_group = nullptr;  // [batches]
    int32_t *d_group_km = nullptr;     // [2 * MAX_GROUPS]: k of each group, then its metric
    int32_t *d_group = nullptr;        // [queries]
    Bucketed Q;
    uint32_t *q_fp2 = nullptr;  // second fingerprints of the patterns (combined-type indexes)
    BucketScratch S{};
    QueryPlan qp;
    int32_t seg_cap = 0;  // segments the arena holds
    int32_t *d_err = nullptr;
    int64_t match_cap = 0;
    uint64_t *matches = nullptr, *tmp = nullptr;
    int64_t *row_ptr = nullptr;  // [queries + 1]
    int32_t *idx = nullptr;      // [match_cap]
};

// Bytes of an arena for runs up to `s`; with base != nullptr (256-byte
// aligned, that many bytes) also points every buffer of *p into it.
size_t pipe_layout(const PipeShape &s, uint8_t *base, Pipe *p);

// Host side of a batch table: batch starts, the group of each batch, and the
// (k, metric) of each group (k in group_km[g], metric in group_km[MAX_GROUPS + g]).
// Validates k (0..15), the metric, and the metric against the index's type.
int group_batches(const fp_index *ix, const fp_batch *batches, int n_batches, int64_t n_queries,
                  int64_t *batch_start, int32_t *batch_group, int32_t *group_km, int *n_groups);

// Host counter block the pipeline copies back: [0..7] QueryPlan::scal
// ([2] pairs, [4] survivors, [5] matches, [6] tile-plan overflow) and the
// input error flag as the first int32 of word 8.
constexpr int PIPE_SCAL_WORDS = 9;

// Enqueues one run on st.  The inputs (d_chars, d_off, the batch table) must
// already be in the arena, ordered before on st.  ev (optional, 4 events) get
// recorded at: start, filter start, filter end, end.
int pipe_enqueue(fp_index *ix, const FilterCfg &cfg, Pipe &p, int64_t n, int64_t total, int n_batches, int n_groups,
                 cudaStream_t st, uint64_t *h_scal, cudaEvent_t *ev);

}  // namespace fpk
