/*
 * fp.h -- C ABI of the GB300 fingerprint-filtered keyword matcher.
 *
 * Method: Cislak and Grabowski, "Lightweight Fingerprints for Fast Approximate
 * Keyword Matching Using Bitwise Operations" (arXiv 1711.08475).  A pattern P
 * is compared with every string of a collection D = [S_1 .. S_|D|] (Sec. 1,
 * keyword / dictionary matching) and every index i with D(P, S_i) <= k is
 * reported, D being the Hamming or the Levenshtein distance (Sec. 1).  Each
 * string carries a fixed-size fingerprint (Sec. 3); a pair is rejected
 * without looking at the strings when ceil(F_D / 2) > k (Eq. 1, Sec. 3.3), and
 * only the remaining pairs are verified explicitly (Sec. 3, Sec. 4).
 *
 * All entry points return 0 (FP_OK) or a negative error code; none aborts or
 * traps.  fp_strerror() describes a code; fp_last_error() gives the text of
 * the most recent failure on the calling thread (including the CUDA error
 * string for FP_E_CUDA).  Strings are byte arrays with explicit lengths given
 * by CSR offsets (string i is chars[offsets[i] .. offsets[i+1]) ); they are
 * not NUL-terminated and may contain any byte.  Lengths must be 0..255.
 *
 * Pointers: "host" arguments are ordinary CPU memory (pinned memory makes the
 * copies asynchronous); "host or device" arguments are accepted from either
 * side, the library asks the CUDA runtime which one it is.  The caller keeps
 * ownership of every input; the library copies what it needs before the call
 * returns.  Objects returned through an out-pointer are owned by the library
 * until the matching *_free call.
 *
 * Streams: cuda_stream is a cudaStream_t (NULL = the legacy default stream).
 * Device work of a call is ordered on that stream.
 */
#ifndef FP_H
#define FP_H

#include <stdint.h>

#if defined(__GNUC__)
#define FP_API __attribute__((visibility("default")))
#else
#define FP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------- */
#define FP_OK 0
#define FP_E_INVAL (-1)       /* null pointer, bad size, width, k, length > 255, offsets not monotone */
#define FP_E_UNSUPPORTED (-2) /* a (fingerprint type, metric) pair the bound does not hold for, or a layout that does not fit the width */
#define FP_E_NOMEM (-3)       /* a device or host allocation failed */
#define FP_E_CUDA (-4)        /* a CUDA runtime call failed; fp_last_error() has the CUDA message */
#define FP_E_TIMEOUT (-5)     /* a bounded wait ran out (serving loop) */
#define FP_E_OVERFLOW (-6)    /* a fixed-capacity buffer (captured plan) was too small; counts are still exact */

/* ---- fingerprint types (Sec. 3) ----------------------------------------- */
/* FP_OCC: bit q set iff a symbol mapped to q occurs (Sec. 3, "Occurrence").
 * FP_OCC_HALVED: occurrence in S[0, floor(n/2)) at bit 2q and in the rest at
 *   bit 2q+1 (Sec. 3, "Occurrence halved"); sound for Hamming only.
 * FP_COUNT: saturating count min(c, 2^b - 1) of the symbols mapped to q in
 *   bits [b q, b q + b) (Sec. 3, "Count").  Stored reflected-Gray coded: with
 *   the paper's plain binary code one edit can change F_D by 3 or 4 (aa vs ab,
 *   aab vs abb), which breaks Theorem 1; with a Gray code every +-1 step of a
 *   counter flips one bit, so Theorem 1 and Eq. 1 hold.
 * FP_POS: 0-indexed first position of the symbol mapped to field j,
 *   saturated at 2^p - 1 (also meaning absent), in bits [p j, p j + p); the
 *   leftover W mod p bits are occurrence bits (Sec. 3, "Position");
 *   Hamming only (Theorem 2).
 * FP_QGRAM: occurrence of q-grams, the paper's future work (Sec. 5): the W
 *   most frequent q-grams of the dictionary (occurrences over all positions;
 *   ties go to the smaller q-gram in byte order) each own one bit, set iff
 *   the q-gram occurs in the string; strings shorter than q get 0.  One edit
 *   touches at most q q-grams on each side, so F_D grows by at most 2q per
 *   edit and D >= ceil(F_D / 2q): a pair is rejected iff F_D > 2qk (Eq. 1 is
 *   q = 1).  Sound for Hamming and Levenshtein.  q = opts->qgram (1..3).
 * FP_COUNT_L1: the count fingerprint in the paper's own binary code
 *   (Sec. 3.2), compared by the distance of the counts themselves, F_D =
 *   sum over fields of |c1 - c2| (the remark after Eq. 1 in Sec. 3.3: the
 *   Hamming weight of the XOR under-counts, 3 (11) against 1 (01) gives 1
 *   instead of 2, and over-counts 1 (01) against 2 (10)).  One edit moves
 *   each of at most two counts by one, so Eq. 1 holds; F_D is never below
 *   the Gray-coded FP_COUNT distance.  b = 2 only.  Tested on every eligible pair (no
 *   weight bands: the weight of a binary count field is not bounded by the
 *   count difference across part boundaries). */
typedef enum { FP_OCC = 0, FP_OCC_HALVED = 1, FP_COUNT = 2, FP_POS = 3, FP_QGRAM = 4, FP_COUNT_L1 = 5 } fp_type;

/* Distances of Sec. 1. */
typedef enum { FP_HAM = 0, FP_LEV = 1 } fp_metric;

/* Symbol sets of Sec. 3: most frequent, least frequent, half of each; or a
 * caller-given map (e.g. a learned one).  Frequencies are byte counts over
 * the whole dictionary; ties go to the smaller byte value. */
typedef enum { FP_SET_COMMON = 0, FP_SET_RARE = 1, FP_SET_MIXED = 2, FP_SET_CUSTOM = 3 } fp_symset;

typedef struct {
    int32_t set;               /* fp_symset; default FP_SET_COMMON */
    int32_t count_bits;        /* b for FP_COUNT, 1..8; 0 = default 2 (Sec. 4) */
    int32_t pos_bits;          /* p for FP_POS, 1..8; 0 = default 3 (Sec. 4) */
    int32_t combined;          /* 1: combined types (occurrence + count in 64 bits): every word and
                                  pattern also gets a 32-bit occurrence fingerprint over the 32 most
                                  frequent symbols, and a pair survives only if both fingerprints
                                  pass Eq. 1 (each is sound alone, Theorem 1).  FP_COUNT at 32 bits
                                  only; used by fp_query / fp_query_ex, batched runs and the server
                                  (fp_query_noalloc tests the count fingerprint alone).  0 = off */
    const int8_t *custom_map;  /* host, [256]: field of each byte value or -1; only for FP_SET_CUSTOM */
    int32_t qgram;             /* q for FP_QGRAM, 1..3; 0 = 2.  The set must be FP_SET_COMMON */
} fp_build_opts;

/* Query execution forms. */
typedef enum {
    FP_MODE_TILED = 0, /* query fingerprints of a tile staged in shared memory, dictionary fingerprints streamed once per tile */
    FP_MODE_PLAIN = 1, /* one query per warp, every dictionary fingerprint read once per query: the plain GPU scan */
    FP_MODE_FUSED = 2  /* tiled filter with verification done inside the same persistent kernel */
} fp_mode;

typedef struct {
    int32_t mode;            /* fp_mode; default FP_MODE_TILED */
    int32_t tile_queries;    /* queries per block for FP_MODE_TILED / FUSED, 1..256; 0 = default (64 with
                                weight bands, i.e. all but position fingerprints; 256 for those) */
    int32_t words_per_thread;/* dictionary fingerprints per thread per tile, 4 or 8; 0 = default */
    int32_t variant;         /* 0 = automatic (k = 1: a quarter of the pair tests use an ALU-only
                                "at most two bits" test, identical decisions); 1 = population count only;
                                2 = tensor cores for occ / occh / count fingerprints: with set bits as +1
                                and clear bits as -1 the dot product of two fingerprints is W - 2 F_D, so
                                FP8 MMA dot products decide Eq. 1 exactly (128 patterns x 1024 words per
                                tile; tile_queries and words_per_thread do not apply; position
                                fingerprints keep the population-count kernel) */
    int32_t flags;           /* FP_OPT_* bits; 0 = none */
} fp_query_opts;
/* fp_plan_create: run the pipeline launch by launch instead of capturing it
 * into a CUDA graph (for timing the stages, or where graphs are unwanted). */
#define FP_OPT_NO_GRAPH 1

typedef struct {
    int64_t n_queries;
    int64_t pairs;        /* eligible (query, word) pairs: equal length (Ham) or lengths within k (Lev) */
    int64_t survivors;    /* pairs not rejected by Eq. 1 */
    int64_t matches;      /* pairs with D <= k */
    int64_t filter_launches;
    float ms_prepare;     /* copy-in, bucketing, query fingerprints, tile plan */
    float ms_filter;      /* fingerprint filter kernel(s) */
    float ms_verify;      /* Hamming / Levenshtein verification */
    float ms_emit;        /* sort and CSR */
    float ms_total;       /* whole call on the device, copy-in included */
    int64_t pairs_tested; /* pairs the filter kernel tested: the eligible pairs less those whose
                             fingerprint weights differ by more than 2k (rejected by Eq. 1
                             without a test; see fp_build) */
} fp_stats;

typedef struct {
    int64_t n_words;
    int32_t type, width_bits, count_bits, pos_bits;
    int32_t n_pos;        /* position fields (FP_POS) */
    int32_t sigma;        /* tracked fields */
    int64_t bucket_count[256]; /* words per length */
    int64_t device_bytes; /* device memory held by the index */
    int32_t qgram;        /* q of FP_QGRAM (1 for the other types) */
    int32_t combined;     /* 1: combined types (fp_build_opts.combined) */
} fp_index_info;

typedef struct fp_index fp_index;
typedef struct fp_result fp_result;

/* ---- build (Sec. 3.2 construction, Sec. 3.4 storage) -------------------- */
/* Copies the dictionary to the device, buckets it by length, chooses the
 * symbol map (Sec. 3 symbol sets) and builds one fingerprint per word
 * (Sec. 3.2).  For occurrence, occurrence-halved and count fingerprints the
 * words of a bucket are then ordered by fingerprint weight (population count;
 * equal weights keep ascending index order) and the first word of every weight
 * is recorded: since popc(a ^ b) >= |popc(a) - popc(b)|, a query tile tests
 * only the words whose weight lies within 2k of its patterns' weights (Eq. 1
 * rejects the rest).  Position fingerprints keep index order.
 *   chars, offsets: host or device; offsets[0] == 0, non-decreasing,
 *     n_words + 1 entries, every length <= 255.
 *   type: fp_type; width_bits: 16 or 32.
 *   opts: NULL for defaults.
 * Errors: FP_E_INVAL (bad pointer/size/width/offsets/length),
 * FP_E_UNSUPPORTED (layout does not fit: b*1 > W, p*1 > W; FP_QGRAM with a
 * set other than FP_SET_COMMON, combined types or more than 2^32 - 1
 * dictionary bytes), FP_E_NOMEM,
 * FP_E_CUDA.  Synchronises cuda_stream before returning. */
FP_API int fp_build(const uint8_t *chars, const int64_t *offsets, int64_t n_words, int type, int width_bits,
             const fp_build_opts *opts, void *cuda_stream, fp_index **out);

/* ---- query (Sec. 3.3 comparison, Eq. 1, Sec. 4 verification) ------------ */
/* For every pattern q, the ascending original indices i with D(P_q, S_i) <= k
 * (Sec. 1).  The query fingerprint is built once per pattern (Sec. 4) and
 * compared with every word of equal length (Ham) or of length within k (Lev).
 *   chars, offsets: host or device, same rules as fp_build.
 *   k: 0..15; metric: fp_metric.
 *   opts: NULL for FP_MODE_TILED with the tuned tile.
 * FP_QGRAM indexes reject a pair iff F_D > 2qk; the other types use Eq. 1.
 * Errors: FP_E_INVAL, FP_E_UNSUPPORTED (FP_OCC_HALVED or FP_POS index with
 * FP_LEV: Eq. 1 does not hold for them), FP_E_NOMEM, FP_E_CUDA.
 * Synchronises cuda_stream once at the end (to size the result). */
FP_API int fp_query(fp_index *ix, const uint8_t *chars, const int64_t *offsets, int64_t n_queries, int k,
             int metric, void *cuda_stream, fp_result **out);
FP_API int fp_query_ex(fp_index *ix, const uint8_t *chars, const int64_t *offsets, int64_t n_queries, int k,
                int metric, const fp_query_opts *opts, void *cuda_stream, fp_result **out);

/* ---- learned symbol-to-bit map (occurrence fingerprints) ----------------- */
/* Sec. 3.2 builds a fingerprint through "a mapping c -> q" and Sec. 3 picks
 * the most frequent symbols.  For occurrence fingerprints Eq. 1 stays valid
 * for ANY map, also many-to-one (one substitution moves at most one symbol
 * out of and one into the set of fields a string touches), so a map can be
 * learned for rejection alone; the result is exact whatever the map.
 *
 * fp_sample_pairs: n_samples pairs drawn by the method from the index and
 * the given patterns (a uniform pattern, then a uniform eligible word: equal
 * length for Ham, length within k for Lev), with: original pattern and word
 * indices (int32, -1 when no eligible word exists), passed = the pair passes
 * Eq. 1 under the index's current map, match = D <= k (Sec. 4 verification),
 * masks = the printable symbols (0x20..0x7E, bit c - 0x20) of the pattern
 * (words 0-1) and of the word (words 2-3).  Outputs all host or all device.
 *
 * Model (FP32, project kernels): per printable symbol c, one-hot input ->
 * 64 ReLU units -> `fields` logits z_c; A_c = softmax(z_c / tau).  Soft
 * F_D = expected Hamming weight of the XOR when symbol c lands on field b
 * with probability A_c,b: sum_b prod_{c in P&W}(1 - A_c,b) (p_b + q_b -
 * 2 p_b q_b), p_b (q_b) = 1 - prod over the symbols only in the pattern
 * (word) of (1 - A_c,b); equal to F_D for one-hot A.  Loss = mean over
 * non-matching samples of softplus(beta (2k+1 - F))/beta.
 * Parameters (fp_mlp_param_count() floats): W1[64][95], b1[64], W2[32][64],
 * b2[32] (rows past `fields` unused).
 *
 * fp_mlp_loss_grad: one forward + backward on the GPU: *loss_sum = summed
 * loss, *n_used = non-matching samples, grad = mean gradient.  params, masks,
 * match, grad: host or device.
 *
 * fp_learn_map: Adam (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) over
 * epochs of mini-batches, tau annealed geometrically from tau0 (first epoch)
 * to tau1 (last; a single epoch uses tau1); map_out[256] (host) = argmax field per printable symbol,
 * -1 elsewhere; params_out (optional, host or device) = trained parameters;
 * loss_curve (optional, host) = mean loss per epoch.  Apply the map with
 * fp_set_symbol_map. */
typedef struct {
    int32_t epochs;  /* 0 = 12 */
    int32_t batch;   /* samples per step; 0 = 65536 */
    float lr;        /* 0 = 3e-3 */
    float tau0;      /* 0 = 1.0 */
    float tau1;      /* 0 = 0.1 */
    float beta;      /* 0 = 2.0 */
    uint64_t seed;   /* 0 = 1711 */
    const float *init_params; /* host or device, fp_mlp_param_count() floats: the starting parameters
                                 (NULL = seeded initialisation: W uniform in +-1/sqrt(fan-in), b = 0) */
} fp_learn_opts;
FP_API int fp_mlp_param_count(void);
FP_API int fp_sample_pairs(fp_index *ix, const uint8_t *chars, const int64_t *offsets, int64_t n_queries, int k,
                           int metric, int64_t n_samples, uint64_t seed, void *cuda_stream, int32_t *out_q,
                           int32_t *out_w, uint8_t *out_passed, uint8_t *out_match, uint64_t *out_masks);
FP_API int fp_mlp_loss_grad(const float *params, int fields, float tau, float beta, int k, const uint64_t *masks,
                            const uint8_t *match, int64_t n_samples, void *cuda_stream, double *loss_sum,
                            int64_t *n_used, float *grad);
FP_API int fp_learn_map(int fields, const uint64_t *masks, const uint8_t *match, int64_t n_samples, int k,
                        const fp_learn_opts *opts, void *cuda_stream, float *params_out, int8_t *map_out,
                        float *loss_curve);

/* ---- autotuner ----------------------------------------------------------- */
/* No paper counterpart.  Times every tile shape (queries per block 32..256,
 * 4 or 8 fingerprints per thread; for k = 1 also the population-count-only
 * variant) on the given sample of patterns, `reps` timed runs each after one
 * warm-up, using the library's stage events (filter + verification time),
 * and returns the fastest in *best (all candidates in all[0 .. *n_all) when
 * all is given).  Every candidate's match lists must equal the first one's,
 * else FP_E_CUDA.  mode: FP_MODE_TILED or FP_MODE_FUSED. */
typedef struct {
    int32_t tile_queries;
    int32_t words_per_thread;
    int32_t variant;
    int32_t mode;
    float ms;
} fp_tune_result;
FP_API int fp_autotune(fp_index *ix, const uint8_t *chars, const int64_t *offsets, int64_t n_queries, int k, int metric,
                       int mode, int reps, void *cuda_stream, fp_tune_result *best, fp_tune_result *all,
                       int32_t max_all, int32_t *n_all);

/* ---- batched queries and captured plans --------------------------------- */
/* The paper answers one pattern at a time (Sec. 4: the query fingerprint is
 * built once and compared with every word).  These entry points answer many
 * batches, each with its own k and metric, in one pass: patterns are bucketed
 * by (k, metric, length), and one persistent kernel filters (Eq. 1) and
 * verifies (Sec. 4) every tile of every batch.  Batches are consecutive
 * ranges of the pattern list (batch b covers the next batches[b].n_queries
 * patterns); the result is one CSR over all patterns in input order. */
typedef struct {
    int64_t n_queries;
    int32_t k;      /* 0..15 */
    int32_t metric; /* fp_metric */
} fp_batch;
typedef struct fp_plan fp_plan;

/* One-off batched query (no graph).  chars, offsets: host or device;
 * batches: host.  Errors as fp_query; FP_E_INVAL if the batch sizes do not
 * add up to n_queries.  Synchronises cuda_stream. */
FP_API int fp_query_batched(fp_index *ix, const uint8_t *chars, const int64_t *offsets, int64_t n_queries,
                            const fp_batch *batches, int32_t n_batches, const fp_query_opts *opts, void *cuda_stream,
                            fp_result **out);
/* A plan owns every device buffer for up to max_queries patterns of
 * max_chars bytes in max_batches batches (allocated here, once).  The first
 * fp_plan_run of a shape (patterns, bytes, batches, distinct (k, metric)
 * groups) records the device pipeline into a CUDA graph on the plan's own
 * stream; later runs of the same shape replay it with one graph launch.
 * opts: tile_queries and variant as for fp_query_ex; flags FP_OPT_NO_GRAPH
 * turns the graph off; mode must be FP_MODE_TILED or FP_MODE_FUSED (both mean
 * the fused pipeline; the plain scan is not a plan form, FP_E_UNSUPPORTED).
 * Runs of one plan must not overlap (one host thread at a time); results do
 * not refer to the plan's memory. */
FP_API int fp_plan_create(fp_index *ix, int64_t max_queries, int64_t max_chars, int32_t max_batches,
                          const fp_query_opts *opts, fp_plan **out);
FP_API int fp_plan_run(fp_plan *plan, const uint8_t *chars, const int64_t *offsets, int64_t n_queries,
                       const fp_batch *batches, int32_t n_batches, void *cuda_stream, fp_result **out);
FP_API void fp_plan_free(fp_plan *plan);

/* ---- serving loop: continuous batching over a resident dictionary ------- */
/* The paper answers one pattern at a time (Sec. 4); this server answers
 * requests (pattern batches, each with its own k and metric) that arrive
 * while others run.  fp_server_submit copies a request into host memory and
 * queues it.  A scheduler thread inside the server keeps up to `lanes`
 * launches in flight, each on its own CUDA stream: whenever a lane is free
 * it takes the oldest queued requests that fit one launch (max_requests,
 * max_queries, max_chars, at most 32 distinct (k, metric)) and whose device
 * footprint fits what is left of memory_budget (oldest first: a request
 * that does not fit waits, and so do the ones behind it), and runs them as
 * one batched launch (the pipeline of fp_plan_run) with its buffers in one
 * stream-ordered allocation of exactly the launch's size, released when the
 * launch's results are back in host memory.  Launches of different lanes
 * overlap on the device.  A request's match lists are the same whether it
 * runs alone or merged with others.
 * The index must outlive the server and must not be changed
 * (fp_set_symbol_map) while the server exists.  The functions may be called
 * from any thread. */
typedef struct fp_server fp_server;
typedef struct {
    int32_t lanes;          /* launches in flight at once; 0 = 4, at most 64 */
    int32_t max_requests;   /* requests merged into one launch; 0 = 64 */
    int64_t max_queries;    /* patterns in one launch (and in one request); 0 = 16384 */
    int64_t max_chars;      /* pattern bytes in one launch; 0 = 128 * max_queries */
    int64_t memory_budget;  /* device bytes the launches in flight may hold; 0 = a quarter of the free memory */
    int32_t tile_queries;   /* as fp_query_opts; 0 = 256 */
    int32_t variant;        /* as fp_query_opts */
} fp_server_opts;
typedef struct {
    int64_t submitted, completed, queries, launches, reruns; /* reruns: launches re-run with a larger match buffer */
    int64_t pairs, survivors, matches;                       /* summed over finished launches */
    int32_t max_lanes_busy;          /* most launches seen in flight at once */
    int32_t max_requests_per_launch; /* most requests merged into one launch */
    int64_t budget_bytes, peak_bytes, in_use_bytes; /* admitted device bytes: budget, peak, now */
    double p50_ms, p99_ms, mean_ms, max_ms;  /* submit -> result ready, over completed requests (nearest rank) */
    double mean_queue_ms;   /* submit -> admission, over admitted requests */
    double busy_seconds;    /* wall time with at least one launch in flight */
} fp_server_stats;
/* opts NULL = defaults.  Errors: FP_E_INVAL, FP_E_NOMEM (budget below one
 * single-pattern launch, pinned staging), FP_E_CUDA. */
FP_API int fp_server_create(fp_index *ix, const fp_server_opts *opts, fp_server **out);
/* chars, offsets: host (copied before the call returns); 1 <= n_queries <=
 * max_queries, offsets[n] <= max_chars.  Returns at once with the request's
 * id.  FP_E_INVAL (bad argument, device pointers, request larger than one
 * launch), FP_E_UNSUPPORTED (Lev on occurrence-halved / position
 * fingerprints), FP_E_NOMEM (the request alone exceeds the budget). */
FP_API int fp_server_submit(fp_server *s, const uint8_t *chars, const int64_t *offsets, int64_t n_queries, int k,
                            int metric, int64_t *request_id);
/* Waits at most timeout_us for the request; on FP_OK *out owns its match
 * lists (host memory: fp_result_csr with on_device = 0; stats.ms_total =
 * latency, stats.matches) and the id is forgotten.  FP_E_TIMEOUT leaves the
 * request pending (wait again later); another code is the launch's error. */
FP_API int fp_server_wait(fp_server *s, int64_t request_id, int64_t timeout_us, fp_result **out);
FP_API int fp_server_stats_get(fp_server *s, fp_server_stats *out);
/* Arrival-time driver: request r (patterns [sum of earlier sizes, + request_sizes[r])
 * of chars/offsets, host) is submitted arrival_us[r] microseconds (non-decreasing)
 * after the call starts, then every request is waited for (timeout_us in
 * total).  latency_ms (optional, host, [n_requests]) gets each request's
 * latency; *out the match lists of all patterns in order. */
FP_API int fp_server_replay(fp_server *s, const uint8_t *chars, const int64_t *offsets, const int64_t *request_sizes,
                            const int64_t *arrival_us, int64_t n_requests, int k, int metric, int64_t timeout_us,
                            double *latency_ms, fp_result **out);
/* Finishes every queued and running request, then frees the server (results
 * not waited for are dropped). */
FP_API void fp_server_free(fp_server *s);

/* ---- query without device allocation ------------------------------------ */
/* The paper has no counterpart to this entry point: it is a deployment aid.
 * Same result as fp_query for small batches, but the call allocates no device
 * memory at all (no cudaMalloc, no stream-ordered pool, no library that
 * allocates): all of its working memory is one fixed scratch array of
 * FP_NOALLOC_SCRATCH_BYTES compiled into the library, which every GPU that
 * loads the library holds until the process exits.  It is meant for callers
 * that cannot allocate once they are serving -- e.g. a process whose device
 * memory is carved up in advance by its own allocator, or a latency-critical
 * loop that must not risk the device-wide synchronisation an allocation can
 * cause.
 *   chars, offsets: DEVICE memory, offsets[0] == 0, n_queries + 1 entries.
 *   n_queries <= FP_NOALLOC_MAX_QUERIES, offsets[n] <= FP_NOALLOC_MAX_CHARS.
 *   row_ptr: DEVICE, n_queries + 1 int64 (written); idx: DEVICE, idx_capacity
 *   int32 (written, ascending per query as in fp_query).
 *   n_matches: host; set to the number of matches (also when it exceeds the
 *   capacity, so the caller can retry with a larger idx buffer).
 * Errors: FP_E_INVAL (sizes beyond the limits, host pointers, bad offsets),
 * FP_E_UNSUPPORTED (as fp_query), FP_E_OVERFLOW (more than
 * FP_NOALLOC_MAX_CANDIDATES pairs passed the filter, or more matches than
 * min(idx_capacity, FP_NOALLOC_MAX_MATCHES); outputs are then not valid),
 * FP_E_CUDA.
 * The first call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  All calls share the one array and it keeps the
 * last call's contents (each call clears what must start at zero).  Calls
 * whose GPU work overlapped would race, so calls are serialised by a
 * process-wide lock and each call synchronises cuda_stream before it
 * returns. */
#define FP_NOALLOC_MAX_QUERIES 4096
#define FP_NOALLOC_MAX_CHARS 262144
#define FP_NOALLOC_MAX_CANDIDATES 1048576
#define FP_NOALLOC_MAX_MATCHES 262144
#define FP_NOALLOC_SCRATCH_BYTES (14 * 1024 * 1024)
FP_API int fp_query_noalloc(fp_index *ix, const uint8_t *chars, const int64_t *offsets, int64_t n_queries, int k,
                            int metric, int64_t *row_ptr, int32_t *idx, int64_t idx_capacity, int64_t *n_matches,
                            void *cuda_stream);

/* ---- results ------------------------------------------------------------ */
/* CSR of match lists: row_ptr[n_queries + 1] (int64) and idx[row_ptr[n]]
 * (int32, strictly ascending within a row; duplicate dictionary strings are
 * separate indices).  on_device = 1 returns device pointers owned by the
 * result; 0 returns host copies owned by the result (copied on first use). */
FP_API int fp_result_csr(fp_result *r, const int64_t **row_ptr, const int32_t **idx, int on_device);
FP_API int fp_result_stats(const fp_result *r, fp_stats *s);
FP_API void fp_result_free(fp_result *r);

/* ---- index utilities ---------------------------------------------------- */
FP_API int fp_index_info_get(const fp_index *ix, fp_index_info *info);
/* The symbol map in use: map[c] = field of byte c or -1 (host, [256]). */
FP_API int fp_index_map(const fp_index *ix, int8_t *map_out);
/* The q-grams of an FP_QGRAM index in field order: grams_out (host, at
 * least 32 * 3 bytes) gets field f's q bytes at [f q, f q + q); *n_grams the
 * number of fields used, *q the gram length.  FP_E_UNSUPPORTED for other
 * types. */
FP_API int fp_index_qgrams(const fp_index *ix, uint8_t *grams_out, int32_t *n_grams, int32_t *q);
/* Replaces the symbol map (Sec. 3.2: the c -> q mapping) and rebuilds every
 * dictionary fingerprint on the device.  Any many-to-one map keeps Eq. 1
 * valid for FP_OCC and FP_COUNT.  map: host, [256], values < sigma or -1.
 * FP_E_UNSUPPORTED for FP_QGRAM indexes (their fields are q-grams). */
FP_API int fp_set_symbol_map(fp_index *ix, const int8_t *map);
/* Fingerprints (Sec. 3.2) of arbitrary strings under the index's type, width
 * and map, in input order.  chars/offsets host or device; out_fp host or
 * device, n_strings uint32 values (16-bit fingerprints zero-extended). */
FP_API int fp_fingerprint(const fp_index *ix, const uint8_t *chars, const int64_t *offsets, int64_t n_strings,
                   uint32_t *out_fp, void *cuda_stream);
FP_API void fp_free(fp_index *ix);

/* ---- diagnostics -------------------------------------------------------- */
FP_API const char *fp_strerror(int code);
FP_API const char *fp_last_error(void);
/* Number of kernels this library has launched in the process so far. */
FP_API int64_t fp_launch_count(void);
/* Library version string. */
FP_API const char *fp_version(void);

/* Integer-pipe throughput probe used to state the filter's arithmetic
 * ceiling.  No paper counterpart: it measures the GPU, not the method.
 *   kind 0: the filter's per-pair work (XOR, population count, minimum,
 *           compare with 2k) on register-resident operands; ops = pair tests
 *   kind 1: independent chains of 3-input logic operations; ops = LOP3s
 *   kind 2: independent chains of population counts; ops = POPCs
 *   kind 3: the filter's k = 1 pattern loop (three XOR + POPC tests and one
 *           ALU-only "at most two bits" test per pattern and thread, minimum,
 *           hit mask, warp sum per 32 patterns), no pair passing; ops = pair tests
 * Every SM runs the same number of resident blocks.  ops_per_clk_per_sm
 * divides the ops by each SM's span of cycles, from its first block's start
 * to its last block's end (the blocks sharing an SM finish at different
 * times, so one block's duration would understate the SM time); seconds come
 * from CUDA events on cuda_stream, sm_clock_mhz = mean span / seconds. */
typedef struct {
    int32_t kind;
    int32_t sm_count;
    double ops;
    double seconds;
    double ops_per_s;
    double ops_per_clk_per_sm;
    double sm_clock_mhz;
} fp_probe_result;
FP_API int fp_probe(int kind, int iters, void *cuda_stream, fp_probe_result *out);

#ifdef __cplusplus
}
#endif
#endif /* FP_H */
