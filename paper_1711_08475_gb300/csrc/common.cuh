// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "fp.h"

namespace fpk {

// ---------------------------------------------------------------------------
// errors and launch accounting
// ---------------------------------------------------------------------------
void set_error(const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);
extern std::atomic<int64_t> g_launches;

#define FP_CUDA(call)                                          \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return ::fpk::cuda_fail(e_, #call); \
    } while (0)

#define FP_TRY(call)               \
    do {                           \
        int rc_ = (call);          \
        if (rc_ != FP_OK) return rc_; \
    } while (0)

// Counts one launch and checks the launch error.
#define FP_LAUNCHED(name)                                       \
    do {                                                        \
        ::fpk::g_launches.fetch_add(1, std::memory_order_relaxed); \
        cudaError_t e_ = cudaGetLastError();                    \
        if (e_ != cudaSuccess) return ::fpk::cuda_fail(e_, name); \
    } while (0)

constexpr int MAX_LEN = 255;
constexpr int SLOT_ALIGN = 8;      // bucket starts are multiples of 8 slots (16-byte fingerprint rows)
constexpr int STR_SLACK = 512;     // readable bytes after the last string row
constexpr int FP_SLACK_SLOTS = 8192; // readable fingerprint slots after the last bucket

// ---------------------------------------------------------------------------
// fingerprint parameters (Sec. 3, Sec. 3.2)
// ---------------------------------------------------------------------------
struct FpParams {
    int32_t type;     // fp_type
    int32_t width;    // 16 or 32
    int32_t b;        // bits per count
    int32_t p;        // bits per position
    int32_t n_pos;    // position fields
    int32_t sigma;    // tracked fields
    uint32_t count_top;  // top bit of every count field (Gray conversion)
    uint32_t pos_low;    // low p-1 bits of every position field
    uint32_t pos_high;   // top bit of every position field
    uint32_t pos_occ;    // occurrence bits above the position fields
    int32_t q;           // q-gram length (FP_QGRAM); 1 for the other types.  A pair is
                         // rejected iff F_D > 2 q k (Eq. 1 is q = 1)
    const int8_t *gmap;  // FP_QGRAM: device table q-gram code (first byte most significant) -> field or -1
};
int make_params(int type, int width, int b, int p, FpParams *out, int q = 0);
// Types whose F_D is the population count of the XOR and whose buckets are
// kept in weight-cell order (weight bands); position fingerprints and the
// count L1 distance are compared field by field and are not banded.
inline bool banded_type(int type) { return type != FP_POS && type != FP_COUNT_L1; }

// ---------------------------------------------------------------------------
// a bucketed set of strings on the device (dictionary or query batch)
// ---------------------------------------------------------------------------
// Slots: bucket (bin) c occupies slots [start[c], start[c] + count[c]); bin c
// holds strings of length c & 255 (bins >= 256 separate query groups).
// Starts are multiples of SLOT_ALIGN; the gaps are padding slots with idx -1.
struct Bucketed {
    int32_t nbins = 0;
    int64_t n = 0;          // strings
    int64_t n_slots = 0;    // slots including padding
    int64_t str_bytes = 0;  // bytes of padded rows
    // device arrays
    void *fp = nullptr;         // uint16 or uint32 per slot (+ FP_SLACK_SLOTS)
    uint32_t *fp2 = nullptr;    // combined types: 32-bit occurrence fingerprint per slot, or null
    int32_t *idx = nullptr;     // original index per slot
    uint8_t *len = nullptr;     // length per slot
    uint32_t *row16 = nullptr;  // row byte offset / 16 per slot
    uint8_t *str = nullptr;     // padded rows (+ STR_SLACK)
    int32_t *b_start = nullptr; // [nbins]
    int32_t *b_count = nullptr; // [nbins]
    bool stream_ordered = false; // allocated with cudaMallocAsync
};

// Copies / bucketizes / fingerprints n strings.  chars and offsets are device
// pointers.  total_chars = offsets[n].  bin of string i = group[i] * 256 + len
// (group may be null).  map is a device int8[256].  cells: order every bin by
// weight cell (fp_cell, stable), as weight_order would; position fingerprints
// keep index order.
int bucketize(const uint8_t *d_chars, const int64_t *d_off, int64_t n, int64_t total_chars,
              const int32_t *d_group, int32_t n_groups, const int8_t *d_map, const FpParams &fp,
              bool stream_ordered, cudaStream_t st, Bucketed *out, int32_t *d_err, bool cells = false);
void free_bucketed(Bucketed *b, cudaStream_t st);
// Rebuilds fingerprints of an existing bucketed set from its rows.
int refingerprint(Bucketed *b, const int8_t *d_map, const FpParams &fp, cudaStream_t st);
// Combined types: (re)computes b->fp2, the 32-bit occurrence fingerprint of
// every slot under map2 (allocated on first use), from the rows in slot order.
int second_fingerprints(Bucketed *b, const int8_t *d_map2, const FpParams &p2, cudaStream_t st);
// Weight cells.  The W bits of a fingerprint are split into three parts of
// ceil / floor(W/3) bits (W = 32: bits 21..31, 10..20, 0..9; W = 16: 10..15,
// 5..9, 0..4); its cell is (x, y, z) = the population counts of the parts,
// numbered (x * R1 + y) * R2 + z with R_i = bits of part i + 1.  Every bit
// that differs between two fingerprints changes one part's count by one, so
// |x - x'| + |y - y'| + |z - z'| <= popc(f ^ f'): a pair whose cells lie more
// than 2k apart (L1) fails Eq. 1.
__host__ __device__ constexpr int cell_part_bits(int width, int i) { return width / 3 + (i < width % 3 ? 1 : 0); }
__host__ __device__ constexpr int cell_part_radix(int width, int i) { return cell_part_bits(width, i) + 1; }
__host__ __device__ constexpr int cell_count(int width) {
    return cell_part_radix(width, 0) * cell_part_radix(width, 1) * cell_part_radix(width, 2);
}
__device__ __forceinline__ int fp_cell(uint32_t f, int width) {
    const int b1 = cell_part_bits(width, 1), b2 = cell_part_bits(width, 2);
    const int x = __popc(f >> (b1 + b2)), y = __popc((f >> b2) & ((1u << b1) - 1u)), z = __popc(f & ((1u << b2) - 1u));
    return (x * (b1 + 1) + y) * (b2 + 1) + z;
}
// Orders the real slots of every bin by weight cell (stable), for occurrence,
// occurrence-halved and count fingerprints (a no-op for position
// fingerprints).  d_wstart (optional, nbins * (cell_count(W) + 1) int32):
// per bin the first slot of every cell 0 .. cell_count(W) (the last: the end
// of the bin's real slots).
int weight_order(Bucketed *b, const FpParams &fp, int32_t *d_wstart, cudaStream_t st);

// Symbol statistics (Sec. 3 symbol sets): byte counts and the field map.
int symbol_map(const uint8_t *d_chars, int64_t total, int set, int sigma, int8_t *d_map,
               unsigned long long *d_counts, cudaStream_t st);
// q-gram fingerprints (Sec. 5): counts every q-gram (1 <= q <= 3) of the n
// strings and writes d_gmap[code] = field for the sigma most frequent ones
// (ties: smaller code; -1 elsewhere; d_gmap has 256^q entries).  h_codes
// (host, sigma) gets the codes in field order, *n_used how many occur.
// Synchronises st.
int qgram_map(const uint8_t *d_chars, const int64_t *d_off, int64_t n, int q, int sigma, int8_t *d_gmap,
              uint32_t *h_codes, int *n_used, cudaStream_t st);

// ---------------------------------------------------------------------------
// radix sort of 64-bit keys (stable LSD) and scans
// ---------------------------------------------------------------------------
// Sorts keys[0 .. *d_n) (or n_host if d_n is null) on bits [0, bits).
// tmp must hold as many keys.  The sorted keys end up in *result (either keys
// or tmp).  max_n bounds *d_n.
int radix_sort_u64(uint64_t *keys, uint64_t *tmp, const uint64_t *d_n, int64_t max_n, int bits_lo,
                   int bits_hi, cudaStream_t st, uint64_t **result);

// ---------------------------------------------------------------------------
// filter + verify + emit
// ---------------------------------------------------------------------------
struct Segment {        // one (query bucket, dictionary bucket) rectangle of pairs
    uint32_t q_start, q_count;
    uint32_t d_start, d_count;
    uint32_t n_qtiles, n_dtiles;
    uint64_t tile_begin;
    int32_t k, metric;
};

struct QueryPlan {
    Segment *seg = nullptr;          // device
    int32_t max_segments = 0;
    // device scalars (one small block)
    uint64_t *scal = nullptr;   // [0] n_segments [1] total tiles [2] pairs [3] tile counter
                                // [4] survivors [5] matches [6] plan overflow [7] pairs tested
    // scratch of the banded planner over many blocks (optional: without it one
    // block plans); units_cap >= ceil(patterns / tq) + bins
    int32_t units_cap = 0;
    int32_t *unit0 = nullptr;     // [bins + 1] first unit of every bin
    int32_t *u_seg = nullptr;     // [units_cap] segments per unit, then their offsets
    uint64_t *u_tiles = nullptr;  // [units_cap] tiles per unit, then their offsets
    uint64_t *acc = nullptr;      // [4] pairs, tested pairs, fall-back flag, units
};
// Bytes of the banded planner's scratch for a plan of units_cap units over nbins
// bins, and the scratch placed at base (256-byte aligned).
size_t plan_scratch_bytes(int64_t units_cap, int nbins);
void plan_scratch_place(QueryPlan *plan, uint8_t *base, int64_t units_cap, int nbins);

struct FilterCfg {
    int mode;      // fp_mode
    int tq;        // queries per tile
    int v;         // 32-bit fingerprint words per thread (4 or 8)
    bool k1mix;    // k = 1: test a quarter of the words with integer ALU ops instead of POPC
    bool mma;      // popcount-type fingerprints: dot products of +-1 vectors on the tensor cores
};

// d_wstart (optional): the dictionary's cell table (weight_order); when
// given, the patterns' bins must be in cell order too, and each tile of tq
// patterns gets segments per dictionary bucket restricted to the cells
// Eq. 1 can pass.  width: fingerprint width in bits.  tmul: a pair can pass
// only if F_D <= 2 tmul k (q for q-gram fingerprints, else 1).
int plan_segments(const Bucketed &q, const Bucketed &d, const int32_t *d_group_k,
                  const int32_t *d_group_metric, int tq, int tw, QueryPlan *plan, cudaStream_t st,
                  const int32_t *d_wstart = nullptr, int width = 32, int tmul = 1);

int launch_filter(const Bucketed &q, const Bucketed &d, const QueryPlan &plan, const FpParams &fp,
                  const FilterCfg &cfg, uint64_t *surv, int64_t surv_cap, cudaStream_t st,
                  int64_t *launches);

// Filter and verification in one persistent kernel: survivors never leave
// the SM; matches (original query << idx_bits | original word) are appended
// to `matches` (counter plan.scal[5]; plan.scal[4] counts the survivors).
int launch_fused(const Bucketed &q, const Bucketed &d, const QueryPlan &plan, const FpParams &fp,
                 const FilterCfg &cfg, int idx_bits, uint64_t *matches, int64_t match_cap, cudaStream_t st,
                 int64_t *launches);

int launch_verify(const Bucketed &q, const Bucketed &d, const uint64_t *surv, const uint64_t *d_n_surv,
                  int64_t surv_cap, int k, int metric, int idx_bits, uint64_t *matches,
                  uint64_t *d_n_matches, int64_t match_cap, cudaStream_t st);
int tile_words(int width, int v);
// Tile of the filter kernel the configuration selects: patterns x words.
void tile_shape(const FilterCfg &cfg, const FpParams &fp, int *tq, int *tw);
int fingerprint_list(const uint8_t *d_chars, const int64_t *d_off, int64_t n, const int8_t *d_map,
                     const FpParams &P, uint32_t *d_out, cudaStream_t st);

int build_csr(uint64_t *keys, uint64_t *tmp, const uint64_t *d_n, int64_t max_n, int q_bits, int idx_bits,
              int64_t n_queries, int64_t *row_ptr, int32_t *idx, cudaStream_t st);

int sm_count();
void init_pool();
int fail(int code, const std::string &msg);
bool is_device_ptr(const void *p);
int bits_for(int64_t n);
int check_host_offsets(const int64_t *off, int64_t n);

// ---------------------------------------------------------------------------
// the same steps on caller-placed buffers (nothing is allocated)
// ---------------------------------------------------------------------------
struct BucketScratch {
    uint64_t *keys, *keys2;  // n keys each
    int32_t *hist, *ustart;  // 256 each
    int64_t *str16;          // 256
    int64_t *tot;            // 2
    uint32_t *radix_hist;    // 256 * radix_blocks(n)
};
int radix_blocks(int64_t max_n);
int radix_sort_u64_into(uint64_t *keys, uint64_t *tmp, uint32_t *hist, const uint64_t *d_n, int64_t max_n,
                        int bits_lo, int bits_hi, cudaStream_t st, uint64_t **result);
int build_csr_into(uint64_t *keys, uint64_t *tmp, uint32_t *hist, const uint64_t *d_n, int64_t max_n, int q_bits,
                   int idx_bits, int64_t n_queries, int64_t *row_ptr, int32_t *idx, cudaStream_t st);
int bucketize_into(const uint8_t *d_chars, const int64_t *d_off, int64_t n, int64_t total_chars,
                   const int32_t *d_group, int32_t n_groups, const int8_t *d_map, const FpParams &P, cudaStream_t st,
                   Bucketed *B, const BucketScratch &S, int32_t *d_err, bool cells = false);
// group[i] = batch_group[b] for every pattern i of batch b (batch b covers
// [batch_start[b], batch_start[b+1]), device arrays).
int fill_groups(const int64_t *d_batch_start, const int32_t *d_batch_group, int n_batches, int32_t *d_group,
                cudaStream_t st);

}  // namespace fpk

// Match lists behind the opaque fp_result handle.
struct fp_result {
    int64_t n_queries = 0;
    int64_t n_matches = 0;
    int64_t *d_row_ptr = nullptr;  // stream-ordered pool memory
    int32_t *d_idx = nullptr;
    std::vector<int64_t> h_row_ptr;
    std::vector<int32_t> h_idx;
    bool host_ready = false;
    void *pin = nullptr;  // pinned host copy: row_ptr then idx (from the pinned pool)
    size_t pin_cap = 0;
    fp_stats stats{};
};

namespace fpk {
// Pinned host blocks for result copies, reused across results.
void *pinned_get(size_t bytes, size_t *cap);
void pinned_put(void *p, size_t cap);
}  // namespace fpk

// The resident dictionary behind the opaque fp_index handle.
struct fp_index {
    fpk::FpParams P{};
    int set = 0;
    int64_t n_words = 0;
    fpk::Bucketed D;
    int8_t *d_map = nullptr;
    int8_t h_map[256];
    int8_t *d_gmap = nullptr;     // FP_QGRAM: q-gram code -> field (256^q entries)
    uint32_t h_gram[32];          // FP_QGRAM: the q-gram of every field (code, first byte most significant)
    int n_grams = 0;
    int32_t *d_wstart = nullptr;  // weight order of the buckets (null: position fingerprints, no weight bands)
    // combined types: a second, 32-bit occurrence fingerprint over the 32 most
    // frequent symbols (null map: off)
    int8_t *d_map2 = nullptr;
    int8_t h_map2[256];
    fpk::FpParams P2{};
    unsigned long long *d_counts = nullptr;
    int32_t h_count[256];
    int32_t h_start[256];
    int idx_bits = 1;
    int64_t device_bytes = 0;
    double surv_ratio = 1.0 / 64.0;  // survivors / pairs of the last query (sizes the next survivor buffer)
};
