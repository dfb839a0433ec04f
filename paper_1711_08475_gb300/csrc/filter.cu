// The fingerprint filter (Sec. 3.3, Eq. 1) over length-bucketed tiles.
//
// Work is a set of segments: one query bucket (equal-length patterns of one
// (k, metric) group) against one dictionary bucket of equal length (Hamming)
// or of length within k (Levenshtein).  A segment is cut into tiles of
// tq queries x tw dictionary words.  A persistent grid pops tiles from a
// device counter; a block stages the tile's query fingerprints in shared
// memory and every thread keeps v 32-bit words of dictionary fingerprints in
// registers (loaded once per tile with coalesced 128-bit loads), so each
// dictionary fingerprint read from memory serves tq queries.
//
// Per pair the work is one XOR and one population count (Sec. 3.3: F_D is
// the Hamming weight of the XOR), or for position fingerprints a SWAR test of
// which p-bit fields differ; the pair passes iff F_D <= 2k, i.e. iff
// ceil(F_D / 2) <= k (Eq. 1).
//
// Passing pairs are rare (well under 1% on the English-like workloads) but a
// warp tests 128 pairs per query, so most warp-steps still hold one.  The hot
// loop therefore only records, per thread, a bit per query saying "one of my
// fingerprints passed" (min over its F_D values, one compare).  After every 32
// queries the lanes append their (lane, query) hits to a warp queue, and the
// warp re-tests the queue exactly in rounds of 32 (one hit per lane, the
// owner's fingerprints fetched by shuffles), appending the passing pairs to a
// per-warp buffer in shared memory.  The buffer is emptied before any round
// whose passes might not fit, with one atomic reservation on the global
// survivor list per flush (or, in the fused form, by verifying it in place).
#include <cuda_fp16.h>

#include "verify_core.cuh"

namespace fpk {

#ifndef FT_THREADS
#define FT_THREADS 128  // threads per block of the tiled filter (measured against 256)
#endif
constexpr int FT_WARPS = FT_THREADS / 32;
constexpr int FT_MAX_TQ = 256;
constexpr int FT_STAGE = 256;  // staged survivors per warp
constexpr int FT_QUEUE = 256;  // queued (lane, tile query) hits per warp

// Tuning constants (compile-time; the defaults come from sweeps on GB300).
// Resident blocks per SM the register budget is set for (blocks of 128
// threads): the 32-bit, 4-words-per-thread filter fits 32 registers (16
// blocks, 64 warps); 32-bit position fingerprints take 64 (8 blocks); the
// other shapes keep 48 (10 blocks); the fused form, which calls the verifier,
// is fastest at 80 registers (6 blocks, no spills to speak of): 13 % faster
// than 8 blocks at 64 registers on mixed k = 1, 2 batches, and 10 blocks or
// more spill hundreds of bytes.  Four-warp blocks beat eight-warp ones by
// 1-2 %: fewer warps wait at a tile's barrier for the slowest one.
#ifndef FT_MIN_BLOCKS
#define FT_MIN_BLOCKS 10
#endif
#ifndef FT_MAIN_MIN_BLOCKS
#define FT_MAIN_MIN_BLOCKS 16
#endif
#ifndef FT_FUSED_MIN_BLOCKS
#define FT_FUSED_MIN_BLOCKS 6
#endif
#ifndef FT_POS_MIN_BLOCKS
#define FT_POS_MIN_BLOCKS 8  // 32-bit position fingerprints: 7 % faster than at 10 (the 16-bit shapes are not)
#endif
#ifndef FT_MIX_DIV
#define FT_MIX_DIV 4  // k = 1 mix: V / FT_MIX_DIV of a thread's words use the ALU-only test
#endif
#ifndef FT_UNROLL
#define FT_UNROLL 1  // groups of four queries unrolled in the loop over a partial batch
#endif
#ifndef FT_COLS
#define FT_COLS 2  // 128-word columns each warp scans per tile (the tile's setup is shared by them)
#endif
#define FT_STR(x) #x
#define FT_UNROLL_PRAGMA(n) _Pragma(FT_STR(unroll n))

// ---------------------------------------------------------------------------
// distance functors
// ---------------------------------------------------------------------------
struct PosMasks {
    uint32_t low, high, occ;
};

// Kinds of F_D (Sec. 3.3): the Hamming weight of the XOR (occurrence,
// occurrence halved, Gray-coded count, q-grams); the number of differing
// p-bit position fields plus the weight of the occurrence bits (position);
// the L1 distance of 2-bit binary-coded counts (count in the paper's code).
constexpr int FDK_POPC = 0, FDK_POS = 1, FDK_L1 = 2;

// F_D of a dictionary fingerprint w and a pattern fingerprint q (32-bit).
// L1 of 2-bit binary counts: with x = w ^ q, a field differs by x0 + 2 x1,
// except that x1 = x0 = 1 means 3 against 0 when the word's two bits are
// equal and 2 against 1 (a difference of 1) when they differ; so F_D =
// popc(x) + popc(x & high bits) - 2 popc(low bits where x1, x0 and w1 ^ w0
// are set).
template <int FDK>
__device__ __forceinline__ uint32_t fd32(uint32_t w, uint32_t q, const PosMasks &M) {
    const uint32_t x = w ^ q;
    if (FDK == FDK_POPC) return __popc(x);
    if (FDK == FDK_POS) {
        // a field is nonzero iff its top bit or the carry out of its low p-1 bits is set
        uint32_t s = (x & M.low) + M.low;
        return __popc(((s | x) & M.high) | (x & M.occ));
    }
    const uint32_t c = x & (x >> 1) & (w ^ (w >> 1)) & 0x55555555u;
    return __popc(x) + __popc(x & 0xAAAAAAAAu) - 2u * __popc(c);
}

// F_D of the two 16-bit fingerprints packed in one 32-bit word of each side
// (masks replicated in both halves; position carries and count fields never
// cross a field, so never the halves).
template <int FDK>
__device__ __forceinline__ void fd16x2(uint32_t w, uint32_t q, const PosMasks &M, uint32_t &lo, uint32_t &hi) {
    const uint32_t x = w ^ q;
    if (FDK == FDK_L1) {
        const uint32_t h = x & 0xAAAAAAAAu, c = x & (x >> 1) & (w ^ (w >> 1)) & 0x55555555u;
        lo = __popc(x & 0xFFFFu) + __popc(h & 0xFFFFu) - 2u * __popc(c & 0xFFFFu);
        hi = __popc(x >> 16) + __popc(h >> 16) - 2u * __popc(c >> 16);
        return;
    }
    uint32_t z = x;
    if (FDK == FDK_POS) {
        uint32_t s = (x & M.low) + M.low;
        z = ((s | x) & M.high) | (x & M.occ);
    }
    lo = __popc(z & 0xFFFFu);
    hi = __popc(z >> 16);
}

struct FilterArgs {
    const uint32_t *qfp32;  // query fingerprints (32-bit slots)
    const uint16_t *qfp16;  // query fingerprints (16-bit slots)
    const uint32_t *dfp;    // dictionary fingerprints viewed as 32-bit words
    const Segment *seg;
    uint64_t *scal;         // [0] n_seg [1] tiles [3] tile counter [4] survivors [5] matches
    uint64_t *surv;
    uint64_t surv_cap;
    PosMasks M;
    int tq;
    int tmul;  // a pair passes iff F_D <= 2 tmul k: tmul = q for q-gram fingerprints, 1 otherwise (Eq. 1)
    // fused form: survivors are verified in the kernel and only matches leave it
    const uint8_t *q_len, *d_len;
    const uint32_t *q_row16, *d_row16;
    const uint8_t *q_str, *d_str;
    const int32_t *q_idx, *d_idx;
    int idx_bits;
    uint64_t *matches;
    uint64_t match_cap;
    // combined types: second fingerprints (32-bit occurrence) of the patterns
    // and the words, or null
    const uint32_t *qfp2, *dfp2;
};

// Explicit check of one surviving pair (Sec. 4): Hamming for equal lengths,
// banded Levenshtein otherwise.  Returns the match key (original query index
// << idx_bits | original word index) through *key.
static __device__ __noinline__ bool verify_one(const FilterArgs &A, uint64_t e, int k, int metric,
                                               uint64_t *key) {
    const uint32_t qs = (uint32_t)(e >> 32), ds = (uint32_t)e;
    const int m = A.q_len[qs], L = A.d_len[ds];
    const uint8_t *qa = A.q_str + (uint64_t)A.q_row16[qs] * 16;
    const uint8_t *da = A.d_str + (uint64_t)A.d_row16[ds] * 16;
    bool hit;  // k = 1 and 2 inline (the common cases), other k through the out-of-line switch
    if (metric == FP_HAM) hit = m == L && ham_within(qa, da, m, k);
    else if (k == 1) hit = lev1_within(qa, m, da, L);
    else if (k == 2) hit = m - L <= 2 && L - m <= 2 && lev_within<2>(qa, m, da, L);
    else hit = m - L <= k && L - m <= k && lev_within_k(k, qa, m, da, L);
    *key = ((uint64_t)(uint32_t)A.q_idx[qs] << A.idx_bits) | (uint64_t)(uint32_t)A.d_idx[ds];
    return hit;
}

// Fused form: verifies the warp's staged survivors, one per lane.  Matches
// are compacted into the front of the same buffer (a round's survivors are in
// registers before any of its matches is written, and a round never writes
// past its own slots) and appended to the match list with one reservation.
__device__ __forceinline__ void verify_stage(const FilterArgs &A, uint64_t *stage, uint32_t *cnt, int lane, int k,
                                             int metric) {
    __syncwarp();
    const uint32_t c = min(*cnt, (uint32_t)FT_STAGE);
    const unsigned lt = (1u << lane) - 1u;
    if (lane == 0 && c) atomicAdd((unsigned long long *)&A.scal[4], (unsigned long long)c);
    uint32_t nm = 0;
    for (uint32_t base = 0; base < c; base += 32) {
        const uint32_t i = base + lane;
        uint64_t key = 0;
        const bool hit = i < c && verify_one(A, stage[i], k, metric, &key);
        const unsigned bal = __ballot_sync(0xffffffffu, hit);
        if (hit) stage[nm + __popc(bal & lt)] = key;
        nm += __popc(bal);
        __syncwarp();
    }
    if (nm) {
        unsigned long long mb = 0;
        if (lane == 0) mb = atomicAdd((unsigned long long *)&A.scal[5], (unsigned long long)nm);
        mb = __shfl_sync(0xffffffffu, mb, 0);
        for (uint32_t j = lane; j < nm; j += 32)
            if (mb + j < A.match_cap) A.matches[mb + j] = stage[j];
    }
    __syncwarp();
    if (lane == 0) *cnt = 0;
    __syncwarp();
}

__device__ __forceinline__ int find_segment(const Segment *seg, int nseg, uint64_t tile) {
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (seg[mid].tile_begin <= tile) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// The same search by a whole warp, 32 probes per step (three dependent loads
// for 32,768 segments instead of fifteen): the segment of `tile` is the last
// one whose tile_begin <= tile; segment 0 begins at tile 0.
__device__ __forceinline__ int find_segment_warp(const Segment *seg, int nseg, uint64_t tile, int lane) {
    int lo = 0, hi = nseg;  // the answer lies in [lo, hi); seg[lo].tile_begin <= tile
    while (hi - lo > 1) {
        const int step = (hi - lo + 31) >> 5;
        const int i = lo + lane * step;
        const bool le = i < hi && seg[i].tile_begin <= tile;
        const unsigned m = __ballot_sync(0xffffffffu, le);  // lane 0 always set
        lo += (31 - __clz(m)) * step;
        hi = min(hi, lo + step);
    }
    return lo;
}

// Lane layout of a column (one warp's load: 32 lanes x NF fingerprints).
// Fingerprints arrive in 128-bit vectors of G fingerprints (G = 4 for 32-bit,
// 8 for 16-bit); vector r of lane l holds the column's fingerprints
// r*(32*G) + l*G + (0..G-1), so one warp-wide load reads 512 contiguous
// bytes.  Fingerprint i of a lane (0 <= i < NF) is at column offset
// (i/G)*(32*G) + lane*G + i%G.
template <int G>
__device__ __forceinline__ uint32_t lane_offset(int i, int lane) {
    return (uint32_t)(i / G) * (uint32_t)(32 * G) + (uint32_t)lane * G + (uint32_t)(i % G);
}

// All F_D values of a thread's fingerprints against query word q.
template <int W, int V, int FDK, int NF>
__device__ __forceinline__ void all_fd(const uint32_t (&w)[V], uint32_t q, const PosMasks &M, uint32_t (&F)[NF]) {
    if (W == 32) {
#pragma unroll
        for (int v = 0; v < V; v++) F[v] = fd32<FDK>(w[v], q, M);
    } else {
#pragma unroll
        for (int v = 0; v < V; v++) fd16x2<FDK>(w[v], q, M, F[2 * v], F[2 * v + 1]);
    }
}

// Combined types: bit i = fingerprint i of lane src (W = 32, so fingerprint
// i is slot wbase + (i/4)*128 + src*4 + i%4) has a second fingerprint within
// 2k of the pattern's second fingerprint q2 (Eq. 1 on the 32-bit occurrence
// fingerprints).  Four slots per 128-bit load: the dictionary's second
// fingerprints carry readable slack past the last slot, like its first.
template <int V>
__device__ __forceinline__ uint32_t second_pass(const uint32_t *dfp2, uint32_t wbase, int src, uint32_t q2, uint32_t T2) {
    uint32_t bits = 0;
#pragma unroll
    for (int r = 0; r < V / 4; r++) {
        const uint4 x = *reinterpret_cast<const uint4 *>(dfp2 + wbase + r * 128 + src * 4);
        bits |= ((uint32_t)(__popc(x.x ^ q2) <= T2) | (uint32_t)(__popc(x.y ^ q2) <= T2) << 1 |
                 (uint32_t)(__popc(x.z ^ q2) <= T2) << 2 | (uint32_t)(__popc(x.w ^ q2) <= T2) << 3) << (4 * r);
    }
    return bits;
}

// Moves the warp's staged survivors to the global list (one reservation).
__device__ __forceinline__ void flush_stage(const FilterArgs &A, uint64_t *stage, uint32_t *cnt, int lane) {
    __syncwarp();
    const uint32_t c = min(*cnt, (uint32_t)FT_STAGE);
    unsigned long long base = 0;
    if (lane == 0 && c) base = atomicAdd((unsigned long long *)&A.scal[4], (unsigned long long)c);
    base = __shfl_sync(0xffffffffu, base, 0);
    for (uint32_t i = lane; i < c; i += 32) {
        const uint64_t g = base + i;
        if (g < A.surv_cap) A.surv[g] = stage[i];
    }
    __syncwarp();
    if (lane == 0) *cnt = 0;
    __syncwarp();
}

// Appends one survivor to the warp's staging buffer.  When it is full the
// survivor goes to the global list directly, or, in the fused form, is
// verified on the spot by this thread.
//
// With combined types (f3: occurrence + count) a pair that passed the first
// fingerprint survives only if its second fingerprints pass Eq. 1 as well;
// each type is sound on its own (Theorem 1), so both must pass for a match.
template <bool FUSED, bool COMB>
__device__ __forceinline__ void stage_push(const FilterArgs &A, uint64_t *stage, uint32_t *cnt, uint64_t e, int k,
                                           int metric) {
    if (COMB && __popc(A.qfp2[(uint32_t)(e >> 32)] ^ A.dfp2[(uint32_t)e]) > 2 * k) return;
    const uint32_t pos = atomicAdd(cnt, 1u);
    if (pos < FT_STAGE) {
        stage[pos] = e;
    } else if (!FUSED) {
        const unsigned long long g = atomicAdd((unsigned long long *)&A.scal[4], 1ull);
        if (g < A.surv_cap) A.surv[g] = e;
    } else {
        atomicAdd((unsigned long long *)&A.scal[4], 1ull);
        uint64_t key;
        if (verify_one(A, e, k, metric, &key)) {
            const unsigned long long g = atomicAdd((unsigned long long *)&A.scal[5], 1ull);
            if (g < A.match_cap) A.matches[g] = key;
        }
    }
}

// x has at most two bits set: clear the lowest set bit twice (integer ALU
// only, no population count).  Used for k = 1 on part of a thread's words so
// that the population-count pipe and the logic pipe share the work.
__device__ __forceinline__ uint32_t clear2(uint32_t x) {
    const uint32_t t = x & (x - 1u);
    return t & (t - 1u);  // zero iff popc(x) <= 2
}

// Minimum of n values with 3-input minima.
template <int N>
__device__ __forceinline__ uint32_t min_tree(const uint32_t *v) {
    if (N == 1) return v[0];
    if (N == 2) return min(v[0], v[1]);
    if (N == 3) return __vimin3_u32(v[0], v[1], v[2]);
    return __vimin3_u32(min_tree<N / 3>(v), min_tree<N / 3>(v + N / 3), min_tree<N - 2 * (N / 3)>(v + 2 * (N / 3)));
}

// A value whose sign bit says "some fingerprint of the thread passes against
// query word q" (min over F_D - (2k+1) < 0).  It may also be negative when
// nothing passes (only with K1MIX, for words of 0xFFFFFFFE or more after the
// two clears): a spurious hit only costs an exact re-test, a missed pass cannot
// happen.  K1MIX (32-bit occ/occh/count, k = 1): the last quarter of the words
// is tested with clear2 instead of the population count (passes iff clear2 == 0,
// i.e. iff (clear2 | 2) <= 2, so it joins the same minimum).
template <int W, int V, int FDK, bool FULL, bool K1MIX>
__device__ __forceinline__ int32_t pass_sign(const uint32_t (&w)[V], uint32_t q, const PosMasks &M,
                                             uint32_t invalid, uint32_t T) {
    if (K1MIX) {
        constexpr int NZ = V / FT_MIX_DIV, NP = V - NZ;  // NP words through POPC, NZ through clear2
        uint32_t f[NP + 1];
#pragma unroll
        for (int v = 0; v < NP; v++) {
            f[v] = __popc(w[v] ^ q);
            if (!FULL && ((invalid >> v) & 1u)) f[v] = 0xFFu;
        }
        uint32_t z[NZ];
#pragma unroll
        for (int v = 0; v < NZ; v++) {
            // clear2 is 0 (pass) or >= 4, so clear2 | 2 is 2 (pass) or >= 6: one
            // 3-input logic op joins it to the F_D scale
            z[v] = clear2(w[NP + v] ^ q) | 2u;
            if (!FULL && ((invalid >> (NP + v)) & 1u)) z[v] = 3u;
        }
        f[NP] = min_tree<NZ>(z);
        return (int32_t)(min_tree<NP + 1>(f) - 3u);
    } else {
        constexpr int NF = (W == 32) ? V : 2 * V;
        uint32_t f[NF];
#pragma unroll
        for (int v = 0; v < V; v++) {
            if (W == 32) {
                f[v] = fd32<FDK>(w[v], q, M);
            } else {
                fd16x2<FDK>(w[v], q, M, f[2 * v], f[2 * v + 1]);
            }
        }
        if (!FULL) {
#pragma unroll
            for (int i = 0; i < NF; i++)
                if ((invalid >> i) & 1u) f[i] = 0xFFu;
        }
        return (int32_t)(min_tree<NF>(f) - (T + 1u));
    }
}

// Four queries (one 128-bit shared load) against the thread's fingerprints;
// each test's sign bit is shifted into the hit mask.
template <int W, int V, int FDK, bool FULL, bool K1MIX>
__device__ __forceinline__ uint32_t four_queries(const uint32_t (&w)[V], uint4 q4, const PosMasks &M, uint32_t invalid,
                                                 uint32_t T, uint32_t hits) {
    const int32_t h0 = pass_sign<W, V, FDK, FULL, K1MIX>(w, q4.x, M, invalid, T);
    const int32_t h1 = pass_sign<W, V, FDK, FULL, K1MIX>(w, q4.y, M, invalid, T);
    const int32_t h2 = pass_sign<W, V, FDK, FULL, K1MIX>(w, q4.z, M, invalid, T);
    const int32_t h3 = pass_sign<W, V, FDK, FULL, K1MIX>(w, q4.w, M, invalid, T);
    hits = __funnelshift_l((uint32_t)h0, hits, 1);
    hits = __funnelshift_l((uint32_t)h1, hits, 1);
    hits = __funnelshift_l((uint32_t)h2, hits, 1);
    return __funnelshift_l((uint32_t)h3, hits, 1);
}

// Empties the warp's stage when it might not hold the passing pairs of one
// more round (32 lanes x NF fingerprints), so that pushes never take the
// slow per-survivor path of a full stage.  Warp-uniform.
template <int NF, bool FUSED>
__device__ __forceinline__ void make_room(const FilterArgs &A, uint64_t *stage, uint32_t *cnt, int lane, int k,
                                          int metric) {
    __syncwarp();
    if (*cnt > (uint32_t)(FT_STAGE - 32 * NF)) {
        if (FUSED) verify_stage(A, stage, cnt, lane, k, metric);
        else flush_stage(A, stage, cnt, lane);
    }
}

// One round of exact re-tests: lane l takes queued hit first + l (if l <
// count), i.e. (owner lane, tile query), fetches the owner's fingerprints with
// shuffles and stages every pair of that query and those fingerprints that
// passes Eq. 1.
template <int W, int V, int FDK, bool FULL, bool FUSED, bool COMB>
__device__ __forceinline__ void retest_round(const FilterArgs &A, const uint32_t *s_q, const uint32_t *s_q2,
                                             const uint16_t *queue,
                                             uint32_t first, uint32_t count, uint32_t q0, const uint32_t (&w)[V],
                                             uint32_t invalid, uint32_t T, uint32_t wbase, uint64_t *stage,
                                             uint32_t *cnt, int lane, int k, int metric) {
    constexpr int G = (W == 32) ? 4 : 8;
    constexpr int NF = (W == 32) ? V : 2 * V;
    const bool has = (uint32_t)lane < count;
    const uint32_t item = has ? queue[first + lane] : ((uint32_t)lane << 8);
    const int src = (int)(item >> 8);
    const uint32_t jq = item & 255u;
    uint32_t ws[V];
#pragma unroll
    for (int v = 0; v < V; v++) ws[v] = __shfl_sync(0xffffffffu, w[v], src);
    const uint32_t inv = FULL ? 0u : __shfl_sync(0xffffffffu, invalid, src);
    if (has) {
        uint32_t F[NF];
        all_fd<W, V, FDK, NF>(ws, s_q[jq], A.M, F);
        uint32_t pass = 0;
#pragma unroll
        for (int i = 0; i < NF; i++) pass |= (uint32_t)(F[i] <= T) << i;
        if (!FULL) pass &= ~inv;
        // combined types: the second check for the whole round's fingerprints at once
        if (COMB && pass) pass &= second_pass<V>(A.dfp2, wbase, src, s_q2[jq], 2u * (uint32_t)k);
#pragma unroll
        for (int i = 0; i < NF; i++)
            if ((pass >> i) & 1u)
                stage_push<FUSED, false>(A, stage, cnt, ((uint64_t)(q0 + jq) << 32) | (uint64_t)(wbase + lane_offset<G>(i, src)),
                                         k, metric);
    }
}

// One tile's pairs for the thread: queries s_q[0 .. nq) against its NF
// fingerprints.  FULL = every fingerprint of the thread lies inside the tile.
// Query fingerprints are read four at a time (one 128-bit shared load), the
// four tests are independent, and each test's sign bit is shifted into the
// hit mask (bit b of a 32-query batch <-> query jn4 - 1 - b).
//
// Hits are re-tested exactly, but not one batch at a time: every lane appends
// its (lane, query) hits to the warp's queue (one shared atomic per lane with
// hits), and the warp re-tests the queue in rounds of 32 whenever it holds a
// full round, so nearly every round keeps all 32 lanes busy; the last partial
// round runs when the tile ends (the fingerprints in registers belong to it).
template <int W, int V, int FDK, bool FULL, bool K1MIX, bool FUSED, bool COMB>
__device__ __forceinline__ void scan_tile(const FilterArgs &A, const uint32_t *s_q, const uint32_t *s_q2, uint32_t nq,
                                          uint32_t q0,
                                          const uint32_t (&w)[V], uint32_t invalid, uint32_t T, uint32_t wbase,
                                          uint64_t *stage, uint32_t *cnt, uint16_t *queue, uint32_t *qcnt, int lane,
                                          int k, int metric) {
    constexpr int G = (W == 32) ? 4 : 8;
    constexpr int NF = (W == 32) ? V : 2 * V;
    const uint4 *s_q4 = reinterpret_cast<const uint4 *>(s_q);
    for (uint32_t jb = 0; jb < nq; jb += 32) {
        const uint32_t jn = min(32u, nq - jb);
        const uint32_t jn4 = (jn + 3u) & ~3u;
        uint32_t hits = 0;
        if (!FUSED && jn == 32u) {  // a whole batch: fully unrolled (the fused form is faster without)
#pragma unroll
            for (uint32_t jj = 0; jj < 32u; jj += 4)
                hits = four_queries<W, V, FDK, true, K1MIX>(w, s_q4[(jb + jj) >> 2], A.M, invalid, T,
                                                                              hits);
        } else {
            FT_UNROLL_PRAGMA(FT_UNROLL)
            for (uint32_t jj = 0; jj < jn; jj += 4)
                hits = four_queries<W, V, FDK, true, K1MIX>(w, s_q4[(jb + jj) >> 2], A.M, invalid, T,
                                                                              hits);
        }
        hits &= ~((1u << (jn4 - jn)) - 1u);  // queries past nq in the last group of four
        const uint32_t c = __popc(hits);
        const uint32_t total = __reduce_add_sync(0xffffffffu, c);
        if (total != 0 && total <= (uint32_t)(FT_QUEUE - 32)) {  // the queue holds < 32 items here
            if (c) {
                uint32_t pos = atomicAdd(qcnt, c);
                for (uint32_t h = hits; h; h &= h - 1)
                    queue[pos++] = (uint16_t)((lane << 8) | (jb + jn4 - 1u - (__ffs(h) - 1)));
            }
            __syncwarp();
            const uint32_t qn = *qcnt;
            uint32_t done = 0;
            for (; qn - done >= 32u; done += 32u) {
                make_room<NF, FUSED>(A, stage, cnt, lane, k, metric);
                retest_round<W, V, FDK, FULL, FUSED, COMB>(A, s_q, s_q2, queue, done, 32u, q0, w, invalid, T, wbase, stage, cnt,
                                                     lane, k, metric);
            }
            if (done) {  // move the rest (< 32) to the front
                const uint32_t rem = qn - done;
                const uint16_t keep = (uint32_t)lane < rem ? queue[done + lane] : (uint16_t)0;
                __syncwarp();
                if ((uint32_t)lane < rem) queue[lane] = keep;
                if (lane == 0) *qcnt = rem;
            }
            __syncwarp();
        } else if (total != 0) {
            // very many hits (large k, short words, dense matches): the batch's
            // queries one at a time, each lane re-testing its own fingerprints,
            // with room in the stage for a whole query's passes
            for (uint32_t jj = 0; jj < jn; jj++) {
                const bool mine = (hits >> (jn4 - 1u - jj)) & 1u;
                if (__ballot_sync(0xffffffffu, mine) == 0u) continue;
                make_room<NF, FUSED>(A, stage, cnt, lane, k, metric);
                if (mine) {
                    uint32_t F[NF];
                    all_fd<W, V, FDK, NF>(w, s_q[jb + jj], A.M, F);
                    uint32_t pass = 0;
#pragma unroll
                    for (int i = 0; i < NF; i++) pass |= (uint32_t)(F[i] <= T) << i;
                    if (!FULL) pass &= ~invalid;
                    if (COMB && pass) pass &= second_pass<V>(A.dfp2, wbase, lane, s_q2[jb + jj], 2u * (uint32_t)k);
#pragma unroll
                    for (int i = 0; i < NF; i++)
                        if ((pass >> i) & 1u)
                            stage_push<FUSED, false>(
                                A, stage, cnt,
                                ((uint64_t)(q0 + jb + jj) << 32) | (uint64_t)(wbase + lane_offset<G>(i, lane)), k, metric);
                }
            }
            __syncwarp();
        }
        if (*cnt >= FT_STAGE / 2) {
            if (FUSED) verify_stage(A, stage, cnt, lane, k, metric);
            else flush_stage(A, stage, cnt, lane);
        }
    }
    // the last partial round of this tile
    const uint32_t qn = *qcnt;
    if (qn) {
        make_room<NF, FUSED>(A, stage, cnt, lane, k, metric);
        retest_round<W, V, FDK, FULL, FUSED, COMB>(A, s_q, s_q2, queue, 0u, qn, q0, w, invalid, T, wbase, stage, cnt, lane, k,
                                             metric);
        __syncwarp();
        if (lane == 0) *qcnt = 0;
        __syncwarp();
    }
}

template <int W, int V, int FDK, bool FUSED>
constexpr int ft_min_blocks() {
    return FUSED ? FT_FUSED_MIN_BLOCKS
                 : ((W == 32 && V == 4 && FDK == FDK_POPC) ? FT_MAIN_MIN_BLOCKS
                                                           : ((W == 32 && FDK == FDK_POS) ? FT_POS_MIN_BLOCKS : FT_MIN_BLOCKS));
}

// W: fingerprint width; V: 32-bit words per thread (multiple of 4).
// COMB: combined types (second fingerprints checked for every pass).
//
// A tile is tq patterns x FT_WARPS * FT_COLS columns of 32 * NF words.  Its
// setup is done once per block: thread 0 claims it, warp 0 finds its segment
// and stages the patterns in shared memory.  The block's work in the tile is
// a list of items (column, batch of 32 patterns), split evenly over the warps
// in order: a warp loads a column's fingerprints into registers once and
// scans its consecutive batches against them.  A short tile (the end of a
// run of weight cells) has fewer columns, and its items spread the same way,
// so no warp idles while there is work.
template <int W, int V, int FDK, bool K1MIX, bool FUSED, bool COMB>
__global__ void __launch_bounds__(FT_THREADS, (ft_min_blocks<W, V, FDK, FUSED>())) k_filter_tiled(FilterArgs A) {
    constexpr int G = (W == 32) ? 4 : 8;             // fingerprints per 128-bit vector
    constexpr int NF = (W == 32) ? V : 2 * V;        // fingerprints per lane
    constexpr int CW = NF * 32;                      // fingerprints per column
    constexpr int TW = CW * FT_WARPS * FT_COLS;      // fingerprints per tile
    __shared__ __align__(16) uint32_t s_q[FT_MAX_TQ];
    __shared__ uint32_t s_q2[COMB ? FT_MAX_TQ : 1];  // combined types: the patterns' second fingerprints
    __shared__ uint64_t s_stage[FT_WARPS][FT_STAGE];
    __shared__ uint32_t s_cnt[FT_WARPS];
    __shared__ uint16_t s_queue[FT_WARPS][FT_QUEUE];
    __shared__ uint32_t s_qcnt[FT_WARPS];
    __shared__ uint64_t s_tile;
    __shared__ Segment s_seg;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nseg = (int)A.scal[0];
    const uint64_t ntiles = A.scal[1];
    uint64_t *stage = s_stage[warp];
    uint32_t *cnt = &s_cnt[warp];
    uint16_t *queue = s_queue[warp];
    uint32_t *qcnt = &s_qcnt[warp];
    if (lane == 0) {
        *cnt = 0;
        *qcnt = 0;
    }
    __syncwarp();
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd((unsigned long long *)&A.scal[3], 1ull);
        __syncthreads();
        const uint64_t tile = s_tile;
        if (tile >= ntiles) break;
        if (warp == 0) {  // the tile's segment and patterns
            const Segment S = A.seg[find_segment_warp(A.seg, nseg, tile, lane)];
            const uint32_t local = (uint32_t)(tile - S.tile_begin);
            const uint32_t qt = S.n_qtiles == 1u ? 0u : local / S.n_dtiles;
            const uint32_t q0 = S.q_start + qt * (uint32_t)A.tq;
            const uint32_t nq = min((uint32_t)A.tq, S.q_count - qt * (uint32_t)A.tq);
            for (uint32_t j = lane; j < nq; j += 32) {
                uint32_t f = (W == 32) ? A.qfp32[q0 + j] : (uint32_t)A.qfp16[q0 + j];
                s_q[j] = (W == 32) ? f : (f | (f << 16));
                if (COMB) s_q2[j] = A.qfp2[q0 + j];
            }
            if (lane == 0) s_seg = S;
        }
        __syncthreads();
        const uint32_t local = (uint32_t)(tile - s_seg.tile_begin);
        const uint32_t ndt = s_seg.n_dtiles;
        const uint32_t qt = s_seg.n_qtiles == 1u ? 0u : local / ndt;
        const uint32_t dt = local - qt * ndt;
        const uint32_t q0 = s_seg.q_start + qt * (uint32_t)A.tq;
        const uint32_t nq = min((uint32_t)A.tq, s_seg.q_count - qt * (uint32_t)A.tq);
        const uint32_t w0 = s_seg.d_start + dt * (uint32_t)TW;  // first fingerprint slot of the tile
        const uint32_t nw = min((uint32_t)TW, s_seg.d_count - dt * (uint32_t)TW);
        const int k = s_seg.k, metric = s_seg.metric;
        const uint32_t T = 2u * (uint32_t)k * (uint32_t)A.tmul;
        const uint32_t nb = (nq + 31u) >> 5;                         // batches of 32 patterns
        const uint32_t nit = ((nw + CW - 1u) / CW) * nb;             // items (column, batch)
        const uint32_t it1 = (uint32_t)(warp + 1) * nit / FT_WARPS;
        for (uint32_t it = (uint32_t)warp * nit / FT_WARPS; it < it1;) {
            const uint32_t col = it / nb, b0 = it - col * nb, b1 = min(nb, b0 + (it1 - it));
            const uint32_t wbase = w0 + col * CW;
            // the column's fingerprints, as 32-bit words (wbase is a multiple of 8
            // slots; slots past the tile end are readable slack or the next run)
            uint32_t w[V];
            const uint32_t word0 = (W == 32) ? wbase : wbase / 2;
#pragma unroll
            for (int r = 0; r < V / 4; r++) {
                const uint4 x = *reinterpret_cast<const uint4 *>(A.dfp + word0 + r * (32 * 4) + lane * 4);
                w[4 * r + 0] = x.x;
                w[4 * r + 1] = x.y;
                w[4 * r + 2] = x.z;
                w[4 * r + 3] = x.w;
            }
            const uint32_t nvalid = nw - col * CW;
            uint32_t invalid = 0;  // bit i: fingerprint i lies past the tile end (masked in the exact re-test)
#pragma unroll
            for (int i = 0; i < NF; i++)
                if (lane_offset<G>(i, lane) >= nvalid) invalid |= 1u << i;
            const uint32_t qa = b0 * 32u, qn = min(nq, b1 * 32u) - qa;
            if (K1MIX && T != 2u)  // a k = 1 variant given another k: exact general path
                scan_tile<W, V, FDK, false, false, FUSED, COMB>(A, s_q + qa, s_q2 + (COMB ? qa : 0u), qn, q0 + qa, w, invalid, T, wbase, stage,
                                                                cnt, queue, qcnt, lane, k, metric);
            else
                scan_tile<W, V, FDK, false, K1MIX, FUSED, COMB>(A, s_q + qa, s_q2 + (COMB ? qa : 0u), qn, q0 + qa, w, invalid, T, wbase, stage,
                                                                cnt, queue, qcnt, lane, k, metric);
            it += b1 - b0;
        }
        // fused: the next tile may have another (k, metric), so verify what is staged
        if (FUSED) verify_stage(A, stage, cnt, lane, k, metric);
        __syncthreads();
    }
    if (!FUSED) flush_stage(A, stage, cnt, lane);
}

// ---------------------------------------------------------------------------
// the same filter on the tensor cores
// ---------------------------------------------------------------------------
// With bit b of a fingerprint mapped to s_b = +1 (set) or -1 (clear), the dot
// product of two fingerprints' sign vectors is W - 2 F_D (every equal bit adds
// one, every differing bit subtracts one; F_D = H_W(x XOR y), Sec. 3.3), so
// F_D <= 2k (Eq. 1) iff dot >= W - 4k.  One mma.sync.m16n8k32 on FP8 (E4M3)
// operands, which hold +1 and -1 exactly, gives a warp 16 x 8 such dot
// products; they are integers of magnitude <= 32, exact in the FP16
// accumulators.  The accumulator starts at 0.5 - (W - 4k), so a pair passes
// iff its result is positive, i.e. iff its FP16 sign bit is clear.  A thread
// ANDs its results together and looks at them one by one only when a sign
// bit survives; passing pairs go to the same per-warp staging as above.
//
// Bit b of the fingerprint is K position (b / 8) * 4 + b % 4 (+16 for
// b % 8 >= 4) in both operands, which puts the eight bits a thread of the
// mma layout needs into one byte: thread t of a quad takes byte t, expanded
// to eight FP8 values by a 256-entry table.  16-bit fingerprints use the
// first 16 positions and leave the other 16 zero.
constexpr int FM_THREADS = 256;  // the tensor-core filter keeps 8 warps per block
constexpr int FM_WARPS = FM_THREADS / 32;
constexpr int FM_TQ = 128;                       // patterns per tile: 8 row tiles of 16
constexpr int FM_RT = FM_TQ / 16;
constexpr int FM_GROUPS = 16;                    // groups of 8 words per warp and tile
constexpr int FM_TW = FM_WARPS * FM_GROUPS * 8;  // 1024 words per tile
#ifndef FM_MIN_BLOCKS
#define FM_MIN_BLOCKS 2
#endif

__device__ __forceinline__ void mma_e4m3_f16(uint32_t &d0, uint32_t &d1, const uint32_t (&a)[4], uint32_t b0,
                                             uint32_t b1, uint32_t c) {
    asm("mma.sync.aligned.m16n8k32.row.col.f16.e4m3.e4m3.f16 {%0,%1}, {%2,%3,%4,%5}, {%6,%7}, {%8,%8};"
        : "=r"(d0), "=r"(d1)
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1), "r"(c));
}

template <int W, bool FUSED, bool COMB>
__global__ void __launch_bounds__(FM_THREADS, FM_MIN_BLOCKS) k_filter_mma(FilterArgs A) {
    __shared__ uint2 s_lut[256];  // byte -> eight E4M3 values (+1 for a set bit, -1 for a clear one)
    __shared__ uint32_t s_q[FM_TQ];
    __shared__ __align__(16) uint32_t s_w[FM_TW];
    __shared__ uint64_t s_stage[FM_WARPS][FT_STAGE];
    __shared__ uint32_t s_cnt[FM_WARPS];
    __shared__ uint64_t s_tile;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    for (int v = threadIdx.x; v < 256; v += FM_THREADS) {
        uint32_t lo = 0, hi = 0;
#pragma unroll
        for (int i = 0; i < 4; i++) {
            lo |= (((v >> i) & 1) ? 0x38u : 0xB8u) << (8 * i);
            hi |= (((v >> (4 + i)) & 1) ? 0x38u : 0xB8u) << (8 * i);
        }
        s_lut[v] = make_uint2(lo, hi);
    }
    const int nseg = (int)A.scal[0];
    const uint64_t ntiles = A.scal[1];
    uint64_t *stage = s_stage[warp];
    uint32_t *cnt = &s_cnt[warp];
    if (lane == 0) *cnt = 0;
    const bool live = W == 32 || t < 2;  // 16-bit fingerprints: bytes 2 and 3 stay zero
    const uint32_t wrel0 = (uint32_t)warp * (FM_GROUPS * 8);
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd((unsigned long long *)&A.scal[3], 1ull);
        __syncthreads();
        const uint64_t tile = s_tile;
        if (tile >= ntiles) break;
        const Segment S = A.seg[find_segment(A.seg, nseg, tile)];
        const uint64_t local = tile - S.tile_begin;
        const uint32_t qt = (uint32_t)(local / S.n_dtiles), dt = (uint32_t)(local % S.n_dtiles);
        const uint32_t q0 = S.q_start + qt * (uint32_t)FM_TQ;
        const uint32_t nq = min((uint32_t)FM_TQ, S.q_count - qt * (uint32_t)FM_TQ);
        const uint32_t w0 = S.d_start + dt * (uint32_t)FM_TW;
        const uint32_t nw = min((uint32_t)FM_TW, S.d_count - dt * (uint32_t)FM_TW);
        for (uint32_t j = threadIdx.x; j < (uint32_t)FM_TQ; j += FM_THREADS)
            s_q[j] = j < nq ? ((W == 32) ? A.qfp32[q0 + j] : (uint32_t)A.qfp16[q0 + j]) : 0u;
        if (W == 32) {
            // w0 is a multiple of 8 slots and the slack after the last bucket is
            // readable, so whole 128-bit vectors may be loaded past nw
            for (uint32_t j = threadIdx.x; j * 4 < nw; j += FM_THREADS)
                *reinterpret_cast<uint4 *>(&s_w[4 * j]) = *reinterpret_cast<const uint4 *>(A.dfp + w0 + 4 * j);
        } else {
            const uint16_t *d16 = reinterpret_cast<const uint16_t *>(A.dfp);
            for (uint32_t j = threadIdx.x; j < nw; j += FM_THREADS) s_w[j] = d16[w0 + j];
        }
        __syncthreads();
        const int nr = (int)((nq + 15u) / 16u);
        const float Tf = (float)((W == 32 ? 32 : 16) - 4 * S.k * A.tmul);  // pass iff dot >= W - 4 tmul k
        const __half2 hb = __float2half2_rn(0.5f - Tf);
        const uint32_t bias = *reinterpret_cast<const uint32_t *>(&hb);
        uint32_t a[FM_RT][4];
#pragma unroll
        for (int r = 0; r < FM_RT; r++) {
            const uint32_t r0 = (uint32_t)(r * 16 + g), r1 = r0 + 8u;
            uint2 x0 = make_uint2(0u, 0u), x1 = make_uint2(0u, 0u);
            if (live && r0 < nq) x0 = s_lut[(s_q[r0] >> (8 * t)) & 0xFFu];
            if (live && r1 < nq) x1 = s_lut[(s_q[r1] >> (8 * t)) & 0xFFu];
            a[r][0] = x0.x;
            a[r][1] = x1.x;
            a[r][2] = x0.y;
            a[r][3] = x1.y;
        }
        for (int gi = 0; gi < FM_GROUPS; gi++) {
            const uint32_t wrel = wrel0 + (uint32_t)gi * 8u;
            if (wrel >= nw) break;  // warp-uniform
            uint32_t b0 = 0u, b1 = 0u;
            if (live && wrel + g < nw) {
                const uint2 x = s_lut[(s_w[wrel + g] >> (8 * t)) & 0xFFu];
                b0 = x.x;
                b1 = x.y;
            }
            uint32_t d[FM_RT][2];
            uint32_t all = 0xFFFFFFFFu;
#pragma unroll
            for (int r = 0; r < FM_RT; r++) {
                if (r < nr) {
                    mma_e4m3_f16(d[r][0], d[r][1], a[r], b0, b1, bias);
                    all &= d[r][0] & d[r][1];
                } else {
                    d[r][0] = d[r][1] = 0xFFFFFFFFu;
                }
            }
            if ((all & 0x80008000u) != 0x80008000u) {  // some result of this thread is positive
#pragma unroll
                for (int r = 0; r < FM_RT; r++) {
                    if (((d[r][0] & d[r][1]) & 0x80008000u) == 0x80008000u) continue;
#pragma unroll
                    for (int h = 0; h < 4; h++) {
                        const uint32_t reg = d[r][h >> 1];
                        if ((reg >> ((h & 1) ? 31 : 15)) & 1u) continue;
                        const uint32_t row = (uint32_t)(r * 16 + g + (h >> 1) * 8);
                        const uint32_t col = wrel + 2u * (uint32_t)t + (uint32_t)(h & 1);
                        if (row < nq && col < nw)
                            stage_push<FUSED, COMB>(A, stage, cnt, ((uint64_t)(q0 + row) << 32) | (uint64_t)(w0 + col), S.k,
                                              S.metric);
                    }
                }
            }
            __syncwarp();
            if (*cnt >= FT_STAGE / 2) {
                if (FUSED) verify_stage(A, stage, cnt, lane, S.k, S.metric);
                else flush_stage(A, stage, cnt, lane);
            }
        }
        if (FUSED) verify_stage(A, stage, cnt, lane, S.k, S.metric);
        __syncthreads();
    }
    if (!FUSED) flush_stage(A, stage, cnt, lane);
}

template <int W, bool FUSED, bool COMB>
static int launch_mma(const FilterArgs &A, cudaStream_t st) {
    static int grid = 0;
    if (grid == 0) {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_filter_mma<W, FUSED, COMB>, FM_THREADS, 0);
        grid = sm_count() * (per_sm > 0 ? per_sm : 1);
    }
    k_filter_mma<W, FUSED, COMB><<<grid, FM_THREADS, 0, st>>>(A);
    FP_LAUNCHED(FUSED ? "k_filter_mma(fused)" : "k_filter_mma");
    return FP_OK;
}

template <int W, int V, int FDK, bool FUSED, bool COMB = false>
static int launch_one(const FilterArgs &A, bool k1mix, cudaStream_t st) {
    constexpr bool MIX = W == 32 && FDK == FDK_POPC;  // the k = 1 mixed POPC / ALU test needs popcount fingerprints
    static int grid[2] = {0, 0};
    int &g = grid[k1mix ? 1 : 0];
    if (g == 0) {
        int per_sm = 0;
        if (k1mix)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_filter_tiled<W, V, FDK, MIX, FUSED, COMB>,
                                                          FT_THREADS, 0);
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_filter_tiled<W, V, FDK, false, FUSED, COMB>,
                                                          FT_THREADS, 0);
        g = sm_count() * (per_sm > 0 ? per_sm : 1);
    }
    if (k1mix) k_filter_tiled<W, V, FDK, MIX, FUSED, COMB><<<g, FT_THREADS, 0, st>>>(A);
    else k_filter_tiled<W, V, FDK, false, FUSED, COMB><<<g, FT_THREADS, 0, st>>>(A);
    FP_LAUNCHED(FUSED ? "k_filter_tiled(fused)" : "k_filter_tiled");
    return FP_OK;
}

// The F_D kind of a fingerprint type.
static int fd_kind(int type) { return type == FP_POS ? FDK_POS : (type == FP_COUNT_L1 ? FDK_L1 : FDK_POPC); }

template <bool FUSED>
static int dispatch(const FilterArgs &A, const FpParams &fp, const FilterCfg &cfg, cudaStream_t st) {
    const int kind = fd_kind(fp.type);
    const bool pos = kind == FDK_POS;
    // combined types (32-bit count fingerprints only): their own instances, so
    // that the other kernels carry no second check
    const bool comb = A.qfp2 != nullptr && fp.width == 32 && kind == FDK_POPC;
    const bool mix = cfg.k1mix && fp.width == 32 && kind == FDK_POPC;
    if (comb) {
        if (cfg.mma) return launch_mma<32, FUSED, true>(A, st);
        return launch_one<32, 4, FDK_POPC, FUSED, true>(A, mix, st);
    }
    if (kind == FDK_L1)  // count L1: 4 words per thread, no mixed test, no tensor-core form
        return fp.width == 32 ? launch_one<32, 4, FDK_L1, FUSED>(A, false, st)
                              : launch_one<16, 4, FDK_L1, FUSED>(A, false, st);
    if (cfg.mma && !pos) return fp.width == 32 ? launch_mma<32, FUSED, false>(A, st) : launch_mma<16, FUSED, false>(A, st);
    if (FUSED) {  // the fused form is built for 4 words per thread only
        if (fp.width == 32)
            return pos ? launch_one<32, 4, FDK_POS, true>(A, false, st) : launch_one<32, 4, FDK_POPC, true>(A, mix, st);
        return pos ? launch_one<16, 4, FDK_POS, true>(A, false, st) : launch_one<16, 4, FDK_POPC, true>(A, false, st);
    }
    if (fp.width == 32) {
        if (cfg.v == 4)
            return pos ? launch_one<32, 4, FDK_POS, false>(A, false, st) : launch_one<32, 4, FDK_POPC, false>(A, mix, st);
        return pos ? launch_one<32, 8, FDK_POS, false>(A, false, st) : launch_one<32, 8, FDK_POPC, false>(A, mix, st);
    }
    if (cfg.v == 4)
        return pos ? launch_one<16, 4, FDK_POS, false>(A, false, st) : launch_one<16, 4, FDK_POPC, false>(A, false, st);
    return pos ? launch_one<16, 8, FDK_POS, false>(A, false, st) : launch_one<16, 8, FDK_POPC, false>(A, false, st);
}

int tile_words(int width, int v) { return (width == 32 ? v : 2 * v) * FT_THREADS * FT_COLS; }

void tile_shape(const FilterCfg &cfg, const FpParams &fp, int *tq, int *tw) {
    if (cfg.mma && fd_kind(fp.type) == FDK_POPC) {
        *tq = FM_TQ;
        *tw = FM_TW;
    } else {
        *tq = cfg.tq < 1 ? 1 : (cfg.tq > FT_MAX_TQ ? FT_MAX_TQ : cfg.tq);
        *tw = tile_words(fp.width, fd_kind(fp.type) == FDK_L1 ? 4 : cfg.v);
    }
}

static FilterArgs make_args(const Bucketed &q, const Bucketed &d, const QueryPlan &plan, const FpParams &fp,
                            const FilterCfg &cfg) {
    FilterArgs A{};
    A.qfp32 = (const uint32_t *)q.fp;
    A.qfp16 = (const uint16_t *)q.fp;
    A.dfp = (const uint32_t *)d.fp;
    A.seg = plan.seg;
    A.scal = plan.scal;
    const bool rep = fp.width == 16;
    A.M.low = fp.pos_low | (rep ? fp.pos_low << 16 : 0u);
    A.M.high = fp.pos_high | (rep ? fp.pos_high << 16 : 0u);
    A.M.occ = fp.pos_occ | (rep ? fp.pos_occ << 16 : 0u);
    A.tq = cfg.tq < 1 ? 1 : (cfg.tq > FT_MAX_TQ ? FT_MAX_TQ : cfg.tq);
    A.tmul = fp.q > 0 ? fp.q : 1;
    A.qfp2 = q.fp2;  // combined types (null otherwise); both sets or neither
    A.dfp2 = q.fp2 ? d.fp2 : nullptr;
    return A;
}

int launch_filter(const Bucketed &q, const Bucketed &d, const QueryPlan &plan, const FpParams &fp,
                  const FilterCfg &cfg, uint64_t *surv, int64_t surv_cap, cudaStream_t st,
                  int64_t *launches) {
    FilterArgs A = make_args(q, d, plan, fp, cfg);
    A.surv = surv;
    A.surv_cap = (uint64_t)surv_cap;
    int rc = dispatch<false>(A, fp, cfg, st);
    if (launches) (*launches)++;
    return rc;
}

int launch_fused(const Bucketed &q, const Bucketed &d, const QueryPlan &plan, const FpParams &fp,
                 const FilterCfg &cfg, int idx_bits, uint64_t *matches, int64_t match_cap, cudaStream_t st,
                 int64_t *launches) {
    FilterArgs A = make_args(q, d, plan, fp, cfg);
    A.q_len = q.len;
    A.d_len = d.len;
    A.q_row16 = q.row16;
    A.d_row16 = d.row16;
    A.q_str = q.str;
    A.d_str = d.str;
    A.q_idx = q.idx;
    A.d_idx = d.idx;
    A.idx_bits = idx_bits;
    A.matches = matches;
    A.match_cap = (uint64_t)match_cap;
    int rc = dispatch<true>(A, fp, cfg, st);
    if (launches) (*launches)++;
    return rc;
}

}  // namespace fpk
