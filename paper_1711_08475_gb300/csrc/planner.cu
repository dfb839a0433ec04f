// The tile planner: turns the bucket counts of a pattern batch and of the
// dictionary into the segments the filter kernels walk (one block of 1024
// threads, two passes: count, block-wide scan, write).
//
// A segment is a run of query slots against a run of dictionary slots of one
// admissible length pair (equal lengths for the Hamming distance, lengths
// within k for Levenshtein, Sec. 3.3) with the (k, metric) of its group; it is
// cut into tiles of tq queries x tw words.  Eq. 1 holds for each pair in a
// segment's range or fails for it, so a plan only decides which pairs are
// tested, never the result.
#include "common.cuh"

namespace fpk {

// ---------------------------------------------------------------------------
// tile planner: one block
// ---------------------------------------------------------------------------
// Without weight bands a segment is (query bin, dictionary bucket) with
// ceil(q/tq) x ceil(d/tw) tiles.  With weight bands the patterns of every
// bin and the words of every bucket are ordered by weight cell (x, y, z)
// (fp_cell: the population counts of the fingerprint's three parts), and a
// segment is (tile of tq patterns, dictionary bucket, run of cells).  From
// the cells of the tile's first and last pattern, (x1, y1, z1) and
// (x2, y2, z2) in cell (lexicographic) order, the tile's box is x in
// [x1, x2], y in [y1, y2] when x1 = x2 (else all), z in [z1, z2] when also
// y1 = y2 (else all).  A word with cell (x', y', z') can pass Eq. 1 for some
// pattern of the tile only if its L1 distance to the box is at most 2k (the
// parts' weight differences add up to at most popc of the XOR).  So for every
// admissible (x', y') the tile tests one run of cells (x', y', z_lo .. z_hi),
// a run of slots in the bucket; each run starts at the 8-slot boundary below
// its first word (the words in between fail the bound too) so that tiles keep
// their aligned vector loads, and runs that then touch or overlap are merged,
// so no pair is tested twice.  "pairs" counts every eligible pair, tested or
// not; "tested" the pairs the tiles test.
struct PlanCounts {
    int32_t nseg = 0;
    uint64_t tiles = 0, pairs = 0, tested = 0;
};

constexpr int PLAN_MAX_BINS = 8192;  // 32 (k, metric) groups x 256 lengths
constexpr int PLAN_CHUNK = 6;  // table loads a planner thread keeps in flight per length
#ifndef PLAN_MERGE_GAP
#define PLAN_MERGE_GAP 0u  // runs closer than this many slots are merged (the gap's words are tested too)
#endif

__device__ __forceinline__ int slot_cell_of(const void *fp, int width, uint32_t s) {
    return fp_cell(width == 16 ? (uint32_t)((const uint16_t *)fp)[s] : ((const uint32_t *)fp)[s], width);
}

template <bool WRITE>
__device__ __forceinline__ void plan_emit(uint32_t q0, int qn, uint32_t nqt, uint32_t ds, uint32_t dn, int tw, int k,
                                          int metric, Segment *seg, int max_segments, int64_t &si, uint64_t &tb,
                                          PlanCounts &pc) {
    const uint32_t ndt = (dn + (uint32_t)tw - 1u) / (uint32_t)tw;
    pc.nseg++;
    pc.tiles += (uint64_t)nqt * ndt;
    pc.tested += (uint64_t)qn * dn;
    if (WRITE) {
        Segment sg;
        sg.q_start = q0;
        sg.q_count = (uint32_t)qn;
        sg.d_start = ds;
        sg.d_count = dn;
        sg.n_qtiles = nqt;
        sg.n_dtiles = ndt;
        sg.tile_begin = tb;
        sg.k = k;
        sg.metric = metric;
        if (si < max_segments) seg[si] = sg;
        si++;
        tb += (uint64_t)nqt * ndt;
    }
}

__device__ __forceinline__ int64_t plan_units(int qc, bool band, int tq) {
    return qc <= 0 ? 0 : (band ? (qc + tq - 1) / tq : 1);
}

// Unit u of bin c: the bin's patterns (no bands) or its u-th tile of tq
// patterns; segments per dictionary bucket within the length window.
template <bool WRITE>
__device__ void plan_unit(int c, int64_t u, const int32_t *__restrict__ qb_start, const int32_t *__restrict__ qb_count,
                          const int32_t *__restrict__ db_start, const int32_t *__restrict__ db_count,
                          const int32_t *__restrict__ group_k, const int32_t *__restrict__ group_metric, int tq,
                          int tw, const void *q_fp, int width, int tmul, const int32_t *__restrict__ d_wstart, bool band,
                          Segment *seg, int max_segments, int64_t &si, uint64_t &tb, PlanCounts &pc) {
    const int qc = qb_count[c];
    const int g = c >> 8, n = c & 255, k = group_k[g], metric = group_metric[g];
    const int L0 = metric == FP_HAM ? n : (n - k < 0 ? 0 : n - k);
    const int L1 = metric == FP_HAM ? n : (n + k > MAX_LEN ? MAX_LEN : n + k);
    const uint32_t q0 = (uint32_t)qb_start[c] + (band ? (uint32_t)(u * tq) : 0u);
    const int qn = band ? min(tq, qc - (int)(u * tq)) : qc;
    const uint32_t nqt = band ? 1u : (uint32_t)((qc + tq - 1) / tq);
    if (!band) {
        for (int L = L0; L <= L1; L++) {
            const int dc = db_count[L];
            if (dc <= 0) continue;
            pc.pairs += (uint64_t)qn * (uint64_t)dc;
            plan_emit<WRITE>(q0, qn, nqt, (uint32_t)db_start[L], (uint32_t)dc, tw, k, metric, seg, max_segments, si, tb,
                             pc);
        }
        return;
    }
    const int R1 = cell_part_radix(width, 1), R2 = cell_part_radix(width, 2), NC = cell_count(width);
    const int H0 = cell_part_bits(width, 0), H1 = R1 - 1, H2 = R2 - 1, r2k = 2 * k * tmul;  // F_D <= 2 tmul k can pass
    const int cf = slot_cell_of(q_fp, width, q0), cl = slot_cell_of(q_fp, width, q0 + (uint32_t)qn - 1u);
    // the tile's box from its first and last pattern (cell order is
    // lexicographic in (x, y, z))
    const int xa = cf / (R1 * R2), xb = cl / (R1 * R2);
    const int y1 = cf / R2 % R1, y2 = cl / R2 % R1, z1 = cf % R2, z2 = cl % R2;
    const int ya = xa == xb ? y1 : 0, yb = xa == xb ? y2 : H1;
    const int za = xa == xb && y1 == y2 ? z1 : 0, zb = xa == xb && y1 == y2 ? z2 : H2;
    const int xlo = max(0, xa - r2k), xhi = min(H0, xb + r2k);
    for (int L = L0; L <= L1; L++) {
        const int dc = db_count[L];
        if (dc <= 0) continue;
        pc.pairs += (uint64_t)qn * (uint64_t)dc;
        const int32_t *tab = d_wstart + (size_t)L * (NC + 1);
        uint32_t ps = 0, pe = 0;  // pending run of slots [ps, pe)
        bool pending = false;
        for (int x = xlo; x <= xhi; x++) {
            const int r1 = r2k - max(0, max(xa - x, x - xb));
            const int ylo = max(0, ya - r1), yhi = min(H1, yb + r1);
            // the runs of PLAN_CHUNK consecutive y' at a time: their table
            // loads are all in flight at once, then merged in order
            for (int yc = ylo; yc <= yhi; yc += PLAN_CHUNK) {
                int32_t fs[PLAN_CHUNK], es[PLAN_CHUNK];
#pragma unroll
                for (int j = 0; j < PLAN_CHUNK; j++) {
                    const int y = yc + j;
                    fs[j] = 0;
                    es[j] = 0;
                    if (y <= yhi) {
                        const int r2 = r1 - max(0, max(ya - y, y - yb));
                        const int zlo = max(0, za - r2), zhi = min(H2, zb + r2);
                        const int cxy = (x * R1 + y) * R2;
                        fs[j] = tab[cxy + zlo];
                        es[j] = tab[cxy + zhi + 1];
                    }
                }
#pragma unroll
                for (int j = 0; j < PLAN_CHUNK; j++) {
                    const int32_t first = fs[j], end = es[j];
                    if (end <= first) continue;
                    const uint32_t s8 = (uint32_t)first & ~(uint32_t)(SLOT_ALIGN - 1);
                    if (pending && s8 <= pe + PLAN_MERGE_GAP) {
                        pe = max(pe, (uint32_t)end);
                    } else {
                        if (pending)
                            plan_emit<WRITE>(q0, qn, 1u, ps, pe - ps, tw, k, metric, seg, max_segments, si, tb, pc);
                        ps = s8;
                        pe = (uint32_t)end;
                        pending = true;
                    }
                }
            }
        }
        if (pending) plan_emit<WRITE>(q0, qn, 1u, ps, pe - ps, tw, k, metric, seg, max_segments, si, tb, pc);
    }
}

// One block of 1024 threads.  The units (bins, or tiles of bins with weight
// bands) are numbered bin by bin; thread t plans units [t U / 1024,
// (t + 1) U / 1024): a counting pass, a block scan of the segment and tile
// counts, and a writing pass.  only_if (optional): plan only when *only_if is
// set (the parallel banded planner's fall-back to whole buckets).
__global__ void __launch_bounds__(1024) k_plan_segments(
    const int32_t *__restrict__ qb_start, const int32_t *__restrict__ qb_count, int q_nbins,
    const int32_t *__restrict__ db_start, const int32_t *__restrict__ db_count,
    const int32_t *__restrict__ group_k, const int32_t *__restrict__ group_metric, int tq, int tw, const void *q_fp,
    int width, int tmul, const int32_t *__restrict__ d_wstart, Segment *__restrict__ seg, int max_segments,
    uint64_t *__restrict__ scal, const uint64_t *only_if) {
    if (only_if && *only_if == 0) return;  // block-uniform
    __shared__ int32_t s_unit0[PLAN_MAX_BINS + 1];  // first unit of every bin
    __shared__ int32_t s_n[1024];
    __shared__ uint64_t s_t[1024];
    __shared__ unsigned long long s_pairs, s_tested;
    const int t = threadIdx.x;
    // a banded plan that does not fit falls back to whole buckets (which fit
    // whenever max_segments >= bins x (2k + 1))
    bool band = q_fp != nullptr && d_wstart != nullptr;
    const int nbins = min(q_nbins, PLAN_MAX_BINS);
    bool too_many = false;
    int64_t u0 = 0, u1 = 0;
    int c0 = 0;
    PlanCounts pc;
    for (;;) {
        if (t == 0) {
            s_pairs = 0;
            s_tested = 0;
        }
        // units per bin and their prefix
        {
            const int per = (nbins + 1023) / 1024;
            const int lo = min(nbins, t * per), hi = min(nbins, lo + per);
            int64_t a = 0;
            for (int c = lo; c < hi; c++) a += plan_units(qb_count[c], band, tq);
            s_t[t] = (uint64_t)a;
            __syncthreads();
            for (int o = 1; o < 1024; o <<= 1) {
                const uint64_t v = t >= o ? s_t[t - o] : 0;
                __syncthreads();
                s_t[t] += v;
                __syncthreads();
            }
            int64_t r = (int64_t)s_t[t] - a;
            for (int c = lo; c < hi; c++) {
                s_unit0[c] = (int32_t)(r < 0x7FFFFFFF ? r : 0x7FFFFFFF);
                r += plan_units(qb_count[c], band, tq);
            }
            if (t == 1023) s_unit0[nbins] = (int32_t)(s_t[1023] < 0x7FFFFFFFull ? s_t[1023] : 0x7FFFFFFFull);
            __syncthreads();
        }
        too_many = s_t[1023] >= 0x7FFFFFFFull;  // units beyond int32: refuse the plan
        const int64_t U = too_many ? 0 : s_unit0[nbins];
        u0 = U * t / 1024;
        u1 = U * (t + 1) / 1024;
        {  // bin of unit u0: last bin whose first unit is <= u0
            int lo = 0, hi = nbins - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (s_unit0[mid] <= u0) lo = mid;
                else hi = mid - 1;
            }
            c0 = lo;
        }
        pc = PlanCounts{};
        int64_t si = 0;
        uint64_t tb = 0;
        for (int64_t u = u0, c = c0; u < u1; u++) {
            while (s_unit0[c + 1] <= u) c++;
            plan_unit<false>((int)c, u - s_unit0[c], qb_start, qb_count, db_start, db_count, group_k, group_metric,
                             tq, tw, q_fp, width, tmul, d_wstart, band, seg, max_segments, si, tb, pc);
        }
        s_n[t] = pc.nseg;
        s_t[t] = pc.tiles;
        atomicAdd(&s_pairs, (unsigned long long)pc.pairs);
        atomicAdd(&s_tested, (unsigned long long)pc.tested);
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            const int32_t a = t >= o ? s_n[t - o] : 0;
            const uint64_t b = t >= o ? s_t[t - o] : 0;
            __syncthreads();
            s_n[t] += a;
            s_t[t] += b;
            __syncthreads();
        }
        if (!(band && s_n[1023] > max_segments)) break;
        band = false;
        __syncthreads();  // everyone has read s_n[1023] before it is reused
    }
    int64_t si;
    uint64_t tb;
    si = (int64_t)s_n[t] - pc.nseg;
    tb = s_t[t] - pc.tiles;
    PlanCounts again;
    for (int64_t u = u0, c = c0; u < u1; u++) {
        while (s_unit0[c + 1] <= u) c++;
        plan_unit<true>((int)c, u - s_unit0[c], qb_start, qb_count, db_start, db_count, group_k, group_metric, tq,
                        tw, q_fp, width, tmul, d_wstart, band, seg, max_segments, si, tb, again);
    }
    if (t == 1023) {
        const int64_t ns = s_n[1023];
        const bool over = ns > max_segments || q_nbins > PLAN_MAX_BINS || too_many;
        scal[0] = (uint64_t)(ns < max_segments ? ns : max_segments);
        scal[1] = over ? 0 : s_t[1023];  // refuse to run an incomplete plan
        scal[2] = s_pairs;
        scal[3] = 0;
        scal[4] = 0;
        scal[5] = 0;
        scal[6] = over ? 1 : 0;
        scal[7] = s_tested;
    }
}

// ---------------------------------------------------------------------------
// the banded planner over many blocks
// ---------------------------------------------------------------------------
// One thread per unit (tile of patterns), so that the chains of table loads of
// different tiles run on the whole GPU instead of one block:
//   k_plan_prefix  (1 block)  first unit of every bin, unit count
//   k_plan_units   (a thread per unit) segments and tiles per unit, pair sums
//   k_plan_offsets (1 block)  exclusive prefix of both, the counters
//   k_plan_units   again, writing each unit's segments at its offsets
// acc: [0] eligible pairs, [1] tested pairs, [2] fall-back flag (the units or
// the segments do not fit: k_plan_segments then plans whole buckets), [3] U.
__global__ void __launch_bounds__(1024) k_plan_prefix(const int32_t *__restrict__ qb_count, int nbins, int tq,
                                                      int32_t *__restrict__ unit0, uint64_t *__restrict__ acc,
                                                      int units_cap) {
    __shared__ uint64_t s_t[1024];
    const int t = threadIdx.x, per = (nbins + 1023) / 1024;
    const int lo = min(nbins, t * per), hi = min(nbins, lo + per);
    uint64_t a = 0;
    for (int c = lo; c < hi; c++) a += (uint64_t)plan_units(qb_count[c], true, tq);
    s_t[t] = a;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const uint64_t v = t >= o ? s_t[t - o] : 0;
        __syncthreads();
        s_t[t] += v;
        __syncthreads();
    }
    const uint64_t U = s_t[1023];
    const bool fits = U <= (uint64_t)units_cap;
    uint64_t r = s_t[t] - a;
    for (int c = lo; c < hi; c++) {
        unit0[c] = fits ? (int32_t)r : 0;
        r += (uint64_t)plan_units(qb_count[c], true, tq);
    }
    if (t == 0) {
        unit0[nbins] = fits ? (int32_t)U : 0;
        acc[0] = 0;
        acc[1] = 0;
        acc[2] = fits ? 0 : 1;
        acc[3] = fits ? U : 0;
    }
}

template <bool WRITE>
__global__ void __launch_bounds__(128) k_plan_units(
    const int32_t *__restrict__ qb_start, const int32_t *__restrict__ qb_count, int nbins,
    const int32_t *__restrict__ db_start, const int32_t *__restrict__ db_count,
    const int32_t *__restrict__ group_k, const int32_t *__restrict__ group_metric, int tq, int tw, const void *q_fp,
    int width, int tmul, const int32_t *__restrict__ d_wstart, Segment *__restrict__ seg, int max_segments,
    const int32_t *__restrict__ unit0, int32_t *__restrict__ u_seg, uint64_t *__restrict__ u_tiles,
    uint64_t *__restrict__ acc) {
    __shared__ unsigned long long s_sum[2];
    const bool fallback = acc[2] != 0;
    const int64_t U = (int64_t)acc[3];
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (!WRITE && threadIdx.x < 2) s_sum[threadIdx.x] = 0;
    if (!WRITE) __syncthreads();
    PlanCounts pc;
    if (!fallback && u < U) {
        int lo = 0, hi = nbins - 1;  // bin of the unit: the last bin whose first unit is <= u
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (unit0[mid] <= u) lo = mid;
            else hi = mid - 1;
        }
        int64_t si = WRITE ? (int64_t)u_seg[u] : 0;
        uint64_t tb = WRITE ? u_tiles[u] : 0;
        plan_unit<WRITE>(lo, u - unit0[lo], qb_start, qb_count, db_start, db_count, group_k, group_metric, tq, tw,
                         q_fp, width, tmul, d_wstart, true, seg, max_segments, si, tb, pc);
        if (!WRITE) {
            u_seg[u] = pc.nseg;
            u_tiles[u] = pc.tiles;
        }
    }
    if (!WRITE) {
        unsigned long long p = pc.pairs, x = pc.tested;
        for (int o = 16; o > 0; o >>= 1) {
            p += __shfl_down_sync(0xffffffffu, p, o);
            x += __shfl_down_sync(0xffffffffu, x, o);
        }
        if ((threadIdx.x & 31) == 0 && (p | x)) {
            atomicAdd(&s_sum[0], p);
            atomicAdd(&s_sum[1], x);
        }
        __syncthreads();
        if (threadIdx.x == 0 && (s_sum[0] | s_sum[1])) {
            atomicAdd((unsigned long long *)&acc[0], s_sum[0]);
            atomicAdd((unsigned long long *)&acc[1], s_sum[1]);
        }
    }
}

// Exclusive prefix of the segments and tiles per unit, in place (one block;
// thread t takes a contiguous run of units), then the plan's counters.
__global__ void __launch_bounds__(1024) k_plan_offsets(int32_t *__restrict__ u_seg, uint64_t *__restrict__ u_tiles,
                                                       uint64_t *__restrict__ acc, int max_segments,
                                                       uint64_t *__restrict__ scal) {
    __shared__ int64_t s_n[1024];
    __shared__ uint64_t s_t[1024];
    if (acc[2] != 0) return;  // block-uniform: the fall-back planner writes the counters
    const int t = threadIdx.x;
    const int64_t U = (int64_t)acc[3], per = (U + 1023) / 1024;
    const int64_t lo = min(U, t * per), hi = min(U, lo + per);
    int64_t n = 0;
    uint64_t ti = 0;
    for (int64_t u = lo; u < hi; u++) {
        n += u_seg[u];
        ti += u_tiles[u];
    }
    s_n[t] = n;
    s_t[t] = ti;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const int64_t a = t >= o ? s_n[t - o] : 0;
        const uint64_t b = t >= o ? s_t[t - o] : 0;
        __syncthreads();
        s_n[t] += a;
        s_t[t] += b;
        __syncthreads();
    }
    const int64_t ns = s_n[1023];
    if (ns > max_segments) {  // does not fit: plan whole buckets instead
        if (t == 0) acc[2] = 1;
        return;
    }
    int64_t rn = s_n[t] - n;
    uint64_t rt = s_t[t] - ti;
    for (int64_t u = lo; u < hi; u++) {
        const int32_t a = u_seg[u];
        const uint64_t b = u_tiles[u];
        u_seg[u] = (int32_t)rn;
        u_tiles[u] = rt;
        rn += a;
        rt += b;
    }
    if (t == 1023) {
        scal[0] = (uint64_t)ns;
        scal[1] = s_t[1023];
        scal[2] = acc[0];
        scal[3] = 0;
        scal[4] = 0;
        scal[5] = 0;
        scal[6] = 0;
        scal[7] = acc[1];
    }
}

static size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

size_t plan_scratch_bytes(int64_t units_cap, int nbins) {
    return al256(4 * (size_t)(nbins + 1)) + al256(4 * (size_t)units_cap) + al256(8 * (size_t)units_cap) + al256(32);
}

void plan_scratch_place(QueryPlan *plan, uint8_t *base, int64_t units_cap, int nbins) {
    size_t off = 0;
    plan->units_cap = (int32_t)units_cap;
    plan->unit0 = (int32_t *)(base + off);
    off += al256(4 * (size_t)(nbins + 1));
    plan->u_seg = (int32_t *)(base + off);
    off += al256(4 * (size_t)units_cap);
    plan->u_tiles = (uint64_t *)(base + off);
    off += al256(8 * (size_t)units_cap);
    plan->acc = (uint64_t *)(base + off);
}

int plan_segments(const Bucketed &q, const Bucketed &d, const int32_t *d_group_k,
                  const int32_t *d_group_metric, int tq, int tw, QueryPlan *plan, cudaStream_t st,
                  const int32_t *d_wstart, int width, int tmul) {
    if (d_wstart && plan->unit0 && plan->units_cap > 0) {
        const unsigned blocks = (unsigned)((plan->units_cap + 127) / 128);
        k_plan_prefix<<<1, 1024, 0, st>>>(q.b_count, q.nbins, tq, plan->unit0, plan->acc, plan->units_cap);
        FP_LAUNCHED("k_plan_prefix");
        k_plan_units<false><<<blocks, 128, 0, st>>>(q.b_start, q.b_count, q.nbins, d.b_start, d.b_count, d_group_k,
                                                    d_group_metric, tq, tw, q.fp, width, tmul, d_wstart, plan->seg,
                                                    plan->max_segments, plan->unit0, plan->u_seg, plan->u_tiles,
                                                    plan->acc);
        FP_LAUNCHED("k_plan_units");
        k_plan_offsets<<<1, 1024, 0, st>>>(plan->u_seg, plan->u_tiles, plan->acc, plan->max_segments, plan->scal);
        FP_LAUNCHED("k_plan_offsets");
        k_plan_units<true><<<blocks, 128, 0, st>>>(q.b_start, q.b_count, q.nbins, d.b_start, d.b_count, d_group_k,
                                                   d_group_metric, tq, tw, q.fp, width, tmul, d_wstart, plan->seg,
                                                   plan->max_segments, plan->unit0, plan->u_seg, plan->u_tiles,
                                                   plan->acc);
        FP_LAUNCHED("k_plan_units");
        // whole buckets, only when the banded plan did not fit
        k_plan_segments<<<1, 1024, 0, st>>>(q.b_start, q.b_count, q.nbins, d.b_start, d.b_count, d_group_k,
                                            d_group_metric, tq, tw, nullptr, width, tmul, nullptr, plan->seg,
                                            plan->max_segments, plan->scal, plan->acc + 2);
        FP_LAUNCHED("k_plan_segments");
        return FP_OK;
    }
    k_plan_segments<<<1, 1024, 0, st>>>(q.b_start, q.b_count, q.nbins, d.b_start, d.b_count, d_group_k,
                                        d_group_metric, tq, tw, d_wstart ? q.fp : nullptr, width, tmul, d_wstart,
                                        plan->seg, plan->max_segments, plan->scal, nullptr);
    FP_LAUNCHED("k_plan_segments");
    return FP_OK;
}

}  // namespace fpk
