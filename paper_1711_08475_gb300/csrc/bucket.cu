// Length bucketing, symbol statistics and fingerprint construction.
//
// Sec. 3.4: the collection is preprocessed once and every word keeps one
// fixed-size fingerprint (O(|D| F + sigma) extra space).  Here the words are
// also grouped by length (Hamming compares only equal lengths, Levenshtein
// only lengths within k), each bucket holding a structure of arrays: the
// fingerprints (16- or 32-bit, 16-byte aligned rows of 8 slots), the original
// index, the length and the byte offset of a zero-padded copy of the string
// whose row length is a multiple of 16 bytes.
//
// Sec. 3.2 (construction): every fingerprint starts at zero and the string is
// read once, left to right; a symbol c whose field is q = map[c] sets or
// updates field q.  Sec. 3 (symbol sets): the map takes the most / least
// frequent symbols of the collection, or half of each.
#include <type_traits>

#include "common.cuh"

namespace fpk {

int make_params(int type, int width, int b, int p, FpParams *o, int q) {
    if (width != 16 && width != 32) return FP_E_INVAL;
    if (type < FP_OCC || type > FP_COUNT_L1) return FP_E_INVAL;
    if (b <= 0) b = 2;
    if (p <= 0) p = 3;
    if (q <= 0) q = 2;
    if (b > 8 || p > 8) return FP_E_UNSUPPORTED;
    if (type == FP_QGRAM && q > 3) return FP_E_UNSUPPORTED;
    if (type == FP_COUNT_L1 && b != 2) return FP_E_UNSUPPORTED;  // the filter's L1 arithmetic is for 2-bit counts
    FpParams P{};
    P.type = type;
    P.width = width;
    P.b = b;
    P.p = p;
    P.q = type == FP_QGRAM ? q : 1;
    switch (type) {
        case FP_OCC: P.sigma = width; break;
        case FP_QGRAM: P.sigma = width; break;
        case FP_OCC_HALVED: P.sigma = width / 2; break;
        case FP_COUNT:
        case FP_COUNT_L1:
            if (b > width) return FP_E_UNSUPPORTED;
            P.sigma = width / b;
            for (int f = 0; f < P.sigma; f++) P.count_top |= 1u << (b * f + b - 1);
            break;
        case FP_POS:
            if (p > width) return FP_E_UNSUPPORTED;
            P.n_pos = width / p;
            P.sigma = P.n_pos + (width - p * P.n_pos);
            for (int j = 0; j < P.n_pos; j++) {
                P.pos_high |= 1u << (p * j + p - 1);
                for (int t = 0; t < p - 1; t++) P.pos_low |= 1u << (p * j + t);
            }
            for (int t = p * P.n_pos; t < width; t++) P.pos_occ |= 1u << t;
            break;
    }
    *o = P;
    return FP_OK;
}

static int grid_for(int64_t n, int threads = 256, int cap = 8192) {
    int64_t g = (n + threads - 1) / threads;
    return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

// Counts one launch and returns its launch error as a status.
static int launched(const char *name) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FP_OK : cuda_fail(e, name);
}

// ---------------------------------------------------------------------------
// fingerprint of one string, byte by byte (Sec. 3.2)
// ---------------------------------------------------------------------------
// For FP_QGRAM (the future work of Sec. 5) a field is a q-gram, not a symbol:
// put() keeps the last q bytes as a rolling code (first byte most
// significant) and, from the q-th byte on, sets the bit of the q-gram ending
// here (P.gmap: code -> field or -1).  The other types map one byte.
template <int TYPE>
struct FpAcc {
    uint32_t v, seen;
    __device__ __forceinline__ void init(const FpParams &P) {
        seen = 0;
        v = (TYPE == FP_POS) ? (P.pos_low | P.pos_high) : 0u;
    }
    // byte ch at position pos of a string of length len (smap: byte -> field)
    __device__ __forceinline__ void put(uint32_t ch, const int8_t *smap, int pos, int len, const FpParams &P) {
        if (TYPE == FP_QGRAM) {
            seen = (seen << 8) | ch;  // rolling code of the last q bytes
            if (pos + 1 >= P.q) {
                const int f = P.gmap[seen & ((1u << (8 * P.q)) - 1u)];
                if (f >= 0) v |= 1u << f;
            }
        } else {
            add(smap[ch], pos, len, P);
        }
    }
    __device__ __forceinline__ void add(int q, int pos, int len, const FpParams &P) {
        if (q < 0) return;
        if (TYPE == FP_OCC) {
            v |= 1u << q;
        } else if (TYPE == FP_OCC_HALVED) {
            v |= 1u << (2 * q + (pos >= (len >> 1) ? 1 : 0));
        } else if (TYPE == FP_COUNT || TYPE == FP_COUNT_L1) {
            uint32_t sat = (1u << P.b) - 1u;
            uint32_t c = (v >> (P.b * q)) & sat;
            if (c < sat) v += 1u << (P.b * q);
        } else {
            if (q < P.n_pos) {
                if (!((seen >> q) & 1u)) {
                    seen |= 1u << q;
                    uint32_t sat = (1u << P.p) - 1u;
                    uint32_t f = (uint32_t)pos < sat ? (uint32_t)pos : sat;
                    v = (v & ~(sat << (P.p * q))) | (f << (P.p * q));
                }
            } else {
                v |= 1u << (P.p * P.n_pos + (q - P.n_pos));
            }
        }
    }
    __device__ __forceinline__ uint32_t finish(const FpParams &P) {
        uint32_t r = v;
        if (TYPE == FP_COUNT) r = r ^ ((r >> 1) & ~P.count_top);  // per-field reflected Gray code
        // FP_COUNT_L1 keeps the paper's plain binary counts
        if (P.width == 16) r &= 0xFFFFu;
        return r;
    }
};

__device__ __forceinline__ void store_fp(void *fp, int width, int64_t slot, uint32_t v) {
    if (width == 16) ((uint16_t *)fp)[slot] = (uint16_t)v;
    else ((uint32_t *)fp)[slot] = v;
}

// ---------------------------------------------------------------------------
// symbol statistics (Sec. 3 symbol sets)
// ---------------------------------------------------------------------------
__global__ void k_byte_hist(const uint8_t *__restrict__ chars, int64_t total,
                            unsigned long long *__restrict__ counts) {
    __shared__ uint32_t h[256];
    for (int t = threadIdx.x; t < 256; t += blockDim.x) h[t] = 0;
    __syncthreads();
    int64_t n16 = total / 16;
    const uint4 *c16 = (const uint4 *)chars;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint4 v = c16[i];
        uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int j = 0; j < 4; j++) {
#pragma unroll
            for (int s = 0; s < 32; s += 8) atomicAdd(&h[(w[j] >> s) & 0xFF], 1u);
        }
    }
    if (blockIdx.x == 0)
        for (int64_t i = n16 * 16 + threadIdx.x; i < total; i += blockDim.x) atomicAdd(&h[chars[i]], 1u);
    __syncthreads();
    for (int t = threadIdx.x; t < 256; t += blockDim.x)
        if (h[t]) atomicAdd(&counts[t], (unsigned long long)h[t]);
}

// One block of 256 threads, thread c decides the field of byte c.
__global__ void k_symbol_rank(const unsigned long long *__restrict__ counts, int set, int sigma,
                              int8_t *__restrict__ map) {
    __shared__ unsigned long long cnt[256];
    __shared__ int crank[256];
    const int c = threadIdx.x;
    cnt[c] = counts[c];
    __syncthreads();
    const unsigned long long mine = cnt[c];
    int cr = 0, rr = 0;
    for (int o = 0; o < 256; o++) {
        unsigned long long x = cnt[o];
        if (x == 0) continue;
        if (x > mine || (x == mine && o < c)) cr++;
        if (x < mine || (x == mine && o < c)) rr++;
    }
    crank[c] = cr;
    __syncthreads();
    int field = -1;
    if (mine > 0) {
        if (set == FP_SET_COMMON) {
            if (cr < sigma) field = cr;
        } else if (set == FP_SET_RARE) {
            if (rr < sigma) field = rr;
        } else {
            const int nc = (sigma + 1) / 2, nr = sigma / 2;
            if (cr < nc) {
                field = cr;
            } else {
                int r2 = 0;  // rank among the symbols not taken by the common half, least frequent first
                for (int o = 0; o < 256; o++) {
                    unsigned long long x = cnt[o];
                    if (x == 0 || crank[o] < nc) continue;
                    if (x < mine || (x == mine && o < c)) r2++;
                }
                if (r2 < nr) field = nc + r2;
            }
        }
    }
    map[c] = (int8_t)field;
}

int symbol_map(const uint8_t *d_chars, int64_t total, int set, int sigma, int8_t *d_map,
               unsigned long long *d_counts, cudaStream_t st) {
    FP_CUDA(cudaMemsetAsync(d_counts, 0, 256 * sizeof(unsigned long long), st));
    if (total > 0) {
        int64_t g = (total / 16 + 255) / 256;
        int grid = (int)(g < 1 ? 1 : (g > 1024 ? 1024 : g));
        k_byte_hist<<<grid, 256, 0, st>>>(d_chars, total, d_counts);
        FP_LAUNCHED("k_byte_hist");
    }
    k_symbol_rank<<<1, 256, 0, st>>>(d_counts, set, sigma, d_map);
    FP_LAUNCHED("k_symbol_rank");
    return FP_OK;
}

// ---------------------------------------------------------------------------
// q-gram statistics (Sec. 5 future work: fingerprints over q-grams)
// ---------------------------------------------------------------------------
// One thread per string: every q-gram occurrence (positions 0 .. len - q).
__global__ void k_qgram_hist(const uint8_t *__restrict__ chars, const int64_t *__restrict__ off, int64_t n, int q,
                             uint32_t *__restrict__ counts) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint8_t *s = chars + off[i];
        const int64_t L = off[i + 1] - off[i];
        uint32_t code = 0;
        for (int64_t j = 0; j < L; j++) {
            code = (code << 8) | s[j];
            if (j + 1 >= q) atomicAdd(&counts[code & ((1u << (8 * q)) - 1u)], 1u);
        }
    }
}

// The most frequent q-gram not yet taken: key (count << 24) | (2^24 - 1 -
// code), so the largest key has the highest count and, among equal counts,
// the smallest code.  Block maxima meet in one atomicMax.
__global__ void __launch_bounds__(256) k_qgram_argmax(const uint32_t *__restrict__ counts, int64_t ncodes,
                                                      unsigned long long *__restrict__ best) {
    unsigned long long m = 0;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncodes; c += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t v = counts[c];
        if (v) {
            const unsigned long long key = ((unsigned long long)v << 24) | (unsigned long long)(0xFFFFFFu - (uint32_t)c);
            m = key > m ? key : m;
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, m, o);
        m = y > m ? y : m;
    }
    __shared__ unsigned long long s_m[8];
    if ((threadIdx.x & 31) == 0) s_m[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; w++) m = s_m[w] > m ? s_m[w] : m;
        if (m) atomicMax(best, m);
    }
}

// Takes the winner of round f: field f, and its count is cleared so the next
// round skips it.  codes[f] = the code, or ~0 when no q-gram is left.
__global__ void k_qgram_take(unsigned long long *__restrict__ best, int f, uint32_t *__restrict__ counts,
                             int8_t *__restrict__ gmap, uint32_t *__restrict__ codes) {
    const unsigned long long m = *best;
    if (m == 0) {
        codes[f] = 0xFFFFFFFFu;
    } else {
        const uint32_t code = 0xFFFFFFu - (uint32_t)(m & 0xFFFFFFu);
        codes[f] = code;
        gmap[code] = (int8_t)f;
        counts[code] = 0;
    }
    *best = 0;
}

int qgram_map(const uint8_t *d_chars, const int64_t *d_off, int64_t n, int q, int sigma, int8_t *d_gmap,
              uint32_t *h_codes, int *n_used, cudaStream_t st) {
    if (q < 1 || q > 3 || sigma < 0 || sigma > 32) return fail(FP_E_INVAL, "q-gram map: q must be 1..3");
    const int64_t ncodes = (int64_t)1 << (8 * q);
    uint32_t *counts = nullptr, *codes = nullptr;
    unsigned long long *best = nullptr;
    int rc = FP_OK;
    cudaError_t e;
    if ((e = cudaMallocAsync((void **)&counts, sizeof(uint32_t) * (size_t)ncodes, st)) != cudaSuccess ||
        (e = cudaMallocAsync((void **)&codes, sizeof(uint32_t) * 32, st)) != cudaSuccess ||
        (e = cudaMallocAsync((void **)&best, sizeof(unsigned long long), st)) != cudaSuccess ||
        (e = cudaMemsetAsync(counts, 0, sizeof(uint32_t) * (size_t)ncodes, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(best, 0, sizeof(unsigned long long), st)) != cudaSuccess ||
        (e = cudaMemsetAsync(d_gmap, 0xFF, (size_t)ncodes, st)) != cudaSuccess) {
        rc = cuda_fail(e, "q-gram map: scratch");
    }
    if (rc == FP_OK && n > 0) {
        k_qgram_hist<<<grid_for(n, 256, 8192), 256, 0, st>>>(d_chars, d_off, n, q, counts);
        rc = launched("k_qgram_hist");
    }
    const int g = (int)std::min<int64_t>(1024, (ncodes + 255) / 256);
    for (int f = 0; rc == FP_OK && f < sigma; f++) {
        k_qgram_argmax<<<g, 256, 0, st>>>(counts, ncodes, best);
        if ((rc = launched("k_qgram_argmax")) != FP_OK) break;
        k_qgram_take<<<1, 1, 0, st>>>(best, f, counts, d_gmap, codes);
        rc = launched("k_qgram_take");
    }
    *n_used = 0;
    if (rc == FP_OK) {
        uint32_t h[32];
        if ((e = cudaMemcpyAsync(h, codes, sizeof(uint32_t) * (size_t)(sigma > 0 ? sigma : 1), cudaMemcpyDeviceToHost,
                                 st)) != cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess) {
            rc = cuda_fail(e, "q-gram map");
        } else {
            for (int f = 0; f < sigma && h[f] != 0xFFFFFFFFu; f++) h_codes[(*n_used)++] = h[f];
        }
    }
    if (counts) cudaFreeAsync(counts, st);
    if (codes) cudaFreeAsync(codes, st);
    if (best) cudaFreeAsync(best, st);
    return rc;
}

// ---------------------------------------------------------------------------
// bucketing
// ---------------------------------------------------------------------------
__global__ void k_bin_keys(const int64_t *__restrict__ off, int64_t n, const int32_t *__restrict__ group,
                           int nbins, uint64_t *__restrict__ keys, int32_t *__restrict__ hist,
                           int32_t *__restrict__ err) {
    extern __shared__ int32_t h[];
    for (int t = threadIdx.x; t < nbins; t += blockDim.x) h[t] = 0;
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t L = off[i + 1] - off[i];
        int g = group ? group[i] : 0;
        int bin;
        if (L < 0 || L > MAX_LEN || g < 0 || (int64_t)g * 256 + L >= nbins) {
            atomicOr(err, 1);
            bin = 0;
        } else {
            bin = g * 256 + (int)L;
        }
        keys[i] = ((uint64_t)bin << 32) | (uint64_t)i;
        atomicAdd(&h[bin], 1);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nbins; t += blockDim.x)
        if (h[t]) atomicAdd(&hist[t], h[t]);
}


constexpr int CELL_BITS = 11;  // cell_count(32) = 12 x 12 x 11 = 1584 < 2048
static_assert(cell_count(32) < (1 << CELL_BITS) && cell_count(16) < (1 << CELL_BITS), "cell keys");

// k_bin_keys with the weight cell of each string's fingerprint between the bin
// and the index, so that the sort leaves every bin in cell order.
template <int TYPE>
__global__ void k_bin_keys_cells(const int64_t *__restrict__ off, const uint8_t *__restrict__ chars, int64_t n,
                                 const int32_t *__restrict__ group, int nbins, const int8_t *__restrict__ map,
                                 FpParams P, uint64_t *__restrict__ keys, int32_t *__restrict__ hist,
                                 int32_t *__restrict__ err) {
    extern __shared__ int32_t h[];
    __shared__ int8_t smap[256];
    for (int t = threadIdx.x; t < nbins; t += blockDim.x) h[t] = 0;
    for (int t = threadIdx.x; t < 256; t += blockDim.x) smap[t] = map[t];
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t L = off[i + 1] - off[i];
        const int g = group ? group[i] : 0;
        int bin = 0, cell = 0;
        if (L < 0 || L > MAX_LEN || g < 0 || (int64_t)g * 256 + L >= nbins) {
            atomicOr(err, 1);
        } else {
            bin = g * 256 + (int)L;
            const uint8_t *src = chars + off[i];
            FpAcc<TYPE> acc;
            acc.init(P);
            for (int pos = 0; pos < (int)L; pos++) acc.put(src[pos], smap, pos, (int)L, P);
            cell = fp_cell(acc.finish(P), P.width);
        }
        keys[i] = ((((uint64_t)bin << CELL_BITS) | (uint64_t)cell) << 32) | (uint64_t)i;
        atomicAdd(&h[bin], 1);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nbins; t += blockDim.x)
        if (h[t]) atomicAdd(&hist[t], h[t]);
}

// One block of 1024 threads: bucket starts (aligned), unaligned starts and
// string-row bases.  tot[0] = slots, tot[1] = 16-byte row units.
__global__ void __launch_bounds__(1024) k_plan_bins(const int32_t *__restrict__ hist, int nbins,
                                                    int32_t *__restrict__ b_start,
                                                    int32_t *__restrict__ b_count,
                                                    int32_t *__restrict__ b_ustart,
                                                    int64_t *__restrict__ b_str16,
                                                    int64_t *__restrict__ tot) {
    __shared__ int64_t s_a[1024], s_u[1024], s_r[1024];
    const int t = threadIdx.x;
    const int per = (nbins + 1023) / 1024;
    const int lo = t * per, hi = lo + per < nbins ? lo + per : nbins;
    int64_t a = 0, u = 0, r = 0;
    for (int c = lo; c < hi; c++) {
        int64_t n = hist[c];
        a += (n + SLOT_ALIGN - 1) / SLOT_ALIGN * SLOT_ALIGN;
        u += n;
        r += n * (((c & 255) + 15) / 16);
    }
    s_a[t] = a;
    s_u[t] = u;
    s_r[t] = r;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        int64_t va = t >= o ? s_a[t - o] : 0, vu = t >= o ? s_u[t - o] : 0, vr = t >= o ? s_r[t - o] : 0;
        __syncthreads();
        s_a[t] += va;
        s_u[t] += vu;
        s_r[t] += vr;
        __syncthreads();
    }
    int64_t ra = s_a[t] - a, ru = s_u[t] - u, rr = s_r[t] - r;
    for (int c = lo; c < hi; c++) {
        int64_t n = hist[c];
        b_start[c] = (int32_t)ra;
        b_count[c] = (int32_t)n;
        b_ustart[c] = (int32_t)ru;
        b_str16[c] = rr;
        ra += (n + SLOT_ALIGN - 1) / SLOT_ALIGN * SLOT_ALIGN;
        ru += n;
        rr += n * (((c & 255) + 15) / 16);
    }
    if (t == 1023) {
        tot[0] = s_a[1023];
        tot[1] = s_r[1023];
    }
}

template <int TYPE>
__global__ void __launch_bounds__(256) k_scatter_fp(const uint64_t *__restrict__ sorted, int64_t n,
                                                    const int64_t *__restrict__ off,
                                                    const uint8_t *__restrict__ chars,
                                                    const int8_t *__restrict__ map, FpParams P,
                                                    const int32_t *__restrict__ b_start,
                                                    const int32_t *__restrict__ b_ustart,
                                                    const int64_t *__restrict__ b_str16, Bucketed B,
                                                    int bin_shift) {
    __shared__ int8_t smap[256];
    for (int t = threadIdx.x; t < 256; t += blockDim.x) smap[t] = map[t];
    __syncthreads();
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        uint64_t key = sorted[p];
        int bin = (int)(key >> (32 + bin_shift));
        int64_t i = (int64_t)(key & 0xffffffffu);
        int L = bin & 255;
        int64_t rank = p - b_ustart[bin];
        int64_t slot = b_start[bin] + rank;
        int64_t row16 = b_str16[bin] + rank * ((L + 15) / 16);
        B.idx[slot] = (int32_t)i;
        B.len[slot] = (uint8_t)L;
        B.row16[slot] = (uint32_t)row16;
        const uint8_t *src = chars + off[i];
        uint4 *dst = (uint4 *)(B.str + row16 * 16);
        FpAcc<TYPE> acc;
        acc.init(P);
        for (int c0 = 0; c0 < L; c0 += 16) {
            uint32_t w[4] = {0, 0, 0, 0};
#pragma unroll
            for (int j = 0; j < 16; j++) {
                int pos = c0 + j;
                if (pos < L) {
                    uint32_t ch = src[pos];
                    w[j >> 2] |= ch << (8 * (j & 3));
                    acc.put(ch, smap, pos, L, P);
                }
            }
            dst[c0 >> 4] = make_uint4(w[0], w[1], w[2], w[3]);
        }
        store_fp(B.fp, P.width, slot, acc.finish(P));
    }
}

template <int TYPE>
__global__ void __launch_bounds__(256) k_refingerprint(Bucketed B, const int8_t *__restrict__ map,
                                                       FpParams P) {
    __shared__ int8_t smap[256];
    for (int t = threadIdx.x; t < 256; t += blockDim.x) smap[t] = map[t];
    __syncthreads();
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < B.n_slots;
         s += (int64_t)gridDim.x * blockDim.x) {
        if (B.idx[s] < 0) continue;
        int L = B.len[s];
        const uint4 *row = (const uint4 *)(B.str + (int64_t)B.row16[s] * 16);
        FpAcc<TYPE> acc;
        acc.init(P);
        for (int c0 = 0; c0 < L; c0 += 16) {
            uint4 v = row[c0 >> 4];
            uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int j = 0; j < 16; j++) {
                int pos = c0 + j;
                if (pos < L) acc.put((w[j >> 2] >> (8 * (j & 3))) & 0xFF, smap, pos, L, P);
            }
        }
        store_fp(B.fp, P.width, s, acc.finish(P));
    }
}

template <int TYPE>
__global__ void __launch_bounds__(256) k_fingerprint_list(const uint8_t *__restrict__ chars,
                                                          const int64_t *__restrict__ off, int64_t n,
                                                          const int8_t *__restrict__ map, FpParams P,
                                                          uint32_t *__restrict__ out) {
    __shared__ int8_t smap[256];
    for (int t = threadIdx.x; t < 256; t += blockDim.x) smap[t] = map[t];
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t L = off[i + 1] - off[i];
        const uint8_t *src = chars + off[i];
        FpAcc<TYPE> acc;
        acc.init(P);
        for (int64_t pos = 0; pos < L; pos++) acc.put(src[pos], smap, (int)pos, (int)L, P);
        out[i] = acc.finish(P);
    }
}

// Calls f(std::integral_constant<int, TYPE>) for the fingerprint type.
template <class F>
static void by_type(int type, F &&f) {
    switch (type) {
        case FP_OCC: f(std::integral_constant<int, FP_OCC>{}); break;
        case FP_OCC_HALVED: f(std::integral_constant<int, FP_OCC_HALVED>{}); break;
        case FP_COUNT: f(std::integral_constant<int, FP_COUNT>{}); break;
        case FP_QGRAM: f(std::integral_constant<int, FP_QGRAM>{}); break;
        case FP_COUNT_L1: f(std::integral_constant<int, FP_COUNT_L1>{}); break;
        default: f(std::integral_constant<int, FP_POS>{}); break;
    }
}


int fingerprint_list(const uint8_t *d_chars, const int64_t *d_off, int64_t n, const int8_t *d_map,
                     const FpParams &P, uint32_t *d_out, cudaStream_t st) {
    if (n <= 0) return FP_OK;
    int g = grid_for(n);
    by_type(P.type, [&](auto tt) {
        k_fingerprint_list<decltype(tt)::value><<<g, 256, 0, st>>>(d_chars, d_off, n, d_map, P, d_out);
    });
    FP_LAUNCHED("k_fingerprint_list");
    return FP_OK;
}

void free_bucketed(Bucketed *b, cudaStream_t st) {
    void *ptrs[] = {b->fp, b->idx, b->len, b->row16, b->str, b->b_start, b->b_count, b->fp2};
    for (void *p : ptrs) {
        if (!p) continue;
        if (b->stream_ordered) cudaFreeAsync(p, st);
        else cudaFree(p);
    }
    *b = Bucketed{};
}

static int dev_alloc(void **p, size_t bytes, bool so, cudaStream_t st) {
    if (bytes == 0) bytes = 16;
    cudaError_t e = so ? cudaMallocAsync(p, bytes, st) : cudaMalloc(p, bytes);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        set_error("device allocation failed");
        return FP_E_NOMEM;
    }
    if (e != cudaSuccess) return cuda_fail(e, "device allocation");
    return FP_OK;
}

// ---------------------------------------------------------------------------
// weight order inside the buckets
// ---------------------------------------------------------------------------
// F_D is the Hamming weight of the XOR of two fingerprints (Sec. 3.3) for
// occurrence, occurrence-halved and count fingerprints, and the weight of an
// XOR is at least the difference of the two weights: |H(x) - H(y)| <=
// H(x XOR y).  With the strings of every bucket ordered by fingerprint weight,
// a tile of patterns with weights [wmin, wmax] can skip every word whose
// weight lies outside [wmin - 2k, wmax + 2k]: Eq. 1 rejects all those pairs.
// weight_order sorts the real slots of each bin by (weight, current slot)
// and, on request, records per bin the first slot of every weight.


__device__ __forceinline__ int slot_cell(const void *fp, int width, int64_t s) {
    return fp_cell(width == 16 ? (uint32_t)((const uint16_t *)fp)[s] : ((const uint32_t *)fp)[s], width);
}

// U[c] = real slots of the bins before c (one block).
__global__ void __launch_bounds__(1024) k_bin_prefix(const int32_t *__restrict__ count, int nbins,
                                                     int64_t *__restrict__ U) {
    __shared__ int64_t s[1024];
    const int t = threadIdx.x, per = (nbins + 1023) / 1024;
    const int lo = min(nbins, t * per), hi = min(nbins, lo + per);
    int64_t a = 0;
    for (int c = lo; c < hi; c++) a += count[c];
    s[t] = a;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const int64_t v = t >= o ? s[t - o] : 0;
        __syncthreads();
        s[t] += v;
        __syncthreads();
    }
    int64_t r = s[t] - a;
    for (int c = lo; c < hi; c++) {
        U[c] = r;
        r += count[c];
    }
}

// One block per bin: key (bin, cell, slot) of every real slot, written at
// the bin's place in slot order.
__global__ void __launch_bounds__(256) k_weight_keys(Bucketed B, int width, const int64_t *__restrict__ U,
                                                     uint64_t *__restrict__ keys) {
    const int c = blockIdx.x;
    const int32_t start = B.b_start[c], count = B.b_count[c];
    for (int i = threadIdx.x; i < count; i += blockDim.x) {
        const int64_t slot = start + i;
        const uint64_t w = (uint64_t)slot_cell(B.fp, width, slot);
        keys[U[c] + i] = ((((uint64_t)c << CELL_BITS) | w) << 32) | (uint64_t)slot;
    }
}

// Moves the slots into cell order: sorted key p of bin c goes to slot
// b_start[c] + (p - U[c]); the old arrays are read from copies.  The string
// rows move with their slots, so that a bin's rows stay contiguous in slot
// order (row of slot s = row of the bin's first slot + (s - first) x rows per
// string), which the verifier relies on.
__global__ void __launch_bounds__(256) k_weight_permute(const uint64_t *__restrict__ keys, int64_t n, Bucketed B,
                                                        int width, const int64_t *__restrict__ U,
                                                        const uint8_t *__restrict__ old_fp,
                                                        const int32_t *__restrict__ old_idx,
                                                        const uint8_t *__restrict__ old_len,
                                                        const uint32_t *__restrict__ old_row16,
                                                        const uint8_t *__restrict__ old_str) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t key = keys[p];
        const int c = (int)(key >> (32 + CELL_BITS));
        const int64_t from = (int64_t)(key & 0xffffffffu);
        const int64_t first = B.b_start[c], to = first + (p - U[c]);
        if (width == 16) ((uint16_t *)B.fp)[to] = ((const uint16_t *)old_fp)[from];
        else ((uint32_t *)B.fp)[to] = ((const uint32_t *)old_fp)[from];
        B.idx[to] = old_idx[from];
        const int L = old_len[from];
        B.len[to] = (uint8_t)L;
        const uint32_t rp = (uint32_t)((L + 15) >> 4);
        const uint32_t row = old_row16[first] + (uint32_t)(to - first) * rp;  // the bin's rows start at its first slot's
        B.row16[to] = row;
        const uint4 *src = (const uint4 *)(old_str + (uint64_t)old_row16[from] * 16);
        uint4 *dst = (uint4 *)(B.str + (uint64_t)row * 16);
        for (uint32_t r = 0; r < rp; r++) dst[r] = src[r];
    }
}

// wstart[c * (NC + 1) + w] = first slot of bin c whose cell is >= w (w = NC:
// the end of the bin's real slots); one thread per (bin, cell).
__global__ void k_weight_table(const uint64_t *__restrict__ keys, const int32_t *__restrict__ b_start,
                               const int32_t *__restrict__ b_count, const int64_t *__restrict__ U, int nbins,
                               int NC, int32_t *__restrict__ wstart) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)nbins * (NC + 1)) return;
    const int c = (int)(t / (NC + 1)), w = (int)(t % (NC + 1));
    int64_t lo = U[c], hi = U[c] + b_count[c];  // first key of the run with cell >= w
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if ((int)((keys[mid] >> 32) & ((1u << CELL_BITS) - 1u)) < w) lo = mid + 1;
        else hi = mid;
    }
    wstart[t] = b_start[c] + (int32_t)(lo - U[c]);
}

int weight_order(Bucketed *B, const FpParams &P, int32_t *d_wstart, cudaStream_t st) {
    if (!banded_type(P.type) || B->n <= 0) {
        if (d_wstart)
            FP_CUDA(cudaMemsetAsync(d_wstart, 0, sizeof(int32_t) * (size_t)B->nbins * (cell_count(P.width) + 1), st));
        return FP_OK;
    }
    const int nbins = B->nbins;
    const int64_t n = B->n, ns = B->n_slots;
    const size_t fpw = P.width == 16 ? 2 : 4;
    int bin_bits = 1;
    while ((1 << bin_bits) < nbins) bin_bits++;
    int64_t *U = nullptr;
    uint64_t *keys = nullptr, *tmp = nullptr, *sorted = nullptr;
    uint8_t *old = nullptr;
    int rc = FP_OK;
    const size_t o_idx = ((size_t)ns * fpw + 255) & ~(size_t)255, o_len = o_idx + (((size_t)ns * 4 + 255) & ~(size_t)255),
                 o_row = o_len + (((size_t)ns + 255) & ~(size_t)255),
                 o_str = o_row + (((size_t)ns * 4 + 255) & ~(size_t)255), total = o_str + (size_t)B->str_bytes;
    cudaError_t e;
    if ((e = cudaMallocAsync((void **)&U, sizeof(int64_t) * (size_t)nbins, st)) != cudaSuccess ||
        (e = cudaMallocAsync((void **)&keys, sizeof(uint64_t) * (size_t)n, st)) != cudaSuccess ||
        (e = cudaMallocAsync((void **)&tmp, sizeof(uint64_t) * (size_t)n, st)) != cudaSuccess ||
        (e = cudaMallocAsync((void **)&old, total, st)) != cudaSuccess) {
        rc = cuda_fail(e, "weight_order: scratch");
    } else if ((e = cudaMemcpyAsync(old, B->fp, (size_t)ns * fpw, cudaMemcpyDeviceToDevice, st)) != cudaSuccess ||
               (e = cudaMemcpyAsync(old + o_idx, B->idx, (size_t)ns * 4, cudaMemcpyDeviceToDevice, st)) != cudaSuccess ||
               (e = cudaMemcpyAsync(old + o_len, B->len, (size_t)ns, cudaMemcpyDeviceToDevice, st)) != cudaSuccess ||
               (e = cudaMemcpyAsync(old + o_row, B->row16, (size_t)ns * 4, cudaMemcpyDeviceToDevice, st)) !=
                   cudaSuccess ||
               (e = cudaMemcpyAsync(old + o_str, B->str, (size_t)B->str_bytes, cudaMemcpyDeviceToDevice, st)) !=
                   cudaSuccess) {
        rc = cuda_fail(e, "weight_order: copies");
    } else {
        k_bin_prefix<<<1, 1024, 0, st>>>(B->b_count, nbins, U);
        if ((rc = launched("k_bin_prefix")) == FP_OK) {
            k_weight_keys<<<nbins, 256, 0, st>>>(*B, P.width, U, keys);
            rc = launched("k_weight_keys");
        }
        if (rc == FP_OK)
            rc = radix_sort_u64(keys, tmp, nullptr, n, 32, 32 + CELL_BITS + bin_bits, st, &sorted);
        if (rc == FP_OK) {
            k_weight_permute<<<grid_for(n, 256, 8192), 256, 0, st>>>(sorted, n, *B, P.width, U, old,
                                                                      (const int32_t *)(old + o_idx), old + o_len,
                                                                      (const uint32_t *)(old + o_row), old + o_str);
            rc = launched("k_weight_permute");
        }
        if (rc == FP_OK && d_wstart) {
            const int64_t nt = (int64_t)nbins * (cell_count(P.width) + 1);
            k_weight_table<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(sorted, B->b_start, B->b_count, U, nbins,
                                                                        cell_count(P.width), d_wstart);
            rc = launched("k_weight_table");
        }
    }
    if (U) cudaFreeAsync(U, st);
    if (keys) cudaFreeAsync(keys, st);
    if (tmp) cudaFreeAsync(tmp, st);
    if (old) cudaFreeAsync(old, st);
    return rc;
}

int bucketize(const uint8_t *d_chars, const int64_t *d_off, int64_t n, int64_t total_chars,
              const int32_t *d_group, int32_t n_groups, const int8_t *d_map, const FpParams &P,
              bool so, cudaStream_t st, Bucketed *out, int32_t *d_err, bool cells) {
    Bucketed B;
    const int shift = cells && banded_type(P.type) ? CELL_BITS : 0;
    B.stream_ordered = so;
    B.n = n;
    B.nbins = 256 * (n_groups < 1 ? 1 : n_groups);
    const int nbins = B.nbins;
    const int64_t slots_ub = n + (int64_t)(SLOT_ALIGN - 1) * nbins;
    const int64_t str_ub = total_chars + 15 * n;
    const size_t fpw = P.width == 16 ? 2 : 4;
    int rc = FP_OK;
    uint64_t *keys = nullptr, *keys2 = nullptr;
    int32_t *hist = nullptr, *ustart = nullptr;
    int64_t *str16 = nullptr, *tot = nullptr;
#define ALLOC(ptr, bytes, soflag)                                      \
    do {                                                               \
        rc = dev_alloc((void **)&(ptr), (size_t)(bytes), soflag, st); \
        if (rc != FP_OK) goto fail;                                    \
    } while (0)
    ALLOC(B.fp, (slots_ub + FP_SLACK_SLOTS) * fpw, so);
    ALLOC(B.idx, slots_ub * 4, so);
    ALLOC(B.len, slots_ub, so);
    ALLOC(B.row16, slots_ub * 4, so);
    ALLOC(B.str, str_ub + STR_SLACK, so);
    ALLOC(B.b_start, nbins * 4, so);
    ALLOC(B.b_count, nbins * 4, so);
    ALLOC(keys, (n > 0 ? n : 1) * 8, true);
    ALLOC(keys2, (n > 0 ? n : 1) * 8, true);
    ALLOC(hist, nbins * 4, true);
    ALLOC(ustart, nbins * 4, true);
    ALLOC(str16, nbins * 8, true);
    ALLOC(tot, 2 * 8, true);
#undef ALLOC
    {
        cudaError_t e;
        if ((e = cudaMemsetAsync(B.fp, 0, (slots_ub + FP_SLACK_SLOTS) * fpw, st)) != cudaSuccess ||
            (e = cudaMemsetAsync(B.idx, 0xFF, slots_ub * 4, st)) != cudaSuccess ||
            (e = cudaMemsetAsync(B.len, 0, slots_ub, st)) != cudaSuccess ||
            (e = cudaMemsetAsync(B.row16, 0, slots_ub * 4, st)) != cudaSuccess ||
            (e = cudaMemsetAsync(B.str + str_ub, 0, STR_SLACK, st)) != cudaSuccess ||
            (e = cudaMemsetAsync(hist, 0, nbins * 4, st)) != cudaSuccess) {
            rc = cuda_fail(e, "cudaMemsetAsync");
            goto fail;
        }
        if (n > 0) {
            int g = grid_for(n, 256, 2048);
            const size_t sh = nbins * sizeof(int32_t);
            if (shift == 0)
                k_bin_keys<<<g, 256, sh, st>>>(d_off, n, d_group, nbins, keys, hist, d_err);
            else
                by_type(P.type, [&](auto tt) {
                    k_bin_keys_cells<decltype(tt)::value>
                        <<<g, 256, sh, st>>>(d_off, d_chars, n, d_group, nbins, d_map, P, keys, hist, d_err);
                });
            g_launches++;
            if ((e = cudaGetLastError()) != cudaSuccess) { rc = cuda_fail(e, "k_bin_keys"); goto fail; }
        }
        k_plan_bins<<<1, 1024, 0, st>>>(hist, nbins, B.b_start, B.b_count, ustart, str16, tot);
        g_launches++;
        if ((e = cudaGetLastError()) != cudaSuccess) { rc = cuda_fail(e, "k_plan_bins"); goto fail; }
        if (n > 0) {
            int bin_bits = 1;
            while ((1 << bin_bits) < nbins) bin_bits++;
            uint64_t *sorted = keys;
            rc = radix_sort_u64(keys, keys2, nullptr, n, 32, 32 + shift + bin_bits, st, &sorted);
            if (rc != FP_OK) goto fail;
            int g = grid_for(n, 256, 8192);
            by_type(P.type, [&](auto tt) {
                k_scatter_fp<decltype(tt)::value>
                    <<<g, 256, 0, st>>>(sorted, n, d_off, d_chars, d_map, P, B.b_start, ustart, str16, B, shift);
            });
            g_launches++;
            if ((e = cudaGetLastError()) != cudaSuccess) { rc = cuda_fail(e, "k_scatter_fp"); goto fail; }
        }
    }
    B.n_slots = slots_ub;
    B.str_bytes = str_ub;
    cudaFreeAsync(keys, st);
    cudaFreeAsync(keys2, st);
    cudaFreeAsync(hist, st);
    cudaFreeAsync(ustart, st);
    cudaFreeAsync(str16, st);
    cudaFreeAsync(tot, st);
    *out = B;
    return FP_OK;
fail:
    if (keys) cudaFreeAsync(keys, st);
    if (keys2) cudaFreeAsync(keys2, st);
    if (hist) cudaFreeAsync(hist, st);
    if (ustart) cudaFreeAsync(ustart, st);
    if (str16) cudaFreeAsync(str16, st);
    if (tot) cudaFreeAsync(tot, st);
    free_bucketed(&B, st);
    return rc;
}

// Combined types: the 32-bit occurrence fingerprint of every real slot from
// its row (padding slots get 0).
__global__ void __launch_bounds__(256) k_second_fp(Bucketed B, const int8_t *__restrict__ map, FpParams P) {
    __shared__ int8_t smap[256];
    for (int t = threadIdx.x; t < 256; t += blockDim.x) smap[t] = map[t];
    __syncthreads();
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < B.n_slots;
         s += (int64_t)gridDim.x * blockDim.x) {
        uint32_t f = 0;
        if (B.idx[s] >= 0) {
            const int L = B.len[s];
            const uint8_t *row = B.str + (uint64_t)B.row16[s] * 16;
            FpAcc<FP_OCC> acc;
            acc.init(P);
            for (int i = 0; i < L; i++) acc.add(smap[row[i]], i, L, P);
            f = acc.finish(P);
        }
        B.fp2[s] = f;
    }
}

int second_fingerprints(Bucketed *B, const int8_t *d_map2, const FpParams &P2, cudaStream_t st) {
    if (!B->fp2) {
        // readable slack after the last slot, as for the first fingerprints: the
        // filter reads a lane's four slots with one 128-bit load
        const size_t bytes = sizeof(uint32_t) * ((size_t)(B->n_slots > 0 ? B->n_slots : 0) + FP_SLACK_SLOTS);
        const cudaError_t e = B->stream_ordered ? cudaMallocAsync((void **)&B->fp2, bytes, st)
                                                : cudaMalloc((void **)&B->fp2, bytes);
        if (e != cudaSuccess) return cuda_fail(e, "second fingerprints");
        const cudaError_t z = cudaMemsetAsync(B->fp2, 0, bytes, st);
        if (z != cudaSuccess) return cuda_fail(z, "second fingerprints");
    }
    if (B->n_slots <= 0) return FP_OK;
    k_second_fp<<<grid_for(B->n_slots, 256, 8192), 256, 0, st>>>(*B, d_map2, P2);
    FP_LAUNCHED("k_second_fp");
    return FP_OK;
}

int refingerprint(Bucketed *B, const int8_t *d_map, const FpParams &P, cudaStream_t st) {
    if (B->n_slots <= 0) return FP_OK;
    int g = grid_for(B->n_slots, 256, 8192);
    by_type(P.type, [&](auto tt) { k_refingerprint<decltype(tt)::value><<<g, 256, 0, st>>>(*B, d_map, P); });
    FP_LAUNCHED("k_refingerprint");
    return FP_OK;
}

}  // namespace fpk

namespace fpk {

// bucketize() into arrays the caller has placed in B (fp, idx, len, row16,
// str, b_start, b_count, sized for n strings of total_chars bytes and
// 256 * n_groups bins) with the temporaries in S; allocates nothing.
int bucketize_into(const uint8_t *d_chars, const int64_t *d_off, int64_t n, int64_t total_chars,
                   const int32_t *d_group, int32_t n_groups, const int8_t *d_map, const FpParams &P, cudaStream_t st,
                   Bucketed *B, const BucketScratch &S, int32_t *d_err, bool cells) {
    const int nbins = 256 * (n_groups < 1 ? 1 : n_groups);
    const int shift = cells && banded_type(P.type) ? CELL_BITS : 0;
    const int64_t slots_ub = n + (int64_t)(SLOT_ALIGN - 1) * nbins;
    const int64_t str_ub = total_chars + 15 * n;
    const size_t fpw = P.width == 16 ? 2 : 4;
    B->nbins = nbins;
    B->n = n;
    B->stream_ordered = false;
    FP_CUDA(cudaMemsetAsync(B->fp, 0, (slots_ub + FP_SLACK_SLOTS) * fpw, st));
    FP_CUDA(cudaMemsetAsync(B->idx, 0xFF, slots_ub * 4, st));
    FP_CUDA(cudaMemsetAsync(B->len, 0, slots_ub, st));
    FP_CUDA(cudaMemsetAsync(B->row16, 0, slots_ub * 4, st));
    FP_CUDA(cudaMemsetAsync(B->str + str_ub, 0, STR_SLACK, st));
    FP_CUDA(cudaMemsetAsync(S.hist, 0, nbins * 4, st));
    if (n > 0) {
        const int g = grid_for(n, 256, 2048);
        const size_t sh = nbins * sizeof(int32_t);
        if (shift == 0)
            k_bin_keys<<<g, 256, sh, st>>>(d_off, n, d_group, nbins, S.keys, S.hist, d_err);
        else
            by_type(P.type, [&](auto tt) {
                k_bin_keys_cells<decltype(tt)::value>
                    <<<g, 256, sh, st>>>(d_off, d_chars, n, d_group, nbins, d_map, P, S.keys, S.hist, d_err);
            });
        FP_LAUNCHED("k_bin_keys");
    }
    k_plan_bins<<<1, 1024, 0, st>>>(S.hist, nbins, B->b_start, B->b_count, S.ustart, S.str16, S.tot);
    FP_LAUNCHED("k_plan_bins");
    if (n > 0) {
        int bin_bits = 1;
        while ((1 << bin_bits) < nbins) bin_bits++;
        uint64_t *sorted = S.keys;
        FP_TRY(radix_sort_u64_into(S.keys, S.keys2, S.radix_hist, nullptr, n, 32, 32 + shift + bin_bits, st, &sorted));
        int g = grid_for(n, 256, 8192);
        by_type(P.type, [&](auto tt) {
            k_scatter_fp<decltype(tt)::value>
                <<<g, 256, 0, st>>>(sorted, n, d_off, d_chars, d_map, P, B->b_start, S.ustart, S.str16, *B, shift);
        });
        FP_LAUNCHED("k_scatter_fp");
    }
    B->n_slots = slots_ub;
    B->str_bytes = str_ub;
    return FP_OK;
}

}  // namespace fpk
