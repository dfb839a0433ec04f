// Stable LSD radix sort of 64-bit keys whose count lives on the device, and
// the CSR builder for sorted match keys.
//
// Used twice on the query path: to bucket strings by length stably (the key
// is bin << 32 | original index) and to turn unordered (query, word) matches
// into per-query ascending match lists (Sec. 1: the answer for a pattern is
// the set of matching dictionary indices; ascending order makes it unique).
//
// Each pass sorts one 8-bit digit with three kernels: block histograms
// (digit-major), one exclusive scan over them, and a stable scatter in which
// every block walks its contiguous range in order, ranking equal digits inside
// a warp with __match_any_sync and across the block's warps with shared
// counters.  The grid is fixed from the caller's capacity bound; each block
// derives its range from the device-side count.
#include "common.cuh"

namespace fpk {

namespace {

constexpr int RB_THREADS = 256;
#ifndef RADIX_MID_BLOCKS
#define RADIX_MID_BLOCKS 256  // blocks per pass below 2^26 keys (measured against 64 and 128)
#endif
constexpr int RB_WARPS = RB_THREADS / 32;

__device__ __forceinline__ void block_range(uint64_t n, int nb, int b, uint64_t *lo, uint64_t *hi) {
    *lo = n * (uint64_t)b / (uint64_t)nb;
    *hi = n * (uint64_t)(b + 1) / (uint64_t)nb;
}

__global__ void __launch_bounds__(RB_THREADS) k_radix_hist(const uint64_t *__restrict__ in,
                                                           const uint64_t *d_n, uint64_t n_host,
                                                           int shift, uint32_t mask,
                                                           uint32_t *__restrict__ hist) {
    __shared__ uint32_t h[256];
    const int nb = gridDim.x, b = blockIdx.x;
    h[threadIdx.x] = 0;
    __syncthreads();
    uint64_t n = d_n ? min(*d_n, n_host) : n_host, lo, hi;
    block_range(n, nb, b, &lo, &hi);
    for (uint64_t i = lo + threadIdx.x; i < hi; i += RB_THREADS)
        atomicAdd(&h[(uint32_t)(in[i] >> shift) & mask], 1u);
    __syncthreads();
    hist[(size_t)threadIdx.x * nb + b] = h[threadIdx.x];
}

// Exclusive scan of n uint32 values in place with one block of 1024 threads,
// in tiles of 8192 values: a tile is loaded with coalesced reads (eight loads
// per thread in flight at once) into shared memory, thread t scans the eight
// consecutive values [8t, 8t + 8) of the tile, the per-thread sums are scanned
// across the block (warp shuffles, then one shared step over the 32 warps),
// and the tile is written back coalesced.  Shared indices are padded by one
// word per 32 so that both access patterns are free of bank conflicts.  The
// next tile's loads are issued before the current tile is scanned, so their
// latency overlaps the scan.
constexpr int SCAN_R = 8, SCAN_TILE = 1024 * SCAN_R;

__device__ __forceinline__ int scan_pad(int j) { return j + (j >> 5); }

__global__ void __launch_bounds__(1024) k_scan_u32(uint32_t *__restrict__ a, int64_t n) {
    __shared__ uint32_t s[SCAN_TILE + SCAN_TILE / 32];
    __shared__ uint32_t s_warp[32];
    __shared__ uint32_t s_carry;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    if (t == 0) s_carry = 0;
    uint32_t pre[SCAN_R];  // the tile about to be scanned, in coalesced order
#pragma unroll
    for (int r = 0; r < SCAN_R; r++) {
        const int64_t i = r * 1024 + t;
        pre[r] = i < n ? a[i] : 0u;
    }
    for (int64_t base = 0; base < n; base += SCAN_TILE) {
#pragma unroll
        for (int r = 0; r < SCAN_R; r++) s[scan_pad(r * 1024 + t)] = pre[r];
#pragma unroll
        for (int r = 0; r < SCAN_R; r++) {  // prefetch the next tile
            const int64_t i = base + SCAN_TILE + r * 1024 + t;
            pre[r] = i < n ? a[i] : 0u;
        }
        __syncthreads();
        uint32_t v[SCAN_R], sum = 0;
#pragma unroll
        for (int r = 0; r < SCAN_R; r++) {
            v[r] = s[scan_pad(t * SCAN_R + r)];
            sum += v[r];
        }
        uint32_t x = sum;  // inclusive scan of the thread sums within the warp
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[w] = x;
        __syncthreads();
        if (w == 0) {
            uint32_t q = s_warp[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, q, o);
                if (lane >= o) q += y;
            }
            s_warp[lane] = q;  // inclusive over warps
        }
        __syncthreads();
        const uint32_t carry = s_carry;
        uint32_t run = carry + (w ? s_warp[w - 1] : 0u) + x - sum;
#pragma unroll
        for (int r = 0; r < SCAN_R; r++) {
            s[scan_pad(t * SCAN_R + r)] = run;
            run += v[r];
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < SCAN_R; r++) {
            const int64_t i = base + r * 1024 + t;
            if (i < n) a[i] = s[scan_pad(r * 1024 + t)];
        }
        if (t == 1023) s_carry = carry + s_warp[31];
        __syncthreads();
    }
}

__global__ void __launch_bounds__(RB_THREADS) k_radix_scatter(const uint64_t *__restrict__ in,
                                                              uint64_t *__restrict__ out,
                                                              const uint64_t *d_n, uint64_t n_host,
                                                              int shift, uint32_t mask,
                                                              const uint32_t *__restrict__ hist) {
    __shared__ uint32_t s_off[256];
    __shared__ uint32_t s_w[RB_WARPS][256];
    const int nb = gridDim.x, b = blockIdx.x;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    s_off[t] = hist[(size_t)t * nb + b];
    uint64_t n = d_n ? min(*d_n, n_host) : n_host, lo, hi;
    block_range(n, nb, b, &lo, &hi);
    const unsigned lt = (1u << lane) - 1u;
    uint64_t next = lo + t < hi ? in[lo + t] : 0;  // keys are loaded one chunk ahead
    for (uint64_t base = lo; base < hi; base += RB_THREADS) {
        uint64_t i = base + t;
        bool valid = i < hi;
        const uint64_t key = next;
        if (i + RB_THREADS < hi) next = in[i + RB_THREADS];
        uint32_t d = valid ? ((uint32_t)(key >> shift) & mask) : 256u;
#pragma unroll
        for (int x = 0; x < RB_WARPS; x++) s_w[x][t] = 0;
        __syncthreads();
        unsigned peers = __match_any_sync(0xffffffffu, d);
        uint32_t rank = __popc(peers & lt);
        if (valid && (peers & lt) == 0) s_w[w][d] = __popc(peers);
        __syncthreads();
        uint32_t run = 0;
#pragma unroll
        for (int x = 0; x < RB_WARPS; x++) {
            uint32_t c = s_w[x][t];
            s_w[x][t] = run;
            run += c;
        }
        __syncthreads();
        if (valid) out[s_off[d] + s_w[w][d] + rank] = key;
        __syncthreads();
        s_off[t] += run;
        __syncthreads();
    }
}

__global__ void k_row_ptr(const uint64_t *__restrict__ keys, const uint64_t *d_n, uint64_t cap,
                          int64_t n_queries, int idx_bits, int64_t *__restrict__ row_ptr) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q > n_queries) return;
    uint64_t n = min(*d_n, cap);
    uint64_t target = (uint64_t)q << idx_bits;
    uint64_t lo = 0, hi = n;  // first position with key >= target
    while (lo < hi) {
        uint64_t mid = (lo + hi) >> 1;
        if (keys[mid] < target) lo = mid + 1;
        else hi = mid;
    }
    row_ptr[q] = (int64_t)lo;
}

__global__ void k_extract_idx(const uint64_t *__restrict__ keys, const uint64_t *d_n, uint64_t cap,
                              int idx_bits, int32_t *__restrict__ idx) {
    uint64_t n = min(*d_n, cap);
    uint64_t mask = (idx_bits >= 64) ? ~0ull : ((1ull << idx_bits) - 1ull);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        idx[i] = (int32_t)(keys[i] & mask);
}

}  // namespace

int radix_sort_u64(uint64_t *keys, uint64_t *tmp, const uint64_t *d_n, int64_t max_n, int bits_lo,
                   int bits_hi, cudaStream_t st, uint64_t **result) {
    *result = keys;
    if (max_n <= 0 || bits_hi <= bits_lo) return FP_OK;
    int64_t nb64 = (max_n + 4095) / 4096;
    const int64_t cap = max_n >= (1LL << 26) ? 4096 : RADIX_MID_BLOCKS;  // more blocks only for very large sorts
    int nb = (int)(nb64 < 1 ? 1 : (nb64 > cap ? cap : nb64));
    uint32_t *hist = nullptr;
    FP_CUDA(cudaMallocAsync((void **)&hist, sizeof(uint32_t) * 256 * (size_t)nb, st));
    uint64_t *src = keys, *dst = tmp;
    const uint64_t n_host = (uint64_t)max_n;  // the count, or the cap of the device count
    for (int s = bits_lo; s < bits_hi; s += 8) {
        int w = bits_hi - s < 8 ? bits_hi - s : 8;
        uint32_t mask = (1u << w) - 1u;
        k_radix_hist<<<nb, RB_THREADS, 0, st>>>(src, d_n, n_host, s, mask, hist);
        FP_LAUNCHED("k_radix_hist");
        k_scan_u32<<<1, 1024, 0, st>>>(hist, 256 * (int64_t)nb);
        FP_LAUNCHED("k_scan_u32");
        k_radix_scatter<<<nb, RB_THREADS, 0, st>>>(src, dst, d_n, n_host, s, mask, hist);
        FP_LAUNCHED("k_radix_scatter");
        uint64_t *t = src;
        src = dst;
        dst = t;
    }
    FP_CUDA(cudaFreeAsync(hist, st));
    *result = src;
    return FP_OK;
}

int build_csr(uint64_t *keys, uint64_t *tmp, const uint64_t *d_n, int64_t max_n, int q_bits, int idx_bits,
              int64_t n_queries, int64_t *row_ptr, int32_t *idx, cudaStream_t st) {
    uint64_t *sorted = keys;
    FP_TRY(radix_sort_u64(keys, tmp, d_n, max_n, 0, q_bits + idx_bits, st, &sorted));
    int64_t nt = n_queries + 1;
    k_row_ptr<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(sorted, d_n, (uint64_t)max_n, n_queries, idx_bits,
                                                            row_ptr);
    FP_LAUNCHED("k_row_ptr");
    if (max_n > 0 && idx) {
        int64_t g = (max_n + 255) / 256;
        int grid = (int)(g > 4096 ? 4096 : (g < 1 ? 1 : g));
        k_extract_idx<<<grid, 256, 0, st>>>(sorted, d_n, (uint64_t)max_n, idx_bits, idx);
        FP_LAUNCHED("k_extract_idx");
    }
    return FP_OK;
}

}  // namespace fpk

namespace fpk {

// Blocks per radix pass for a capacity of max_n keys (the digit histogram
// holds 256 entries per block).
int radix_blocks(int64_t max_n) {
    int64_t nb64 = (max_n + 4095) / 4096;
    const int64_t cap = max_n >= (1LL << 26) ? 4096 : RADIX_MID_BLOCKS;  // more blocks only for very large sorts
    return (int)(nb64 < 1 ? 1 : (nb64 > cap ? cap : nb64));
}

// radix_sort_u64 with the digit histogram supplied by the caller
// (256 * radix_blocks(max_n) uint32 values); allocates nothing.
int radix_sort_u64_into(uint64_t *keys, uint64_t *tmp, uint32_t *hist, const uint64_t *d_n, int64_t max_n,
                        int bits_lo, int bits_hi, cudaStream_t st, uint64_t **result) {
    *result = keys;
    if (max_n <= 0 || bits_hi <= bits_lo) return FP_OK;
    const int nb = radix_blocks(max_n);
    uint64_t *src = keys, *dst = tmp;
    const uint64_t n_host = (uint64_t)max_n;
    for (int s = bits_lo; s < bits_hi; s += 8) {
        int w = bits_hi - s < 8 ? bits_hi - s : 8;
        uint32_t mask = (1u << w) - 1u;
        k_radix_hist<<<nb, RB_THREADS, 0, st>>>(src, d_n, n_host, s, mask, hist);
        FP_LAUNCHED("k_radix_hist");
        k_scan_u32<<<1, 1024, 0, st>>>(hist, 256 * (int64_t)nb);
        FP_LAUNCHED("k_scan_u32");
        k_radix_scatter<<<nb, RB_THREADS, 0, st>>>(src, dst, d_n, n_host, s, mask, hist);
        FP_LAUNCHED("k_radix_scatter");
        uint64_t *t = src;
        src = dst;
        dst = t;
    }
    *result = src;
    return FP_OK;
}

// build_csr with caller-supplied sort scratch; allocates nothing.
int build_csr_into(uint64_t *keys, uint64_t *tmp, uint32_t *hist, const uint64_t *d_n, int64_t max_n, int q_bits,
                   int idx_bits, int64_t n_queries, int64_t *row_ptr, int32_t *idx, cudaStream_t st) {
    uint64_t *sorted = keys;
    FP_TRY(radix_sort_u64_into(keys, tmp, hist, d_n, max_n, 0, q_bits + idx_bits, st, &sorted));
    int64_t nt = n_queries + 1;
    k_row_ptr<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(sorted, d_n, (uint64_t)max_n, n_queries, idx_bits,
                                                            row_ptr);
    FP_LAUNCHED("k_row_ptr");
    if (max_n > 0 && idx) {
        int64_t g = (max_n + 255) / 256;
        int grid = (int)(g > 4096 ? 4096 : (g < 1 ? 1 : g));
        k_extract_idx<<<grid, 256, 0, st>>>(sorted, d_n, (uint64_t)max_n, idx_bits, idx);
        FP_LAUNCHED("k_extract_idx");
    }
    return FP_OK;
}

}  // namespace fpk
