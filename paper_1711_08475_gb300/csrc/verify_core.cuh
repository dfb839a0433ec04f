// Device-side verification routines shared by the verification kernels and
// the fused filter + verify kernel.  See verify.cu for the method.
#pragma once

#include "common.cuh"

namespace fpk {

// 0x80 in each zero byte of x, 0 elsewhere
__device__ __forceinline__ uint32_t zero_byte_mask(uint32_t x) {
    return ~(((x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | x | 0x7F7F7F7Fu);  // 0x80 in each zero byte
}

__device__ __forceinline__ bool ham_within(const uint8_t *a, const uint8_t *b, int len, int k) {
    const uint4 *A = (const uint4 *)a, *B = (const uint4 *)b;
    int mism = 0;
    for (int c = 0; c < len; c += 16) {
        uint4 x = A[c >> 4], y = B[c >> 4];
        // mismatching bytes = 4 - zero bytes of the XOR (padding is zero on both sides)
        mism += __popc(~zero_byte_mask(x.x ^ y.x) & 0x80808080u) + __popc(~zero_byte_mask(x.y ^ y.y) & 0x80808080u) +
                __popc(~zero_byte_mask(x.z ^ y.z) & 0x80808080u) + __popc(~zero_byte_mask(x.w ^ y.w) & 0x80808080u);
        if (mism > k) return false;
    }
    return true;
}

// ham_within with the first 16 bytes of both rows already loaded (x, y).
__device__ __forceinline__ bool ham_within_first(uint4 x, uint4 y, const uint8_t *a, const uint8_t *b, int len, int k) {
    int mism = __popc(~zero_byte_mask(x.x ^ y.x) & 0x80808080u) + __popc(~zero_byte_mask(x.y ^ y.y) & 0x80808080u) +
               __popc(~zero_byte_mask(x.z ^ y.z) & 0x80808080u) + __popc(~zero_byte_mask(x.w ^ y.w) & 0x80808080u);
    if (mism > k) return false;
    const uint4 *A = (const uint4 *)a, *B = (const uint4 *)b;
    for (int c = 16; c < len; c += 16) {
        const uint4 p = A[c >> 4], q = B[c >> 4];
        mism += __popc(~zero_byte_mask(p.x ^ q.x) & 0x80808080u) + __popc(~zero_byte_mask(p.y ^ q.y) & 0x80808080u) +
                __popc(~zero_byte_mask(p.z ^ q.z) & 0x80808080u) + __popc(~zero_byte_mask(p.w ^ q.w) & 0x80808080u);
        if (mism > k) return false;
    }
    return true;
}

// Bytes [lo, hi) of a little-endian 32-bit word, 0 <= lo <= hi <= 4.
__device__ __forceinline__ uint32_t byte_range_mask(int lo, int hi) {
    const uint32_t up = hi >= 4 ? 0xFFFFFFFFu : ((1u << (8 * hi)) - 1u);
    const uint32_t low = lo <= 0 ? 0u : ((1u << (8 * lo)) - 1u);
    return up & ~low;
}

// Lev(a, b) <= 1 without the strip DP.  Equal lengths: one edit can only be a
// substitution, so Lev <= 1 iff at most one byte differs.  Lengths differing
// by one: the shorter string must be the longer one with one byte deleted,
// i.e. the two agree before their first mismatch p (p = the shorter length
// if there is none) and the longer string's bytes after p equal the shorter
// one's bytes from p on.  Strings sit in zero-padded 16-byte rows with
// readable bytes after them; bytes outside a string are masked off.
__device__ __forceinline__ bool lev1_within(const uint8_t *a, int m, const uint8_t *b, int n) {
    if (m == n) return ham_within(a, b, m, 1);
    if (m < n) {  // a is the longer one
        const uint8_t *t = a;
        a = b;
        b = t;
        const int u = m;
        m = n;
        n = u;
    }
    if (m != n + 1) return false;
    const uint32_t *A = (const uint32_t *)a, *B = (const uint32_t *)b;
    int p = n;  // first mismatch among bytes [0, n)
    for (int j = 0; 4 * j < n; j++) {
        const uint32_t x = (A[j] ^ B[j]) & byte_range_mask(0, n - 4 * j);
        if (x) {
            p = 4 * j + ((__ffs(x) - 1) >> 3);
            break;
        }
    }
    // a[i + 1] == b[i] for every i in [p, n)
    for (int j = p >> 2; 4 * j < n; j++) {
        const uint32_t shifted = __funnelshift_r(A[j], A[j + 1], 8);  // bytes 4j+1 .. 4j+4 of a
        if ((shifted ^ B[j]) & byte_range_mask(p - 4 * j, n - 4 * j)) return false;
    }
    return true;
}

template <int K>
__device__ __forceinline__ bool lev_within(const uint8_t *a, int m, const uint8_t *b, int n) {
    constexpr int BAND = 2 * K + 1;
    constexpr uint32_t BM = BAND >= 32 ? 0xFFFFFFFFu : ((1u << BAND) - 1u);
    constexpr int PADW = (K + 3) / 4;  // zero words in front of A so that window offsets are >= 0
    constexpr int NWIN = (BAND + 3) / 4;
    constexpr int NREG = ((3 - K + 4 * PADW + 4 * (NWIN - 1)) >> 2) + 2;
    const uint32_t *A32 = (const uint32_t *)a;
    const uint32_t *B32 = (const uint32_t *)b;
    uint32_t R[K + 1];
#pragma unroll
    for (int e = 0; e <= K; e++) R[e] = ((((e + 1) >= 32 ? 0xFFFFFFFFu : ((1u << (e + 1)) - 1u))) << K) & BM;
    uint32_t w[NREG];
#pragma unroll
    for (int x = 0; x < NREG; x++) w[x] = x < PADW ? 0u : A32[x - PADW];
    const int iters = (n + 3) >> 2;
    for (int it = 0; it < iters; it++) {
        const uint32_t bw = B32[it];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            if (4 * it + u < n) {
                const uint32_t tt = ((bw >> (8 * u)) & 0xFFu) * 0x01010101u;
                uint32_t eq = 0;
#pragma unroll
                for (int q = 0; q < NWIN; q++) {
                    const int off = u - K + 4 * PADW + 4 * q;  // byte offset of the window word
                    const int wi = off >> 2, sh = (off & 3) * 8;
                    const uint32_t win = sh ? __funnelshift_r(w[wi], w[wi + 1], sh) : w[wi];
                    const uint32_t z = zero_byte_mask(win ^ tt) >> 7;  // bits 0, 8, 16, 24
                    eq |= ((z * 0x00204081u) >> 21 & 0xFu) << (4 * q);
                }
                eq &= BM;
                uint32_t prev = R[0];
                uint32_t cur = prev & eq;
                R[0] = cur;
#pragma unroll
                for (int e = 1; e <= K; e++) {
                    const uint32_t old = R[e];
                    const uint32_t nv = ((old & eq) | prev | (prev >> 1) | (cur << 1)) & BM;
                    prev = old;
                    cur = nv;
                    R[e] = nv;
                }
            }
        }
        if (R[K] == 0u) return false;
#pragma unroll
        for (int x = 0; x + 1 < NREG; x++) w[x] = w[x + 1];
        const int nx = it + NREG - PADW;
        w[NREG - 1] = nx < 0 ? 0u : A32[nx];
    }
    return (R[K] >> (m - n + K)) & 1u;
}

// Each banded test compiled once per translation unit, out of line, so that
// kernels calling it for a runtime k do not carry sixteen inlined copies.
template <int K>
static __device__ __noinline__ bool lev_within_outline(const uint8_t *a, int m, const uint8_t *b, int n) {
    return lev_within<K>(a, m, b, n);
}

// Lev(a, b) <= k for a runtime k in 0..15 (warp-uniform in every caller, so
// the switch does not diverge).
static __device__ __noinline__ bool lev_within_k(int k, const uint8_t *a, int m, const uint8_t *b, int n) {
    switch (k) {
        case 0: return lev_within_outline<0>(a, m, b, n);
        case 1: return lev_within_outline<1>(a, m, b, n);
        case 2: return lev_within_outline<2>(a, m, b, n);
        case 3: return lev_within_outline<3>(a, m, b, n);
        case 4: return lev_within_outline<4>(a, m, b, n);
        case 5: return lev_within_outline<5>(a, m, b, n);
        case 6: return lev_within_outline<6>(a, m, b, n);
        case 7: return lev_within_outline<7>(a, m, b, n);
        case 8: return lev_within_outline<8>(a, m, b, n);
        case 9: return lev_within_outline<9>(a, m, b, n);
        case 10: return lev_within_outline<10>(a, m, b, n);
        case 11: return lev_within_outline<11>(a, m, b, n);
        case 12: return lev_within_outline<12>(a, m, b, n);
        case 13: return lev_within_outline<13>(a, m, b, n);
        case 14: return lev_within_outline<14>(a, m, b, n);
        default: return lev_within_outline<15>(a, m, b, n);
    }
}

}  // namespace fpk
