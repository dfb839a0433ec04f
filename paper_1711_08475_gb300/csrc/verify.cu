// Explicit verification of the pairs the fingerprint bound could not reject
// (Sec. 3: "when the fingerprint comparison is not decisive, we still have to
// perform an explicit verification"; Sec. 4 for the two routines).
//
// Hamming (Sec. 4: compare characters until more than k mismatches): both
// strings sit in zero-padded 16-byte rows of equal length, so the compare
// runs over 128-bit words; a 32-bit word's mismatching bytes are counted with
// the exact zero-byte test ((x & 0x7f..) + 0x7f.. | x) & 0x80.. on x = a ^ b,
// and the loop stops as soon as the count exceeds k.
//
// Levenshtein (Sec. 4 uses the 2k+1 diagonal strip, Ukkonen 1985): cells
// (i, j) with |i - j| > k cannot lie on an edit path of cost <= k, so only the
// 2k+1 diagonals are kept, here as bits of a word.  The test is the anchored
// Wu-Manber recurrence (Wu and Manber, "Fast text searching allowing errors",
// CACM 1992) on that band: R_e holds the cells (i, j) of the current column
// with D(i, j) <= e, bit b standing for row i = j - k + b.  Tying the bit to
// the diagonal makes the diagonal move (match or substitution) shift-free,
// the insertion move a right shift and the deletion move a left shift:
//   R_0' = R_0 & Eq
//   R_e' = (R_e & Eq) | R_{e-1} | (R_{e-1} >> 1) | (R_{e-1}' << 1)
// Eq bit b says A[j-k+b-1] == B[j-1]; it is computed for all 2k+1 rows at once
// with the zero-byte test on a byte window of A that slides one byte per
// column.  Every move keeps or increases i, so bits for rows beyond |A| never
// reach row |A| and need no mask.  Lev(A, B) <= k iff bit |A| - |B| + k of
// R_k is set after the last column; the scan stops early once R_k is empty.
//
// For k = 1 the recurrence is not needed: with equal lengths one edit is a
// substitution (at most one differing byte), and with lengths differing by
// one the shorter string is the longer one minus one byte, which one pass
// over the first mismatch and the shifted suffix decides (lev1_within).
#include "verify_core.cuh"

namespace fpk {

struct VerifyArgs {
    const uint64_t *surv;
    const uint64_t *n_surv;
    uint64_t surv_cap;
    const uint8_t *q_len;
    const uint32_t *q_row16;
    const uint8_t *q_str;
    const int32_t *q_idx;
    const uint8_t *d_len;
    const uint32_t *d_row16;
    const uint8_t *d_str;
    const int32_t *d_idx;
    // rows by slot: both sets have one group of 256 length bins whose rows are
    // contiguous in slot order (bucketing writes them so, the weight order
    // moves them with their slots), so the row of a slot follows from its
    // length and the bin's first slot and row, kept in shared memory: one
    // gather fewer per string
    const int32_t *q_bstart, *q_bcount, *d_bstart, *d_bcount;
    int rows_by_slot;
    int idx_bits;
    uint64_t *matches;
    uint64_t *n_matches;
    uint64_t match_cap;
};

// Survivors per thread: a thread gathers the records, lengths and row offsets
// of VU survivors (and, for Hamming, the first 16 bytes of both rows) before
// it verifies any of them, so that VU independent chains of dependent loads
// are in flight instead of one.
#ifndef VERIFY_U
#define VERIFY_U 4
#endif

// metric 0: Hamming with runtime k; metric 1: Levenshtein with K.
// Matches are staged per warp in shared memory and appended to the global
// list with one atomic reservation per VSTAGE / 2 or more, not one per round.
constexpr int VSTAGE = 256;

__device__ __forceinline__ void flush_matches(const VerifyArgs &A, uint64_t *stage, uint32_t *cnt, int lane) {
    __syncwarp();
    const uint32_t c = min(*cnt, (uint32_t)VSTAGE);
    unsigned long long base = 0;
    if (lane == 0 && c) base = atomicAdd((unsigned long long *)A.n_matches, (unsigned long long)c);
    base = __shfl_sync(0xffffffffu, base, 0);
    for (uint32_t i = lane; i < c; i += 32) {
        const uint64_t pos = base + i;
        if (pos < A.match_cap) A.matches[pos] = stage[i];
    }
    __syncwarp();
    if (lane == 0) *cnt = 0;
    __syncwarp();
}

// Resident blocks per SM the register budget is set for.
#ifndef VERIFY_MIN_BLOCKS
#define VERIFY_MIN_BLOCKS 4  // measured against 1 and 3 (Hamming keeps 64 registers instead of 80)
#endif
#ifndef VERIFY_LEV1_MIN_BLOCKS
#define VERIFY_LEV1_MIN_BLOCKS 4  // the direct k = 1 test: 48 registers; 6 and 8 blocks measured no faster
#endif
template <int METRIC, int K>
constexpr int verify_min_blocks() {
    return METRIC == FP_LEV && K == 1 ? VERIFY_LEV1_MIN_BLOCKS : VERIFY_MIN_BLOCKS;
}

template <int METRIC, int K>
__global__ void __launch_bounds__(256, (verify_min_blocks<METRIC, K>())) k_verify(VerifyArgs A, int k) {
    constexpr int U = VERIFY_U;
    __shared__ uint64_t s_stage[8][VSTAGE];
    __shared__ uint32_t s_cnt[8];
    __shared__ uint32_t s_first[2][256], s_row0[2][256];  // per length bin: first slot, its row
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t *stage = s_stage[warp];
    uint32_t *cnt = &s_cnt[warp];
    if (lane == 0) *cnt = 0;
    if (A.rows_by_slot) {
        const int t = threadIdx.x;  // blockDim.x == 256
        const int32_t qf = A.q_bstart[t], df = A.d_bstart[t];
        s_first[0][t] = (uint32_t)qf;
        s_row0[0][t] = A.q_bcount[t] > 0 ? A.q_row16[qf] : 0u;
        s_first[1][t] = (uint32_t)df;
        s_row0[1][t] = A.d_bcount[t] > 0 ? A.d_row16[df] : 0u;
    }
    __syncthreads();
    const uint64_t n0 = *A.n_surv;
    const uint64_t n = n0 < A.surv_cap ? n0 : A.surv_cap;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x * U;
    const unsigned lt = (1u << lane) - 1u;
    static_assert(VSTAGE / 2 + 32 * VERIFY_U <= VSTAGE, "a round of matches must fit the stage");
    for (uint64_t base = ((uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u)) * U; base < n; base += stride) {
        // survivor base + 32 u + lane for u < U: each of the U loads is coalesced
        uint64_t s[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const uint64_t i = base + 32u * u + lane;
            s[u] = i < n ? A.surv[i] : ~0ull;
        }
        int m[U], L[U];
        uint32_t qr[U], dr[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            if (s[u] != ~0ull) {
                const uint32_t qs = (uint32_t)(s[u] >> 32), ds = (uint32_t)s[u];
                m[u] = A.q_len[qs];
                L[u] = A.d_len[ds];
                if (A.rows_by_slot) {
                    qr[u] = s_row0[0][m[u]] + (qs - s_first[0][m[u]]) * (uint32_t)((m[u] + 15) >> 4);
                    dr[u] = s_row0[1][L[u]] + (ds - s_first[1][L[u]]) * (uint32_t)((L[u] + 15) >> 4);
                } else {
                    qr[u] = A.q_row16[qs];
                    dr[u] = A.d_row16[ds];
                }
            } else {
                m[u] = -1;
                L[u] = -2;
                qr[u] = dr[u] = 0;
            }
        }
        bool hit[U];
        if (METRIC == FP_HAM) {
            uint4 x[U], y[U];
#pragma unroll
            for (int u = 0; u < U; u++) {
                if (m[u] == L[u] && m[u] > 0) {
                    x[u] = *(const uint4 *)(A.q_str + (uint64_t)qr[u] * 16);
                    y[u] = *(const uint4 *)(A.d_str + (uint64_t)dr[u] * 16);
                } else {
                    x[u] = y[u] = make_uint4(0u, 0u, 0u, 0u);
                }
            }
#pragma unroll
            for (int u = 0; u < U; u++)
                hit[u] = m[u] == L[u] && ham_within_first(x[u], y[u], A.q_str + (uint64_t)qr[u] * 16,
                                                          A.d_str + (uint64_t)dr[u] * 16, m[u], k);
        } else {
#pragma unroll
            for (int u = 0; u < U; u++)
                hit[u] = m[u] >= 0 && m[u] - L[u] <= K && L[u] - m[u] <= K &&
                         (K == 1 ? lev1_within(A.q_str + (uint64_t)qr[u] * 16, m[u], A.d_str + (uint64_t)dr[u] * 16,
                                               L[u])
                                 : lev_within<K>(A.q_str + (uint64_t)qr[u] * 16, m[u],
                                                 A.d_str + (uint64_t)dr[u] * 16, L[u]));
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            const unsigned bal = __ballot_sync(0xffffffffu, hit[u]);
            if (bal) {
                const uint32_t at = *cnt;  // < VSTAGE / 2 + 32 * U <= VSTAGE
                if (hit[u]) {
                    const uint32_t qs = (uint32_t)(s[u] >> 32), ds = (uint32_t)s[u];
                    stage[at + __popc(bal & lt)] =
                        ((uint64_t)(uint32_t)A.q_idx[qs] << A.idx_bits) | (uint64_t)(uint32_t)A.d_idx[ds];
                }
                __syncwarp();
                if (lane == 0) *cnt = at + __popc(bal);
                __syncwarp();
            }
        }
        if (*cnt >= VSTAGE / 2) flush_matches(A, stage, cnt, lane);
    }
    flush_matches(A, stage, cnt, lane);
}

template <int METRIC, int K>
static int launch_verify_k(const VerifyArgs &A, int k, cudaStream_t st) {
    static int grid = 0;
    if (grid == 0) {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_verify<METRIC, K>, 256, 0);
        grid = sm_count() * (per_sm > 0 ? per_sm : 1);
    }
    k_verify<METRIC, K><<<grid, 256, 0, st>>>(A, k);
    FP_LAUNCHED("k_verify");
    return FP_OK;
}

int launch_verify_args(const VerifyArgs &A, int k, int metric, cudaStream_t st) {
    if (metric == FP_HAM) return launch_verify_k<FP_HAM, 0>(A, k, st);
    switch (k) {
        case 0: return launch_verify_k<FP_LEV, 0>(A, k, st);
        case 1: return launch_verify_k<FP_LEV, 1>(A, k, st);
        case 2: return launch_verify_k<FP_LEV, 2>(A, k, st);
        case 3: return launch_verify_k<FP_LEV, 3>(A, k, st);
        case 4: return launch_verify_k<FP_LEV, 4>(A, k, st);
        case 5: return launch_verify_k<FP_LEV, 5>(A, k, st);
        case 6: return launch_verify_k<FP_LEV, 6>(A, k, st);
        case 7: return launch_verify_k<FP_LEV, 7>(A, k, st);
        case 8: return launch_verify_k<FP_LEV, 8>(A, k, st);
        case 9: return launch_verify_k<FP_LEV, 9>(A, k, st);
        case 10: return launch_verify_k<FP_LEV, 10>(A, k, st);
        case 11: return launch_verify_k<FP_LEV, 11>(A, k, st);
        case 12: return launch_verify_k<FP_LEV, 12>(A, k, st);
        case 13: return launch_verify_k<FP_LEV, 13>(A, k, st);
        case 14: return launch_verify_k<FP_LEV, 14>(A, k, st);
        case 15: return launch_verify_k<FP_LEV, 15>(A, k, st);
    }
    return FP_E_INVAL;
}

int launch_verify(const Bucketed &q, const Bucketed &d, const uint64_t *surv, const uint64_t *d_n_surv,
                  int64_t surv_cap, int k, int metric, int idx_bits, uint64_t *matches,
                  uint64_t *d_n_matches, int64_t match_cap, cudaStream_t st) {
    VerifyArgs A;
    A.surv = surv;
    A.n_surv = d_n_surv;
    A.surv_cap = (uint64_t)surv_cap;
    A.q_len = q.len;
    A.q_row16 = q.row16;
    A.q_str = q.str;
    A.q_idx = q.idx;
    A.d_len = d.len;
    A.d_row16 = d.row16;
    A.d_str = d.str;
    A.d_idx = d.idx;
    A.q_bstart = q.b_start;
    A.q_bcount = q.b_count;
    A.d_bstart = d.b_start;
    A.d_bcount = d.b_count;
    A.rows_by_slot = q.nbins == 256 && d.nbins == 256;
    A.idx_bits = idx_bits;
    A.matches = matches;
    A.n_matches = d_n_matches;
    A.match_cap = (uint64_t)match_cap;
    return launch_verify_args(A, k, metric, st);
}

}  // namespace fpk
