// Integer-pipe throughput probe (no counterpart in the paper: it measures the
// GPU the filter runs on, to state the filter's arithmetic ceiling).
//
// kind 0 mirrors the filter's inner loop without its memory traffic: eight
// register-resident dictionary fingerprints per thread, query fingerprints
// read from shared memory, XOR + population count per pair, a minimum over
// the eight, one compare with 2k.  kind 1 is independent chains of 3-input
// logic operations, kind 2 independent chains of population counts.  kind 3
// is the filter's own k = 1 pattern loop: four fingerprints per thread, three
// through XOR + population count and one through the two-clear test, a
// 3-input minimum, the sign of (minimum - 3) shifted into a 32-pattern hit
// mask, patterns read four at a time from shared memory (128-bit loads), a
// warp sum of the hits after every 32 patterns; the data never passes, so it
// is the loop's ceiling without re-tests.
// Each block records its SM's cycle counter before and after the loop and the
// SM it ran on.  The blocks sharing an SM do not progress evenly (the warp
// schedulers favour some of them, which finish early while the others still
// run), so one block's own duration understates the SM time the blocks take
// together; the rate per SM per clock is therefore taken over each SM's span,
// from its first block's start to its last block's end (cycle counters are
// per SM, so starts and ends compare within one SM only).
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace fpk {

constexpr int PR_THREADS = 256;

__device__ __forceinline__ uint32_t sm_id() {
    uint32_t s;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(s));
    return s;
}

// rec[3 b .. 3 b + 2] = block b's start cycle, end cycle and SM
__global__ void __launch_bounds__(PR_THREADS) k_probe(int kind, int iters, uint32_t seed,
                                                     unsigned long long *rec, uint32_t *sink) {
    __shared__ __align__(16) uint32_t s_q[64];
    const uint32_t t = blockIdx.x * PR_THREADS + threadIdx.x;
    if (threadIdx.x < 64) s_q[threadIdx.x] = (seed * 2654435761u) ^ (threadIdx.x * 0x9E3779B9u);
    __syncthreads();
    uint32_t w[8];
#pragma unroll
    for (int v = 0; v < 8; v++) w[v] = (t * 0x85EBCA6Bu) ^ (v * 0xC2B2AE35u) ^ seed;
    uint32_t acc = 0;
    const long long c0 = clock64();
    if (kind == 0) {
        for (int it = 0; it < iters; it++) {
#pragma unroll 4
            for (int j = 0; j < 64; j++) {
                const uint32_t q = s_q[j];
                uint32_t m = __popc(w[0] ^ q);
#pragma unroll
                for (int v = 1; v < 8; v++) m = min(m, (uint32_t)__popc(w[v] ^ q));
                acc += m <= 2u;
            }
            w[it & 7] ^= acc;  // keeps the rounds from being folded together
        }
    } else if (kind == 1) {
        uint32_t a[8];
#pragma unroll
        for (int v = 0; v < 8; v++) a[v] = w[v];
        for (int it = 0; it < iters; it++) {
#pragma unroll 8
            for (int j = 0; j < 64; j++) {
                // eight independent 3-input logic operations per step, each reading
                // the previous step's values of other chains (nothing to fold)
                uint32_t b[8];
#pragma unroll
                for (int v = 0; v < 8; v++) b[v] = (a[v] & a[(v + 1) & 7]) ^ a[(v + 3) & 7];
#pragma unroll
                for (int v = 0; v < 8; v++) a[v] = b[v];
            }
        }
#pragma unroll
        for (int v = 0; v < 8; v++) acc ^= a[v];
    } else if (kind == 2) {
        uint32_t a[8];
#pragma unroll
        for (int v = 0; v < 8; v++) a[v] = w[v];
        for (int it = 0; it < iters; it++) {
#pragma unroll 8
            for (int j = 0; j < 64; j++) {
#pragma unroll
                for (int v = 0; v < 8; v++) a[v] = __popc(a[v]);  // one POPC each
            }
        }
#pragma unroll
        for (int v = 0; v < 8; v++) acc ^= a[v];
    } else {
        const uint4 *q4 = reinterpret_cast<const uint4 *>(s_q);
        for (int it = 0; it < iters; it++) {
            for (int jb = 0; jb < 64; jb += 32) {
                uint32_t hits = 0;
#pragma unroll
                for (int jj = 0; jj < 32; jj += 4) {
                    const uint4 q = q4[(jb + jj) >> 2];
                    const uint32_t qs[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
                    for (int u = 0; u < 4; u++) {
                        const uint32_t f0 = __popc(w[0] ^ qs[u]), f1 = __popc(w[1] ^ qs[u]),
                                       f2 = __popc(w[2] ^ qs[u]);
                        const uint32_t x = w[3] ^ qs[u], t = x & (x - 1u), z = (t & (t - 1u)) | 2u;
                        const uint32_t m = __vimin3_u32(f0, f1, min(f2, z));
                        hits = __funnelshift_l(m - 3u, hits, 1);
                    }
                }
                acc += __reduce_add_sync(0xffffffffu, __popc(hits));
            }
            w[0] ^= acc;
        }
    }
    const long long c1 = clock64();
    if (threadIdx.x == 0) {
        rec[3 * blockIdx.x + 0] = (unsigned long long)c0;
        rec[3 * blockIdx.x + 1] = (unsigned long long)c1;
        rec[3 * blockIdx.x + 2] = sm_id();
    }
    if (acc == 0x12345678u) sink[t] = acc;
}

}  // namespace fpk

using namespace fpk;

extern "C" int fp_probe(int kind, int iters, void *cuda_stream, fp_probe_result *out) {
    if (!out || kind < 0 || kind > 3 || iters <= 0) return FP_E_INVAL;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int per_sm = 0;
    FP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_probe, PR_THREADS, 0));
    if (per_sm < 1) per_sm = 1;
    const int sms = sm_count();
    const int grid = sms * per_sm;
    unsigned long long *cyc = nullptr;
    uint32_t *sink = nullptr;
    FP_CUDA(cudaMalloc((void **)&cyc, sizeof(unsigned long long) * 3 * grid));
    FP_CUDA(cudaMalloc((void **)&sink, sizeof(uint32_t) * grid * PR_THREADS));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_probe<<<grid, PR_THREADS, 0, st>>>(kind, iters / 8 + 1, 7u, cyc, sink);  // warm-up
    g_launches++;
    cudaEventRecord(e0, st);
    k_probe<<<grid, PR_THREADS, 0, st>>>(kind, iters, 11u, cyc, sink);
    g_launches++;
    cudaEventRecord(e1, st);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    std::vector<unsigned long long> h(3 * (size_t)grid);
    if (e == cudaSuccess) e = cudaMemcpy(h.data(), cyc, sizeof(unsigned long long) * 3 * grid, cudaMemcpyDeviceToHost);
    cudaFree(cyc);
    cudaFree(sink);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(e, "fp_probe");
    // per SM: blocks, first start, last end
    std::vector<long long> nblk(sms, 0);
    std::vector<unsigned long long> first(sms, ~0ull), last(sms, 0);
    for (int b = 0; b < grid; b++) {
        const unsigned long long sm = h[3 * b + 2];
        if (sm >= (unsigned long long)sms) return fail(FP_E_CUDA, "fp_probe: SM id out of range");
        nblk[sm]++;
        first[sm] = std::min(first[sm], h[3 * b]);
        last[sm] = std::max(last[sm], h[3 * b + 1]);
    }
    double blocks = 0, span = 0;  // over the SMs that ran blocks
    int used = 0;
    for (int i = 0; i < sms; i++)
        if (nblk[i]) {
            blocks += (double)nblk[i];
            span += (double)(last[i] - first[i]);
            used++;
        }
    const double per_thread = (double)iters * 64.0 * (kind == 3 ? 4.0 : 8.0);  // pair tests, LOP3s or POPCs
    out->kind = kind;
    out->sm_count = sms;
    out->ops = per_thread * PR_THREADS * grid;
    out->seconds = ms * 1e-3;
    out->ops_per_s = out->ops / out->seconds;
    out->ops_per_clk_per_sm = per_thread * PR_THREADS * blocks / span;  // ops per SM-cycle of the spans
    out->sm_clock_mhz = used ? span / used / out->seconds * 1e-6 : 0.0;
    return FP_OK;
}
