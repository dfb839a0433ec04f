// fp_query_noalloc: the query path for small batches, running entirely in a
// fixed scratch area that is part of the library image, so the call never
// allocates device memory.
//
// Who needs it: callers that must not allocate while they serve -- a process
// whose device memory is handed out up front by its own allocator (the CUDA
// pool must stay untouched once it starts answering), code that runs between
// the capture-free set-up and a latency-critical loop where an allocation
// could stall on a device-wide synchronisation, or hosts that forbid new
// device allocations after start-up.  They pass device inputs and outputs and
// the library works in the scratch array below.
//
// The scratch array is a file-scope __device__ array: every GPU that loads
// the library holds it (FP_NOALLOC_SCRATCH_BYTES, about 14 MB) until the
// process exits.  In host code the array's name is only a host-side stand-in,
// so its device address is obtained once per device with
// cudaGetSymbolAddress, on the first call made with that device current;
// that first call should therefore come before any stream capture.  Every
// call shares the array and it keeps the last call's contents; everything
// that must start at zero is cleared by the call itself.  Two calls whose GPU
// work overlapped would race on the array, so this entry point holds a
// process-wide lock and waits for its stream before it returns.
#include <mutex>

#include "common.cuh"

namespace fpk {
namespace {

constexpr int64_t MAXQ = FP_NOALLOC_MAX_QUERIES;
constexpr int64_t MAXC = FP_NOALLOC_MAX_CHARS;
constexpr int64_t MAXS = FP_NOALLOC_MAX_CANDIDATES;
constexpr int64_t MAXM = FP_NOALLOC_MAX_MATCHES;
constexpr int64_t SLOTS = MAXQ + (int64_t)(SLOT_ALIGN - 1) * 256;
constexpr int64_t STRB = MAXC + 15 * MAXQ + STR_SLACK;
constexpr int64_t MAXSEG = 256 * 31;
constexpr int64_t al(int64_t x) { return (x + 255) / 256 * 256; }

constexpr int64_t O_KEYS = 0;
constexpr int64_t O_KEYS2 = O_KEYS + al(8 * MAXQ);
constexpr int64_t O_HIST = O_KEYS2 + al(8 * MAXQ);
constexpr int64_t O_USTART = O_HIST + al(4 * 256);
constexpr int64_t O_STR16 = O_USTART + al(4 * 256);
constexpr int64_t O_TOT = O_STR16 + al(8 * 256);
constexpr int64_t O_QFP = O_TOT + al(16);
constexpr int64_t O_QIDX = O_QFP + al(4 * (SLOTS + FP_SLACK_SLOTS));
constexpr int64_t O_QLEN = O_QIDX + al(4 * SLOTS);
constexpr int64_t O_QROW = O_QLEN + al(SLOTS);
constexpr int64_t O_QSTR = O_QROW + al(4 * SLOTS);
constexpr int64_t O_BSTART = O_QSTR + al(STRB);
constexpr int64_t O_BCOUNT = O_BSTART + al(4 * 256);
constexpr int64_t O_SEG = O_BCOUNT + al(4 * 256);
constexpr int64_t O_SCAL = O_SEG + al((int64_t)sizeof(Segment) * MAXSEG);
constexpr int64_t O_GROUP = O_SCAL + al(8 * 8);
constexpr int64_t O_ERR = O_GROUP + al(8);
constexpr int64_t O_SURV = O_ERR + al(4);
constexpr int64_t O_MATCH = O_SURV + al(8 * MAXS);
constexpr int64_t O_TMP = O_MATCH + al(8 * MAXM);
constexpr int64_t O_RHIST = O_TMP + al(8 * MAXM);
constexpr int64_t SCRATCH_BYTES = O_RHIST + al(4 * 256 * 256);
static_assert(SCRATCH_BYTES <= FP_NOALLOC_SCRATCH_BYTES, "scratch layout exceeds the stated size");

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
unsigned char *g_base[MAX_DEVICES] = {};

int nfail(int code, const char *msg) {
    set_error(msg);
    return code;
}

bool on_device(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int bits_for_count(int64_t n) {
    int b = 1;
    while (b < 63 && ((int64_t)1 << b) < n) b++;
    return b;
}

}  // namespace

// The scratch area itself (device memory reserved with the library image).
static __device__ __align__(256) unsigned char g_noalloc_scratch[FP_NOALLOC_SCRATCH_BYTES];

// Device address of the scratch array on the current device (looked up once
// per device, with that device current).  Caller holds g_mu.
static int scratch_base(unsigned char **out) {
    int dev = 0;
    FP_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= MAX_DEVICES) return nfail(FP_E_UNSUPPORTED, "device ordinal out of range");
    if (!g_base[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(e != cudaSuccess ? e : cudaErrorInvalidSymbol,
                                                     "cudaGetSymbolAddress(scratch)");
        g_base[dev] = (unsigned char *)p;
    }
    *out = g_base[dev];
    return FP_OK;
}

}  // namespace fpk

using namespace fpk;

extern "C" int fp_query_noalloc(fp_index *ix, const uint8_t *chars, const int64_t *offsets, int64_t n_queries,
                                int k, int metric, int64_t *row_ptr, int32_t *idx, int64_t idx_capacity,
                                int64_t *n_matches, void *cuda_stream) {
    if (!ix || !offsets || !row_ptr || !n_matches || idx_capacity < 0 || (idx_capacity > 0 && !idx))
        return nfail(FP_E_INVAL, "fp_query_noalloc: null pointer or negative capacity");
    *n_matches = 0;
    if (n_queries < 0 || n_queries > MAXQ)
        return nfail(FP_E_INVAL, "fp_query_noalloc: at most FP_NOALLOC_MAX_QUERIES (4096) patterns per call");
    if (k < 0 || k > 15) return nfail(FP_E_INVAL, "k must be in 0..15");
    if (metric != FP_HAM && metric != FP_LEV) return nfail(FP_E_INVAL, "bad metric");
    if (metric == FP_LEV && (ix->P.type == FP_OCC_HALVED || ix->P.type == FP_POS))
        return nfail(FP_E_UNSUPPORTED, "occurrence-halved and position fingerprints bound only the Hamming distance");
    if (!on_device(offsets) || !on_device(row_ptr) || (idx_capacity > 0 && !on_device(idx)))
        return nfail(FP_E_INVAL, "fp_query_noalloc: offsets, row_ptr and idx must be device memory");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    std::lock_guard<std::mutex> lock(g_mu);
    unsigned char *base = nullptr;
    FP_TRY(scratch_base(&base));
    if (n_queries == 0) {
        FP_CUDA(cudaMemsetAsync(row_ptr, 0, sizeof(int64_t), st));
        FP_CUDA(cudaStreamSynchronize(st));
        return FP_OK;
    }
    int64_t ends[2] = {0, 0};
    FP_CUDA(cudaMemcpyAsync(&ends[0], offsets, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    FP_CUDA(cudaMemcpyAsync(&ends[1], offsets + n_queries, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    FP_CUDA(cudaStreamSynchronize(st));
    if (ends[0] != 0 || ends[1] < 0) return nfail(FP_E_INVAL, "offsets[0] must be 0 and offsets non-decreasing");
    if (ends[1] > MAXC)
        return nfail(FP_E_INVAL, "fp_query_noalloc: at most FP_NOALLOC_MAX_CHARS (262144) pattern bytes per call");
    if (ends[1] > 0 && (!chars || !on_device(chars)))
        return nfail(FP_E_INVAL, "fp_query_noalloc: chars must be device memory");

    Bucketed Q;
    Q.fp = base + O_QFP;
    Q.idx = (int32_t *)(base + O_QIDX);
    Q.len = base + O_QLEN;
    Q.row16 = (uint32_t *)(base + O_QROW);
    Q.str = base + O_QSTR;
    Q.b_start = (int32_t *)(base + O_BSTART);
    Q.b_count = (int32_t *)(base + O_BCOUNT);
    BucketScratch S;
    S.keys = (uint64_t *)(base + O_KEYS);
    S.keys2 = (uint64_t *)(base + O_KEYS2);
    S.hist = (int32_t *)(base + O_HIST);
    S.ustart = (int32_t *)(base + O_USTART);
    S.str16 = (int64_t *)(base + O_STR16);
    S.tot = (int64_t *)(base + O_TOT);
    S.radix_hist = (uint32_t *)(base + O_RHIST);
    int32_t *d_group = (int32_t *)(base + O_GROUP);
    int32_t *d_err = (int32_t *)(base + O_ERR);
    uint64_t *surv = (uint64_t *)(base + O_SURV);
    uint64_t *matches = (uint64_t *)(base + O_MATCH);
    uint64_t *tmp = (uint64_t *)(base + O_TMP);
    QueryPlan plan;
    plan.seg = (Segment *)(base + O_SEG);
    plan.max_segments = 256 * (2 * k + 1);
    plan.scal = (uint64_t *)(base + O_SCAL);

    // From the first enqueue on, every exit goes through finish(): a failure
    // still waits for the work already queued on st, so that no later call
    // (on any stream) can meet this call's kernels in the shared scratch.
    uint64_t scal[8] = {0};
    int32_t h_err = 0;
    const int64_t cap = idx_capacity < MAXM ? idx_capacity : MAXM;
    auto enqueue = [&]() -> int {
        const int32_t group[2] = {k, metric};
        FP_CUDA(cudaMemsetAsync(d_err, 0, sizeof(int32_t), st));
        FP_CUDA(cudaMemcpyAsync(d_group, group, sizeof(group), cudaMemcpyHostToDevice, st));
        FP_TRY(bucketize_into(chars, offsets, n_queries, ends[1], nullptr, 1, ix->d_map, ix->P, st, &Q, S, d_err));
        FilterCfg cfg{};
        cfg.mode = FP_MODE_TILED;
        cfg.tq = 256;
        cfg.v = 4;
        cfg.k1mix = k == 1;
        cfg.mma = false;
        int tq = 0, tw = 0;
        tile_shape(cfg, ix->P, &tq, &tw);
        FP_TRY(plan_segments(Q, ix->D, d_group, d_group + 1, tq, tw, &plan, st));
        FP_TRY(launch_filter(Q, ix->D, plan, ix->P, cfg, surv, MAXS, st, nullptr));
        FP_TRY(launch_verify(Q, ix->D, surv, plan.scal + 4, MAXS, k, metric, ix->idx_bits, matches, plan.scal + 5,
                             MAXM, st));
        FP_TRY(build_csr_into(matches, tmp, S.radix_hist, plan.scal + 5, cap, bits_for_count(n_queries),
                              ix->idx_bits, n_queries, row_ptr, idx, st));
        FP_CUDA(cudaMemcpyAsync(scal, plan.scal, sizeof(scal), cudaMemcpyDeviceToHost, st));
        FP_CUDA(cudaMemcpyAsync(&h_err, d_err, sizeof(h_err), cudaMemcpyDeviceToHost, st));
        return FP_OK;
    };
    const int rc = enqueue();
    const cudaError_t se = cudaStreamSynchronize(st);  // on every path, success or not
    if (rc != FP_OK) return rc;  // the first error is the one reported
    if (se != cudaSuccess) return cuda_fail(se, "cudaStreamSynchronize");
    if (h_err) return nfail(FP_E_INVAL, "string longer than 255 bytes or offsets not monotone");
    if (scal[6])  // the planner's overflow flag: no tile ran, so the lists would be incomplete
        return nfail(FP_E_OVERFLOW, "fp_query_noalloc: tile plan overflow");
    if ((int64_t)scal[4] > MAXS)
        return nfail(FP_E_OVERFLOW, "fp_query_noalloc: more than FP_NOALLOC_MAX_CANDIDATES pairs passed the filter");
    *n_matches = (int64_t)scal[5];
    if ((int64_t)scal[5] > cap)
        return nfail(FP_E_OVERFLOW, "fp_query_noalloc: more matches than idx_capacity / FP_NOALLOC_MAX_MATCHES");
    return FP_OK;
}
