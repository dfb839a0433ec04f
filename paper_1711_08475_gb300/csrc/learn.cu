// Learned symbol-to-bit map for occurrence fingerprints (a10 of the build
// plan).  Sec. 3.2 builds the fingerprint through "a mapping c -> q"; the
// paper takes the most frequent symbols (Sec. 3, "Common").  Any map, also a
// many-to-one one, keeps Eq. 1 valid for occurrence fingerprints (a
// substitution moves at most one symbol out of and one into the string's
// field set), so a map may be chosen purely for how many non-matching pairs
// it rejects.  This file learns one from pairs the method itself produces.
//
// Model (FP32): for each printable symbol c (0x20..0x7E, 95 symbols),
//   h_c = ReLU(W1[:, c] + b1)            (64 hidden units; one-hot input)
//   z_c = W2 h_c + b2                    (one logit per field, F <= 32)
//   A_c = softmax(z_c / tau)             (soft assignment of c to the fields)
// Soft F_D of a pair (pattern symbols P, word symbols W): the expected
// Hamming weight of the XOR of the two fingerprints when every symbol c lands
// on field b with probability A_c,b, independently.  With I = P & W,
// P' = P \ W, W' = W \ P, bit b differs iff no symbol of I lands on b and
// exactly one of P', W' has a symbol landing on b:
//   f_b = prod_{c in I} (1 - A_c,b) * (p_b + q_b - 2 p_b q_b),
//   p_b = 1 - prod_{c in P'} (1 - A_c,b),  q_b likewise over W',
// and F = sum_b f_b.  With one-hot A_c this is exactly the Hamming weight of
// the XOR (Sec. 3.3); for near-identical strings it is near zero, which is
// where the loss has to act.
// Loss on non-matching pairs (matches carry no constraint: the bound stays
// sound for any map):  softplus(beta (2k + 1 - F)) / beta, i.e. a smooth
// push of F_D to at least 2k + 1, the rejection threshold of Eq. 1.
// Forward, backward and Adam are the kernels below; the hard map is
// map[0x20 + c] = argmax_b A_c,b.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "verify_core.cuh"

namespace fpk {
namespace {

constexpr int NSYM = 95;   // printable ASCII
constexpr int HID = 64;
constexpr int MAXF = 32;
constexpr int NPARAM = HID * NSYM + HID + MAXF * HID + MAXF;  // W1, b1, W2, b2

// parameter offsets
constexpr int P_W1 = 0;                       // [HID][NSYM]
constexpr int P_B1 = P_W1 + HID * NSYM;       // [HID]
constexpr int P_W2 = P_B1 + HID;              // [MAXF][HID]
constexpr int P_B2 = P_W2 + MAXF * HID;       // [MAXF]

__device__ __forceinline__ uint64_t mix64(uint64_t z) {  // SplitMix64 finaliser
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// ---------------------------------------------------------------------------
// sampling: uniform pattern, then a uniform eligible word (equal length for
// Hamming, length within k for Levenshtein)
// ---------------------------------------------------------------------------
struct SampleArgs {
    Bucketed Q, D;
    FpParams P;
    int k, metric;
    uint64_t seed;
    int64_t n;
    int32_t *out_q, *out_w;
    uint8_t *out_passed, *out_match;
    uint64_t *out_masks;  // [n][4]: pattern symbols (2 words), word symbols (2 words)
};

__device__ __forceinline__ void symbol_mask(const uint8_t *row, int len, uint64_t &lo, uint64_t &hi) {
    lo = hi = 0;
    for (int i = 0; i < len; i++) {
        int c = (int)row[i] - 0x20;
        if (c < 0 || c >= NSYM) continue;
        if (c < 64) lo |= 1ull << c;
        else hi |= 1ull << (c - 64);
    }
}

__global__ void k_sample_pairs(SampleArgs A) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < A.n; s += (int64_t)gridDim.x * blockDim.x) {
        int32_t qs = -1, ds = -1;
        for (int attempt = 0; attempt < 64 && ds < 0; attempt++) {
            const uint64_t r1 = mix64(A.seed + (uint64_t)s * 0x9E3779B97F4A7C15ull + 2 * attempt + 1);
            const uint64_t r2 = mix64(r1 ^ 0xD1B54A32D192ED03ull);
            const int64_t slot = (int64_t)(r1 % (uint64_t)A.Q.n_slots);
            if (A.Q.idx[slot] < 0) continue;
            const int n = A.Q.len[slot];
            const int lo = A.metric == FP_HAM ? n : max(0, n - A.k), hi = A.metric == FP_HAM ? n : min(MAX_LEN, n + A.k);
            int64_t tot = 0;
            for (int L = lo; L <= hi; L++) tot += A.D.b_count[L];
            if (tot == 0) continue;
            int64_t r = (int64_t)(r2 % (uint64_t)tot);
            for (int L = lo; L <= hi; L++) {
                const int64_t c = A.D.b_count[L];
                if (r < c) {
                    ds = (int32_t)(A.D.b_start[L] + r);
                    break;
                }
                r -= c;
            }
            qs = (int32_t)slot;
        }
        if (ds < 0) {  // no eligible pair found: an empty sample (never a training signal)
            A.out_q[s] = -1;
            A.out_w[s] = -1;
            A.out_passed[s] = 0;
            A.out_match[s] = 1;
            for (int j = 0; j < 4; j++) A.out_masks[4 * s + j] = 0;
            continue;
        }
        const uint32_t fq = A.P.width == 16 ? ((const uint16_t *)A.Q.fp)[qs] : ((const uint32_t *)A.Q.fp)[qs];
        const uint32_t fw = A.P.width == 16 ? ((const uint16_t *)A.D.fp)[ds] : ((const uint32_t *)A.D.fp)[ds];
        const uint32_t x = fq ^ fw;
        uint32_t F;
        if (A.P.type == FP_POS) {
            const uint32_t t = (x & A.P.pos_low) + A.P.pos_low;
            F = __popc(((t | x) & A.P.pos_high) | (x & A.P.pos_occ));
        } else {
            F = __popc(x);
        }
        const int m = A.Q.len[qs], L = A.D.len[ds];
        const uint8_t *qa = A.Q.str + (uint64_t)A.Q.row16[qs] * 16;
        const uint8_t *da = A.D.str + (uint64_t)A.D.row16[ds] * 16;
        const bool match = A.metric == FP_HAM ? (m == L && ham_within(qa, da, m, A.k))
                                              : lev_within_k(A.k, qa, m, da, L);
        A.out_q[s] = A.Q.idx[qs];
        A.out_w[s] = A.D.idx[ds];
        A.out_passed[s] = F <= 2u * (uint32_t)A.k;
        A.out_match[s] = match;
        uint64_t a, b, c, d;
        symbol_mask(qa, m, a, b);
        symbol_mask(da, L, c, d);
        A.out_masks[4 * s + 0] = a;
        A.out_masks[4 * s + 1] = b;
        A.out_masks[4 * s + 2] = c;
        A.out_masks[4 * s + 3] = d;
    }
}

// ---------------------------------------------------------------------------
// forward: per symbol hidden units, logits, assignment and log(1 - A)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_mlp_forward(const float *__restrict__ prm, int F, float tau,
                                                     float *__restrict__ H, float *__restrict__ Aout,
                                                     float *__restrict__ logA1) {
    __shared__ float sh[NSYM * HID];
    for (int t = threadIdx.x; t < NSYM * HID; t += blockDim.x) {
        const int c = t / HID, i = t % HID;
        const float v = prm[P_W1 + i * NSYM + c] + prm[P_B1 + i];
        sh[t] = v > 0.f ? v : 0.f;
        H[t] = sh[t];
    }
    __syncthreads();
    // one thread per symbol: logits, softmax (F <= 32 fields)
    for (int c = threadIdx.x; c < NSYM; c += blockDim.x) {
        float z[MAXF];
        float zmax = -1e30f;
        for (int j = 0; j < F; j++) {
            float acc = prm[P_B2 + j];
            for (int i = 0; i < HID; i++) acc += prm[P_W2 + j * HID + i] * sh[c * HID + i];
            z[j] = acc / tau;
            zmax = fmaxf(zmax, z[j]);
        }
        float sum = 0.f;
        for (int j = 0; j < F; j++) {
            z[j] = expf(z[j] - zmax);
            sum += z[j];
        }
        for (int j = 0; j < MAXF; j++) {
            float a = j < F ? z[j] / sum : 0.f;
            Aout[c * MAXF + j] = a;
            // log(1 - A), with A kept below 1 so a product without c stays finite
            logA1[c * MAXF + j] = log1pf(-fminf(a, 1.f - 1e-6f));
        }
    }
}

// ---------------------------------------------------------------------------
// loss and dLoss/dA over a batch of samples: one warp per sample, lane = field
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_loss_grad(const float *__restrict__ logA1g, int F, float T, float beta,
                                                   const uint64_t *__restrict__ masks,
                                                   const uint8_t *__restrict__ match, int64_t n,
                                                   float *__restrict__ dA, double *__restrict__ loss,
                                                   unsigned long long *__restrict__ n_used) {
    __shared__ float s_l[NSYM * MAXF];
    __shared__ float s_d[NSYM * MAXF];
    __shared__ double s_loss;
    __shared__ unsigned long long s_used;
    for (int t = threadIdx.x; t < NSYM * MAXF; t += blockDim.x) {
        s_l[t] = logA1g[t];
        s_d[t] = 0.f;
    }
    if (threadIdx.x == 0) {
        s_loss = 0.0;
        s_used = 0;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const bool on = lane < F;
    for (int64_t s = warp; s < n; s += nwarps) {
        if (match[s]) continue;  // warp-uniform
        const uint64_t p0 = masks[4 * s], p1 = masks[4 * s + 1], w0 = masks[4 * s + 2], w1 = masks[4 * s + 3];
        // shared symbols I, symbols only in the pattern P', only in the word W'
        const uint64_t i0 = p0 & w0, i1 = p1 & w1, a0 = p0 & ~w0, a1 = p1 & ~w1, b0 = w0 & ~p0, b1 = w1 & ~p1;
        float lI = 0.f, lA = 0.f, lB = 0.f;  // sums of log(1 - A_c,b)
        if (on) {
            for (uint64_t m = i0; m; m &= m - 1) lI += s_l[(__ffsll(m) - 1) * MAXF + lane];
            for (uint64_t m = i1; m; m &= m - 1) lI += s_l[(64 + __ffsll(m) - 1) * MAXF + lane];
            for (uint64_t m = a0; m; m &= m - 1) lA += s_l[(__ffsll(m) - 1) * MAXF + lane];
            for (uint64_t m = a1; m; m &= m - 1) lA += s_l[(64 + __ffsll(m) - 1) * MAXF + lane];
            for (uint64_t m = b0; m; m &= m - 1) lB += s_l[(__ffsll(m) - 1) * MAXF + lane];
            for (uint64_t m = b1; m; m &= m - 1) lB += s_l[(64 + __ffsll(m) - 1) * MAXF + lane];
        }
        const float nI = expf(lI), p = 1.f - expf(lA), q = 1.f - expf(lB);
        const float x = p + q - 2.f * p * q;  // one of P', W' lands on b, the other not
        float f = on ? nI * x : 0.f;           // and no shared symbol does
#pragma unroll
        for (int o = 16; o; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
        const float t = beta * (T - f);
        const float dLdF = -1.f / (1.f + expf(-t));  // -sigmoid(t)
        if (lane == 0) {
            const float sp = t > 20.f ? t : log1pf(expf(t));
            atomicAdd(&s_loss, (double)(sp / beta));
            atomicAdd(&s_used, 1ull);
        }
        if (on) {
            // dF_b/dA_c,b = [c in I] (-nI x) / (1 - A_c,b) + [c in P'] nI (1 - 2q) (1 - p) / (1 - A_c,b)
            //             + [c in W'] nI (1 - 2p) (1 - q) / (1 - A_c,b)
            const float gI = -dLdF * nI * x, gA = dLdF * nI * (1.f - 2.f * q) * (1.f - p),
                        gB = dLdF * nI * (1.f - 2.f * p) * (1.f - q);
            for (uint64_t m = i0; m; m &= m - 1) {
                const int c = __ffsll(m) - 1;
                atomicAdd(&s_d[c * MAXF + lane], gI * __expf(-s_l[c * MAXF + lane]));
            }
            for (uint64_t m = i1; m; m &= m - 1) {
                const int c = 64 + __ffsll(m) - 1;
                atomicAdd(&s_d[c * MAXF + lane], gI * __expf(-s_l[c * MAXF + lane]));
            }
            for (uint64_t m = a0; m; m &= m - 1) {
                const int c = __ffsll(m) - 1;
                atomicAdd(&s_d[c * MAXF + lane], gA * __expf(-s_l[c * MAXF + lane]));
            }
            for (uint64_t m = a1; m; m &= m - 1) {
                const int c = 64 + __ffsll(m) - 1;
                atomicAdd(&s_d[c * MAXF + lane], gA * __expf(-s_l[c * MAXF + lane]));
            }
            for (uint64_t m = b0; m; m &= m - 1) {
                const int c = __ffsll(m) - 1;
                atomicAdd(&s_d[c * MAXF + lane], gB * __expf(-s_l[c * MAXF + lane]));
            }
            for (uint64_t m = b1; m; m &= m - 1) {
                const int c = 64 + __ffsll(m) - 1;
                atomicAdd(&s_d[c * MAXF + lane], gB * __expf(-s_l[c * MAXF + lane]));
            }
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < NSYM * MAXF; t += blockDim.x)
        if (s_d[t] != 0.f) atomicAdd(&dA[t], s_d[t]);
    if (threadIdx.x == 0) {
        atomicAdd(loss, s_loss);
        atomicAdd(n_used, s_used);
    }
}

// ---------------------------------------------------------------------------
// backward through softmax, W2/b2, ReLU, W1/b1 (one block); grads are scaled
// by 1 / (number of non-matching samples)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_mlp_backward(const float *__restrict__ prm, int F, float tau,
                                                      const float *__restrict__ H, const float *__restrict__ Aa,
                                                      const float *__restrict__ dA,
                                                      const unsigned long long *__restrict__ n_used,
                                                      float *__restrict__ grad) {
    __shared__ float dz[NSYM * MAXF];
    __shared__ float dh[NSYM * HID];
    const float scale = *n_used ? 1.f / (float)*n_used : 0.f;
    for (int c = threadIdx.x; c < NSYM; c += blockDim.x) {
        float dot = 0.f;
        for (int j = 0; j < F; j++) dot += Aa[c * MAXF + j] * dA[c * MAXF + j];
        for (int j = 0; j < MAXF; j++)
            dz[c * MAXF + j] = j < F ? scale * Aa[c * MAXF + j] * (dA[c * MAXF + j] - dot) / tau : 0.f;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < NSYM * HID; t += blockDim.x) {
        const int c = t / HID, i = t % HID;
        float acc = 0.f;
        for (int j = 0; j < F; j++) acc += prm[P_W2 + j * HID + i] * dz[c * MAXF + j];
        dh[t] = H[t] > 0.f ? acc : 0.f;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < MAXF * HID; t += blockDim.x) {  // dW2[j][i] = sum_c dz[c][j] h[c][i]
        const int j = t / HID, i = t % HID;
        float acc = 0.f;
        if (j < F)
            for (int c = 0; c < NSYM; c++) acc += dz[c * MAXF + j] * H[c * HID + i];
        grad[P_W2 + t] = acc;
    }
    for (int j = threadIdx.x; j < MAXF; j += blockDim.x) {
        float acc = 0.f;
        for (int c = 0; c < NSYM; c++) acc += dz[c * MAXF + j];
        grad[P_B2 + j] = acc;
    }
    for (int t = threadIdx.x; t < HID * NSYM; t += blockDim.x) {  // dW1[i][c] = dh[c][i]
        const int i = t / NSYM, c = t % NSYM;
        grad[P_W1 + t] = dh[c * HID + i];
    }
    for (int i = threadIdx.x; i < HID; i += blockDim.x) {
        float acc = 0.f;
        for (int c = 0; c < NSYM; c++) acc += dh[c * HID + i];
        grad[P_B1 + i] = acc;
    }
}

__global__ void k_adam(float *__restrict__ prm, const float *__restrict__ grad, float *__restrict__ m1,
                       float *__restrict__ m2, int n, float lr, float b1, float b2, float eps, int step) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = grad[i];
    const float a = b1 * m1[i] + (1.f - b1) * g;
    const float v = b2 * m2[i] + (1.f - b2) * g * g;
    m1[i] = a;
    m2[i] = v;
    const float ah = a / (1.f - powf(b1, (float)step)), vh = v / (1.f - powf(b2, (float)step));
    prm[i] -= lr * ah / (sqrtf(vh) + eps);
}

struct Work {
    float *prm = nullptr, *grad = nullptr, *m1 = nullptr, *m2 = nullptr, *H = nullptr, *A = nullptr,
          *logA1 = nullptr, *dA = nullptr;
    double *loss = nullptr;
    unsigned long long *used = nullptr;
    int alloc(cudaStream_t st) {
        FP_CUDA(cudaMallocAsync((void **)&prm, 4 * NPARAM, st));
        FP_CUDA(cudaMallocAsync((void **)&grad, 4 * NPARAM, st));
        FP_CUDA(cudaMallocAsync((void **)&m1, 4 * NPARAM, st));
        FP_CUDA(cudaMallocAsync((void **)&m2, 4 * NPARAM, st));
        FP_CUDA(cudaMallocAsync((void **)&H, 4 * NSYM * HID, st));
        FP_CUDA(cudaMallocAsync((void **)&A, 4 * NSYM * MAXF, st));
        FP_CUDA(cudaMallocAsync((void **)&logA1, 4 * NSYM * MAXF, st));
        FP_CUDA(cudaMallocAsync((void **)&dA, 4 * NSYM * MAXF, st));
        FP_CUDA(cudaMallocAsync((void **)&loss, 8, st));
        FP_CUDA(cudaMallocAsync((void **)&used, 8, st));
        return FP_OK;
    }
    void release(cudaStream_t st) {
        void *ps[] = {prm, grad, m1, m2, H, A, logA1, dA, loss, used};
        for (void *p : ps)
            if (p) cudaFreeAsync(p, st);
    }
};

// forward, loss/dA over samples [0, n), backward into w.grad
int loss_grad(Work &w, int F, float tau, float T, float beta, const uint64_t *masks, const uint8_t *match, int64_t n,
              cudaStream_t st) {
    k_mlp_forward<<<1, 256, 0, st>>>(w.prm, F, tau, w.H, w.A, w.logA1);
    FP_LAUNCHED("k_mlp_forward");
    FP_CUDA(cudaMemsetAsync(w.dA, 0, 4 * NSYM * MAXF, st));
    FP_CUDA(cudaMemsetAsync(w.loss, 0, 8, st));
    FP_CUDA(cudaMemsetAsync(w.used, 0, 8, st));
    if (n > 0) {
        const int64_t warps = (n + 7) / 8;  // up to 8 samples per warp
        int grid = (int)std::min<int64_t>((warps + 7) / 8, 4 * sm_count());
        if (grid < 1) grid = 1;
        k_loss_grad<<<grid, 256, 0, st>>>(w.logA1, F, T, beta, masks, match, n, w.dA, w.loss, w.used);
        FP_LAUNCHED("k_loss_grad");
    }
    k_mlp_backward<<<1, 256, 0, st>>>(w.prm, F, tau, w.H, w.A, w.dA, w.used, w.grad);
    FP_LAUNCHED("k_mlp_backward");
    return FP_OK;
}

}  // namespace
}  // namespace fpk

using namespace fpk;

extern "C" {

int fp_mlp_param_count(void) { return NPARAM; }

int fp_sample_pairs(fp_index *ix, const uint8_t *chars, const int64_t *offsets, int64_t n_queries, int k,
                    int metric, int64_t n_samples, uint64_t seed, void *cuda_stream, int32_t *out_q, int32_t *out_w,
                    uint8_t *out_passed, uint8_t *out_match, uint64_t *out_masks) {
    if (!ix || !offsets || !out_q || !out_w || !out_passed || !out_match || !out_masks || n_queries < 1 ||
        n_samples < 0 || k < 0 || k > 15 || (metric != FP_HAM && metric != FP_LEV))
        return fail(FP_E_INVAL, "fp_sample_pairs: bad argument");
    if (metric == FP_LEV && (ix->P.type == FP_OCC_HALVED || ix->P.type == FP_POS))
        return fail(FP_E_UNSUPPORTED, "occurrence-halved and position fingerprints bound only the Hamming distance");
    if (ix->P.type == FP_QGRAM || ix->P.type == FP_COUNT_L1)
        return fail(FP_E_UNSUPPORTED, "pair sampling: symbol fingerprints compared by their Hamming weight only");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int64_t total = 0;
    int64_t *d_off = nullptr;
    uint8_t *d_chars = nullptr;
    const bool dev = is_device_ptr(offsets);
    if (dev) {
        FP_CUDA(cudaMemcpy(&total, offsets + n_queries, 8, cudaMemcpyDeviceToHost));
    } else {
        FP_TRY(check_host_offsets(offsets, n_queries));
        total = offsets[n_queries];
    }
    FP_CUDA(cudaMallocAsync((void **)&d_off, 8 * (size_t)(n_queries + 1), st));
    FP_CUDA(cudaMallocAsync((void **)&d_chars, (size_t)total + 16, st));
    FP_CUDA(cudaMemcpyAsync(d_off, offsets, 8 * (size_t)(n_queries + 1), cudaMemcpyDefault, st));
    if (total) FP_CUDA(cudaMemcpyAsync(d_chars, chars, (size_t)total, cudaMemcpyDefault, st));
    int32_t *d_err = nullptr;
    FP_CUDA(cudaMallocAsync((void **)&d_err, 4, st));
    FP_CUDA(cudaMemsetAsync(d_err, 0, 4, st));
    SampleArgs A{};
    int rc = bucketize(d_chars, d_off, n_queries, total, nullptr, 1, ix->d_map, ix->P, true, st, &A.Q, d_err);
    if (rc != FP_OK) return rc;
    A.D = ix->D;
    A.P = ix->P;
    A.k = k;
    A.metric = metric;
    A.seed = seed;
    A.n = n_samples;
    const bool dev_out = is_device_ptr(out_q);
    std::vector<void *> tmp;
    auto place = [&](void *user, size_t bytes) -> void * {
        if (dev_out) return user;
        void *p = nullptr;
        if (cudaMallocAsync(&p, bytes ? bytes : 16, st) != cudaSuccess) return nullptr;
        tmp.push_back(p);
        return p;
    };
    A.out_q = (int32_t *)place(out_q, 4 * (size_t)n_samples);
    A.out_w = (int32_t *)place(out_w, 4 * (size_t)n_samples);
    A.out_passed = (uint8_t *)place(out_passed, (size_t)n_samples);
    A.out_match = (uint8_t *)place(out_match, (size_t)n_samples);
    A.out_masks = (uint64_t *)place(out_masks, 32 * (size_t)n_samples);
    if (!A.out_q || !A.out_w || !A.out_passed || !A.out_match || !A.out_masks) rc = FP_E_NOMEM;
    if (rc == FP_OK && n_samples > 0) {
        int grid = (int)std::min<int64_t>((n_samples + 255) / 256, 8 * sm_count());
        k_sample_pairs<<<grid, 256, 0, st>>>(A);
        g_launches++;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_fail(e, "k_sample_pairs");
    }
    if (rc == FP_OK && !dev_out) {
        cudaMemcpyAsync(out_q, A.out_q, 4 * (size_t)n_samples, cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(out_w, A.out_w, 4 * (size_t)n_samples, cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(out_passed, A.out_passed, (size_t)n_samples, cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(out_match, A.out_match, (size_t)n_samples, cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(out_masks, A.out_masks, 32 * (size_t)n_samples, cudaMemcpyDeviceToHost, st);
    }
    for (void *p : tmp) cudaFreeAsync(p, st);
    free_bucketed(&A.Q, st);
    cudaFreeAsync(d_off, st);
    cudaFreeAsync(d_chars, st);
    cudaFreeAsync(d_err, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (rc == FP_OK && e != cudaSuccess) rc = cuda_fail(e, "fp_sample_pairs");
    return rc;
}

int fp_mlp_loss_grad(const float *params, int fields, float tau, float beta, int k, const uint64_t *masks,
                     const uint8_t *match, int64_t n_samples, void *cuda_stream, double *loss_sum,
                     int64_t *n_used, float *grad) {
    if (!params || !masks || !match || !grad || fields < 1 || fields > MAXF || tau <= 0.f || beta <= 0.f || k < 0 ||
        n_samples < 0)
        return fail(FP_E_INVAL, "fp_mlp_loss_grad: bad argument");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    Work w;
    FP_TRY(w.alloc(st));
    FP_CUDA(cudaMemcpyAsync(w.prm, params, 4 * NPARAM, cudaMemcpyDefault, st));
    int rc = loss_grad(w, fields, tau, 2.f * k + 1.f, beta, masks, match, n_samples, st);
    unsigned long long used = 0;
    if (rc == FP_OK) {
        cudaMemcpyAsync(grad, w.grad, 4 * NPARAM, cudaMemcpyDefault, st);
        cudaMemcpyAsync(loss_sum, w.loss, 8, cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(&used, w.used, 8, cudaMemcpyDeviceToHost, st);
    }
    w.release(st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (rc == FP_OK && e != cudaSuccess) rc = cuda_fail(e, "fp_mlp_loss_grad");
    if (n_used) *n_used = (int64_t)used;
    return rc;
}

int fp_learn_map(int fields, const uint64_t *masks, const uint8_t *match, int64_t n_samples, int k,
                 const fp_learn_opts *opts, void *cuda_stream, float *params_out, int8_t *map_out,
                 float *loss_curve) {
    if (!masks || !match || !map_out || fields < 1 || fields > MAXF || n_samples < 1 || k < 0)
        return fail(FP_E_INVAL, "fp_learn_map: bad argument");
    fp_learn_opts o{};
    if (opts) o = *opts;
    if (o.epochs <= 0) o.epochs = 12;
    if (o.batch <= 0) o.batch = 65536;
    if (o.lr <= 0.f) o.lr = 3e-3f;
    if (o.tau0 <= 0.f) o.tau0 = 1.0f;
    if (o.tau1 <= 0.f) o.tau1 = 0.1f;
    if (o.beta <= 0.f) o.beta = 2.0f;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // masks / match may be host or device; training reads them from the device
    const bool dev = is_device_ptr(masks);
    uint64_t *d_masks = (uint64_t *)masks;
    uint8_t *d_match = (uint8_t *)match;
    if (!dev) {
        FP_CUDA(cudaMallocAsync((void **)&d_masks, 32 * (size_t)n_samples, st));
        FP_CUDA(cudaMallocAsync((void **)&d_match, (size_t)n_samples, st));
        FP_CUDA(cudaMemcpyAsync(d_masks, masks, 32 * (size_t)n_samples, cudaMemcpyHostToDevice, st));
        FP_CUDA(cudaMemcpyAsync(d_match, match, (size_t)n_samples, cudaMemcpyHostToDevice, st));
    }
    Work w;
    FP_TRY(w.alloc(st));
    // seeded initialisation (SplitMix64 uniforms): W ~ U(-1/sqrt(fan_in), +), b = 0
    std::vector<float> h(NPARAM, 0.f);
    uint64_t state = o.seed ? o.seed : 1711;
    auto uni = [&]() {
        state += 0x9E3779B97F4A7C15ull;
        uint64_t z = state;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return (float)((z >> 11) * (1.0 / 9007199254740992.0)) * 2.f - 1.f;
    };
    for (int i = 0; i < HID * NSYM; i++) h[P_W1 + i] = uni() * 1.0f;  // fan_in 1 (one-hot input)
    for (int i = 0; i < MAXF * HID; i++) h[P_W2 + i] = uni() * (1.0f / sqrtf((float)HID));
    if (o.init_params)  // the caller's starting point instead (host or device)
        FP_CUDA(cudaMemcpyAsync(w.prm, o.init_params, 4 * NPARAM, cudaMemcpyDefault, st));
    else
        FP_CUDA(cudaMemcpyAsync(w.prm, h.data(), 4 * NPARAM, cudaMemcpyHostToDevice, st));
    FP_CUDA(cudaMemsetAsync(w.m1, 0, 4 * NPARAM, st));
    FP_CUDA(cudaMemsetAsync(w.m2, 0, 4 * NPARAM, st));
    int rc = FP_OK;
    int step = 0;
    const float T = 2.f * k + 1.f;
    for (int ep = 0; ep < o.epochs && rc == FP_OK; ep++) {
        const float tau = o.epochs > 1 ? o.tau0 * powf(o.tau1 / o.tau0, (float)ep / (float)(o.epochs - 1)) : o.tau1;
        double ep_loss = 0.0;
        int64_t ep_used = 0;
        for (int64_t b0 = 0; b0 < n_samples && rc == FP_OK; b0 += o.batch) {
            const int64_t nb = std::min<int64_t>(o.batch, n_samples - b0);
            rc = loss_grad(w, fields, tau, T, o.beta, d_masks + 4 * b0, d_match + b0, nb, st);
            if (rc != FP_OK) break;
            step++;
            k_adam<<<(NPARAM + 255) / 256, 256, 0, st>>>(w.prm, w.grad, w.m1, w.m2, NPARAM, o.lr, 0.9f, 0.999f, 1e-8f,
                                                         step);
            g_launches++;
            if (loss_curve) {
                double l = 0;
                unsigned long long u = 0;
                cudaMemcpyAsync(&l, w.loss, 8, cudaMemcpyDeviceToHost, st);
                cudaMemcpyAsync(&u, w.used, 8, cudaMemcpyDeviceToHost, st);
                cudaStreamSynchronize(st);
                ep_loss += l;
                ep_used += (int64_t)u;
            }
        }
        if (loss_curve) loss_curve[ep] = ep_used ? (float)(ep_loss / (double)ep_used) : 0.f;
    }
    if (rc == FP_OK) {
        // hard map: argmax field per symbol at the final temperature
        k_mlp_forward<<<1, 256, 0, st>>>(w.prm, fields, o.tau1, w.H, w.A, w.logA1);
        g_launches++;
        std::vector<float> a(NSYM * MAXF);
        cudaMemcpyAsync(a.data(), w.A, 4 * NSYM * MAXF, cudaMemcpyDeviceToHost, st);
        if (params_out) cudaMemcpyAsync(params_out, w.prm, 4 * NPARAM, cudaMemcpyDefault, st);
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = cuda_fail(e, "fp_learn_map");
        for (int c = 0; c < 256; c++) map_out[c] = -1;
        for (int c = 0; c < NSYM && rc == FP_OK; c++) {
            int best = 0;
            for (int j = 1; j < fields; j++)
                if (a[c * MAXF + j] > a[c * MAXF + best]) best = j;
            map_out[0x20 + c] = (int8_t)best;
        }
    }
    w.release(st);
    if (!dev) {
        cudaFreeAsync(d_masks, st);
        cudaFreeAsync(d_match, st);
    }
    cudaStreamSynchronize(st);
    return rc;
}

}  // extern "C"
