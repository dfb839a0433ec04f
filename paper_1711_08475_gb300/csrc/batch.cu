// Batched queries: many pattern batches, each with its own k and metric,
// answered by one pass of the pipeline (the paper is
// single-query, Sec. 4).  Batches that share (k, metric) form one group;
// patterns are bucketed by (group, length), so every tile of the fused
// filter + verify kernel has one k and one metric.
#include "common.cuh"

namespace fpk {

// group[i] for every pattern i of batch b (batches are consecutive ranges).
__global__ void k_fill_groups(const int64_t *__restrict__ batch_start, const int32_t *__restrict__ batch_group,
                              int32_t *__restrict__ group) {
    const int b = blockIdx.x;
    const int64_t lo = batch_start[b], hi = batch_start[b + 1];
    const int32_t g = batch_group[b];
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) group[i] = g;
}

int fill_groups(const int64_t *d_batch_start, const int32_t *d_batch_group, int n_batches, int32_t *d_group,
                cudaStream_t st) {
    if (n_batches <= 0) return FP_OK;
    k_fill_groups<<<n_batches, 256, 0, st>>>(d_batch_start, d_batch_group, d_group);
    FP_LAUNCHED("k_fill_groups");
    return FP_OK;
}

}  // namespace fpk
