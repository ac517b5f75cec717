// FP32 instantiations of the per-edge series kernels.
#include "s3_series.cuh"

namespace s3 {

cudaError_t launch_edge_bucket_f32(const EdgeBucketArgs &b, const float *x, const EdgeOutArgs &o,
                                   int thread_max_w, int block_threads, cudaStream_t st) {
    return launch_edge_bucket_t<float>(b, x, o, thread_max_w, block_threads, st);
}

cudaError_t launch_edge_tail_f32(const TailEntry *tab, int ntab, int64_t nblocks, int bs, size_t smem,
                                 const float *x, const EdgeOutArgs &o, cudaStream_t st) {
    return launch_edge_tail_t<float>(tab, ntab, nblocks, bs, smem, x, o, st);
}

cudaError_t prepare_edge_kernels_f32() { return prepare_edge_kernels_t<float>(); }

}  // namespace s3
