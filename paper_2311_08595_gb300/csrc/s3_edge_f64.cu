// FP64 instantiations of the per-edge series kernels.
#include "s3_series.cuh"

namespace s3 {

cudaError_t launch_edge_bucket_f64(const EdgeBucketArgs &b, const double *x, const EdgeOutArgs &o,
                                   int thread_max_w, int block_threads, cudaStream_t st) {
    return launch_edge_bucket_t<double>(b, x, o, thread_max_w, block_threads, st);
}

cudaError_t launch_edge_tail_f64(const TailEntry *tab, int ntab, int64_t nblocks, int bs, size_t smem,
                                 const double *x, const EdgeOutArgs &o, cudaStream_t st) {
    return launch_edge_tail_t<double>(tab, ntab, nblocks, bs, smem, x, o, st);
}

cudaError_t prepare_edge_kernels_f64() { return prepare_edge_kernels_t<double>(); }

}  // namespace s3
