// Wide-window kernels (eight lanes per edge) for FP32.  FP64 buckets with wide
// windows keep the one-warp-per-edge kernel: at FP64 the lanes' register
// windows and the per-edge shared memory double, and the group kernel measured
// slower there.
#include "s3_group.cuh"

namespace s3 {

cudaError_t launch_edge_group(const EdgeBucketArgs &b, const float *x, const EdgeOutArgs &o, int W, cudaStream_t st,
                              int *launched) {
    return launch_group_t<float>(b, x, o, W, st, launched);
}

cudaError_t launch_edge_group(const EdgeBucketArgs &, const double *, const EdgeOutArgs &, int, cudaStream_t,
                              int *launched) {
    *launched = 0;
    return cudaSuccess;
}

cudaError_t prepare_edge_group(float) { return prepare_group_t<float>(); }
cudaError_t prepare_edge_group(double) { return cudaSuccess; }

}  // namespace s3
