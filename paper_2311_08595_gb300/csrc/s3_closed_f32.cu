// float instantiations of the closed-form small-edge kernels.
#include "s3_closed.cuh"

namespace s3 {

cudaError_t launch_edge_closed_f32(const EdgeBucketArgs &b, const float *x, const EdgeOutArgs &o,
                                   const ClosedArgs &c, cudaStream_t st) {
    return launch_edge_closed_t<float>(b, x, o, c, st);
}

}  // namespace s3
