// double instantiations of the closed-form small-edge kernels.
#include "s3_closed.cuh"

namespace s3 {

cudaError_t launch_edge_closed_f64(const EdgeBucketArgs &b, const double *x, const EdgeOutArgs &o,
                                   const ClosedArgs &c, cudaStream_t st) {
    return launch_edge_closed_t<double>(b, x, o, c, st);
}

}  // namespace s3
