// Double-float series kernels for windows W = 21..24 (one translation unit per range
// of W, compiled in parallel).
#include "s3_edge_df.h"

namespace s3 {

cudaError_t launch_df_range4(const EdgeBucketArgs &b, const double *x, const EdgeOutArgs &o, int W, int bs, bool pair,
                              cudaStream_t st, int *handled) {
    *handled = 1;
    switch (W) {
        case 21: return pair ? launch_pair_w<DF, 21>(b, x, o, st) : launch_thread_w<DF, 21>(b, x, o, bs, st);
        case 22: return pair ? launch_pair_w<DF, 22>(b, x, o, st) : launch_thread_w<DF, 22>(b, x, o, bs, st);
        case 23: return pair ? launch_pair_w<DF, 23>(b, x, o, st) : launch_thread_w<DF, 23>(b, x, o, bs, st);
        case 24: return pair ? launch_pair_w<DF, 24>(b, x, o, st) : launch_thread_w<DF, 24>(b, x, o, bs, st);
        default: break;
    }
    *handled = 0;
    return cudaSuccess;
}

cudaError_t prepare_df_range4() {
    cudaError_t err = cudaSuccess;
    if (err == cudaSuccess) err = prepare_thread_w<DF, 21>();
    if (err == cudaSuccess) err = prepare_thread_w<DF, 22>();
    if (err == cudaSuccess) err = prepare_thread_w<DF, 23>();
    if (err == cudaSuccess) err = prepare_thread_w<DF, 24>();
    return err;
}

}  // namespace s3
