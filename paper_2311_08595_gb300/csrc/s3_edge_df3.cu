// Double-float series kernels for windows W = 17..20 (one translation unit per range
// of W, compiled in parallel).
#include "s3_edge_df.h"

namespace s3 {

cudaError_t launch_df_range3(const EdgeBucketArgs &b, const double *x, const EdgeOutArgs &o, int W, int bs, bool pair,
                              cudaStream_t st, int *handled) {
    *handled = 1;
    switch (W) {
        case 17: return pair ? launch_pair_w<DF, 17>(b, x, o, st) : launch_thread_w<DF, 17>(b, x, o, bs, st);
        case 18: return pair ? launch_pair_w<DF, 18>(b, x, o, st) : launch_thread_w<DF, 18>(b, x, o, bs, st);
        case 19: return pair ? launch_pair_w<DF, 19>(b, x, o, st) : launch_thread_w<DF, 19>(b, x, o, bs, st);
        case 20: return pair ? launch_pair_w<DF, 20>(b, x, o, st) : launch_thread_w<DF, 20>(b, x, o, bs, st);
        default: break;
    }
    *handled = 0;
    return cudaSuccess;
}

cudaError_t prepare_df_range3() {
    cudaError_t err = cudaSuccess;
    if (err == cudaSuccess) err = prepare_thread_w<DF, 17>();
    if (err == cudaSuccess) err = prepare_thread_w<DF, 18>();
    if (err == cudaSuccess) err = prepare_thread_w<DF, 19>();
    if (err == cudaSuccess) err = prepare_thread_w<DF, 20>();
    return err;
}

}  // namespace s3
