// Double-float series kernels for windows W = 11..16 (one translation unit per range
// of W, compiled in parallel).
#include "s3_edge_df.h"

namespace s3 {

cudaError_t launch_df_range2(const EdgeBucketArgs &b, const double *x, const EdgeOutArgs &o, int W, int bs, bool pair,
                              cudaStream_t st, int *handled) {
    *handled = 1;
    switch (W) {
        case 11: return pair ? launch_pair_w<DF, 11>(b, x, o, st) : launch_thread_w<DF, 11>(b, x, o, bs, st);
        case 12: return pair ? launch_pair_w<DF, 12>(b, x, o, st) : launch_thread_w<DF, 12>(b, x, o, bs, st);
        case 13: return pair ? launch_pair_w<DF, 13>(b, x, o, st) : launch_thread_w<DF, 13>(b, x, o, bs, st);
        case 14: return pair ? launch_pair_w<DF, 14>(b, x, o, st) : launch_thread_w<DF, 14>(b, x, o, bs, st);
        case 15: return pair ? launch_pair_w<DF, 15>(b, x, o, st) : launch_thread_w<DF, 15>(b, x, o, bs, st);
        case 16: return pair ? launch_pair_w<DF, 16>(b, x, o, st) : launch_thread_w<DF, 16>(b, x, o, bs, st);
        default: break;
    }
    *handled = 0;
    return cudaSuccess;
}

cudaError_t prepare_df_range2() {
    cudaError_t err = cudaSuccess;
    if (err == cudaSuccess) err = prepare_thread_w<DF, 11>();
    if (err == cudaSuccess) err = prepare_thread_w<DF, 12>();
    if (err == cudaSuccess) err = prepare_thread_w<DF, 13>();
    if (err == cudaSuccess) err = prepare_thread_w<DF, 14>();
    if (err == cudaSuccess) err = prepare_thread_w<DF, 15>();
    if (err == cudaSuccess) err = prepare_thread_w<DF, 16>();
    return err;
}

}  // namespace s3
