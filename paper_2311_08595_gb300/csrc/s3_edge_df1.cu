// Double-float series kernels for windows W = 1..10 (one translation unit per range
// of W, compiled in parallel).
#include "s3_edge_df.h"

namespace s3 {

cudaError_t launch_df_range1(const EdgeBucketArgs &b, const double *x, const EdgeOutArgs &o, int W, int bs, bool pair,
                              cudaStream_t st, int *handled) {
    *handled = 1;
    switch (W) {
        case 1: return pair ? launch_pair_w<DF, 1>(b, x, o, st) : launch_thread_w<DF, 1>(b, x, o, bs, st);
        case 2: return pair ? launch_pair_w<DF, 2>(b, x, o, st) : launch_thread_w<DF, 2>(b, x, o, bs, st);
        case 3: return pair ? launch_pair_w<DF, 3>(b, x, o, st) : launch_thread_w<DF, 3>(b, x, o, bs, st);
        case 4: return pair ? launch_pair_w<DF, 4>(b, x, o, st) : launch_thread_w<DF, 4>(b, x, o, bs, st);
        case 5: return pair ? launch_pair_w<DF, 5>(b, x, o, st) : launch_thread_w<DF, 5>(b, x, o, bs, st);
        case 6: return pair ? launch_pair_w<DF, 6>(b, x, o, st) : launch_thread_w<DF, 6>(b, x, o, bs, st);
        case 7: return pair ? launch_pair_w<DF, 7>(b, x, o, st) : launch_thread_w<DF, 7>(b, x, o, bs, st);
        case 8: return pair ? launch_pair_w<DF, 8>(b, x, o, st) : launch_thread_w<DF, 8>(b, x, o, bs, st);
        case 9: return pair ? launch_pair_w<DF, 9>(b, x, o, st) : launch_thread_w<DF, 9>(b, x, o, bs, st);
        case 10: return pair ? launch_pair_w<DF, 10>(b, x, o, st) : launch_thread_w<DF, 10>(b, x, o, bs, st);
        default: break;
    }
    *handled = 0;
    return cudaSuccess;
}

cudaError_t prepare_df_range1() {
    cudaError_t err = cudaSuccess;
    if (err == cudaSuccess) err = prepare_thread_w<DF, 1>();
    if (err == cudaSuccess) err = prepare_thread_w<DF, 2>();
    if (err == cudaSuccess) err = prepare_thread_w<DF, 3>();
    if (err == cudaSuccess) err = prepare_thread_w<DF, 4>();
    if (err == cudaSuccess) err = prepare_thread_w<DF, 5>();
    if (err == cudaSuccess) err = prepare_thread_w<DF, 6>();
    if (err == cudaSuccess) err = prepare_thread_w<DF, 7>();
    if (err == cudaSuccess) err = prepare_thread_w<DF, 8>();
    if (err == cudaSuccess) err = prepare_thread_w<DF, 9>();
    if (err == cudaSuccess) err = prepare_thread_w<DF, 10>();
    return err;
}

}  // namespace s3
