// Double-float S^3TTVc (S3_DF64): FP64 x and results, series arithmetic in pairs of
// FP32 numbers (struct DF in s3_series.cuh).  Buckets of size 1, buckets whose window
// is wider than kDfMaxW or than a thread's shared-memory share, run the FP64 kernels.
#include "s3_edge_df.h"

namespace s3 {

cudaError_t launch_edge_bucket_df(const EdgeBucketArgs &b, const double *x, const EdgeOutArgs &o, int thread_max_w,
                                  int block_threads, cudaStream_t st) {
    if (b.m <= 0) return cudaSuccess;
    const int W = b.N - b.s + 1;
    const int tmw = (thread_max_w <= 0 || thread_max_w > kMaxThreadW) ? kMaxThreadW : thread_max_w;
    const bool pair = b.s == 2;
    const int bs = thread_block_size<DF>(b.s, W, block_threads <= 0 ? 128 : block_threads);
    if (b.s == 1 || W > tmw || W > kDfMaxW || (!pair && bs == 0))
        return launch_edge_bucket_f64(b, x, o, thread_max_w, block_threads, st);
    int handled = 0;
    cudaError_t e = launch_df_range1(b, x, o, W, bs, pair, st, &handled);
    if (!handled) e = launch_df_range2(b, x, o, W, bs, pair, st, &handled);
    if (!handled) e = launch_df_range3(b, x, o, W, bs, pair, st, &handled);
    if (!handled) e = launch_df_range4(b, x, o, W, bs, pair, st, &handled);
    if (!handled) return launch_edge_bucket_f64(b, x, o, thread_max_w, block_threads, st);
    return e;
}

cudaError_t prepare_edge_kernels_df() {
    cudaError_t err = prepare_df_range1();
    if (err == cudaSuccess) err = prepare_df_range2();
    if (err == cudaSuccess) err = prepare_df_range3();
    if (err == cudaSuccess) err = prepare_df_range4();
    return err;
}

}  // namespace s3
