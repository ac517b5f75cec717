// Double-float (pairs of FP32) series kernels: declarations shared by their translation units.
#pragma once

#include "s3_series.cuh"

namespace s3 {

// Windows handled with double-float arithmetic; wider ones (and size-1 edges) use FP64.
constexpr int kDfMaxW = 24;

// Launch the thread-per-edge (pair = false) or size-2 (pair = true) kernel of window W if
// it is in the unit's range (*handled = 1), else do nothing (*handled = 0).
cudaError_t launch_df_range1(const EdgeBucketArgs &b, const double *x, const EdgeOutArgs &o, int W, int bs, bool pair,
                              cudaStream_t st, int *handled);
cudaError_t prepare_df_range1();
cudaError_t launch_df_range2(const EdgeBucketArgs &b, const double *x, const EdgeOutArgs &o, int W, int bs, bool pair,
                              cudaStream_t st, int *handled);
cudaError_t prepare_df_range2();
cudaError_t launch_df_range3(const EdgeBucketArgs &b, const double *x, const EdgeOutArgs &o, int W, int bs, bool pair,
                              cudaStream_t st, int *handled);
cudaError_t prepare_df_range3();
cudaError_t launch_df_range4(const EdgeBucketArgs &b, const double *x, const EdgeOutArgs &o, int W, int bs, bool pair,
                              cudaStream_t st, int *handled);
cudaError_t prepare_df_range4();

}  // namespace s3
