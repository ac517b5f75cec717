// Batched S^3TTVc kernels, double instantiation.
#include "s3_batch_kernels.cuh"

namespace s3 {

s3_status record_batch_f64(s3_batch_s *bt, cudaStream_t st) { return batch_detail::record_batch_t<double>(bt, st); }

cudaError_t prepare_batch_f64() {
    return cudaFuncSetAttribute(batch_detail::batch_edge_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                200 * 1024);
}

}  // namespace s3
