// FP32 instantiation of the Bernoulli-series kernels (the biased output mode of NQZ).
#include "s3_bern.cuh"

namespace s3 {

cudaError_t launch_edge_bern_f32_bias(const TailEntry *tab, int ntab, int64_t nblocks, int lane_elems, int fb_elems,
                                      const float *x, const EdgeOutArgs &o, const BernArgs &c, cudaStream_t st) {
    return launch_edge_bern_t<float, true>(tab, ntab, nblocks, lane_elems, fb_elems, x, o, c, st);
}

cudaError_t prepare_edge_bern_f32_bias() { return prepare_edge_bern_t<float, true>(); }

}  // namespace s3
