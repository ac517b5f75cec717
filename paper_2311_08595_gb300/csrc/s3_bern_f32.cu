// FP32 instantiation of the Bernoulli-series kernels (unbiased output modes).
#include "s3_bern.cuh"

namespace s3 {

cudaError_t launch_edge_bern_f32(const TailEntry *tab, int ntab, int64_t nblocks, int lane_elems, int fb_elems,
                                 const float *x, const EdgeOutArgs &o, const BernArgs &c, cudaStream_t st) {
    if (o.bias) return launch_edge_bern_f32_bias(tab, ntab, nblocks, lane_elems, fb_elems, x, o, c, st);
    return launch_edge_bern_t<float, false>(tab, ntab, nblocks, lane_elems, fb_elems, x, o, c, st);
}

cudaError_t prepare_edge_bern_f32() {
    cudaError_t e = prepare_edge_bern_t<float, false>();
    return e == cudaSuccess ? prepare_edge_bern_f32_bias() : e;
}

}  // namespace s3
