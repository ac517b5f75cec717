// FMA-chain throughput probe: the FP32 and FP64 multiply-add rates of the device,
// the denominators of the ALU rooflines of the series kernels (which are bound by
// multiply-add issue, not by memory).
//
// Every thread runs kChains independent chains v <- v * a + b (a, b runtime values,
// so nothing folds), enough independent work per warp to hide the FMA latency; the
// grid fills every SM with 2048 threads.  One FMA counts as two flops.
#include <cuda_runtime.h>

#include "s3_graph.h"

namespace s3 {
namespace {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kPeakThreads) fma_chain_kernel(T *out, int iters, T a, T b) {
    T v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = T(threadIdx.x) * T(1e-3) + T(c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) v[c] = fma(v[c], a, b);
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += v[c];
    // a value the chains never produce for |a| < 1: keeps the stores (and so the chains) alive
    if (s == T(-12345.0)) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
s3_status run_peak(int32_t reps, s3_peak_result *res, cudaStream_t st) {
    int dev = 0, sms = 0, clk = 0;
    S3_CUDA(cudaGetDevice(&dev));
    S3_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev) != cudaSuccess) {
        cudaGetLastError();
        clk = 0;
    }
    int per_sm = 0;
    S3_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_chain_kernel<T>, kPeakThreads, 0));
    if (per_sm <= 0) per_sm = 1;
    const int blocks = sms * per_sm;
    // about 1 ms of FP32 work per launch; FP64 units are far fewer on this device class
    const int iters = sizeof(T) == 4 ? 8192 : 256;
    T *out = nullptr;  // never written for these inputs; a 1-element guard is still valid memory
    S3_CUDA(cudaMallocAsync((void **)&out, sizeof(T) * (size_t)blocks * kPeakThreads, st));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    S3_CUDA(cudaEventCreate(&e0));
    S3_CUDA(cudaEventCreate(&e1));
    const T a = T(0.999999), b = T(1e-7);
    fma_chain_kernel<T><<<blocks, kPeakThreads, 0, st>>>(out, iters, a, b);  // warm-up
    cudaError_t err = cudaGetLastError();
    float best = 0.f;
    for (int r = 0; r < reps && err == cudaSuccess; ++r) {
        cudaEventRecord(e0, st);
        fma_chain_kernel<T><<<blocks, kPeakThreads, 0, st>>>(out, iters, a, b);
        cudaEventRecord(e1, st);
        err = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
        if (err == cudaSuccess && (best == 0.f || ms < best)) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(out, st);
    if (err != cudaSuccess) return cuda_fail(err, "FMA probe");
    const double flops = 2.0 * kChains * (double)iters * (double)blocks * kPeakThreads;
    res->flops_per_launch = flops;
    res->ms = best;
    res->tflops = flops / ((double)best * 1e-3) / 1e12;
    res->sm_count = sms;
    res->threads_per_sm = per_sm * kPeakThreads;
    res->clock_mhz = clk / 1000;
    return S3_OK;
}

}  // namespace
}  // namespace s3

using namespace s3;

extern "C" s3_status s3_fma_peak(s3_dtype dt, int32_t reps, s3_peak_result *res, void *stream) {
    if (!res) return fail(S3_EINVAL, "res is NULL");
    if (dt != S3_F32 && dt != S3_F64) return fail(S3_EINVAL, "dtype must be S3_F32 or S3_F64");
    if (reps < 1 || reps > 10000) return fail(S3_EINVAL, "reps must be in 1..10000");
    *res = s3_peak_result{};
    cudaStream_t st = (cudaStream_t)stream;
    return dt == S3_F32 ? run_peak<float>(reps, res, st) : run_peak<double>(reps, res, st);
}
