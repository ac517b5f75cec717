// S^3TTVc for callers that must not allocate device memory.
//
// Who needs this: code that runs where cudaMalloc is not allowed or not
// wanted -- for example a real-time or embedded pipeline that fixes all of its
// memory up front, a runtime whose own allocator owns every byte of the
// device, or a latency-critical loop that must not risk an allocation's
// implicit device synchronisation.  Such callers cannot build a graph
// handle (s3_build_format allocates) and cannot hand the library a workspace.
//
// s3_sttsvc_f32_noalloc therefore takes the hypergraph directly as device CSR
// arrays plus x and y, and keeps its only scratch -- the FP32 two-sum
// compensation term of every node -- in a fixed array that lives in this file
// (`g_comp`, S3_NOALLOC_MAX_NODES floats).  The CUDA module holds that array
// on every GPU that loads the library until the process exits.  The kernel
// runs the warp-per-edge series of the handle-based path on each edge's CSR
// slice and adds its results with atomics plus compensation.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "s3_graph.h"
#include "s3_series.cuh"

namespace s3 {
namespace {

// Scratch: one compensation float per node, shared by every call on a device.
static __device__ __align__(256) float g_comp[S3_NOALLOC_MAX_NODES];

struct NoallocTables {
    double K[S3_MAX_RANK + 1];      // K(s,N), s = 1..N
    float Km[S3_MAX_RANK + 1];      // K = Km 2^Ke
    int32_t Ke[S3_MAX_RANK + 1];
    float target[S3_MAX_RANK + 1];  // rescaling target T(s,N)
};

// Fill the per-size constants without touching the heap: R(n,k) = k! S(n,k)/n!
// obeys R(n,k) = (k/n)(R(n-1,k) + R(n-1,k-1)); K(s,N) = s/(N R(N,s)), and the
// rescaling target uses R(N-1,s) exactly as the handle-based path does.
void fill_tables(int N, NoallocTables &t) {
    double R[S3_MAX_RANK + 2], Rprev[S3_MAX_RANK + 2];
    for (int k = 0; k <= S3_MAX_RANK + 1; ++k) Rprev[k] = 0.0;
    Rprev[0] = 1.0;
    double RNm1[S3_MAX_RANK + 2];
    for (int k = 0; k <= S3_MAX_RANK + 1; ++k) RNm1[k] = N == 1 ? Rprev[k] : 0.0;
    for (int n = 1; n <= N; ++n) {
        R[0] = 0.0;
        for (int k = 1; k <= n; ++k) R[k] = (double)k / (double)n * (Rprev[k] + Rprev[k - 1]);
        for (int k = n + 1; k <= S3_MAX_RANK + 1; ++k) R[k] = 0.0;
        for (int k = 0; k <= S3_MAX_RANK + 1; ++k) Rprev[k] = R[k];
        if (n == N - 1)
            for (int k = 0; k <= S3_MAX_RANK + 1; ++k) RNm1[k] = R[k];
    }
    for (int s = 0; s <= S3_MAX_RANK; ++s) {
        t.K[s] = 0.0;
        t.Km[s] = 0.f;
        t.Ke[s] = 0;
        t.target[s] = 1.f;
    }
    for (int s = 1; s <= N; ++s) {
        double K = (double)s / ((double)N * Rprev[s]);
        int e = 0;
        double m = std::frexp(K, &e);
        t.K[s] = K;
        t.Km[s] = (float)m;
        t.Ke[s] = e;
        if (N <= 1) t.target[s] = 1.f;
        else if (s >= N || !(RNm1[s] > 0.0)) t.target[s] = (float)s;
        else t.target[s] = (float)(std::pow(1.0 / RNm1[s], 1.0 / (double)(N - 1)) * s);
    }
}

// One warp per edge over CSR input; results added to y with atomics and the
// rounding error of each addition added to comp (both zeroed by the caller).
// Edges of size >= 2 run the warp-per-edge series of the handle-based path
// (warp_edge_compute) with the edge's CSR slice as a one-edge bucket.
__global__ void __launch_bounds__(128) noalloc_edge_kernel(int64_t n, int64_t m, int32_t N,
                                                           const int64_t *__restrict__ edge_ptr,
                                                           const int32_t *__restrict__ members,
                                                           const float *__restrict__ x, float *__restrict__ y,
                                                           float *__restrict__ comp, int64_t per_warp,
                                                           NoallocTables tab) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    float *base = reinterpret_cast<float *>(smem_raw) + (int64_t)wib * per_warp;
    EdgeOutArgs o{};
    o.out = y;
    o.comp = comp;
    o.mode = kOutAtomicComp;
    for (int64_t e = (int64_t)blockIdx.x * wpb + wib; e < m; e += (int64_t)gridDim.x * wpb) {
        const int64_t e0 = edge_ptr[e];
        const int64_t len = edge_ptr[e + 1] - e0;
        // malformed edges (size outside 1..N, or an id outside [0, n)) are skipped
        if (len < 1 || len > N) continue;
        const int s = (int)len;
        bool ok = true;
        for (int i = lane; i < s; i += 32) {
            int v = __ldg(members + e0 + i);
            if (v < 0 || v >= n) ok = false;
        }
        if (!__all_sync(0xffffffffu, ok)) continue;
        EdgeBucketArgs b{};
        b.ids = members + e0;   // member i at ids[i * ld + 0]
        b.m = 1;
        b.ld = 1;
        b.s = s;
        b.N = N;
        b.target = tab.target[s];
        b.K = tab.K[s];
        b.Km = tab.Km[s];
        b.Ke = tab.Ke[s];
        if (s >= 2) {
            warp_edge_compute<float>(b, x, o, 0, N - s + 1, base);
            continue;
        }
        // size 1: c = K(1,N) [t^(N-1)] e^(x t) = x^(N-1), the series with an empty product,
        // formed as (g x)^(N-1)/(N-1)! and scaled back by K(1,N) g^-(N-1)
        if (lane == 0) {
            const int v = __ldg(members + e0);
            const float X = __ldg(x + v);
            const int p = scale_exponent<float>(fabsf(X), b.target);
            const float gx = X * Arith<float>::pow2(p);
            float r = 1.f;
            for (int k = 1; k < N; ++k) r = r * (gx / (float)k);
            const float c = finalize_value<float>(r, b, p, 0, nullptr);
            const float old = atomicAdd(y + v, c);
            float sm, er;
            two_sum(old, c, sm, er);
            if (er != 0.f) atomicAdd(comp + v, er);
        }
        __syncwarp();
    }
}

__global__ void noalloc_fold_kernel(float *__restrict__ y, const float *__restrict__ comp, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] += comp[i];
}

// Shared memory per warp for edges of every size up to rank N (floats).
int64_t per_warp_floats(int N) {
    int64_t best = 0;
    for (int s = 1; s <= N; ++s) {
        int64_t W = N - s + 1;
        int64_t need = 2 * (int64_t)s + (int64_t)(s > 2 ? s - 2 : 0) * W + 4 * W;
        if (need > best) best = need;
    }
    return (best + 3) / 4 * 4;
}

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
float *g_comp_addr[kMaxDevices] = {nullptr};

}  // namespace
}  // namespace s3

using namespace s3;

extern "C" s3_status s3_sttsvc_f32_noalloc(int64_t n, int64_t m, int32_t rank, const int64_t *edge_ptr,
                                           const int32_t *members, const float *x, float *y, void *stream) {
    if (n < 1 || m < 0) return fail(S3_EINVAL, "n must be >= 1 and m >= 0");
    if (n > S3_NOALLOC_MAX_NODES) return fail(S3_EINVAL, "n exceeds S3_NOALLOC_MAX_NODES");
    if (rank < 1 || rank > S3_MAX_RANK) return fail(S3_EINVAL, "rank must be in 1..S3_MAX_RANK");
    if (!x || !y || (m > 0 && (!edge_ptr || !members))) return fail(S3_EINVAL, "NULL argument");
    int dev = 0;
    S3_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(S3_EINVAL, "device ordinal out of range");
    const int64_t per_warp = per_warp_floats(rank);
    const int wpb = 4;
    const size_t smem = (size_t)wpb * (size_t)per_warp * sizeof(float);
    float *comp = nullptr;
    {
        // once per device: resolve the scratch array's device address (a host-side
        // name is not a device pointer) and raise the kernel's shared-memory limit
        std::lock_guard<std::mutex> lock(g_setup_mu);
        if (!g_comp_addr[dev]) {
            void *p = nullptr;
            S3_CUDA(cudaGetSymbolAddress(&p, g_comp));
            S3_CUDA(cudaFuncSetAttribute(noalloc_edge_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         200 * 1024));
            g_comp_addr[dev] = reinterpret_cast<float *>(p);
        }
        comp = g_comp_addr[dev];
    }
    if (smem > 200 * 1024) return fail(S3_EINVAL, "rank too large for the shared-memory budget");
    cudaStream_t st = (cudaStream_t)stream;
    NoallocTables tab;
    fill_tables(rank, tab);
    // y and the compensation terms accumulate from zero on every call
    S3_CUDA(cudaMemsetAsync(y, 0, sizeof(float) * (size_t)n, st));
    S3_CUDA(cudaMemsetAsync(comp, 0, sizeof(float) * (size_t)n, st));
    if (m > 0) {
        int64_t grid = (m + wpb - 1) / wpb;
        if (grid > (1 << 22)) grid = 1 << 22;
        noalloc_edge_kernel<<<(unsigned)grid, wpb * 32, smem, st>>>(n, m, rank, edge_ptr, members, x, y, comp,
                                                                  per_warp, tab);
        S3_CUDA(cudaGetLastError());
    }
    noalloc_fold_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(y, comp, n);
    S3_CUDA(cudaGetLastError());
    return S3_OK;
}
