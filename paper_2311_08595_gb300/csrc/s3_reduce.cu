// Deterministic segmented reduce: y_v = sum of the per-(edge, node) values
// that the edge kernels wrote into the slot buffer.  The buffer is laid out
// by node so that every node's values can be summed without atomics, and the
// work is split by degree so that hubs do not serialise on one thread:
//   degree <= 32          groups of 32 nodes of similar degree in sliced-ELL
//                         layout (the k-th value of lane l at off + 32 k + l):
//                         one warp per group, lane l sums its own node, and
//                         every load of the warp is one coalesced 128-byte row;
//   degree <= 4096        one warp per node over its contiguous segment;
//   larger                pieces of 4096 slots, one block each, then one
//                         warp per node adds its pieces in a fixed order.
// Every thread/warp/block adds in a fixed order, so the result does not
// depend on scheduling.  FP32 sums carry a two-sum compensation term.
#include <cuda_runtime.h>

#include "s3_internal.h"
#include "s3_kernels.h"

namespace s3 {
namespace {

struct AccF {
    float s = 0.f, c = 0.f;
    __device__ void add(float v) {
        float t = s + v;
        float bb = t - s;
        c += (s - (t - bb)) + (v - bb);
        s = t;
    }
    __device__ void merge(const AccF &o) {
        add(o.s);
        c += o.c;
    }
    __device__ float value() const { return s + c; }
};

struct AccD {
    double s = 0.0;
    __device__ void add(double v) { s += v; }
    __device__ void merge(const AccD &o) { s += o.s; }
    __device__ double value() const { return s; }
};

template <typename T> struct AccOf;
template <> struct AccOf<float> { using type = AccF; };
template <> struct AccOf<double> { using type = AccD; };

__device__ __forceinline__ AccF shfl_down_acc(const AccF &a, int d) {
    AccF r;
    r.s = __shfl_down_sync(0xffffffffu, a.s, d);
    r.c = __shfl_down_sync(0xffffffffu, a.c, d);
    return r;
}
__device__ __forceinline__ AccD shfl_down_acc(const AccD &a, int d) {
    AccD r;
    r.s = __shfl_down_sync(0xffffffffu, a.s, d);
    return r;
}

template <typename A>
__device__ __forceinline__ A warp_reduce(A a) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) a.merge(shfl_down_acc(a, d));
    return a;  // lane 0 holds the total
}

__device__ __forceinline__ void store_partial(void *p, int64_t i, const AccF &a) {
    reinterpret_cast<float2 *>(p)[i] = make_float2(a.s, a.c);
}
__device__ __forceinline__ void store_partial(void *p, int64_t i, const AccD &a) {
    reinterpret_cast<double *>(p)[i] = a.s;
}
__device__ __forceinline__ void load_partial(const void *p, int64_t i, AccF &a) {
    float2 v = reinterpret_cast<const float2 *>(p)[i];
    AccF t;
    t.s = v.x;
    t.c = v.y;
    a.merge(t);
}
__device__ __forceinline__ void load_partial(const void *p, int64_t i, AccD &a) {
    a.s += reinterpret_cast<const double *>(p)[i];
}

constexpr int kRedThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kRedThreads) reduce_kernel(ReduceArgs r, const T *__restrict__ buf, T *__restrict__ y,
                                                             int64_t nb_grp, int64_t nb_med) {
    if (r.skip && *r.skip) return;
    using A = typename AccOf<T>::type;
    const int64_t bid = blockIdx.x;
    const int tid = threadIdx.x;
    if (bid < nb_grp) {
        const int64_t gi = bid * (kRedThreads / 32) + (tid >> 5);
        if (gi >= r.n_grp) return;
        const int lane = tid & 31;
        const int node = r.grp_node[gi * 32 + lane];
        const int d = r.grp_deg[gi * 32 + lane];
        const T *p = buf + r.grp_off[gi] + lane;
        A a;
        int k = 0;
        for (; k + 4 <= d; k += 4) {  // four coalesced rows in flight, added in order
            T v0 = p[32 * k], v1 = p[32 * k + 32], v2 = p[32 * k + 64], v3 = p[32 * k + 96];
            a.add(v0);
            a.add(v1);
            a.add(v2);
            a.add(v3);
        }
        for (; k < d; ++k) a.add(p[32 * k]);
        if (node >= 0) y[node] = (T)a.value();
    } else if (bid < nb_grp + nb_med) {
        int64_t i = (bid - nb_grp) * (kRedThreads / 32) + (tid >> 5);
        if (i >= r.n_med) return;
        const int lane = tid & 31;
        const int v = r.med_nodes[i];
        const int64_t b = r.med_off[i], t = b + r.med_len[i];
        A a;
        int64_t k = b + lane;
        for (; k + 96 < t; k += 128) {  // four loads in flight per lane, added in order
            T v0 = buf[k], v1 = buf[k + 32], v2 = buf[k + 64], v3 = buf[k + 96];
            a.add(v0);
            a.add(v1);
            a.add(v2);
            a.add(v3);
        }
        for (; k < t; k += 32) a.add(buf[k]);
        a = warp_reduce(a);
        if (lane == 0) y[v] = (T)a.value();
    } else {
        __shared__ A part[kRedThreads / 32];
        int64_t pc = bid - nb_grp - nb_med;
        int64_t b = r.piece_start[pc];
        int len = r.piece_len[pc];
        A a;
        int k = tid;
        for (; k + 3 * kRedThreads < len; k += 4 * kRedThreads) {
            T v0 = buf[b + k], v1 = buf[b + k + kRedThreads], v2 = buf[b + k + 2 * kRedThreads],
              v3 = buf[b + k + 3 * kRedThreads];
            a.add(v0);
            a.add(v1);
            a.add(v2);
            a.add(v3);
        }
        for (; k < len; k += kRedThreads) a.add(buf[b + k]);
        a = warp_reduce(a);
        if ((tid & 31) == 0) part[tid >> 5] = a;
        __syncthreads();
        if (tid == 0) {
            A tot = part[0];
            for (int w = 1; w < kRedThreads / 32; ++w) tot.merge(part[w]);
            store_partial(r.partial, pc, tot);
        }
    }
}

// one warp per big node: lane l adds pieces l, l+32, ... in order, then a fixed shuffle tree
template <typename T>
__global__ void finalize_big_kernel(ReduceArgs r, T *__restrict__ y) {
    if (r.skip && *r.skip) return;
    using A = typename AccOf<T>::type;
    int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= r.n_big) return;
    A a;
    for (int p = r.big_piece_ptr[i] + lane; p < r.big_piece_ptr[i + 1]; p += 32) load_partial(r.partial, p, a);
    a = warp_reduce(a);
    if (lane == 0) y[r.big_nodes[i]] = (T)a.value();
}

template <typename T>
cudaError_t launch_reduce_t(const ReduceArgs &r, const T *buf, T *y, cudaStream_t st) {
    int64_t nb_grp = (r.n_grp + (kRedThreads / 32) - 1) / (kRedThreads / 32);
    int64_t nb_med = (r.n_med + (kRedThreads / 32) - 1) / (kRedThreads / 32);
    int64_t grid = nb_grp + nb_med + r.n_pieces;
    if (grid > 0) {
        reduce_kernel<T><<<(unsigned)grid, kRedThreads, 0, st>>>(r, buf, y, nb_grp, nb_med);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (r.n_big > 0) {
        finalize_big_kernel<T><<<(unsigned)((r.n_big * 32 + 127) / 128), 128, 0, st>>>(r, y);
        return cudaGetLastError();
    }
    return cudaSuccess;
}

__global__ void add_comp_kernel(float *y, const float *comp, int64_t n, const int32_t *skip) {
    if (skip && *skip) return;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] += comp[i];
}

}  // namespace

cudaError_t launch_reduce_f32(const ReduceArgs &r, const float *buf, float *y, cudaStream_t st) {
    return launch_reduce_t<float>(r, buf, y, st);
}
cudaError_t launch_reduce_f64(const ReduceArgs &r, const double *buf, double *y, cudaStream_t st) {
    return launch_reduce_t<double>(r, buf, y, st);
}
cudaError_t launch_add_comp(float *y, const float *comp, int64_t n, const int32_t *skip, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    add_comp_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(y, comp, n, skip);
    return cudaGetLastError();
}

}  // namespace s3
