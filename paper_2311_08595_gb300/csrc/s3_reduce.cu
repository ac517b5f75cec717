// Deterministic segmented reduce: y_v = sum of the per-(edge, node) values
// that the edge kernels wrote into the slot buffer.  The buffer is laid out
// by node so that every node's values can be summed without atomics, and the
// work is split by degree so that hubs do not serialise on one thread:
//   degree <= 32          groups of 32 nodes of similar degree in sliced-ELL
//                         layout (the k-th value of lane l at off + 32 k + l):
//                         one warp per group, lane l sums its own node, and
//                         every load of the warp is one coalesced 128-byte row;
//   degree <= 128         eight lanes per node over its contiguous segment;
//   degree <= 1024        one warp per node over its contiguous segment;
//   larger                pieces of 2048 slots, one block each; the block that
//                         finishes a node's last piece (a per-node counter)
//                         adds the node's piece sums in a fixed order.
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

// Sum over each aligned group of 8 lanes (all 32 lanes take part); the group's
// first lane holds its total.
template <typename A>
__device__ __forceinline__ A group8_reduce(A a) {
#pragma unroll
    for (int d = 4; d > 0; d >>= 1) a.merge(shfl_down_acc(a, d));
    return a;
}

__device__ __forceinline__ void store_partial(void *p, int64_t i, const AccF &a) {
    reinterpret_cast<float2 *>(p)[i] = make_float2(a.s, a.c);
}
__device__ __forceinline__ void store_partial(void *p, int64_t i, const AccD &a) {
    reinterpret_cast<double *>(p)[i] = a.s;
}
__device__ __forceinline__ void load_partial(const void *p, int64_t i, AccF &a) {
    float2 v = __ldcg(reinterpret_cast<const float2 *>(p) + i);
    AccF t;
    t.s = v.x;
    t.c = v.y;
    a.merge(t);
}
__device__ __forceinline__ void load_partial(const void *p, int64_t i, AccD &a) {
    a.s += __ldcg(reinterpret_cast<const double *>(p) + i);
}

// Per-node warm-start features from per-(edge, node) records (s3_mlp.cu writes them):
// bits 0-7 the edge size s, bits 8-10 its histogram bin, bits 16-63 the sum of the
// other members' degrees; 0 is no record (a padded load).  Integer sums: exact.
struct __align__(8) FeatAcc {
    unsigned h[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    unsigned smax = 0;
    unsigned long long ssum = 0, nbr = 0;
    __device__ void add(unsigned long long rec) {
        const unsigned sz = (unsigned)(rec & 0xffu), b = (unsigned)(rec >> 8) & 7u;
        const unsigned one = rec != 0ull;
#pragma unroll
        for (int k = 0; k < 8; ++k) h[k] += (b == (unsigned)k) ? one : 0u;
        smax = max(smax, sz);
        ssum += sz;
        nbr += rec >> 16;
    }
    __device__ void merge(const FeatAcc &o) {
#pragma unroll
        for (int k = 0; k < 8; ++k) h[k] += o.h[k];
        smax = max(smax, o.smax);
        ssum += o.ssum;
        nbr += o.nbr;
    }
};

__device__ __forceinline__ FeatAcc shfl_down_acc(const FeatAcc &a, int d) {
    FeatAcc r;
#pragma unroll
    for (int k = 0; k < 8; ++k) r.h[k] = __shfl_down_sync(0xffffffffu, a.h[k], d);
    r.smax = __shfl_down_sync(0xffffffffu, a.smax, d);
    r.ssum = __shfl_down_sync(0xffffffffu, a.ssum, d);
    r.nbr = __shfl_down_sync(0xffffffffu, a.nbr, d);
    return r;
}

__device__ __forceinline__ void store_partial(void *p, int64_t i, const FeatAcc &a) {
    reinterpret_cast<FeatAcc *>(p)[i] = a;
}
__device__ __forceinline__ void load_partial(const void *p, int64_t i, FeatAcc &a) {
    const FeatAcc *q = reinterpret_cast<const FeatAcc *>(p) + i;
    FeatAcc t;
#pragma unroll
    for (int k = 0; k < 8; ++k) t.h[k] = __ldcg(&q->h[k]);
    t.smax = __ldcg(&q->smax);
    t.ssum = __ldcg(&q->ssum);
    t.nbr = __ldcg(&q->nbr);
    a.merge(t);
}

// the 12 features of node v (row v of feat), log1p-scaled in FP32: degree; mean and max
// size of its edges; the 8-bin size histogram; the other members' degree sum
struct FeatSink {
    float *feat;
    bool vec;   // feat 16-byte aligned: rows written as three float4
    __device__ void put(int v, const FeatAcc &a) const {
        unsigned d = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) d += a.h[k];
        float f[12];
        const float df = (float)d;
        f[0] = log1pf(df);
        f[1] = log1pf(d ? (float)a.ssum / df : 0.f);
        f[2] = log1pf((float)a.smax);
#pragma unroll
        for (int k = 0; k < 8; ++k) f[3 + k] = log1pf((float)a.h[k]);
        f[11] = log1pf((float)a.nbr);
        static_assert(sizeof(FeatAcc) <= 64, "feature partials hold 64 bytes");
        float *row = feat + (int64_t)v * 12;
        if (vec) {
#pragma unroll
            for (int q = 0; q < 3; ++q)
                reinterpret_cast<float4 *>(row)[q] = make_float4(f[4 * q], f[4 * q + 1], f[4 * q + 2], f[4 * q + 3]);
        } else {
#pragma unroll
            for (int k = 0; k < 12; ++k) row[k] = f[k];
        }
    }
};

constexpr int kRedThreads = 256;

// Eight loads in flight per thread, predicated at the end of a segment (a
// missing value is 0, and adding 0 leaves a sum unchanged), then added in
// order: the kernel is bound by memory latency, not by its few flops.
constexpr int kRedUnroll = 8;

// Blocks [0, n_pieces): one hub piece each (the longest-running blocks start
// first); then one warp per medium node of degree > 128; then eight lanes per
// medium node of degree <= 128; then one warp per group of 32 small nodes.
// T: the slot values; A: the accumulator (add, merge, a shuffle and a partial-sum store
// of its own); Sink: writes a node's result (put(node, acc)).
template <typename T, typename A, typename Sink>
__global__ void __launch_bounds__(kRedThreads) reduce_kernel(ReduceArgs r, const T *__restrict__ buf, Sink y,
                                                             int64_t nb_med, int64_t nb_med8, int64_t nb_grp) {
    if (r.skip && *r.skip) return;
    constexpr int U = kRedUnroll;
    const int64_t bid = blockIdx.x;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    if (bid < r.n_pieces) {
        __shared__ A part[kRedThreads / 32];
        const int64_t pc = bid;
        const T *p = buf + r.piece_start[pc];
        const int len = r.piece_len[pc];
        A a;
        for (int k = tid; k < len; k += U * kRedThreads) {
            T v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) v[u] = k + u * kRedThreads < len ? p[k + u * kRedThreads] : T(0);
#pragma unroll
            for (int u = 0; u < U; ++u) a.add(v[u]);
        }
        a = warp_reduce(a);
        if (lane == 0) part[tid >> 5] = a;
        __syncthreads();
        __shared__ int last;
        const int hb = r.piece_big[pc];
        if (tid == 0) {
            A tot = part[0];
            for (int w = 1; w < kRedThreads / 32; ++w) tot.merge(part[w]);
            store_partial(r.partial, pc, tot);
            __threadfence();
            const int npc = r.big_piece_ptr[hb + 1] - r.big_piece_ptr[hb];
            last = atomicAdd(r.big_count + hb, 1) == npc - 1;
        }
        __syncthreads();
        // the block that completes a node's last piece adds the node's partials, lane l
        // taking pieces l, l+32, ... in order and a fixed shuffle tree after: the same
        // sum whichever block gets there last
        if (last && tid < 32) {
            __threadfence();
            if (lane == 0) r.big_count[hb] = 0;  // ready for the next call
            A t;
            for (int q = r.big_piece_ptr[hb] + lane; q < r.big_piece_ptr[hb + 1]; q += 32) load_partial(r.partial, q, t);
            t = warp_reduce(t);
            if (lane == 0) y.put(r.big_nodes[hb], t);
        }
    } else if (bid < r.n_pieces + nb_med) {
        const int64_t i = (bid - r.n_pieces) * (kRedThreads / 32) + (tid >> 5);
        if (i >= r.n_med) return;
        const int v = r.med_nodes[i];
        const T *p = buf + r.med_off[i];
        const int len = r.med_len[i];
        A a;
        for (int k = lane; k < len; k += U * 32) {
            T w[U];
#pragma unroll
            for (int u = 0; u < U; ++u) w[u] = k + u * 32 < len ? p[k + u * 32] : T(0);
#pragma unroll
            for (int u = 0; u < U; ++u) a.add(w[u]);  // adding 0 leaves the sum unchanged
        }
        a = warp_reduce(a);
        if (lane == 0) y.put(v, a);
    } else if (bid < r.n_pieces + nb_med + nb_med8) {
        // eight lanes per node; lanes of a missing node read nothing but join the shuffles
        const int64_t i = (bid - r.n_pieces - nb_med) * (kRedThreads / 8) + (tid >> 3);
        const bool has = i < r.n_med8;
        const int sl = tid & 7;
        const T *p = has ? buf + r.med8_off[i] : buf;
        const int len = has ? r.med8_len[i] : 0;
        A a;
        for (int k = sl; k < len; k += U * 8) {
            T w[U];
#pragma unroll
            for (int u = 0; u < U; ++u) w[u] = k + u * 8 < len ? p[k + u * 8] : T(0);
#pragma unroll
            for (int u = 0; u < U; ++u) a.add(w[u]);
        }
        a = group8_reduce(a);
        if (has && sl == 0) y.put(r.med8_nodes[i], a);
    } else {
        const int64_t gi = (bid - r.n_pieces - nb_med - nb_med8) * (kRedThreads / 32) + (tid >> 5);
        if (gi >= r.n_grp) return;
        const int node = r.grp_node[gi * 32 + lane];
        const int d = r.grp_deg[gi * 32 + lane];
        const T *p = buf + r.grp_off[gi] + lane;
        A a;
        for (int k = 0; k < d; k += U) {  // U coalesced rows in flight, added in order
            T w[U];
#pragma unroll
            for (int u = 0; u < U; ++u) w[u] = k + u < d ? p[32 * (k + u)] : T(0);
#pragma unroll
            for (int u = 0; u < U; ++u) a.add(w[u]);
        }
        if (node >= 0) y.put(node, a);
    }
}

// y_v = the sum of node v's values
template <typename T>
struct SumSink {
    T *y;
    __device__ void put(int v, const typename AccOf<T>::type &a) const { y[v] = (T)a.value(); }
};

template <typename T, typename A, typename Sink>
cudaError_t launch_reduce_t(const ReduceArgs &r, const T *buf, Sink y, cudaStream_t st) {
    int64_t nb_grp = (r.n_grp + (kRedThreads / 32) - 1) / (kRedThreads / 32);
    int64_t nb_med = (r.n_med + (kRedThreads / 32) - 1) / (kRedThreads / 32);
    int64_t nb_med8 = (r.n_med8 + (kRedThreads / 8) - 1) / (kRedThreads / 8);
    int64_t grid = nb_grp + nb_med + nb_med8 + r.n_pieces;
    if (grid > 0) {
        reduce_kernel<T, A, Sink><<<(unsigned)grid, kRedThreads, 0, st>>>(r, buf, y, nb_med, nb_med8, nb_grp);
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
    return launch_reduce_t<float, AccF>(r, buf, SumSink<float>{y}, st);
}
cudaError_t launch_reduce_f64(const ReduceArgs &r, const double *buf, double *y, cudaStream_t st) {
    return launch_reduce_t<double, AccD>(r, buf, SumSink<double>{y}, st);
}
cudaError_t launch_feature_reduce(const ReduceArgs &r, const unsigned long long *rec, float *feat, cudaStream_t st) {
    return launch_reduce_t<unsigned long long, FeatAcc>(
        r, rec, FeatSink{feat, (reinterpret_cast<uintptr_t>(feat) & 15) == 0}, st);
}
cudaError_t launch_add_comp(float *y, const float *comp, int64_t n, const int32_t *skip, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    add_comp_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(y, comp, n, skip);
    return cudaGetLastError();
}

}  // namespace s3
