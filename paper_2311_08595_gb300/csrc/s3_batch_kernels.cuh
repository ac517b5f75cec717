// Batched S^3TTVc kernels (included by the per-type translation units).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>

#include "s3_batch.h"
#include "s3_bern.cuh"
#include "s3_series.cuh"

namespace s3 {
namespace batch_detail {

// ------------------------------------------------------------ edge tiles --

template <typename T, int W>
__device__ __forceinline__ void batch_thread_tile(const BatchEdgeArgs &a, const BatchBucket &bb, const Tile &tl,
                                                  unsigned char *smem_raw) {
    const EdgeBucketArgs &b = bb.b;
    const int BS = blockDim.x;
    const int tid = threadIdx.x, lane = tid & 31;
    const int s = b.s;
    const int nv = a.nvec;
    // per-warp regions, as in edge_thread_kernel
    const size_t words = thread_smem_words<T>(s, W);
    T *wb = reinterpret_cast<T *>(smem_raw + (size_t)(tid >> 5) * words * 4 * kLS);
    T *Xb0 = wb + lane;
    T *Xb1 = Xb0 + s * kLS;
    T *Pre = Xb0 + 2 * s * kLS;
    int32_t *ibase = reinterpret_cast<int32_t *>(wb + (2 * s + (s > 2 ? (s - 2) * W : 0)) * kLS) + lane;
    auto ids_of = [&](int r) { return ibase + r * s * kLS; };
    auto slots_of = [&](int r) { return ibase + (3 + r) * s * kLS; };
    const int64_t end = tl.e0 + tl.count;
    int64_t e = tl.e0 + tid;
    if (e >= end) return;
    // edges of this thread: e, e + BS, ...; items (edge k, vector v), k-major
    const int64_t nedges = (end - e + BS - 1) / BS;
    const int64_t nitems = nedges * nv;
    auto edge_at = [&](int64_t k) { return e + k * BS; };
    auto issue_ids = [&](int64_t k, int r) {
        const int64_t ee = edge_at(k);
        int32_t *ib = ids_of(r), *sb = slots_of(r);
        for (int i = 0; i < s; ++i) {
            cp_async<4>(ib + i * kLS, b.ids + (int64_t)i * b.ld + ee);
            cp_async<4>(sb + i * kLS, b.slot + (int64_t)i * b.ld + ee);
        }
    };
    auto issue_x = [&](int64_t item, T *xb) {
        const int64_t k = item / nv;
        const int v = (int)(item - k * nv);
        const T *x = reinterpret_cast<const T *>(a.xs[(size_t)bb.graph * nv + v]);
        const int32_t *ib = ids_of((int)(k % 3));
        for (int i = 0; i < s; ++i) cp_async<(int)sizeof(T)>(xb + i * kLS, x + ib[i * kLS]);
    };
    issue_ids(0, 0);
    cp_async_commit();
    cp_async_wait_all();
    issue_x(0, Xb0);
    if (nedges > 1) issue_ids(1, 1);
    cp_async_commit();
    EdgeOutArgs o{};
    o.mode = kOutBuffer;
    o.range_events = a.range_events;
    for (int64_t j = 0; j < nitems; ++j) {
        const int64_t k = j / nv;
        const int v = (int)(j - k * nv);
        T *xc = (j & 1) ? Xb1 : Xb0;
        T *xn = (j & 1) ? Xb0 : Xb1;
        cp_async_wait_all();
        if (j + 1 < nitems) issue_x(j + 1, xn);
        if (v == 0 && k + 2 < nedges) issue_ids(k + 2, (int)((k + 2) % 3));
        cp_async_commit();
        o.out = a.bufs[(size_t)bb.graph * nv + v];
        edge_compute<T, W, true>(b, o, xc, Pre, ids_of((int)(k % 3)), slots_of((int)(k % 3)), s);
    }
    cp_async_wait_all();
}

template <typename T>
__device__ __forceinline__ void batch_warp_tile(const BatchEdgeArgs &a, const BatchBucket &bb, const Tile &tl,
                                                unsigned char *smem_raw) {
    const int wib = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    T *base = reinterpret_cast<T *>(smem_raw) + (int64_t)wib * a.per_warp;
    EdgeOutArgs o{};
    o.mode = kOutBuffer;
    o.range_events = a.range_events;
    for (int64_t e = tl.e0 + wib; e < tl.e0 + tl.count; e += wpb) {
        for (int v = 0; v < a.nvec; ++v) {
            o.out = a.bufs[(size_t)bb.graph * a.nvec + v];
            const T *x = reinterpret_cast<const T *>(a.xs[(size_t)bb.graph * a.nvec + v]);
            warp_edge_compute<T>(bb.b, x, o, e, bb.W, base);
        }
    }
}

// Bernoulli-form tiles (s3_bern.cuh): one edge per thread, every vector of the graph in
// turn; each warp's region holds a.bern_lane values per lane and a.bern_fb for the fallback.
template <typename T, int W>
__device__ __forceinline__ void batch_bern_tile(const BatchEdgeArgs &a, const BatchBucket &bb, const Tile &tl,
                                                unsigned char *smem_raw) {
    T *base = reinterpret_cast<T *>(smem_raw) +
              (size_t)(threadIdx.x >> 5) * ((size_t)kLS * a.bern_lane + (size_t)a.bern_fb);
    T *fb = base + (size_t)kLS * a.bern_lane;
    EdgeOutArgs o{};
    o.mode = kOutBuffer;
    o.range_events = a.range_events;
    const int64_t end = tl.e0 + tl.count;
    for (int64_t e0 = tl.e0; e0 < end; e0 += blockDim.x) {
        const int64_t e = e0 + threadIdx.x;
        const bool valid = e < end;
        if (__all_sync(0xffffffffu, !valid)) break;
        for (int v = 0; v < a.nvec; ++v) {
            o.out = a.bufs[(size_t)bb.graph * a.nvec + v];
            const T *x = reinterpret_cast<const T *>(a.xs[(size_t)bb.graph * a.nvec + v]);
            bern_edge<T, W, true, false>(bb.b, x, o, a.bern, e, valid, base, fb);
        }
    }
}

// Size-1 edges: c(e, v) = x_v^(N-1), one thread per edge and vector.
template <typename T>
__device__ __forceinline__ void batch_single_tile(const BatchEdgeArgs &a, const BatchBucket &bb, const Tile &tl) {
    const EdgeBucketArgs &b = bb.b;
    for (int64_t e = tl.e0 + threadIdx.x; e < tl.e0 + tl.count; e += blockDim.x) {
        const int node = __ldg(b.ids + e);
        const int sl = __ldg(b.slot + e);
        for (int v = 0; v < a.nvec; ++v) {
            const T X = reinterpret_cast<const T *>(a.xs[(size_t)bb.graph * a.nvec + v])[node];
            const int ex = Arith<T>::expo(X);
            const T mm = X * Arith<T>::pow2(-ex);
            T r = T(1), base = mm;
            for (int k = b.N - 1; k > 0; k >>= 1) {
                if (k & 1) r *= base;
                base *= base;
            }
            reinterpret_cast<T *>(a.bufs[(size_t)bb.graph * a.nvec + v])[sl] = Arith<T>::scale2(r, (b.N - 1) * ex);
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(256) batch_edge_kernel(BatchEdgeArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ long long tile_id;
    while (true) {
        if (threadIdx.x == 0) tile_id = (long long)atomicAdd(a.counter, 1ull);
        __syncthreads();
        const long long t = tile_id;
        __syncthreads();
        if (t >= a.ntiles) return;
        const Tile tl = a.tiles[t];
        const BatchBucket bb = a.buckets[tl.bucket];
        if (bb.warp == 2) {
            batch_single_tile<T>(a, bb, tl);
        } else if (bb.warp == 3) {
            switch (bb.W) {
#define S3_BB_CASE(w) \
    case w: batch_bern_tile<T, w>(a, bb, tl, smem_raw); break;
                S3_W_CASES(S3_BB_CASE)
#undef S3_BB_CASE
                default: break;
            }
        } else if (bb.warp) {
            batch_warp_tile<T>(a, bb, tl, smem_raw);
        } else {
            switch (bb.W) {
#define S3_BT_CASE(w) \
    case w: batch_thread_tile<T, w>(a, bb, tl, smem_raw); break;
                S3_W_CASES(S3_BT_CASE)
#undef S3_BT_CASE
                default: break;
            }
        }
        __syncthreads();
    }
}

// --------------------------------------------------------------- reduce --

struct RAccF {
    float s = 0.f, c = 0.f;
    __device__ void add(float v) {
        float t = s + v;
        float bb = t - s;
        c += (s - (t - bb)) + (v - bb);
        s = t;
    }
    __device__ void merge(const RAccF &o) {
        add(o.s);
        c += o.c;
    }
    __device__ float value() const { return s + c; }
    __device__ RAccF down(int d) const {
        RAccF r;
        r.s = __shfl_down_sync(0xffffffffu, s, d);
        r.c = __shfl_down_sync(0xffffffffu, c, d);
        return r;
    }
    __device__ void store(void *p, int64_t i) const { reinterpret_cast<float2 *>(p)[i] = make_float2(s, c); }
    __device__ void load_merge(const void *p, int64_t i) {
        float2 v = reinterpret_cast<const float2 *>(p)[i];
        RAccF t;
        t.s = v.x;
        t.c = v.y;
        merge(t);
    }
};
struct RAccD {
    double s = 0.0;
    __device__ void add(double v) { s += v; }
    __device__ void merge(const RAccD &o) { s += o.s; }
    __device__ double value() const { return s; }
    __device__ RAccD down(int d) const {
        RAccD r;
        r.s = __shfl_down_sync(0xffffffffu, s, d);
        return r;
    }
    __device__ void store(void *p, int64_t i) const { reinterpret_cast<double *>(p)[i] = s; }
    __device__ void load_merge(const void *p, int64_t i) { s += reinterpret_cast<const double *>(p)[i]; }
};
template <typename T> struct RAcc;
template <> struct RAcc<float> { using type = RAccF; };
template <> struct RAcc<double> { using type = RAccD; };

template <typename T>
__global__ void __launch_bounds__(256) batch_reduce_kernel(BatchReduceArgs a) {
    using A = typename RAcc<T>::type;
    __shared__ long long tile_id;
    __shared__ A part[8];
    const int tid = threadIdx.x;
    while (true) {
        if (tid == 0) tile_id = (long long)atomicAdd(a.counter, 1ull);
        __syncthreads();
        const long long t = tile_id;
        __syncthreads();
        if (t >= a.ntiles) return;
        const ReduceTile rt = a.tiles[t];
        const ReduceGraph g = a.graphs[rt.graph];
        for (int v = 0; v < a.nvec; ++v) {
            const size_t jv = (size_t)rt.graph * a.nvec + v;
            const T *buf = reinterpret_cast<const T *>(a.bufs[jv]);
            T *y = reinterpret_cast<T *>(a.ys[jv]);
            if (rt.kind == 0) {
                const int64_t gi = rt.first + (tid >> 5);
                if (gi < g.n_grp) {
                    const int lane = tid & 31;
                    const int node = g.grp_node[gi * 32 + lane];
                    const int d = g.grp_deg[gi * 32 + lane];
                    const T *p = buf + g.grp_off[gi] + lane;
                    A acc;
                    int k = 0;
                    for (; k + 4 <= d; k += 4) {
                        T v0 = p[32 * k], v1 = p[32 * k + 32], v2 = p[32 * k + 64], v3 = p[32 * k + 96];
                        acc.add(v0);
                        acc.add(v1);
                        acc.add(v2);
                        acc.add(v3);
                    }
                    for (; k < d; ++k) acc.add(p[32 * k]);
                    if (node >= 0) y[node] = (T)acc.value();
                }
            } else if (rt.kind == 1) {
                int64_t i = rt.first + (tid >> 5);
                if (i < g.n_med) {
                    const int lane = tid & 31;
                    const int node = g.med_nodes[i];
                    const int64_t b = g.med_off[i], e = b + g.med_len[i];
                    A acc;
                    int64_t k = b + lane;
                    for (; k + 96 < e; k += 128) {
                        T v0 = buf[k], v1 = buf[k + 32], v2 = buf[k + 64], v3 = buf[k + 96];
                        acc.add(v0);
                        acc.add(v1);
                        acc.add(v2);
                        acc.add(v3);
                    }
                    for (; k < e; k += 32) acc.add(buf[k]);
#pragma unroll
                    for (int d = 16; d > 0; d >>= 1) acc.merge(acc.down(d));
                    if (lane == 0) y[node] = (T)acc.value();
                }
            } else if (rt.kind == 3) {
                // eight lanes per node; lanes of a missing node join the shuffles only
                const int64_t i = rt.first + (tid >> 3);
                const bool has = i < g.n_med8;
                const int sl = tid & 7;
                const int64_t b = has ? g.med8_off[i] : 0;
                const int len = has ? g.med8_len[i] : 0;
                A acc;
                for (int k = sl; k < len; k += 8) acc.add(buf[b + k]);
#pragma unroll
                for (int d = 4; d > 0; d >>= 1) acc.merge(acc.down(d));
                if (has && sl == 0) y[g.med8_nodes[i]] = (T)acc.value();
            } else {
                const int64_t pc = rt.first;
                int64_t b = g.piece_start[pc];
                int len = g.piece_len[pc];
                A acc;
                for (int k = tid; k < len; k += 256) acc.add(buf[b + k]);
#pragma unroll
                for (int d = 16; d > 0; d >>= 1) acc.merge(acc.down(d));
                if ((tid & 31) == 0) part[tid >> 5] = acc;
                __syncthreads();
                if (tid == 0) {
                    A tot = part[0];
                    for (int w = 1; w < 8; ++w) tot.merge(part[w]);
                    tot.store(a.partials[jv], pc);
                }
                __syncthreads();
            }
        }
        __syncthreads();
    }
}

template <typename T>
__global__ void batch_final_kernel(BatchReduceArgs a) {
    using A = typename RAcc<T>::type;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.nfinals * a.nvec) return;
    const int64_t f = i / a.nvec;
    const int v = (int)(i - f * a.nvec);
    const FinalTile ft = a.finals[f];
    const ReduceGraph g = a.graphs[ft.graph];
    const size_t jv = (size_t)ft.graph * a.nvec + v;
    A acc;
    for (int p = g.big_piece_ptr[ft.big]; p < g.big_piece_ptr[ft.big + 1]; ++p) acc.load_merge(a.partials[jv], p);
    reinterpret_cast<T *>(a.ys[jv])[g.big_nodes[ft.big]] = (T)acc.value();
}



template <typename T>
s3_status record_batch_t(s3_batch_s *bt, cudaStream_t st) {
    const int which = sizeof(T) == 4 ? 0 : 1;
    // pointer tables: xs, ys from the pinned staging; buffers and partials
    const size_t J = bt->graphs.size() * (size_t)bt->nvec;
    S3_CUDA(cudaMemcpyAsync(bt->d_xs, bt->h_ptrs, sizeof(void *) * 2 * J, cudaMemcpyHostToDevice, st));
    S3_CUDA(cudaMemsetAsync(bt->d_counters, 0, (kBatchClasses + 1) * sizeof(unsigned long long), st));
    int32_t per_warp = 0;
    for (auto &bb : bt->h_buckets)
        if (bb.warp == 1) per_warp = std::max<int32_t>(per_warp, (int32_t)warp_smem_elems(bb.b.s, bb.W));
    // fork: one persistent kernel per shared-memory class
    S3_CUDA(cudaEventRecord(bt->ev_fork, st));
    for (int c = 0; c < kBatchClasses; ++c) {
        const int64_t nt = bt->cls[c].end - bt->cls[c].begin;
        cudaStream_t cs = bt->aux[c];
        S3_CUDA(cudaStreamWaitEvent(cs, bt->ev_fork, 0));
        if (nt > 0) {
            BatchEdgeArgs ea{};
            ea.buckets = bt->d_buckets;
            ea.tiles = bt->d_tiles + bt->cls[c].begin;
            ea.ntiles = nt;
            ea.xs = bt->d_xs;
            ea.bufs = bt->d_bufs + which * J;
            ea.nvec = bt->nvec;
            ea.per_warp = per_warp;
            ea.counter = bt->d_counters + c;
            ea.range_events = bt->graphs.empty() ? nullptr : bt->graphs[0]->d_range;
            ea.bern_lane = bt->bern_lane;
            ea.bern_fb = bt->bern_fb;
            if (!bt->graphs.empty()) ea.bern = bt->graphs[0]->bern_args;   // constants; rejections counted there
            int per_sm = 0;
            S3_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_edge_kernel<T>, bt->bs,
                                                                  bt->cls[c].smem));
            if (per_sm <= 0) return fail(S3_ENOTSUP, "batched kernel does not fit on an SM with this configuration");
            int grid = (int)std::min<int64_t>((int64_t)bt->sms * per_sm, nt);
            batch_edge_kernel<T><<<grid, bt->bs, bt->cls[c].smem, cs>>>(ea);
            S3_CUDA(cudaGetLastError());
        }
        S3_CUDA(cudaEventRecord(bt->ev_join[c], cs));
        S3_CUDA(cudaStreamWaitEvent(st, bt->ev_join[c], 0));
    }
    BatchReduceArgs ra{};
    ra.graphs = bt->d_rgraphs;
    ra.tiles = bt->d_rtiles;
    ra.ntiles = bt->nrtiles;
    ra.finals = bt->d_finals;
    ra.nfinals = bt->nfinals;
    ra.bufs = bt->d_bufs + which * J;
    ra.ys = bt->d_ys;
    ra.partials = bt->d_parts;
    ra.nvec = bt->nvec;
    ra.counter = bt->d_counters + kBatchClasses;
    int rper = 0;
    S3_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&rper, batch_reduce_kernel<T>, 256, 0));
    int rgrid = (int)std::min<int64_t>((int64_t)bt->sms * std::max(rper, 1), std::max<int64_t>(bt->nrtiles, 1));
    batch_reduce_kernel<T><<<rgrid, 256, 0, st>>>(ra);
    S3_CUDA(cudaGetLastError());
    if (bt->nfinals > 0) {
        int64_t nf = bt->nfinals * bt->nvec;
        batch_final_kernel<T><<<(unsigned)((nf + 127) / 128), 128, 0, st>>>(ra);
        S3_CUDA(cudaGetLastError());
    }
    return S3_OK;
}


}  // namespace batch_detail
}  // namespace s3
