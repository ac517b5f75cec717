// Batched S^3TTVc: many hypergraphs x many vectors in one persistent launch.
//
// A batch holds `count` graph handles and `nvec` input vectors per graph.  The
// per-edge work of every (graph, size bucket) is cut into tiles of
// block_threads * edges_per_thread edges; one persistent kernel (a grid that
// fills the GPU once) takes tiles from a device work list (heaviest first,
// atomic counter) and, for each edge of a tile, computes the contributions for
// all nvec vectors of that graph: member ids and incidence slots are loaded once
// per edge and shared by the vectors, and the x gathers of the next
// (edge, vector) item are in flight while the current one is computed.  A
// second persistent kernel reduces every (graph, vector) buffer in
// node-sorted order (deterministic), a third one adds the hub pieces.  The
// whole sequence is captured once into a CUDA graph and replayed; tile shape,
// block size and the thread-vs-warp window threshold come from a built-in
// autotuner that times candidate configurations on the caller's data.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <new>
#include <sstream>
#include <string>
#include <vector>

#include "s3_graph.h"
#include "s3_series.cuh"

namespace s3 {
namespace {

constexpr int kBatchClasses = 4;

struct BatchBucket {
    EdgeBucketArgs b;
    int32_t graph;
    int32_t W;
    int32_t warp;  // 1: one warp per edge
    int32_t pad;
};

struct Tile {
    int32_t bucket;
    int32_t count;
    int64_t e0;
};

struct BatchEdgeArgs {
    const BatchBucket *buckets;
    const Tile *tiles;
    int64_t ntiles;
    const void *const *xs;  // count * nvec input pointers (graph-major)
    void *const *bufs;      // count * nvec per-(edge, node) buffers
    int32_t nvec;
    int32_t per_warp;       // warp tiles: elements of T per warp
    unsigned long long *counter;
    unsigned long long *range_events;
};

struct ReduceGraph {
    const int64_t *inc_ptr;
    const int32_t *small_nodes, *med_nodes, *big_nodes, *big_piece_ptr, *piece_len;
    const int64_t *piece_start;
    int64_t n_small, n_med, n_big, n_pieces;
};

struct ReduceTile {
    int32_t graph;
    int32_t kind;   // 0: 256 small nodes, 1: 8 medium nodes, 2: one hub piece
    int64_t first;
};

struct FinalTile {
    int32_t graph;
    int32_t big;    // index into the graph's hub list
};

struct BatchReduceArgs {
    const ReduceGraph *graphs;
    const ReduceTile *tiles;
    int64_t ntiles;
    const FinalTile *finals;
    int64_t nfinals;
    const void *const *bufs;
    void *const *ys;
    void *const *partials;  // count * nvec partial arrays (hub pieces)
    int32_t nvec;
    unsigned long long *counter;
};

// ------------------------------------------------------------ edge tiles --

template <typename T, int W>
__device__ __forceinline__ void batch_thread_tile(const BatchEdgeArgs &a, const BatchBucket &bb, const Tile &tl,
                                                  unsigned char *smem_raw) {
    const EdgeBucketArgs &b = bb.b;
    const int BS = blockDim.x;
    const int tid = threadIdx.x;
    const int s = b.s;
    const int nv = a.nvec;
    T *tb = reinterpret_cast<T *>(smem_raw);
    T *Xb0 = tb + tid;
    T *Xb1 = tb + (size_t)s * BS + tid;
    T *Pre = tb + (size_t)2 * s * BS + tid;
    int32_t *ibase = reinterpret_cast<int32_t *>(tb + (size_t)(2 * s + (s > 2 ? (s - 2) * W : 0)) * BS) + tid;
    auto ids_of = [&](int r) { return ibase + (size_t)r * s * BS; };
    auto slots_of = [&](int r) { return ibase + (size_t)(3 + r) * s * BS; };
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
            cp_async<4>(ib + (size_t)i * BS, b.ids + (int64_t)i * b.ld + ee);
            cp_async<4>(sb + (size_t)i * BS, b.slot + (int64_t)i * b.ld + ee);
        }
    };
    auto issue_x = [&](int64_t item, T *xb) {
        const int64_t k = item / nv;
        const int v = (int)(item - k * nv);
        const T *x = reinterpret_cast<const T *>(a.xs[(size_t)bb.graph * nv + v]);
        const int32_t *ib = ids_of((int)(k % 3));
        for (int i = 0; i < s; ++i) cp_async<(int)sizeof(T)>(xb + (size_t)i * BS, x + ib[(size_t)i * BS]);
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
        edge_compute<T, W>(b, o, xc, Pre, ids_of((int)(k % 3)), slots_of((int)(k % 3)), BS, s);
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
                int64_t i = rt.first + tid;
                if (i < g.n_small) {
                    int node = g.small_nodes[i];
                    int64_t b = g.inc_ptr[node], e = g.inc_ptr[node + 1];
                    A acc;
                    int64_t k = b;
                    for (; k + 4 <= e; k += 4) {
                        T v0 = buf[k], v1 = buf[k + 1], v2 = buf[k + 2], v3 = buf[k + 3];
                        acc.add(v0);
                        acc.add(v1);
                        acc.add(v2);
                        acc.add(v3);
                    }
                    for (; k < e; ++k) acc.add(buf[k]);
                    y[node] = (T)acc.value();
                }
            } else if (rt.kind == 1) {
                int64_t i = rt.first + (tid >> 5);
                if (i < g.n_med) {
                    const int lane = tid & 31;
                    int node = g.med_nodes[i];
                    int64_t b = g.inc_ptr[node], e = g.inc_ptr[node + 1];
                    A acc;
                    for (int64_t k = b + lane; k < e; k += 32) acc.add(buf[k]);
#pragma unroll
                    for (int d = 16; d > 0; d >>= 1) acc.merge(acc.down(d));
                    if (lane == 0) y[node] = (T)acc.value();
                }
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
cudaError_t prepare_batch_kernels() {
    return cudaFuncSetAttribute(batch_edge_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

}  // namespace
}  // namespace s3

using namespace s3;

struct s3_batch_s {
    int device = 0;
    std::vector<s3_graph_t> graphs;
    int32_t nvec = 0;
    s3_batch_options opt{};
    // current configuration
    int32_t bs = 128, ept = 4, thread_max_w = 32;
    int sms = 0;
    // device tables
    std::vector<void *> allocations;
    BatchBucket *d_buckets = nullptr;
    Tile *d_tiles = nullptr;
    int64_t ntiles = 0, tiles_cap = 0;
    ReduceGraph *d_rgraphs = nullptr;
    ReduceTile *d_rtiles = nullptr;
    int64_t nrtiles = 0;
    FinalTile *d_finals = nullptr;
    int64_t nfinals = 0;
    void **d_xs = nullptr, **d_ys = nullptr, **d_bufs = nullptr, **d_parts = nullptr;
    void **h_ptrs = nullptr;  // pinned staging: xs then ys
    bool staged = false;
    unsigned long long *d_counters = nullptr;  // [0..kBatchClasses) edge tile classes, [kBatchClasses] reduce
    void *d_buf_mem[2] = {nullptr, nullptr};   // per dtype: all per-(graph, vector) buffers
    void *d_part_mem = nullptr;
    std::vector<int64_t> buf_off;              // element offset of each (graph, vector) buffer
    std::vector<int64_t> part_off;
    int64_t buf_elems = 0, part_elems = 0;
    size_t smem = 0;
    int built_eb = 0, built_cfg = -1;
    struct Cls {
        int64_t begin = 0, end = 0;
        size_t smem = 0;
    } cls[kBatchClasses];
    cudaStream_t aux[kBatchClasses] = {nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t ev_fork = nullptr, ev_join[kBatchClasses] = {nullptr, nullptr, nullptr, nullptr};
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    cudaStream_t cap_stream = nullptr;
    std::vector<BatchBucket> h_buckets;
    std::vector<double> bucket_cost;
};

namespace {

s3_status batch_alloc(s3_batch_s *bt, void **p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(S3_ENOMEM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
    }
    bt->allocations.push_back(*p);
    return S3_OK;
}

void free_streams(s3_batch_s *bt) {
    for (int c = 0; c < kBatchClasses; ++c) {
        if (bt->aux[c]) cudaStreamDestroy(bt->aux[c]);
        if (bt->ev_join[c]) cudaEventDestroy(bt->ev_join[c]);
        bt->aux[c] = nullptr;
        bt->ev_join[c] = nullptr;
    }
    if (bt->ev_fork) cudaEventDestroy(bt->ev_fork);
    bt->ev_fork = nullptr;
}

void drop_graphs(s3_batch_s *bt) {
    for (auto &x : bt->exec)
        if (x) {
            cudaGraphExecDestroy(x);
            x = nullptr;
        }
}

// Bucket table, tiles (heaviest first) and launch shape for the current configuration.
s3_status build_tiles(s3_batch_s *bt, int elem_bytes) {
    bt->h_buckets.clear();
    bt->bucket_cost.clear();
    size_t smem = 0;
    const int bs = bt->bs;
    for (size_t gi = 0; gi < bt->graphs.size(); ++gi) {
        s3_graph_s *g = bt->graphs[gi];
        for (size_t k = 0; k < g->buckets.size(); ++k) {
            const HostBucket &hb = g->buckets[k];
            if (hb.m <= 0) continue;
            BatchBucket bb{};
            bb.b.ids = g->d_ids + hb.offset;
            bb.b.slot = g->d_slot + hb.offset;
            bb.b.m = hb.m;
            bb.b.ld = hb.ld;
            bb.b.s = hb.s;
            bb.b.N = g->N;
            bb.b.target = g->target[k];
            bb.b.K = g->K[k];
            bb.b.Km = g->Km[k];
            bb.b.Ke = g->Ke[k];
            bb.graph = (int32_t)gi;
            bb.W = g->N - hb.s + 1;
            size_t need_thread = (size_t)(2 * hb.s + (hb.s > 2 ? (hb.s - 2) * bb.W : 0)) * elem_bytes +
                                 (size_t)24 * hb.s;  // per thread
            bb.warp = (bb.W > bt->thread_max_w || need_thread * bs > 200 * 1024) ? 1 : 0;
            if (hb.s == 1) bb.warp = 2;
            if (bb.warp == 1) {
                int64_t pw = warp_smem_elems(std::max(hb.s, 1), bb.W);
                smem = std::max(smem, (size_t)(bs / 32) * (size_t)pw * elem_bytes);
            } else {
                smem = std::max(smem, need_thread * bs);
            }
            double W = bb.W;
            double fma = hb.s >= 3 ? (2.0 * hb.s - 5.0) * W * (W + 1) / 2 + hb.s * W : 2 * W;
            bt->bucket_cost.push_back(fma + 60.0 * hb.s);
            bt->h_buckets.push_back(bb);
        }
    }
    if (smem > 200 * 1024) return fail(S3_ENOTSUP, "batched tile needs more than 200 KiB of shared memory");
    // tiles are grouped into shared-memory classes, one persistent kernel each (run
    // concurrently), so that tiles of small edges are not held to the occupancy of the
    // widest tile; per-thread byte limits of the classes:
    const size_t class_limit[kBatchClasses] = {128, 320, 768, (size_t)1 << 40};
    std::vector<int> bucket_class(bt->h_buckets.size(), 0);
    std::vector<size_t> class_smem(kBatchClasses, 0);
    for (size_t bi = 0; bi < bt->h_buckets.size(); ++bi) {
        const BatchBucket &bb = bt->h_buckets[bi];
        size_t per_block;
        if (bb.warp == 2) per_block = 0;
        else if (bb.warp == 1) per_block = (size_t)(bs / 32) * (size_t)warp_smem_elems(bb.b.s, bb.W) * elem_bytes;
        else per_block = ((size_t)(2 * bb.b.s + (bb.b.s > 2 ? (bb.b.s - 2) * bb.W : 0)) * elem_bytes +
                          (size_t)24 * bb.b.s) * bs;
        const size_t per_thread = per_block / bs;
        int c = 0;
        while (c < kBatchClasses - 1 && per_thread > class_limit[c]) ++c;
        // every warp tile indexes its warp's region with the largest per-warp size, so all
        // warp tiles share the last class, whose reservation covers that size
        if (bb.warp == 1) c = kBatchClasses - 1;
        bucket_class[bi] = c;
        class_smem[c] = std::max(class_smem[c], per_block);
    }
    std::vector<std::vector<Tile>> tiles(kBatchClasses);
    std::vector<std::vector<double>> cost(kBatchClasses);
    const int64_t span = (int64_t)bs * bt->ept;
    for (size_t bi = 0; bi < bt->h_buckets.size(); ++bi) {
        const BatchBucket &bb = bt->h_buckets[bi];
        const int c = bucket_class[bi];
        const int64_t step = bb.warp == 1 ? (int64_t)(bs / 32) * bt->ept : span;
        for (int64_t e0 = 0; e0 < bb.b.m; e0 += step) {
            Tile t{};
            t.bucket = (int32_t)bi;
            t.e0 = e0;
            t.count = (int32_t)std::min<int64_t>(step, bb.b.m - e0);
            tiles[c].push_back(t);
            cost[c].push_back(bt->bucket_cost[bi] * t.count);
        }
    }
    std::vector<Tile> sorted;
    for (int c = 0; c < kBatchClasses; ++c) {
        std::vector<size_t> order(tiles[c].size());
        for (size_t i = 0; i < order.size(); ++i) order[i] = i;
        std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return cost[c][a] > cost[c][b]; });
        bt->cls[c].begin = (int64_t)sorted.size();
        for (size_t i = 0; i < order.size(); ++i) sorted.push_back(tiles[c][order[i]]);
        bt->cls[c].end = (int64_t)sorted.size();
        bt->cls[c].smem = class_smem[c];
    }
    // upload
    if ((int64_t)sorted.size() > bt->tiles_cap) {
        void *p = nullptr;
        s3_status st = batch_alloc(bt, &p, sizeof(Tile) * sorted.size());
        if (st != S3_OK) return st;
        bt->d_tiles = reinterpret_cast<Tile *>(p);
        bt->tiles_cap = (int64_t)sorted.size();
    }
    if (!bt->d_buckets) {
        void *p = nullptr;
        s3_status st = batch_alloc(bt, &p, sizeof(BatchBucket) * std::max<size_t>(1, bt->h_buckets.size()));
        if (st != S3_OK) return st;
        bt->d_buckets = reinterpret_cast<BatchBucket *>(p);
    }
    if (!sorted.empty())
        S3_CUDA(cudaMemcpy(bt->d_tiles, sorted.data(), sizeof(Tile) * sorted.size(), cudaMemcpyHostToDevice));
    if (!bt->h_buckets.empty())
        S3_CUDA(cudaMemcpy(bt->d_buckets, bt->h_buckets.data(), sizeof(BatchBucket) * bt->h_buckets.size(),
                           cudaMemcpyHostToDevice));
    bt->ntiles = (int64_t)sorted.size();
    bt->smem = smem;
    bt->built_eb = elem_bytes;
    bt->built_cfg = (bt->bs << 16) ^ (bt->ept << 8) ^ bt->thread_max_w;
    return S3_OK;
}

// Rebuild the tiles (and drop captured graphs) only when the configuration or element size changed.
s3_status ensure_tiles(s3_batch_s *bt, int elem_bytes) {
    const int cfg = (bt->bs << 16) ^ (bt->ept << 8) ^ bt->thread_max_w;
    if (bt->built_eb == elem_bytes && bt->built_cfg == cfg) return S3_OK;
    drop_graphs(bt);
    return build_tiles(bt, elem_bytes);
}

s3_status ensure_buffers(s3_batch_s *bt, int which, int elem_bytes) {
    if (bt->d_buf_mem[which]) return S3_OK;
    void *p = nullptr;
    s3_status st = batch_alloc(bt, &p, (size_t)bt->buf_elems * elem_bytes);
    if (st != S3_OK) return st;
    bt->d_buf_mem[which] = p;
    const size_t J = bt->graphs.size() * (size_t)bt->nvec;
    std::vector<void *> bufs(J);
    for (size_t j = 0; j < J; ++j) bufs[j] = (char *)p + (size_t)bt->buf_off[j] * elem_bytes;
    S3_CUDA(cudaMemcpy(bt->d_bufs + which * J, bufs.data(), sizeof(void *) * J, cudaMemcpyHostToDevice));
    return S3_OK;
}

template <typename T>
s3_status record_batch(s3_batch_s *bt, cudaStream_t st) {
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

s3_status capture(s3_batch_s *bt, int which) {
    if (bt->exec[which]) return S3_OK;
    if (!bt->cap_stream) S3_CUDA(cudaStreamCreateWithFlags(&bt->cap_stream, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    S3_CUDA(cudaStreamBeginCapture(bt->cap_stream, cudaStreamCaptureModeThreadLocal));
    s3_status s = which == 0 ? record_batch<float>(bt, bt->cap_stream) : record_batch<double>(bt, bt->cap_stream);
    cudaError_t ce = cudaStreamEndCapture(bt->cap_stream, &graph);
    if (s != S3_OK) {
        if (graph) cudaGraphDestroy(graph);
        return s;
    }
    S3_CUDA(ce);
    ce = cudaGraphInstantiate(&bt->exec[which], graph, 0);
    cudaGraphDestroy(graph);
    S3_CUDA(ce);
    return S3_OK;
}

s3_status run_batch(s3_batch_s *bt, s3_dtype dt, const void *const *x, void *const *y, cudaStream_t st) {
    const int which = dt == S3_F32 ? 0 : 1;
    const int eb = dt == S3_F32 ? 4 : 8;
    s3_status s = ensure_buffers(bt, which, eb);
    if (s != S3_OK) return s;
    const size_t J = bt->graphs.size() * (size_t)bt->nvec;
    // the pinned pointer staging is read by the first copy of every replay: when the
    // caller passes new pointers, wait for earlier replays before overwriting it
    bool same = bt->staged;
    for (size_t j = 0; j < J && same; ++j) same = bt->h_ptrs[j] == x[j] && bt->h_ptrs[J + j] == y[j];
    if (!same) {
        S3_CUDA(cudaStreamSynchronize(st));
        if (bt->cap_stream) S3_CUDA(cudaStreamSynchronize(bt->cap_stream));
        for (size_t j = 0; j < J; ++j) {
            bt->h_ptrs[j] = const_cast<void *>(x[j]);
            bt->h_ptrs[J + j] = y[j];
        }
        bt->staged = true;
    }
    if (bt->opt.use_graph) {
        s = capture(bt, which);
        if (s != S3_OK) return s;
        S3_CUDA(cudaGraphLaunch(bt->exec[which], st));
        return S3_OK;
    }
    return which == 0 ? record_batch<float>(bt, st) : record_batch<double>(bt, st);
}

}  // namespace

extern "C" {

s3_status s3_batch_options_init(s3_batch_options *opt) {
    if (!opt) return fail(S3_EINVAL, "opt is NULL");
    std::memset(opt, 0, sizeof(*opt));
    opt->use_graph = 1;
    return S3_OK;
}

s3_status s3_batch_create(int32_t count, const s3_graph_t *graphs, int32_t nvec, const s3_batch_options *opt_in,
                          s3_batch_t *out) {
    if (!out) return fail(S3_EINVAL, "out is NULL");
    *out = nullptr;
    if (count < 1 || !graphs) return fail(S3_EINVAL, "count must be >= 1 and graphs non-NULL");
    if (nvec < 1 || nvec > 1024) return fail(S3_EINVAL, "nvec must be in 1..1024");
    s3_batch_options opt;
    if (opt_in) opt = *opt_in;
    else s3_batch_options_init(&opt);
    for (int32_t i = 0; i < count; ++i) {
        if (!graphs[i]) return fail(S3_EINVAL, "NULL graph in the batch");
        if (graphs[i]->device != graphs[0]->device) return fail(S3_EINVAL, "graphs live on different devices");
        if (graphs[i]->opt.reduce != S3_REDUCE_SEGMENTED) return fail(S3_EINVAL, "batched calls need the segmented reduce");
    }
    s3_batch_s *bt = new (std::nothrow) s3_batch_s();
    if (!bt) return fail(S3_ENOMEM, "host allocation failed");
    bt->device = graphs[0]->device;
    DeviceGuard guard(bt->device);
    bt->graphs.assign(graphs, graphs + count);
    bt->nvec = nvec;
    bt->opt = opt;
    bt->bs = opt.block_threads > 0 ? opt.block_threads : 128;
    bt->ept = opt.edges_per_thread > 0 ? opt.edges_per_thread : 4;
    bt->thread_max_w = opt.thread_max_w > 0 ? std::min(opt.thread_max_w, 32) : 32;
    auto bail = [&](s3_status s) {
        drop_graphs(bt);
        free_streams(bt);
        for (void *p : bt->allocations) cudaFree(p);
        if (bt->h_ptrs) cudaFreeHost(bt->h_ptrs);
        delete bt;
        return s;
    };
    if (bt->bs % 32 || bt->bs > 256) return bail(fail(S3_EINVAL, "block_threads must be a multiple of 32 up to 256"));
    if (cudaEventCreateWithFlags(&bt->ev_fork, cudaEventDisableTiming) != cudaSuccess)
        return bail(cuda_fail(cudaGetLastError(), "cudaEventCreate"));
    for (int c = 0; c < kBatchClasses; ++c)
        if (cudaStreamCreateWithFlags(&bt->aux[c], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&bt->ev_join[c], cudaEventDisableTiming) != cudaSuccess)
            return bail(cuda_fail(cudaGetLastError(), "cudaStreamCreate"));
    if (cudaDeviceGetAttribute(&bt->sms, cudaDevAttrMultiProcessorCount, bt->device) != cudaSuccess)
        return bail(cuda_fail(cudaGetLastError(), "cudaDeviceGetAttribute"));
    s3_status s = S3_OK;
    if (cudaFuncSetAttribute(batch_edge_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) !=
            cudaSuccess ||
        cudaFuncSetAttribute(batch_edge_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) !=
            cudaSuccess)
        return bail(cuda_fail(cudaGetLastError(), "cudaFuncSetAttribute"));
    const size_t J = (size_t)count * nvec;
    // buffers and partial offsets per (graph, vector)
    for (int32_t gi = 0; gi < count; ++gi)
        for (int32_t v = 0; v < nvec; ++v) {
            bt->buf_off.push_back(bt->buf_elems);
            bt->buf_elems += std::max<int64_t>(graphs[gi]->nnz, 1);
            bt->part_off.push_back(bt->part_elems);
            bt->part_elems += std::max<int64_t>(graphs[gi]->n_pieces, 1);
        }
    void *p = nullptr;
    if ((s = batch_alloc(bt, &p, sizeof(void *) * J * 2)) != S3_OK) return bail(s);
    bt->d_xs = reinterpret_cast<void **>(p);
    bt->d_ys = bt->d_xs + J;
    if ((s = batch_alloc(bt, &p, sizeof(void *) * J * 2)) != S3_OK) return bail(s);
    bt->d_bufs = reinterpret_cast<void **>(p);
    if ((s = batch_alloc(bt, &p, sizeof(void *) * J)) != S3_OK) return bail(s);
    bt->d_parts = reinterpret_cast<void **>(p);
    if ((s = batch_alloc(bt, &p, (size_t)bt->part_elems * 8)) != S3_OK) return bail(s);
    bt->d_part_mem = p;
    {
        std::vector<void *> parts(J);
        for (size_t j = 0; j < J; ++j) parts[j] = (char *)bt->d_part_mem + (size_t)bt->part_off[j] * 8;
        if (cudaMemcpy(bt->d_parts, parts.data(), sizeof(void *) * J, cudaMemcpyHostToDevice) != cudaSuccess)
            return bail(cuda_fail(cudaGetLastError(), "cudaMemcpy"));
    }
    if ((s = batch_alloc(bt, &p, (kBatchClasses + 1) * sizeof(unsigned long long))) != S3_OK) return bail(s);
    bt->d_counters = reinterpret_cast<unsigned long long *>(p);
    if (cudaHostAlloc(reinterpret_cast<void **>(&bt->h_ptrs), sizeof(void *) * J * 2, cudaHostAllocDefault) !=
        cudaSuccess)
        return bail(cuda_fail(cudaGetLastError(), "cudaHostAlloc"));
    // reduce tables
    std::vector<ReduceGraph> rg(count);
    std::vector<ReduceTile> rtiles;
    std::vector<FinalTile> finals;
    for (int32_t gi = 0; gi < count; ++gi) {
        s3_graph_s *g = graphs[gi];
        ReduceGraph r{};
        r.inc_ptr = g->d_inc_ptr;
        r.small_nodes = g->d_small;
        r.med_nodes = g->d_med;
        r.big_nodes = g->d_big_nodes;
        r.big_piece_ptr = g->d_big_piece_ptr;
        r.piece_len = g->d_piece_len;
        r.piece_start = g->d_piece_start;
        r.n_small = g->n_small;
        r.n_med = g->n_med;
        r.n_big = g->n_big;
        r.n_pieces = g->n_pieces;
        rg[gi] = r;
        for (int64_t f = 0; f < g->n_pieces; ++f) rtiles.push_back({gi, 2, f});
        for (int64_t f = 0; f < g->n_med; f += 8) rtiles.push_back({gi, 1, f});
        for (int64_t f = 0; f < g->n_small; f += 256) rtiles.push_back({gi, 0, f});
        for (int64_t k = 0; k < g->n_big; ++k) finals.push_back({gi, (int32_t)k});
    }
    if ((s = batch_alloc(bt, &p, sizeof(ReduceGraph) * rg.size())) != S3_OK) return bail(s);
    bt->d_rgraphs = reinterpret_cast<ReduceGraph *>(p);
    if ((s = batch_alloc(bt, &p, sizeof(ReduceTile) * std::max<size_t>(1, rtiles.size()))) != S3_OK) return bail(s);
    bt->d_rtiles = reinterpret_cast<ReduceTile *>(p);
    if ((s = batch_alloc(bt, &p, sizeof(FinalTile) * std::max<size_t>(1, finals.size()))) != S3_OK) return bail(s);
    bt->d_finals = reinterpret_cast<FinalTile *>(p);
    if (cudaMemcpy(bt->d_rgraphs, rg.data(), sizeof(ReduceGraph) * rg.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        (!rtiles.empty() && cudaMemcpy(bt->d_rtiles, rtiles.data(), sizeof(ReduceTile) * rtiles.size(),
                                       cudaMemcpyHostToDevice) != cudaSuccess) ||
        (!finals.empty() && cudaMemcpy(bt->d_finals, finals.data(), sizeof(FinalTile) * finals.size(),
                                       cudaMemcpyHostToDevice) != cudaSuccess))
        return bail(cuda_fail(cudaGetLastError(), "cudaMemcpy"));
    bt->nrtiles = (int64_t)rtiles.size();
    bt->nfinals = (int64_t)finals.size();
    if ((s = ensure_tiles(bt, 4)) != S3_OK) return bail(s);
    *out = bt;
    return S3_OK;
}

s3_status s3_sttsvc_batched(s3_batch_t bt, s3_dtype dt, const void *const *x, void *const *y, void *stream) {
    if (!bt || !x || !y) return fail(S3_EINVAL, "NULL argument");
    if (dt != S3_F32 && dt != S3_F64) return fail(S3_EINVAL, "bad dtype");
    const size_t J = bt->graphs.size() * (size_t)bt->nvec;
    for (size_t j = 0; j < J; ++j)
        if (!x[j] || !y[j]) return fail(S3_EINVAL, "NULL vector pointer");
    DeviceGuard guard(bt->device);
    // the shared-memory need depends on the element size
    s3_status s = ensure_tiles(bt, dt == S3_F32 ? 4 : 8);
    if (s != S3_OK) return s;
    return run_batch(bt, dt, x, y, (cudaStream_t)stream);
}

s3_status s3_batch_autotune(s3_batch_t bt, s3_dtype dt, const void *const *x, void *const *y, s3_tune_result *res,
                            void *stream) {
    if (!bt || !x || !y || !res) return fail(S3_EINVAL, "NULL argument");
    DeviceGuard guard(bt->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int eb = dt == S3_F32 ? 4 : 8;
    std::memset(res, 0, sizeof(*res));
    const int bss[] = {64, 128, 256};
    const int epts[] = {1, 4, 16};
    const int tws[] = {16, 32};
    cudaEvent_t e0, e1;
    S3_CUDA(cudaEventCreate(&e0));
    S3_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    int best_bs = bt->bs, best_ept = bt->ept, best_tw = bt->thread_max_w;
    int tried = 0;
    for (int tw : tws)
        for (int bs : bss)
            for (int ept : epts) {
                bt->bs = bs;
                bt->ept = ept;
                bt->thread_max_w = tw;
                s3_status s = ensure_tiles(bt, eb);
                if (s != S3_OK) continue;  // configuration does not fit
                s = run_batch(bt, dt, x, y, st);  // warm-up (and capture)
                if (s != S3_OK) continue;
                float ms_sum = 0.f;
                bool ok = true;
                for (int r = 0; r < 3 && ok; ++r) {
                    cudaEventRecord(e0, st);
                    ok = run_batch(bt, dt, x, y, st) == S3_OK;
                    cudaEventRecord(e1, st);
                    cudaEventSynchronize(e1);
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    ms_sum += ms;
                }
                if (!ok) continue;
                float ms = ms_sum / 3.f;
                if (tried < 32) {
                    res->candidates[tried].block_threads = bs;
                    res->candidates[tried].edges_per_thread = ept;
                    res->candidates[tried].thread_max_w = tw;
                    res->candidates[tried].ms = ms;
                }
                ++tried;
                if (ms < best) {
                    best = ms;
                    best_bs = bs;
                    best_ept = ept;
                    best_tw = tw;
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (tried == 0) return fail(S3_ENOTSUP, "no batched configuration could run");
    bt->bs = best_bs;
    bt->ept = best_ept;
    bt->thread_max_w = best_tw;
    s3_status s = ensure_tiles(bt, eb);
    if (s != S3_OK) return s;
    res->block_threads = best_bs;
    res->edges_per_thread = best_ept;
    res->thread_max_w = best_tw;
    res->ms = best;
    res->tried = tried;
    if (bt->opt.cache_path[0]) {
        std::ofstream f(bt->opt.cache_path, std::ios::app);
        if (f) {
            int64_t tot = 0;
            for (auto *g : bt->graphs) tot += g->nnz;
            f << "s3_batch count=" << bt->graphs.size() << " nvec=" << bt->nvec << " nnz=" << tot << " dtype=" << eb
              << " block_threads=" << best_bs << " edges_per_thread=" << best_ept << " thread_max_w=" << best_tw
              << " ms=" << best << "\n";
        }
    }
    return S3_OK;
}

s3_status s3_batch_destroy(s3_batch_t bt) {
    if (!bt) return S3_OK;
    {
        DeviceGuard guard(bt->device);
        cudaDeviceSynchronize();
        drop_graphs(bt);
        free_streams(bt);
        if (bt->cap_stream) cudaStreamDestroy(bt->cap_stream);
        for (void *p : bt->allocations) cudaFree(p);
        if (bt->h_ptrs) cudaFreeHost(bt->h_ptrs);
    }
    delete bt;
    return S3_OK;
}

}  // extern "C"
