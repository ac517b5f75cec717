// Batched S^3TTVc: declarations shared by the host side and the per-type kernel units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "s3_graph.h"

namespace s3 {


constexpr int kBatchClasses = 4;

struct BatchBucket {
    EdgeBucketArgs b;
    int32_t graph;
    int32_t W;
    int32_t warp;  // 0: one thread per edge (series), 1: one warp per edge, 2: size 1, 3: Bernoulli form
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
    int32_t bern_lane;      // Bernoulli tiles: values per lane of a warp's region
    int32_t bern_fb;        // Bernoulli tiles: values of the warp's series-fallback region
    BernArgs bern;          // Bernoulli constants (s3_bern.cuh)
};

// per-graph reduce tables (the partial and skip fields are unused here)
using ReduceGraph = ReduceArgs;

struct ReduceTile {
    int32_t graph;
    int32_t kind;   // 0: 8 groups of 32 small nodes, 1: 8 medium nodes, 2: one hub piece,
                    // 3: 32 medium nodes of degree <= 128
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

}  // namespace s3

using s3::BatchBucket;
using s3::FinalTile;
using s3::kBatchClasses;
using s3::ReduceGraph;
using s3::ReduceTile;
using s3::Tile;

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
    int32_t bern_lane = 0, bern_fb = 0;        // Bernoulli tiles' per-warp shared memory (values)
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

namespace s3 {
// record one batched call (edge classes, reduce, hub pass) on st
s3_status record_batch_f32(s3_batch_s *bt, cudaStream_t st);
s3_status record_batch_f64(s3_batch_s *bt, cudaStream_t st);
cudaError_t prepare_batch_f32();
cudaError_t prepare_batch_f64();
}  // namespace s3
