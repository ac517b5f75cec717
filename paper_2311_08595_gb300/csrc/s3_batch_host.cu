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

#include "s3_batch.h"
#include "s3_series.cuh"

using namespace s3;

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
    // the buckets each graph evaluates in the Bernoulli form for this element type, and the
    // per-warp shared memory those tiles need (one size for all of them)
    const int bern_bit = elem_bytes == 4 ? 1 : 2;
    bt->bern_lane = 0;
    bt->bern_fb = 0;
    for (s3_graph_s *g : bt->graphs)
        for (size_t k = 0; k < g->buckets.size(); ++k)
            if (k < g->bern_mask.size() && (g->bern_mask[k] & bern_bit) && g->buckets[k].m > 0) {
                const int s = g->buckets[k].s;
                bt->bern_lane = std::max(bt->bern_lane, elem_bytes == 4 ? s : s + (s + 1) / 2);
                bt->bern_fb = std::max(bt->bern_fb, (int32_t)warp_smem_elems(s, g->N - s + 1));
            }
    const size_t bern_block = (size_t)(bs / 32) * ((size_t)32 * bt->bern_lane + bt->bern_fb) * elem_bytes;
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
            if (k < g->bern_mask.size() && (g->bern_mask[k] & bern_bit) && bern_block <= 200 * 1024) bb.warp = 3;
            if (bb.warp == 3) {
                smem = std::max(smem, bern_block);
            } else if (bb.warp == 1) {
                int64_t pw = warp_smem_elems(std::max(hb.s, 1), bb.W);
                smem = std::max(smem, (size_t)(bs / 32) * (size_t)pw * elem_bytes);
            } else {
                smem = std::max(smem, need_thread * bs);
            }
            double W = bb.W;
            double fma = bb.warp == 3 ? (elem_bytes == 4 ? hb.s * W * (W - 1) / 2 : 2.0 * hb.s * W + W * (W - 1))
                         : hb.s >= 3 ? (2.0 * hb.s - 5.0) * W * (W + 1) / 2 + hb.s * W : 2 * W;
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
        else if (bb.warp == 3) per_block = bern_block;
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

s3_status capture(s3_batch_s *bt, int which) {
    if (bt->exec[which]) return S3_OK;
    if (!bt->cap_stream) S3_CUDA(cudaStreamCreateWithFlags(&bt->cap_stream, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    S3_CUDA(cudaStreamBeginCapture(bt->cap_stream, cudaStreamCaptureModeThreadLocal));
    s3_status s = which == 0 ? record_batch_f32(bt, bt->cap_stream) : record_batch_f64(bt, bt->cap_stream);
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
    return which == 0 ? record_batch_f32(bt, st) : record_batch_f64(bt, st);
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
    if (prepare_batch_f32() != cudaSuccess || prepare_batch_f64() != cudaSuccess)
        return bail(cuda_fail(cudaGetLastError(), "cudaFuncSetAttribute"));
    const size_t J = (size_t)count * nvec;
    // buffers and partial offsets per (graph, vector)
    for (int32_t gi = 0; gi < count; ++gi)
        for (int32_t v = 0; v < nvec; ++v) {
            bt->buf_off.push_back(bt->buf_elems);
            bt->buf_elems += std::max<int64_t>(graphs[gi]->buf_len, 1);
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
        rg[gi] = reduce_args(g, nullptr);
        for (int64_t f = 0; f < g->n_pieces; ++f) rtiles.push_back({gi, 2, f});
        for (int64_t f = 0; f < g->n_med; f += 8) rtiles.push_back({gi, 1, f});
        for (int64_t f = 0; f < g->n_med8; f += 32) rtiles.push_back({gi, 3, f});
        for (int64_t f = 0; f < g->n_grp; f += 8) rtiles.push_back({gi, 0, f});
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
    s = run_batch(bt, dt, x, y, (cudaStream_t)stream);
    if (s != S3_OK) return s;
    // the batch writes the first graph's range counter: later queries on it wait for this call
    return bt->graphs.empty() ? S3_OK : mark_done(bt->graphs[0], (cudaStream_t)stream);
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
