// The graph handle (internal).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "s3_internal.h"
#include "s3_kernels.h"

struct s3_graph_s {
    int device = 0;
    s3_options opt{};
    int64_t n = 0, m = 0, nnz = 0;
    int32_t N = 0;
    s3_format_info info{};

    // size buckets (host copy of the layout) and per-bucket constants
    std::vector<s3::HostBucket> buckets;
    std::vector<double> K;        // per bucket
    std::vector<float> Km;
    std::vector<int32_t> Ke;
    std::vector<float> target;

    // device format
    int32_t *d_ids = nullptr, *d_slot = nullptr;
    int64_t *d_inc_ptr = nullptr;
    int64_t *d_grp_off = nullptr;
    int32_t *d_grp_node = nullptr;
    uint8_t *d_grp_deg = nullptr;
    int32_t *d_med8 = nullptr, *d_med8_len = nullptr;
    int64_t *d_med8_off = nullptr;
    int32_t *d_med = nullptr, *d_med_len = nullptr;
    int64_t *d_med_off = nullptr;
    int32_t *d_big_nodes = nullptr, *d_big_piece_ptr = nullptr, *d_piece_big = nullptr;
    int32_t *d_big_count = nullptr;  // n_big, zero between calls
    int64_t *d_piece_start = nullptr;
    int32_t *d_piece_len = nullptr;
    int64_t n_grp = 0, n_med8 = 0, n_med = 0, n_big = 0, n_pieces = 0;
    int64_t buf_len = 0;            // slots of the per-(edge, node) buffer (nnz plus group padding)

    // scratch owned by the handle (reused by every call)
    void *d_buf = nullptr;          // buf_len values (8 bytes each) for the segmented reduce
    void *d_partial = nullptr;      // n_pieces partial sums (8 bytes each)
    float *d_comp = nullptr;        // n FP32 compensation terms (atomic mode)
    unsigned long long *d_range = nullptr;
    void *d_xh = nullptr, *d_yh = nullptr;   // n values each, staging for s3_sttsvc_host

    // CCSS forest on the device (S3_LAYOUT_CCSS)
    bool has_ccss = false;
    struct CcssSeg { int32_t level, width; int64_t begin, end; };
    struct CcssLeaf { int32_t s; int64_t begin, end; double K; float Km; int32_t Ke; };
    std::vector<CcssSeg> ccss_segs;
    std::vector<CcssLeaf> ccss_leaves;
    std::vector<float> cc_level_target;  // per-level rescaling targets
    int32_t *d_cc_vertex = nullptr, *d_cc_parent = nullptr, *d_cc_width = nullptr;
    int64_t *d_cc_off = nullptr;
    int32_t *d_leaf_node = nullptr, *d_leaf_vertex = nullptr, *d_leaf_slot = nullptr;
    void *d_cc_values = nullptr;    // value_len coefficients (8 bytes each)
    int64_t cc_value_len = 0;
    int32_t *d_cc_scale = nullptr;  // global rescaling exponent of the last CCSS call

    // NQZ scratch
    double *d_nqz = nullptr;        // 4 n doubles: x, u, z (FP64), spare
    float *d_x32 = nullptr, *d_z32 = nullptr;
    double *d_red = nullptr;        // reduction partials
    int32_t *d_flags = nullptr;     // [0] done, [1] phase-switch, ...
    double *d_hist = nullptr;       // per-iteration (lmin, lmax)
    double *d_zeig = nullptr;       // SS-HOPM / symmetric CP reduction partials and scalars
    int32_t hist_cap = 0;
    int64_t first_isolated = -1;    // a node of degree 0 (NQZ rejects the handle), or -1
    // captured NQZ passes, kept for later calls with the same settings: one per series type
    struct NqzExec {
        cudaGraphExec_t exec = nullptr;
        double tol = 0.0;
        int32_t max_iter = 0, check_every = 0;
        const double *hist = nullptr;
    } nqz_exec[3];

    int32_t last_launches = 0;       // kernels launched by the last S^3TTVc call
    // completion of the handle's last call (recorded on that call's stream unless the stream
    // was being captured), the stream of the counter queries, and two pinned words that a
    // range-checked call reads the range counter into (before, after)
    cudaEvent_t ev_done = nullptr;
    cudaStream_t qstream = nullptr;
    // the host-buffer entry point's call, captured once per series type (x and y are the
    // handle's staging buffers, so the graph never changes); the stream it was captured on
    cudaGraphExec_t host_exec[3] = {nullptr, nullptr, nullptr};
    cudaStream_t cap_stream = nullptr;
    unsigned long long *h_range = nullptr;
    uint32_t *d_feat_scratch = nullptr;  // warm-start feature partials (64 bytes per hub piece)
    s3::TailEntry *d_feat_tab = nullptr; // buckets of the fused feature launch (size bin in W)
    int32_t n_feat_tab = 0;
    int64_t feat_blocks = 0;
    float *d_ws = nullptr;               // warm-start features, predictions, partials
    // concurrent buckets: forked streams and events, bucket order (heaviest first) and cost
    int n_streams = 1;
    cudaStream_t aux[8] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t ev_fork = nullptr;
    cudaEvent_t ev_join[8] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    std::vector<size_t> bucket_order;
    std::vector<double> bucket_cost;
    // small buckets fused into one launch (one edge per thread)
    std::vector<char> in_tail;          // per bucket
    s3::TailEntry *d_tail = nullptr;    // device table, ascending block0
    int32_t n_tail = 0;
    int32_t tail_bs = 64;
    int64_t tail_blocks = 0;
    size_t tail_smem[2] = {0, 0};       // dynamic shared memory of the launch (FP32, FP64)
    double tail_cost = 0.0;
    // closed-form evaluation of small buckets: per bucket a bit mask of the call types
    // that use it (1 = FP32, 2 = FP64) and its constants; d_closed_list holds every such
    // bucket's rejected-edge list, d_closed_count four counters per bucket ([0] list
    // length, cleared at the start of every call; [2..3] rejected edges in total)
    std::vector<int32_t> closed_mask;
    // Bernoulli-form buckets (s3_bern.cuh): per bucket a bit mask of the call types that use
    // it (1 = FP32, 2 = FP64); per call type a device table of those buckets (ascending
    // block0, heaviest first) for the one launch that evaluates them all
    std::vector<int32_t> bern_mask;
    s3::TailEntry *d_bern[2] = {nullptr, nullptr};
    int32_t n_bern[2] = {0, 0};
    int64_t bern_blocks[2] = {0, 0};
    int32_t bern_lane[2] = {0, 0}, bern_fb[2] = {0, 0};
    double bern_cost[2] = {0.0, 0.0};
    s3::BernArgs bern_args{};
    unsigned long long *d_bern_rejected = nullptr;
    std::vector<s3::ClosedArgs> closed_args;
    int32_t *d_closed_list = nullptr;
    int32_t *d_closed_count = nullptr;
    std::vector<void *> allocations;
    int64_t device_bytes = 0;
};

namespace s3 {

// Allocate count elements on the handle's device and remember the block.
template <typename T>
s3_status dev_alloc(s3_graph_s *g, T **p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(S3_ENOMEM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
    }
    g->allocations.push_back(q);
    g->device_bytes += (int64_t)(count * sizeof(T));
    *p = reinterpret_cast<T *>(q);
    return S3_OK;
}

// RAII: make the handle's device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    bool changed = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) {
            changed = cudaSetDevice(dev) == cudaSuccess;
        }
    }
    ~DeviceGuard() {
        if (changed) cudaSetDevice(prev);
    }
};

s3_status cuda_fail(cudaError_t e, const char *what);
s3_status prepare_device(int dev);
// Record the completion of a call's work on st (skipped while st is being captured).
s3_status mark_done(s3_graph_s *g, cudaStream_t st);
// mid (optional) is recorded on st between the edge kernels and the reduce; bern (optional,
// two events) around the Bernoulli launch on the stream it runs on
s3_status run_edges(s3_graph_s *g, s3_dtype dt, const void *x, void *y, int bias, const int32_t *skip,
                    cudaStream_t st, cudaEvent_t mid = nullptr, cudaEvent_t *bern = nullptr);
s3_status run_ccss(s3_graph_s *g, s3_dtype dt, const void *x, void *y, int bias, const int32_t *skip,
                   cudaStream_t st);
s3_status upload_ccss(s3_graph_s *g, const HostFormat &f);

// Arguments of the segmented reduce over the handle's slot buffer.
inline ReduceArgs reduce_args(const s3_graph_s *g, const int32_t *skip) {
    ReduceArgs r{};
    r.grp_off = g->d_grp_off;
    r.grp_node = g->d_grp_node;
    r.grp_deg = g->d_grp_deg;
    r.n_grp = g->n_grp;
    r.med8_nodes = g->d_med8;
    r.med8_off = g->d_med8_off;
    r.med8_len = g->d_med8_len;
    r.n_med8 = g->n_med8;
    r.med_nodes = g->d_med;
    r.med_off = g->d_med_off;
    r.med_len = g->d_med_len;
    r.n_med = g->n_med;
    r.piece_start = g->d_piece_start;
    r.piece_len = g->d_piece_len;
    r.n_pieces = g->n_pieces;
    r.big_nodes = g->d_big_nodes;
    r.big_piece_ptr = g->d_big_piece_ptr;
    r.piece_big = g->d_piece_big;
    r.big_count = g->d_big_count;
    r.n_big = g->n_big;
    r.partial = g->d_partial;
    r.skip = skip;
    return r;
}

}  // namespace s3

#define S3_CUDA(expr)                                   \
    do {                                                \
        cudaError_t _e = (expr);                        \
        if (_e != cudaSuccess) return s3::cuda_fail(_e, #expr); \
    } while (0)
