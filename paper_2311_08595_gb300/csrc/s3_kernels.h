// Host-callable launchers of the device kernels (internal to the library).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace s3 {

// One size bucket as the edge kernels see it.
struct EdgeBucketArgs {
    const int32_t *ids;   // member i of bucket edge k at ids[i * ld + k] (sorted members)
    const int32_t *slot;  // same layout: node-sorted incidence slot (segmented reduce), or nullptr
    int64_t m;            // edges in the bucket
    int64_t ld;
    int32_t s, N;         // edge size and rank
    float target;         // rescaling target T(s,N)
    double K;             // K(s,N) = s (N-1)! / (s! S(N,s))
    float Km;             // K = Km * 2^Ke with Km in [0.5, 1)
    int32_t Ke;
    // list mode (the thread-per-edge and size-2 kernels): process only the bucket
    // edges list[0 .. count[0]) instead of all m; count[2..3] is a running total of
    // the list lengths
    const int32_t *list;
    int32_t *count;
};

// The closed-form (inclusion-exclusion) kernels of s3_closed.cuh.  Edges whose
// error bound fails are appended to fail_list (bucket edge indices; fail_count[0]
// entries) for the series kernels in list mode.
struct ClosedArgs {
    int32_t *fail_list;
    int32_t *fail_count;
    double Ki;            // K(s,N) / (N-1)!
    float Kim;            // Ki = Kim * 2^Kie with Kim in [0.5, 1)
    int32_t Kie;
    double gate;          // an edge passes when every R_v > gate * sum_U |p_U|
};

// One small bucket of the fused small-bucket launch (device table, built once
// per handle): its edges occupy blocks [block0, block0 + ceil(m / threads)).
struct TailEntry {
    EdgeBucketArgs b;
    int32_t W;            // N - s + 1
    int32_t pad;
    int64_t block0;
};

// Elements per warp of the shared memory of one warp-per-edge series evaluation
// (warp_edge_compute in s3_series.cuh): Xs[s] | C[s] | Pre[(s-2) W] | 4 windows of W.
__host__ __device__ constexpr int64_t warp_smem_elems(int s, int W) {
    return ((2 * (int64_t)s + (int64_t)(s > 2 ? s - 2 : 0) * W + 4 * (int64_t)W) + 3) / 4 * 4;
}

// Constants of the Bernoulli-series kernels (s3_bern.cuh): beta_k = B_k^+ / k!
// (Bernoulli numbers, B_1 = +1/2; zero for odd k >= 3), k < 32, and the largest
// accepted amplification (P + Q) / (P - Q) of the alternating sum.
struct BernArgs {
    float beta32[32];
    double beta64[32];
    float kmax32;
    double kmax64;
    unsigned long long *rejected;   // running count of edges sent back to the series
};
constexpr int kBernThreads = 128;   // threads per block of the Bernoulli launch (one edge each)
// Dynamic shared memory of a Bernoulli launch: per warp 32 lanes x lane_elems values plus
// fb_elems values for the series fallback.
inline size_t bern_smem_bytes(int lane_elems, int fb_elems, size_t value_bytes) {
    return (size_t)(kBernThreads / 32) * ((size_t)32 * lane_elems + (size_t)fb_elems) * value_bytes;
}

enum OutMode : int32_t {
    kOutBuffer = 0,       // out[slot] = c
    kOutAtomic = 1,       // out[v] += c (atomics)
    kOutAtomicComp = 2    // FP32: out[v] += c with a two-sum compensation term in comp[v]
};

struct EdgeOutArgs {
    void *out;                          // buffer (nnz) or y (n), element type of the call
    float *comp;                        // FP32 compensation (n) for kOutAtomicComp
    int32_t mode;                       // OutMode
    int32_t bias;                       // 1: scale node v's results by 2^(-(N-1) e_v), x_v = m 2^e_v, m in [0.5,1)
    unsigned long long *range_events;   // incremented for results that leave the normal range
    const int32_t *skip;                // if non-null and *skip != 0 the kernel returns at once
};

// Launch the kernel for one bucket (s >= 1).  thread_max_w: windows up to this
// use one thread per edge; block_threads: threads per block of that kernel.
cudaError_t launch_edge_bucket_f32(const EdgeBucketArgs &b, const float *x, const EdgeOutArgs &o,
                                   int thread_max_w, int block_threads, cudaStream_t st);
cudaError_t launch_edge_bucket_f64(const EdgeBucketArgs &b, const double *x, const EdgeOutArgs &o,
                                   int thread_max_w, int block_threads, cudaStream_t st);
// FP64 x and results, series in double-float (pairs of FP32); size-1 edges and windows
// wider than 24 go to the FP64 kernels.  Small buckets are not fused for it.
cudaError_t launch_edge_bucket_df(const EdgeBucketArgs &b, const double *x, const EdgeOutArgs &o,
                                  int thread_max_w, int block_threads, cudaStream_t st);
// Fused launch of small buckets: tab (device) lists ntab buckets by ascending
// block0; nblocks blocks of bs threads; smem bytes of dynamic shared memory,
// bs * the largest edge_tail_smem_words of the entries * 4.
cudaError_t launch_edge_tail_f32(const TailEntry *tab, int ntab, int64_t nblocks, int bs, size_t smem,
                                 const float *x, const EdgeOutArgs &o, cudaStream_t st);
cudaError_t launch_edge_tail_f64(const TailEntry *tab, int ntab, int64_t nblocks, int bs, size_t smem,
                                 const double *x, const EdgeOutArgs &o, cudaStream_t st);
// 4-byte words of shared memory per thread of the fused launch for an edge of size s
// and window W, values of value_bytes bytes.
inline size_t edge_tail_smem_words(int s, int W, int value_bytes) {
    return (size_t)(s + (s > 2 ? (s - 2) * W : 0)) * (size_t)value_bytes / 4 + (size_t)2 * s;
}
constexpr size_t kEdgeSmemCap = 96 * 1024;   // dynamic shared memory per block of the thread kernels
// Buckets with wide windows: eight lanes per edge (s3_group.cuh; FP32 only).  Sets
// *launched = 1 if it launched, 0 if it did not (FP64, or edges too large for the
// kernel's shared memory): the caller then uses one warp per edge.
cudaError_t launch_edge_group(const EdgeBucketArgs &b, const float *x, const EdgeOutArgs &o, int W, cudaStream_t st,
                              int *launched);
cudaError_t launch_edge_group(const EdgeBucketArgs &b, const double *x, const EdgeOutArgs &o, int W, cudaStream_t st,
                              int *launched);
cudaError_t prepare_edge_group(float);
cudaError_t prepare_edge_group(double);
// Closed-form evaluation of one bucket (2 <= s <= 6, 2 <= N-1 <= 127); edges that
// fail the error gate go to c.fail_list.  FP32 and FP64.
cudaError_t launch_edge_closed_f32(const EdgeBucketArgs &b, const float *x, const EdgeOutArgs &o,
                                   const ClosedArgs &c, cudaStream_t st);
cudaError_t launch_edge_closed_f64(const EdgeBucketArgs &b, const double *x, const EdgeOutArgs &o,
                                   const ClosedArgs &c, cudaStream_t st);
constexpr int kClosedMaxS = 6;
// One launch of every Bernoulli bucket of a call (tab: device, ascending block0,
// kBernThreads threads per block, one edge per thread).  FP32 and FP64.
cudaError_t launch_edge_bern_f32(const TailEntry *tab, int ntab, int64_t nblocks, int lane_elems, int fb_elems,
                                 const float *x, const EdgeOutArgs &o, const BernArgs &c, cudaStream_t st);
cudaError_t launch_edge_bern_f64(const TailEntry *tab, int ntab, int64_t nblocks, int lane_elems, int fb_elems,
                                 const double *x, const EdgeOutArgs &o, const BernArgs &c, cudaStream_t st);
// the biased output mode (o.bias != 0), each in a translation unit of its own
cudaError_t launch_edge_bern_f32_bias(const TailEntry *tab, int ntab, int64_t nblocks, int lane_elems, int fb_elems,
                                      const float *x, const EdgeOutArgs &o, const BernArgs &c, cudaStream_t st);
cudaError_t launch_edge_bern_f64_bias(const TailEntry *tab, int ntab, int64_t nblocks, int lane_elems, int fb_elems,
                                      const double *x, const EdgeOutArgs &o, const BernArgs &c, cudaStream_t st);
cudaError_t prepare_edge_bern_f32_bias();
cudaError_t prepare_edge_bern_f64_bias();
cudaError_t prepare_edge_bern_f32();
cudaError_t prepare_edge_bern_f64();
// One-time per-device set-up (shared-memory limits of the kernels).
cudaError_t prepare_edge_kernels_f32();
cudaError_t prepare_edge_kernels_f64();
cudaError_t prepare_edge_kernels_df();

// Deterministic segmented reduce of a node-sorted buffer into y.
struct ReduceArgs {
    // nodes of degree <= 32: groups of 32 lanes in sliced-ELL layout
    const int64_t *grp_off;        // n_grp: first slot of the group
    const int32_t *grp_node;       // 32 n_grp: node of each lane, -1 for padding
    const uint8_t *grp_deg;        // 32 n_grp: degree of each lane's node
    int64_t n_grp;
    // nodes of degree 33..128: one contiguous segment each, eight lanes per node
    const int32_t *med8_nodes;
    const int64_t *med8_off;
    const int32_t *med8_len;
    int64_t n_med8;
    // nodes of degree 129..1024: one contiguous segment each, a warp per node
    const int32_t *med_nodes;
    const int64_t *med_off;
    const int32_t *med_len;
    int64_t n_med;
    const int64_t *piece_start;    // pieces of big nodes
    const int32_t *piece_len;
    int64_t n_pieces;
    const int32_t *big_nodes;
    const int32_t *big_piece_ptr;  // n_big + 1
    const int32_t *piece_big;      // n_pieces: the big node (index into big_nodes) of each piece
    int32_t *big_count;            // n_big counters, zero between calls: pieces done this call
    int64_t n_big;
    void *partial;                 // n_pieces partial sums (float2 for FP32, double for FP64)
    const int32_t *skip;
};
cudaError_t launch_reduce_f32(const ReduceArgs &r, const float *buf, float *y, cudaStream_t st);
cudaError_t launch_reduce_f64(const ReduceArgs &r, const double *buf, double *y, cudaStream_t st);
// Warm-start features (12 floats per node, row-major) from the per-(edge, node) records in the
// slot buffer; r.partial must hold n_pieces * 64 bytes for this call.
cudaError_t launch_feature_reduce(const ReduceArgs &r, const unsigned long long *rec, float *feat, cudaStream_t st);

// y[v] += comp[v] (FP32 atomic mode), v < n
cudaError_t launch_add_comp(float *y, const float *comp, int64_t n, const int32_t *skip, cudaStream_t st);

}  // namespace s3
