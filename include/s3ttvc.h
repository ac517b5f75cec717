/*
 * s3ttvc.h -- C ABI of the GB300 (sm_103a) S^3TTVc library.
 *
 * The operation (Sec. II, Eq. 1-2): for a rank-N hypergraph H = (V, E) with
 * edge weights w(e) = |e|, the order-N blowup tensor B has, for every edge e,
 * the value w(e)/|beta(e)| at every N-tuple of nodes of e that uses each node
 * of e at least once (|beta(e)| = |e|! S(N,|e|), footnote to Sec. II).  The
 * library computes
 *
 *     y = B x^(N-1),   y_v = sum_{e containing v} c(e, v),
 *     c(e, v) = |e| (N-1)! / |beta(e)| * [t^(N-1)] e^(x_v t) prod_{u in e, u != v} (e^(x_u t) - 1)
 *
 * which is the per-(edge, node) generating-function value of Algorithm 2,
 * evaluated with truncated power-series products, leave-one-out prefix and
 * suffix products (Sec. IV), or the level-by-level CCSS forest of Sec. III
 * and Algorithm 4 (layout S3_LAYOUT_CCSS).  s3_hcentrality runs Algorithm 1
 * (NQZ) for the H-eigenvector centrality of Sec. II.
 *
 * Conventions shared by every entry point
 *   - Node ids are 0-based int32.  Hypergraphs are CSR: edge_ptr (int64, m+1
 *     entries, edge_ptr[0] = 0, non-decreasing) and members (int32,
 *     edge_ptr[m] entries).  The order of members inside an edge and of the
 *     edges themselves does not matter.
 *   - "device" pointers are CUDA global-memory pointers on the graph's device
 *     (any allocator: cudaMalloc, PyTorch, ...); "host" pointers are ordinary
 *     CPU memory.  The caller owns every buffer it passes; the library owns
 *     the graph handle and everything the handle allocated.
 *   - ``stream`` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Unless stated otherwise a call only enqueues work on that
 *     stream and returns; results are ready when the stream is.
 *   - Every entry point returns an s3_status and never aborts.  On failure
 *     s3_last_error() returns a message for the calling thread; outputs are
 *     then unspecified.
 *   - A graph handle may be used by one host thread at a time, and calls that
 *     share a handle must be ordered on one stream (the handle owns scratch
 *     memory that every call reuses).
 */
#ifndef S3TTVC_H
#define S3TTVC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define S3_VERSION 1
#define S3_MAX_RANK 128

typedef enum {
    S3_OK = 0,
    S3_EINVAL = 1,    /* invalid argument or malformed hypergraph */
    S3_ENOMEM = 2,    /* device or host allocation failed */
    S3_ECUDA = 3,     /* a CUDA call failed (message in s3_last_error) */
    S3_ENOCONV = 4,   /* NQZ did not reach the tolerance within max_iter */
    S3_ETIMEOUT = 5,  /* a bounded device wait ran out (the MMA-completion wait of
                         s3_mlp_forward; reported by the next s3_warmstart or s3_mlp_get_params) */
    S3_ERANGE = 6,    /* results left the range of the arithmetic type (synchronous and
                         range-checked calls, s3_options.range_check) */
    S3_ENOTSUP = 7    /* configuration not supported by this build */
} s3_status;

/*
 * Arithmetic of a call.  S3_F32 / S3_F64: x, y and the series in that type.
 * S3_DF64: x and y are FP64 (double); the series of the edges run in
 * double-float -- each value an unevaluated sum of two FP32 numbers, about 44
 * significant bits -- on the FP32 units (GB300 runs FP32 many times faster than
 * FP64).  Size-1 edges, windows N-|e|+1 wider than 24 and the CCSS layout use
 * FP64.  Relative error per node is of order 1e-13 for non-negative x.
 */
typedef enum { S3_F32 = 0, S3_F64 = 1, S3_DF64 = 2 } s3_dtype;

typedef enum {
    /* y_v is summed node by node from a per-(edge, node) buffer laid out by
     * node (groups of 32 low-degree nodes interleaved, one segment per other
     * node, hubs in fixed pieces), each sum in a fixed order: deterministic,
     * bit-identical run to run. */
    S3_REDUCE_SEGMENTED = 0,
    /* contributions are added with warp-aggregated atomics; the FP32 path
     * keeps a two-sum compensation term per node that is folded in at the
     * end.  Summation order (hence rounding) varies run to run. */
    S3_REDUCE_ATOMIC = 1
} s3_reduce;

typedef enum {
    /* each edge recomputes its own prefix and suffix products (Sec. IV with
     * the leave-one-out identity E = Ebar + 1) */
    S3_LAYOUT_EDGE = 0,
    /* the trimmed CCSS forest of Sec. III evaluated level by level: every
     * forest node multiplies its parent's truncated product by one series
     * (the memoisation of Algorithm 4) and every special leaf (e, v) takes a
     * dot product with E_N(x_v) */
    S3_LAYOUT_CCSS = 1
} s3_layout;

typedef struct {
    int32_t rank;          /* N; 0 = largest edge size.  Must be >= largest edge size, <= S3_MAX_RANK */
    int32_t reduce;        /* s3_reduce */
    int32_t layout;        /* s3_layout used by s3_sttsvc */
    int32_t build_ccss;    /* 1 = also build the CCSS forest (implied by layout = CCSS) */
    int32_t device;        /* CUDA device ordinal; -1 = the calling thread's current device */
    int32_t thread_max_w;  /* edges whose window N-|e|+1 is <= this use one thread per edge, wider ones
                              eight lanes (FP32) or one warp (FP64) per edge; 0 = library default (32),
                              range 1..32 */
    int32_t block_threads; /* threads per block of the thread-per-edge kernels; 0 = default (128) */
    int32_t order;         /* order of the nodes inside every edge (the sequence the prefix products
                              and the CCSS forest follow) and of the edges inside a size bucket:
                              S3_ORDER_DEGREE (default) = decreasing degree, ties by id, edges sorted
                              lexicographically; S3_ORDER_INDEX = increasing node id (the index
                              order of Sec. II-B / Fig. 2), edges in input order */
    int32_t streams;       /* size buckets are spread over this many CUDA streams forked from the
                              caller's stream (1..8); 0 = default (4) */
    int32_t small_bucket_edges; /* thread-per-edge buckets of size >= 2 with at most this many edges
                              share one fused launch (one edge per thread); 0 = default (40000),
                              negative = every bucket gets its own launch */
    int32_t closed_form_max_s; /* FP32/FP64 buckets of edges of size 2..this (at most 6) that run
                              their own launch are evaluated in closed form -- the inclusion-exclusion
                              expansion of E(x_v) prod_{u != v} Ebar(x_u) (Sec. II-A) -- where that
                              costs fewer operations than the series products (and, for FP64 from
                              size 6 on, fewer FP64 operations than the Bernoulli form); every edge whose
                              error bound (relative 2^-17 FP32, 2^-42 FP64) does not hold is
                              recomputed by the series kernels.  0 = default (6), -1 = never */
    int32_t range_check;   /* 1 = s3_sttsvc / s3_sttsvc_layout read the handle's range counter
                              (s3_range_events) on the call's stream before and after the call,
                              synchronise that stream and return S3_ERANGE when this call's
                              results left the normal range of the call's type (y is still
                              written).  Not allowed while the stream is being captured into a
                              CUDA graph (S3_ENOTSUP).  0 = default: asynchronous, such results
                              are only counted */
    int32_t bernoulli;     /* FP32/FP64 buckets of edges of size 6..64 whose window N-|e|+1 is at most
                              thread_max_w and that do not use the closed form are evaluated in one
                              launch by the Bernoulli form of the leave-one-out: the product G of the
                              series (e^(x_u t) - 1)/(x_u t) over the whole edge, then for each member
                              v the sum over k of G's coefficients times B_k x_v^k / k! (Bernoulli
                              numbers; E(x_v)/Ebar(x_v) = 1/(1 - e^(-x_v t)), Sec. II-A), where it
                              costs fewer operations than the prefix/suffix products.  Edges whose
                              alternating sum would amplify rounding errors more than 4x (FP32) or
                              64x (FP64), or that hold x < 0, are recomputed with the series.
                              0 = default (on), -1 = never */
    int32_t reserved[3];
} s3_options;

typedef enum { S3_ORDER_DEGREE = 0, S3_ORDER_INDEX = 1 } s3_order;

typedef struct s3_graph_s *s3_graph_t;

/* Host-side description of a built format (s3_format_inspect / s3_graph_query). */
typedef struct {
    int64_t n, m, nnz;                 /* nodes, edges, sum of edge sizes */
    int32_t rank;                      /* N */
    int32_t max_edge;                  /* largest edge size */
    int64_t max_degree;                /* largest node degree */
    int64_t edges_per_size[S3_MAX_RANK + 1];   /* bucket sizes, index = |e| */
    int64_t ccss_levels;               /* number of non-empty CCSS levels (0 if not built) */
    int64_t ccss_nodes_per_level[S3_MAX_RANK + 1]; /* trimmed forest, index = level (1-based) */
    int64_t ccss_nodes;                /* total forest nodes */
    int64_t ccss_special_leaves;       /* = nnz */
    int64_t ccss_products;             /* series products (one per forest node at level >= 2) */
    int64_t device_bytes;              /* device memory held by the handle (0 for inspect) */
} s3_format_info;

/* Fill *opt with defaults (rank 0, segmented reduce, edge layout, current device). */
s3_status s3_options_init(s3_options *opt);

/*
 * Validate and lay out a hypergraph on the host without touching any GPU
 * (no CUDA call is made).  Checks: n >= 1, m >= 0, edge_ptr[0] = 0 and
 * non-decreasing, every edge non-empty, ids in [0, n), no node repeated inside
 * an edge, rank >= largest edge size, rank <= S3_MAX_RANK, edge_ptr[m] < 2^31.
 * Returns S3_EINVAL with a message if a check fails.  With opt->build_ccss
 * (or layout CCSS) the trimmed CCSS forest of Sec. III is built and counted.
 * edge_ptr, members: host.  info: host, written on success.
 */
s3_status s3_format_inspect(int64_t n, int64_t m, const int64_t *edge_ptr, const int32_t *members,
                            const s3_options *opt, s3_format_info *info);

/*
 * Build the device format (Sec. III layouts) and return a handle in *out.
 * Performs the checks of s3_format_inspect, sorts every edge (index-ordered
 * form, footnote to Sec. II-B), buckets edges by size, builds the
 * node-sorted incidence used by the deterministic reduce and (if requested)
 * the CCSS forest, then uploads everything once and allocates the handle's
 * scratch memory.  Synchronous.  edge_ptr, members: host, only read.
 */
s3_status s3_build_format(int64_t n, int64_t m, const int64_t *edge_ptr, const int32_t *members,
                          const s3_options *opt, s3_graph_t *out);

/* Describe a built handle.  info: host. */
s3_status s3_graph_query(s3_graph_t g, s3_format_info *info);

/*
 * y = B x^(N-1) (Eq. 1).  x: device, n elements of dt (float or double).
 * y: device, n elements of dt, overwritten.  x and y must not overlap.
 * Arithmetic is in dt throughout the series products; per edge the vector is
 * rescaled by an exact power of two before the products and the result is
 * rescaled back, so intermediate terms stay in range.  Per-(edge, node)
 * results that underflow or overflow dt are counted on the device
 * (s3_range_events).  By default the call stays asynchronous and does not
 * report them; a handle built with s3_options.range_check = 1 synchronises
 * the stream and returns S3_ERANGE when this call produced any (y written).
 * Small edges may be evaluated in closed form (s3_options.closed_form_max_s)
 * within its stated error bound.  Uses the handle's layout and reduce mode.
 * Calls on one handle share its scratch memory (reduce buffer, closed-form
 * lists): calls that could run at the same time on the GPU (unordered
 * streams) must use different handles.
 */
s3_status s3_sttsvc(s3_graph_t g, s3_dtype dt, const void *x, void *y, void *stream);

/* As s3_sttsvc with an explicit layout (s3_layout); CCSS needs a handle built with the forest. */
s3_status s3_sttsvc_layout(s3_graph_t g, s3_dtype dt, int32_t layout, const void *x, void *y, void *stream);

/*
 * End-to-end variant: x_host and y_host are HOST buffers (n elements of dt,
 * pinned memory recommended).  Copies x to the device, computes as
 * s3_sttsvc, copies y back and synchronises ``stream`` before returning.
 * Being synchronous it always checks the range counter: S3_ERANGE (y_host
 * written) when a result of this call left the normal range of dt.
 */
s3_status s3_sttsvc_host(s3_graph_t g, s3_dtype dt, const void *x_host, void *y_host, void *stream);

/* Device time of one s3_sttsvc call, split into the per-edge series kernels and the reduce. */
typedef struct {
    float edge_ms;     /* all per-edge (size bucket) kernels */
    float reduce_ms;   /* segmented reduce, or the compensation pass of the atomic mode */
    float total_ms;
    int32_t launches;  /* kernels launched by the call */
    float bern_ms;     /* the Bernoulli-form launch alone (events on its own stream); 0 if none */
    int32_t reserved[3];
} s3_profile;

/*
 * Run s3_sttsvc once (edge layout) with CUDA events recorded on ``stream``
 * before the edge kernels, between them and the reduce, and after the
 * reduce, and around the Bernoulli-form launch on the stream it runs on;
 * synchronises ``stream`` and writes the elapsed times to *prof (host).
 * Arguments as s3_sttsvc.
 */
s3_status s3_sttsvc_profile(s3_graph_t g, s3_dtype dt, const void *x, void *y, s3_profile *prof, void *stream);

/*
 * Number of per-(edge, node) results since the handle was built (or since the
 * last reset) that came out as zero, subnormal or non-finite although their
 * exact value is a positive normal number of the call's type.  Waits for the
 * handle's last call (an event recorded on that call's stream), not for the
 * rest of the device.  reset != 0 clears the counter.  count: host.
 */
s3_status s3_range_events(s3_graph_t g, int64_t *count, int32_t reset);

/*
 * Closed-form evaluation (s3_options.closed_form_max_s) on this handle:
 * *sizes_f32 / *sizes_f64 = bit mask of the edge sizes s (bit s) whose bucket
 * uses it for FP32 / FP64 calls; *rejected = edges that failed its error bound
 * and went back to the series kernels, summed over all calls since the handle
 * was built (waits for the handle's last call only).  Any pointer may be NULL.  All
 * host.
 */
s3_status s3_closed_form_query(s3_graph_t g, uint64_t *sizes_f32, uint64_t *sizes_f64, int64_t *rejected);

/*
 * Bernoulli-form evaluation (s3_options.bernoulli) on this handle:
 * *sizes_f32 / *sizes_f64 = bit mask of the edge sizes s (bit s-1, s <= 64)
 * whose bucket uses it for FP32 / FP64 calls; *rejected = edges that failed
 * its amplification gate and were recomputed with the series, summed over all
 * calls since the handle was built (waits for the handle's last call only).
 * Any pointer may be NULL.  All host.
 */
s3_status s3_bernoulli_query(s3_graph_t g, uint64_t *sizes_f32, uint64_t *sizes_f64, int64_t *rejected);

/* ------------------------------------------------------------------ NQZ --- */

typedef struct {
    double tol;            /* stop when (lambda_max - lambda_min)/lambda_min < tol (Algorithm 1) */
    int32_t max_iter;      /* passes through the repeat body; <= 0 = 10000 */
    int32_t precision;     /* 0 = FP64 throughout; 1 = FP32 series until the gap is below
                              switch_tol (or stops shrinking), then FP64 to tol; 2 = as 1 with
                              double-float series (S3_DF64) instead of FP64 after the switch;
                              3 = double-float series throughout.  Norms, roots, ratios and
                              the bracket are FP64 in every mode. */
    double switch_tol;     /* FP32 -> FP64 hand-over gap for precision 1 and 2; <= 0 = 1e-5 */
    int32_t check_every;   /* iterations per captured CUDA graph between host checks; <= 0 = 8.
                              The graphs are kept on the handle for later calls with the same
                              tol, max_iter and check_every (freed by s3_destroy). */
    int32_t reserved[7];
} s3_nqz_options;

typedef struct {
    double lambda_min, lambda_max;  /* bracket of the H-eigenvalue at the last iteration */
    int32_t iters;                  /* passes through the repeat body (all precisions) */
    int32_t iters_fp32;             /* of which in FP32 */
    int32_t converged;              /* 1 if the gap reached tol */
    int32_t reserved;
    double seconds;                 /* wall time of the call */
} s3_nqz_result;

s3_status s3_nqz_options_init(s3_nqz_options *opt);

/*
 * H-eigenvector centrality by Algorithm 1 (NQZ) on the device.
 * x0: device, n doubles, positive (NULL = the uniform start of Algorithm 1).
 * x_out: device, n doubles, written with the last iterate (1-norm 1).
 * res: host.  Every node must belong to at least one edge (S3_EINVAL
 * otherwise: the ratio z/x^(N-1) is undefined there), and rank >= 2.
 * The (N-1)-th roots and the ratios are FP64-accurate (double-float arithmetic on
 * the FP32 units, relative error below 1e-11 at any rank), the 1-norm, the min/max
 * and the test FP64.  Synchronous on ``stream``; returns S3_ENOCONV (x_out and res still
 * written) if max_iter passes do not reach tol.
 */
s3_status s3_hcentrality(s3_graph_t g, const s3_nqz_options *opt, const double *x0, double *x_out,
                         s3_nqz_result *res, void *stream);

/* ------------------------------------- Z-eigenpairs and symmetric CP --- */

typedef struct {
    double alpha;          /* shift (>= 0); 0 = plain higher-order power method */
    double tol;            /* stop when |lambda_k - lambda_(k-1)| < tol max(1, |lambda_k|); default 1e-12 */
    int32_t max_iter;      /* <= 0 = 10000 */
    int32_t reserved[7];
} s3_zeig_options;

typedef struct {
    double lambda;         /* x . B x^(N-1) at the returned x */
    int32_t iters;         /* normalisation steps taken */
    int32_t converged;
    double seconds;
    int32_t reserved[4];
} s3_zeig_result;

s3_status s3_zeig_options_init(s3_zeig_options *opt);

/*
 * A Z-eigenpair B x^(N-1) = lambda x, ||x||_2 = 1, of the blowup tensor by the
 * shifted symmetric higher-order power method (the shifted-power method the
 * paper names as a consumer of S^3TTVc, Sec. I):
 *     x <- (B x^(N-1) + alpha x) / ||B x^(N-1) + alpha x||_2.
 * Each step is one FP64 S^3TTVc (on x / max|x|, so any rank stays in range)
 * and FP64 vector kernels; the host checks lambda after each step.
 * x0: device, n doubles (any nonzero start; NULL = the uniform unit vector).
 * x_out: device, n doubles, written.  res: host.  Synchronous on ``stream``;
 * S3_ENOCONV (x_out, res written) if max_iter steps do not reach tol,
 * S3_ERANGE if lambda leaves the FP64 range.
 */
s3_status s3_zeigenpair(s3_graph_t g, const s3_zeig_options *opt, const double *x0, double *x_out,
                        s3_zeig_result *res, void *stream);

/*
 * Greedy rank-R symmetric CP approximation B ~ sum_r lambda_r x_r^(outer N)
 * (the paper names symmetric CP decomposition as a consumer of S^3TTVc, Sec. I):
 * component r is the s3_zeigenpair of B - sum_{q<r} lambda_q x_q^(outer N),
 * whose product with x^(N-1) is B x^(N-1) - sum_q lambda_q (x_q . x)^(N-1) x_q.
 * R: 1..32.  X0: device, R rows of n doubles (start of each component) or NULL
 * (uniform starts).  X: device, R rows of n doubles, written (unit vectors).
 * lambdas: host, R doubles, written.  iters: host, R ints, or NULL.
 * Synchronous on ``stream``; S3_ENOCONV if some component did not converge.
 */
s3_status s3_symmetric_cp(s3_graph_t g, int32_t R, const s3_zeig_options *opt, const double *X0, double *X,
                          double *lambdas, int32_t *iters, void *stream);

/*
 * One update of Algorithm 1 from a complete z = B xhat^(N-1) that the caller
 * assembled -- e.g. the sum over GPUs of the partial results of handles built
 * on disjoint edge sets of one hypergraph (edge-sharded S^3TTVc, FP64):
 * lambda[0], lambda[1] = min and max over v of z_v / xhat_v^(N-1) (the bracket
 * of this iterate; it does not depend on the scale of xhat), and the next
 * iterate r = z^[1/(N-1)] written twice: x_next with 1-norm 1 (Algorithm 1's
 * x) and xhat_next = r / max(r) (max 1: the input of the next S^3TTVc, which
 * keeps z in range).  FP64 throughout.  z, xhat, x_next, xhat_next: device,
 * n doubles (x_next and xhat_next distinct; either may alias xhat).  lambda:
 * host, 2 doubles.  Synchronous on ``stream``; S3_ERANGE if a ratio or a root
 * leaves the FP64 range (a node in no edge, or x_v = 0).
 */
s3_status s3_nqz_update(s3_graph_t g, const double *z, const double *xhat, double *x_next, double *xhat_next,
                        double *lambda, void *stream);

/* -------------------------------------------------------------- batches --- */

typedef struct s3_batch_s *s3_batch_t;

typedef struct {
    int32_t block_threads;     /* threads per block of the persistent kernels; 0 = 128 */
    int32_t edges_per_thread;  /* a tile holds block_threads * edges_per_thread edges of one bucket; 0 = 4 */
    int32_t thread_max_w;      /* windows up to this use one thread per edge, wider ones a warp; 0 = 32 */
    int32_t use_graph;         /* 1 (default) = replay one captured CUDA graph per call */
    char cache_path[256];      /* non-empty: s3_batch_autotune appends its choice to this text file */
    int32_t reserved[8];
} s3_batch_options;

typedef struct {
    int32_t block_threads, edges_per_thread, thread_max_w;
    float ms;
} s3_tune_candidate;

typedef struct {
    int32_t block_threads, edges_per_thread, thread_max_w; /* the configuration chosen */
    int32_t tried;                                         /* configurations timed */
    float ms;                                              /* its device time per batched call */
    int32_t reserved;
    s3_tune_candidate candidates[32];                      /* every configuration timed (first 32) */
} s3_tune_result;

s3_status s3_batch_options_init(s3_batch_options *opt);

/*
 * Group `count` graph handles (built with the segmented reduce, same device)
 * and `nvec` vectors per graph for s3_sttsvc_batched.  The handles must outlive
 * the batch.  Allocates the per-(graph, vector) buffers and work lists.
 * graphs: host array of count handles.
 */
s3_status s3_batch_create(int32_t count, const s3_graph_t *graphs, int32_t nvec, const s3_batch_options *opt,
                          s3_batch_t *out);

/*
 * y_{g,v} = B_g x_{g,v}^(N_g - 1) for every graph g and vector v of the batch,
 * in one persistent edge kernel, one persistent reduce kernel and one hub
 * pass, replayed from a captured CUDA graph.  Every edge's member ids and
 * incidence slots are loaded once for all nvec vectors of its graph.
 * x, y: HOST arrays of count*nvec DEVICE pointers, graph-major
 * (x[g*nvec + v] holds n_g elements of dt; y likewise, overwritten).
 * Results equal nvec*count separate s3_sttsvc calls up to summation order
 * inside edges (deterministic run to run).  When the pointer arrays differ
 * from the previous call the call first waits for that call to finish.
 */
s3_status s3_sttsvc_batched(s3_batch_t b, s3_dtype dt, const void *const *x, void *const *y, void *stream);

/*
 * Time candidate configurations (block_threads x edges_per_thread x
 * thread_max_w) of s3_sttsvc_batched on these inputs (each: one warm-up and
 * three timed calls, CUDA events on `stream`), keep the fastest for later
 * calls and report all of them in *res (host).  Synchronous.
 */
s3_status s3_batch_autotune(s3_batch_t b, s3_dtype dt, const void *const *x, void *const *y, s3_tune_result *res,
                            void *stream);

/* Release a batch (not its graphs).  NULL is allowed. */
s3_status s3_batch_destroy(s3_batch_t b);

/* ------------------------------------------------- learned warm start --- */

/* Per-node features and the 12-64-64-1 MLP of the warm start (no counterpart in the paper: it
 * speeds up Algorithm 1 by starting it near its fixed point; the uniform start stays the
 * fallback and the reference). */
#define S3_MLP_FEATURES 12
#define S3_MLP_HIDDEN 64
#define S3_MLP_PARAMS 5057   /* W1[64][12] b1[64] W2[64][64] b2[64] W3[64] b3, row-major */

typedef struct s3_mlp_s *s3_mlp_t;

/*
 * feat: device, n x 12 floats, row-major, written.  Features of node v, each
 * log1p(.)-scaled: degree; mean and max size of the edges containing v; the
 * 8-bin histogram of those sizes (bin b collects sizes s with
 * floor(8 log(s/2)/log(N/2)) = b, clamped to 0..7); the sum over v's edges of
 * the other members' degrees.  Integer accumulation: bit-reproducible.
 */
s3_status s3_features(s3_graph_t g, float *feat, void *stream);

/* New model on the current device.  params: host, S3_MLP_PARAMS floats (FP32
 * master weights), or NULL for a deterministic He-style initialisation from seed. */
s3_status s3_mlp_create(const float *params, uint64_t seed, s3_mlp_t *out);

/* Copy the FP32 master weights (bf16 = 0) or their BF16 copies widened to FP32
 * (bf16 = 1) to params (host, S3_MLP_PARAMS floats).  Synchronises the device. */
s3_status s3_mlp_get_params(s3_mlp_t m, float *params, int32_t bf16);

/* out[v] = W3 relu(W2 relu(W1 feat_v + b1) + b2) + b3 with the BF16 weights and
 * FP32 accumulation; both hidden layers on the tensor cores, their inputs split into two
 * BF16 terms each (relative error about 2^-17 against FP32 inputs).  feat: device n x 12;
 * out: device n floats.  Asynchronous; a tensor-core wait that runs out (bounded, well
 * under a second) is reported as S3_ETIMEOUT by the next synchronising call on the model. */
s3_status s3_mlp_forward(s3_mlp_t m, const float *feat, int64_t n, float *out, void *stream);

/*
 * Loss L = (1/n) sum_v (out_v - target_v)^2 over the n given nodes (forward with
 * the BF16 weights) and its gradient with respect to the weights (FP32,
 * accumulated per block and summed in a fixed order), kept in the model for
 * s3_mlp_adam_step.  feat: device n x 12; target: device n.  loss (host,
 * double) and grad (host, S3_MLP_PARAMS floats) are optional; when given the
 * call synchronises `stream`.
 */
s3_status s3_mlp_loss_grad(s3_mlp_t m, const float *feat, const float *target, int64_t n, double *loss,
                           float *grad, void *stream);

/* One Adam step (bias-corrected) on the FP32 master weights with the last gradient;
 * refreshes the BF16 copies. */
s3_status s3_mlp_adam_step(s3_mlp_t m, float lr, float beta1, float beta2, float eps, void *stream);

/*
 * Warm start for s3_hcentrality: x0 = exp(MLP(features)) normalised to 1-norm 1.
 * x0: device, n doubles, written.  Synchronises `stream` once (to shift the
 * exponent by the largest prediction).
 */
s3_status s3_warmstart(s3_graph_t g, s3_mlp_t m, double *x0, void *stream);

/* Training target of the warm start: target_v = log x_v - (1/n) sum_u log x_u for a positive
 * centrality x (device, n doubles); target: device, n floats. */
s3_status s3_mlp_target(s3_graph_t g, const double *x, float *target, void *stream);

s3_status s3_mlp_destroy(s3_mlp_t m);

/* ----------------------------------------------- allocation-free call --- */

/* Largest node count s3_sttsvc_f32_noalloc accepts (its fixed scratch: 4 bytes per node). */
#define S3_NOALLOC_MAX_NODES (1 << 22)

/*
 * FP32 y = B x^(N-1) for callers that cannot allocate device memory:
 * pipelines that fix all their memory up front, hosts whose own allocator
 * owns the device, or latency-critical loops that must not risk an
 * allocation's implicit device synchronisation.  Such callers can neither build a graph handle nor pass a
 * workspace, so this entry point takes the hypergraph as plain device arrays
 * and allocates nothing: its only scratch (one FP32 two-sum compensation term
 * per node) is a fixed array of S3_NOALLOC_MAX_NODES floats (16 MiB) compiled
 * into the library, which every GPU that loads the library holds until the
 * process exits.  The paper has no counterpart of this entry point.
 *
 * n: nodes, 1 <= n <= S3_NOALLOC_MAX_NODES (S3_EINVAL otherwise).
 * m: edges.  rank: N, 1..S3_MAX_RANK.
 * edge_ptr: device, m+1 int64 CSR offsets.  members: device, int32 node ids
 *   (any order inside an edge, no repeats).  Edges whose size is outside
 *   1..rank or that hold an id outside [0, n) are skipped, not reported.
 * x: device, n floats.  y: device, n floats, overwritten (must not overlap x).
 * stream: cudaStream_t as void*; the call only enqueues work.
 * Contributions are added with atomics (summation order varies run to run)
 * and each addition's rounding error is kept in the scratch array and folded
 * into y at the end; the call zeroes y and the scratch itself.
 * The first call on a device resolves the scratch array's device address
 * (cudaGetSymbolAddress) and sets a kernel attribute, so make that first call
 * before any stream capture.  Every call on a device shares the one scratch
 * array: calls whose work overlaps on the GPU (different streams, or several
 * host threads) race and give wrong results -- order them.
 */
s3_status s3_sttsvc_f32_noalloc(int64_t n, int64_t m, int32_t rank, const int64_t *edge_ptr,
                                const int32_t *members, const float *x, float *y, void *stream);

/* --------------------------------------------------------- measurement --- */

typedef struct {
    double tflops;            /* multiply-add throughput, 2 flops per FMA */
    double flops_per_launch;
    float ms;                 /* fastest launch (CUDA events on the stream) */
    int32_t sm_count;         /* cudaDevAttrMultiProcessorCount of the current device */
    int32_t threads_per_sm;   /* resident threads per SM of the probe */
    int32_t clock_mhz;        /* cudaDevAttrClockRate (the device's rated maximum), MHz */
    int32_t reserved[4];
} s3_peak_result;

/*
 * Measured FP32 (dt = S3_F32) or FP64 (S3_F64) FMA throughput of the current
 * device: independent chains v = v * a + b in every thread of a grid that fills
 * all SMs, timed with CUDA events on ``stream`` (one warm-up launch, then `reps`
 * timed launches, 1..10000; the fastest is reported).  These are the peaks the
 * ALU-bound series kernels are compared with; the paper has no counterpart of
 * this entry point.  Synchronises ``stream``.  res: host.
 */
s3_status s3_fma_peak(s3_dtype dt, int32_t reps, s3_peak_result *res, void *stream);

/* ------------------------------------------------------------- cleanup --- */

/* Release the handle and its device memory (synchronises its device).  NULL is allowed. */
s3_status s3_destroy(s3_graph_t g);

/* Message for the last failing call on this host thread ("" if none). */
const char *s3_last_error(void);

/* Constant name of a status code. */
const char *s3_status_string(s3_status st);

/* S3_VERSION of the built library. */
int32_t s3_version(void);

#ifdef __cplusplus
}
#endif

#endif /* S3TTVC_H */
