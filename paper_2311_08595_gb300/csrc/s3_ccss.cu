// S^3TTVc on the trimmed CCSS forest (Sec. III), level by level.
//
// The forest's root-to-node paths are the distinct sorted prefixes of the
// sequences e minus v.  Each node stores the truncated product of Ebar(x_u)
// over its path, kept on a window of `width` coefficients starting at degree
// `level` (the memo W of Algorithm 4, one column per node).  Level 1 windows
// are power tables; a node at level l >= 2 multiplies its parent's window by
// one Ebar series -- one convolution per forest edge, computed once and shared
// by every special leaf below it (the memoisation of Algorithm 4, in
// breadth-first order so that every level is one parallel sweep).  A special
// leaf (e, v) hanging at the node for e minus v then needs one dot product:
//     c(e, v) = K(s,N) sum_{k=0}^{w-1} x_v^k/k! * win[w-1-k],  w = N-s+1.
// Every level l uses its own exact power-of-two scale 2^p_l of x (p_l from the
// largest |x| and a per-level target), so that windows of long paths stay in
// range; the results are scaled back by 2^(-p_l (N-1)).
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>

#include "s3_graph.h"
#include "s3_series.cuh"

namespace s3 {
namespace {

// d_scale[0] = max over v of expo(|x_v|) (x = m 2^e, m in [0.5,1)); 0 entries ignored.
template <typename T>
__global__ void max_expo_kernel(const T *__restrict__ x, int64_t n, int32_t *d_scale, const int32_t *skip) {
    if (skip && *skip) return;
    int best = INT_MIN;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        T v = x[i];
        if (v != T(0)) best = max(best, Arith<T>::expo(Arith<T>::absv(v)));
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, d));
    if ((threadIdx.x & 31) == 0 && best != INT_MIN) atomicMax(d_scale, best);
}

__device__ __forceinline__ int ccss_p(const int32_t *d_scale, float target) {
    int mx = d_scale[0];
    if (mx < -100000) return 0;  // no non-zero entry (the counter starts at 0x80808080)
    return Arith<float>::expo(target) - mx;
}

// level 1: win[j] = (g x_v)^(j+1)/(j+1)!
template <typename T>
__global__ void ccss_level1_kernel(const int32_t *__restrict__ vertex, const int64_t *__restrict__ off,
                                   const int32_t *__restrict__ width, int64_t begin, int64_t end,
                                   const T *__restrict__ x, T *__restrict__ val, const int32_t *d_scale,
                                   float target, const int32_t *skip) {
    if (skip && *skip) return;
    int64_t k = begin + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= end) return;
    int p = ccss_p(d_scale, target);
    T X = x[vertex[k]] * Arith<T>::pow2(p);
    T *w = val + off[k];
    T a = X;
    int W = width[k];
    for (int j = 0; j < W; ++j) {
        w[j] = a;
        a = a * (X / T(j + 2));
    }
}

// level >= 2, one width segment, window width W known at compile time.  The
// parent's window was stored for scale 2^p_par (level l-1); its coefficient
// of degree d is brought to this level's scale 2^p by the exact factor
// 2^((p - p_par) d) before the product.
template <typename T, int W>
__global__ void ccss_level_kernel(const int32_t *__restrict__ vertex, const int32_t *__restrict__ parent,
                                  const int64_t *__restrict__ off, int64_t begin, int64_t end, int level,
                                  const T *__restrict__ x, T *__restrict__ val, const int32_t *d_scale,
                                  float target, float target_par, const int32_t *skip) {
    if (skip && *skip) return;
    int64_t k = begin + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= end) return;
    int p = ccss_p(d_scale, target);
    int dp = p - ccss_p(d_scale, target_par);
    T X = x[vertex[k]] * Arith<T>::pow2(p);
    const T *pw = val + off[parent[k]];
    T P[W];
#pragma unroll
    for (int j = 0; j < W; ++j) P[j] = Arith<T>::scale2(pw[j], dp * (level - 1 + j));
    T a[W];
    power_table<T, W>(X, a);
    toeplitz_inplace<T, W>(P, a);
    T *w = val + off[k];
#pragma unroll
    for (int j = 0; j < W; ++j) w[j] = P[j];
}

// level >= 2, any width (reads the parent window from memory)
template <typename T>
__global__ void ccss_level_generic_kernel(const int32_t *__restrict__ vertex, const int32_t *__restrict__ parent,
                                          const int64_t *__restrict__ off, int64_t begin, int64_t end, int W,
                                          int level, const T *__restrict__ x, T *__restrict__ val,
                                          const int32_t *d_scale, float target, float target_par,
                                          const int32_t *skip) {
    if (skip && *skip) return;
    int64_t k = begin + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= end) return;
    int p = ccss_p(d_scale, target);
    int dp = p - ccss_p(d_scale, target_par);
    T X = x[vertex[k]] * Arith<T>::pow2(p);
    const T *pw = val + off[parent[k]];
    T a[S3_MAX_RANK], P[S3_MAX_RANK];
    a[0] = X;
    for (int j = 1; j < W; ++j) a[j] = a[j - 1] * (X / T(j + 1));
    for (int j = 0; j < W; ++j) P[j] = Arith<T>::scale2(pw[j], dp * (level - 1 + j));
    T *w = val + off[k];
    for (int j = 0; j < W; ++j) {
        T acc = T(0);
        for (int jp = 0; jp <= j; ++jp) acc = Arith<T>::fma_(a[j - jp], P[jp], acc);
        w[j] = acc;
    }
}

// special leaves of edges of size s (window w = N-s+1)
template <typename T>
__global__ void ccss_leaf_kernel(const int32_t *__restrict__ leaf_node, const int32_t *__restrict__ leaf_vertex,
                                 const int32_t *__restrict__ leaf_slot, int64_t begin, int64_t end,
                                 const int64_t *__restrict__ off, const T *__restrict__ x,
                                 const T *__restrict__ val, EdgeBucketArgs b, EdgeOutArgs o,
                                 const int32_t *d_scale) {
    if (o.skip && *o.skip) return;
    int64_t k = begin + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= end) return;
    const int W = b.N - b.s + 1;
    int p = ccss_p(d_scale, b.target);
    int v = leaf_vertex[k];
    T X = x[v] * Arith<T>::pow2(p);
    const T *w = val + off[leaf_node[k]];
    T acc = w[W - 1];
    T a = T(1);
    for (int kk = 1; kk < W; ++kk) {
        a = a * (X / T(kk));
        acc = Arith<T>::fma_(a, w[W - 1 - kk], acc);
    }
    int bias_e = o.bias ? (Arith<T>::expo(X) - p) : 0;
    T c = finalize_value<T>(acc, b, p, bias_e, o.range_events);
    if (o.mode == kOutBuffer) {
        reinterpret_cast<T *>(o.out)[leaf_slot[k]] = c;
    } else {
        scatter_atomic<T>(o, v, c);
    }
}

// Scale target of CCSS level l: the per-node value a with a^(N-1) s! S(N-1,s)/(N-1)! = 1
// for s = l + 1 (the size of the edges whose special leaves hang at level l).
float level_target(int level, int N) { return scale_target(level + 1, N) / (float)(level + 1); }
float cached_level_target(const s3_graph_s *g, int level) { return g->cc_level_target[level]; }

template <typename T>
cudaError_t launch_level(const s3_graph_s *g, const s3_graph_s::CcssSeg &sg, const T *x, T *val,
                         const int32_t *skip, cudaStream_t st) {
    int64_t cnt = sg.end - sg.begin;
    if (cnt <= 0) return cudaSuccess;
    const int bs = 128;
    unsigned grid = (unsigned)((cnt + bs - 1) / bs);
    const float target = cached_level_target(g, sg.level);
    if (sg.level == 1) {
        ccss_level1_kernel<T><<<grid, bs, 0, st>>>(g->d_cc_vertex, g->d_cc_off, g->d_cc_width,
                                                    sg.begin, sg.end, x, val, g->d_cc_scale, target, skip);
        return cudaGetLastError();
    }
    const float target_par = cached_level_target(g, sg.level - 1);
    switch (sg.width) {
#define S3_CC_CASE(w)                                                                                       \
    case w:                                                                                                 \
        ccss_level_kernel<T, w><<<grid, bs, 0, st>>>(g->d_cc_vertex, g->d_cc_parent, g->d_cc_off, sg.begin,  \
                                                     sg.end, sg.level, x, val, g->d_cc_scale, target,       \
                                                     target_par, skip);                                     \
        return cudaGetLastError();
        S3_W_CASES(S3_CC_CASE)
#undef S3_CC_CASE
        default:
            ccss_level_generic_kernel<T><<<grid, bs, 0, st>>>(g->d_cc_vertex, g->d_cc_parent, g->d_cc_off, sg.begin,
                                                              sg.end, sg.width, sg.level, x, val, g->d_cc_scale,
                                                              target, target_par, skip);
            return cudaGetLastError();
    }
}

template <typename T>
s3_status run_ccss_t(s3_graph_s *g, const T *x, T *y, int bias, const int32_t *skip, cudaStream_t st) {
    const bool seg = g->opt.reduce == S3_REDUCE_SEGMENTED;
    EdgeOutArgs o{};
    o.bias = bias;
    o.range_events = g->d_range;
    o.skip = skip;
    if (seg) {
        o.out = g->d_buf;
        o.mode = kOutBuffer;
    } else {
        o.out = y;
        o.mode = sizeof(T) == 4 ? kOutAtomicComp : kOutAtomic;
        o.comp = g->d_comp;
        S3_CUDA(cudaMemsetAsync(y, 0, sizeof(T) * (size_t)g->n, st));
        if (sizeof(T) == 4) S3_CUDA(cudaMemsetAsync(g->d_comp, 0, sizeof(float) * (size_t)g->n, st));
    }
    // global exponent of max |x|
    S3_CUDA(cudaMemsetAsync(g->d_cc_scale, 0x80, sizeof(int32_t), st));
    max_expo_kernel<T><<<(unsigned)std::min<int64_t>((g->n + 255) / 256, 1024), 256, 0, st>>>(x, g->n, g->d_cc_scale,
                                                                                              skip);
    S3_CUDA(cudaGetLastError());
    T *val = reinterpret_cast<T *>(g->d_cc_values);
    for (const auto &sg : g->ccss_segs) S3_CUDA(launch_level<T>(g, sg, x, val, skip, st));
    for (const auto &lc : g->ccss_leaves) {
        EdgeBucketArgs b{};
        b.s = lc.s;
        b.N = g->N;
        b.K = lc.K;
        b.Km = lc.Km;
        b.Ke = lc.Ke;
        b.target = cached_level_target(g, lc.s - 1);
        int64_t cnt = lc.end - lc.begin;
        if (cnt <= 0) continue;
        ccss_leaf_kernel<T><<<(unsigned)((cnt + 127) / 128), 128, 0, st>>>(
            g->d_leaf_node, g->d_leaf_vertex, g->d_leaf_slot, lc.begin, lc.end, g->d_cc_off, x, val, b, o,
            g->d_cc_scale);
        S3_CUDA(cudaGetLastError());
    }
    // size-1 edges go through the edge path's single-member kernel
    for (size_t k = 0; k < g->buckets.size(); ++k) {
        const HostBucket &hb = g->buckets[k];
        if (hb.s != 1) continue;
        EdgeBucketArgs b{};
        b.ids = g->d_ids + hb.offset;
        b.slot = g->d_slot + hb.offset;
        b.m = hb.m;
        b.ld = hb.ld;
        b.s = 1;
        b.N = g->N;
        b.target = g->target[k];
        b.K = g->K[k];
        b.Km = g->Km[k];
        b.Ke = g->Ke[k];
        cudaError_t e = sizeof(T) == 4 ? launch_edge_bucket_f32(b, (const float *)x, o, 0, 0, st)
                                       : launch_edge_bucket_f64(b, (const double *)x, o, 0, 0, st);
        if (e != cudaSuccess) return cuda_fail(e, "single-member launch");
    }
    if (seg) {
        const ReduceArgs r = reduce_args(g, skip);
        cudaError_t e = sizeof(T) == 4 ? launch_reduce_f32(r, (const float *)g->d_buf, (float *)y, st)
                                       : launch_reduce_f64(r, (const double *)g->d_buf, (double *)y, st);
        if (e != cudaSuccess) return cuda_fail(e, "reduce launch");
    } else if (sizeof(T) == 4) {
        cudaError_t e = launch_add_comp((float *)y, g->d_comp, g->n, skip, st);
        if (e != cudaSuccess) return cuda_fail(e, "compensation launch");
    }
    return S3_OK;
}

}  // namespace

s3_status run_ccss(s3_graph_s *g, s3_dtype dt, const void *x, void *y, int bias, const int32_t *skip,
                   cudaStream_t st) {
    if (dt == S3_F32) return run_ccss_t<float>(g, (const float *)x, (float *)y, bias, skip, st);
    return run_ccss_t<double>(g, (const double *)x, (double *)y, bias, skip, st);
}

s3_status upload_ccss(s3_graph_s *g, const HostFormat &f) {
    const HostCCSS &c = f.ccss;
    s3_status st;
    auto up32 = [&](int32_t **d, const std::vector<int32_t> &h) -> s3_status {
        s3_status s = dev_alloc(g, d, h.size());
        if (s != S3_OK) return s;
        if (!h.empty()) S3_CUDA(cudaMemcpy(*d, h.data(), h.size() * 4, cudaMemcpyHostToDevice));
        return S3_OK;
    };
    if ((st = up32(&g->d_cc_vertex, c.vertex)) != S3_OK) return st;
    if ((st = up32(&g->d_cc_parent, c.parent)) != S3_OK) return st;
    if ((st = up32(&g->d_cc_width, c.width)) != S3_OK) return st;
    if ((st = up32(&g->d_leaf_node, c.leaf_node)) != S3_OK) return st;
    if ((st = up32(&g->d_leaf_vertex, c.leaf_vertex)) != S3_OK) return st;
    if ((st = up32(&g->d_leaf_slot, c.leaf_slot)) != S3_OK) return st;
    if ((st = dev_alloc(g, &g->d_cc_off, c.value_off.size())) != S3_OK) return st;
    if (!c.value_off.empty())
        S3_CUDA(cudaMemcpy(g->d_cc_off, c.value_off.data(), c.value_off.size() * 8, cudaMemcpyHostToDevice));
    double *vals = nullptr;
    if ((st = dev_alloc(g, &vals, (size_t)c.value_len)) != S3_OK) return st;
    g->d_cc_values = vals;
    g->cc_value_len = c.value_len;
    if ((st = dev_alloc(g, &g->d_cc_scale, 2)) != S3_OK) return st;
    for (const auto &sg : c.segs) g->ccss_segs.push_back({sg.level, sg.width, sg.begin, sg.end});
    for (const auto &lc : c.leaf_classes) {
        double K = scale_K(lc.s, f.N);
        int e = 0;
        double mant = std::frexp(K, &e);
        g->ccss_leaves.push_back({lc.s, lc.begin, lc.end, K, (float)mant, e});
    }
    g->cc_level_target.assign(S3_MAX_RANK + 2, 1.0f);
    for (int l = 1; l <= S3_MAX_RANK && l < f.N; ++l) g->cc_level_target[l] = level_target(l, f.N);
    g->has_ccss = true;
    return S3_OK;
}

}  // namespace s3
