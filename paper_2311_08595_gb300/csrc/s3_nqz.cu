// H-eigenvector centrality by Algorithm 1 (NQZ) on the device.
//
//   y = 1/n;  z = TTSV1(y)
//   repeat  x = z^[1/(N-1)] / ||z^[1/(N-1)]||_1 ;  z = TTSV1(x)
//           lambda_min/max = min/max z ./ x^[N-1]
//   until   (lambda_max - lambda_min) / lambda_min < tau
//
// z is never formed directly: TTSV1 runs in "biased" mode and returns
// zt_v = z_v 2^(-(N-1) e_v), where x_v = m_v 2^(e_v), m_v in [0.5, 1), is the
// vector the call used.  Then z_v^(1/(N-1)) = zt_v^(1/(N-1)) 2^(e_v) and
// z_v / x_v^(N-1) = zt_v / m_v^(N-1), so neither tiny x (x_v ~ 1/n) nor large
// ranks push anything out of range.  Roots and ratios are FP64-accurate (double-float
// on the FP32 units), the 1-norm and the bracket FP64; the series products are FP64, or FP32 until the gap stops
// shrinking or drops below switch_tol and then FP64 or double-float (pairs of
// FP32, S3_DF64), or double-float throughout (the precision option).
// Iterations run in captured CUDA graphs of `check_every` steps; a device flag
// turns the remaining launches of a graph into no-ops once the test passes.  The
// instantiated graphs stay on the handle and are replayed by later calls with
// the same tolerance, iteration cap and graph length.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "s3_graph.h"
#include "s3_series.cuh"

namespace s3 {
namespace {

constexpr int kNqzThreads = 256;
constexpr int kNqzBlocks = 592;   // 4 x 148..152 SMs; fixed so sums are reproducible

// flags: [0] done, [1] iterations, [2] hit max_iter, [3] range trouble, [4] block counter
enum { F_DONE = 0, F_ITERS = 1, F_MAXED = 2, F_RANGE = 3 };

// 1/y for y > 0 to FP32 accuracy (relative error below 2^-22), as a double: the FP32
// reciprocal of y's mantissa, scaled back by y's exponent (exact), so no range is lost.
__device__ __forceinline__ double rcp_seed(double y) {
    const int ey = Arith<double>::expo(y);
    const float my = (float)(y * Arith<double>::pow2(-ey));   // [0.5, 1)
    return (double)__frcp_rn(my) * Arith<double>::pow2(-ey);
}

// r = a^(1/k) for a > 0: FP32 guess then one Newton step in FP64.
__device__ __forceinline__ double root_k(double a, int k) {
    if (!(a > 0.0)) return 0.0;
    if (k == 1) return a;
    // a = ma 2^ea; a^(1/k) = ma^(1/k) 2^(ea/k) with ea/k split into integer and fraction
    int ea = Arith<double>::expo(a);
    double ma = a * Arith<double>::pow2(-ea);                  // [0.5, 1)
    int q = ea >= 0 ? ea / k : -((-ea + k - 1) / k);           // floor(ea / k)
    int rem = ea - q * k;                                      // 0..k-1
    double b = ma * Arith<double>::pow2(rem);                  // a = b 2^(q k), b in [0.5, 2^(k-1))
    double r = (double)powf((float)b, 1.0f / (float)k);        // ~1e-7 relative
    // Newton on r^k = b: r <- r - (r^k - b) / (k r^(k-1))
    double rk1 = 1.0, base = r;
    for (int e = k - 1; e > 0; e >>= 1) {
        if (e & 1) rk1 *= base;
        base *= base;
    }
    // the step's own size is ~1e-7 r, so its divisor needs FP32 accuracy only
    r = r - fma(rk1, r, -b) * rcp_seed((double)k * rk1);
    return r * Arith<double>::pow2(q);
}

// ---- the per-node pass in double-float arithmetic (pairs of FP32, struct DF) -------------
// GB300 runs FP32 at 64x its FP64 rate, so the roots and ratios of the per-node pass are
// computed on the FP32 units with about 46 significant bits; only the iterate's store and
// its 1-norm stay FP64.

// a positive normal number as a double-float mantissa in [0.5, 1) and its exponent, by
// integer operations on its bits (the lower 29 bits of a double's significand go to lo)
__device__ __forceinline__ DF mant_df(double a, int &ea) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(a);
    ea = (int)((bits >> 52) & 0x7ff) - 1022;
    const unsigned long long M = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const float hi = __uint_as_float((126u << 23) | (unsigned)((M >> 29) & 0x7FFFFFull));
    const float lo = __fmul_rn(__uint2float_rn((unsigned)(M & 0x1FFFFFFFull)), 0x1p-53f);
    return DF{hi, lo};
}
__device__ __forceinline__ DF mant_df(float a, int &ea) {
    const unsigned bits = __float_as_uint(a);
    ea = (int)((bits >> 23) & 0xffu) - 126;
    return DF{__uint_as_float((126u << 23) | (bits & 0x7FFFFFu)), 0.f};
}
__device__ __forceinline__ bool pos_normal(double a) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(a);
    const unsigned ef = (unsigned)((bits >> 52) & 0x7ff);
    return (bits >> 63) == 0 && ef != 0 && ef != 0x7ff;
}
__device__ __forceinline__ bool pos_normal(float a) {
    const unsigned bits = __float_as_uint(a);
    const unsigned ef = (bits >> 23) & 0xffu;
    return (bits >> 31) == 0 && ef != 0 && ef != 0xff;
}

// 2^p as a float, -126 <= p <= 127
__device__ __forceinline__ float pow2f(int p) { return __uint_as_float((unsigned)(p + 127) << 23); }

// h^k, k >= 1, by left-to-right binary powering
__device__ __forceinline__ DF df_pow(DF h, int k) {
    DF r = h;
    for (int b = 30 - __clz(k); b >= 0; --b) {
        r = r * r;
        if ((k >> b) & 1) r = r * h;
    }
    return r;
}

// a / b for b > 0: the FP32 quotient and one correction from the double-float residual
__device__ __forceinline__ DF df_div(DF a, DF b) {
    const float rb = __frcp_rn(b.hi);
    const float q0 = __fmul_rn(a.hi, rb);
    const DF p = DF{q0, 0.f} * b;
    const DF r = a + DF{-p.hi, -p.lo};
    return df_fast_two_sum(q0, __fmul_rn(__fadd_rn(r.hi, r.lo), rb));
}

// b^(1/k) for b in [0.5, 2^(k-1)): FP32 seed (relative error e of a few 2^-24), then one Newton
// step r <- r - (r^k - b) / (k r^(k-1)) with the residual in double-float (the divisor needs FP32
// accuracy only): relative error about (k-1) e^2 / 2, about 7e-13 at rank 25 and 4e-12 at rank
// 128 -- inside what the iteration's 1e-8 bracket and its FP64 results need (a second step, a
// third of the per-node pass's dependent chain, would not change the iterate that matters)
__device__ __forceinline__ DF root_df(DF b, int k) {
    if (k == 1) return b;
    DF r{powf(b.hi, 1.0f / (float)k), 0.f};
    {
        const DF rk1 = df_pow(r, k - 1);
        const DF res = rk1 * r + DF{-b.hi, -b.lo};
        // rk1 < 2^(k-1) <= 2^126: its reciprocal is a normal float; 1/k separately (k rk1 may overflow)
        const float corr = __fmul_rn(__fmul_rn(__fadd_rn(res.hi, res.lo), __frcp_rn(rk1.hi)), __frcp_rn((float)k));
        r = r + DF{-corr, 0.f};
    }
    return r;
}

// ratio m 2^E with m (double-float) in [0.5, 1): ordered by E, then m
struct DFE {
    DF m;
    int E;
};
__device__ __forceinline__ bool dfe_less(const DFE &a, const DFE &b) {
    return a.E < b.E || (a.E == b.E && (a.m.hi < b.m.hi || (a.m.hi == b.m.hi && a.m.lo < b.m.lo)));
}

// z / x^k from the biased zt = zm 2^ez and x = m 2^ex (zm, m in [0.5, 1)): zt / m^k =
// (zm / (2m)^k) 2^(ez + k), with (2m)^k in [1, 2^127) kept in FP32 range
__device__ __forceinline__ DFE ratio_df(DF zm, int ez, DF m, int k) {
    const DF pk = df_pow(DF{m.hi * 2.f, m.lo * 2.f}, k);
    const int pe = (int)((__float_as_uint(pk.hi) >> 23) & 0xffu) - 127;   // pk = pkm 2^pe, pkm in [1, 2)
    const float sc = pow2f(-pe);
    DF q = df_div(zm, DF{pk.hi * sc, pk.lo * sc});                          // in (0.25, 1)
    int E = ez + k - pe;
    if (q.hi < 0.5f) {
        q = DF{q.hi * 2.f, q.lo * 2.f};
        --E;
    }
    return DFE{q, E};
}

__device__ __forceinline__ double dfe_to_double(const DFE &a) {
    return ((double)a.m.hi + (double)a.m.lo) * Arith<double>::pow2(a.E);
}

// flags[F_COUNT]: blocks of the current after-kernel that have stored their partials
enum { F_COUNT = 4 };

// Sum (fixed order: warp trees, then warps in order) of one value per thread; thread 0 gets it.
__device__ __forceinline__ double block_sum(double v, double *sh) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kNqzThreads / 32; ++w) t += sh[w];
    return t;
}

__device__ __forceinline__ void block_minmax(double &lo, double &hi, double *sl, double *sh) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        lo = fmin(lo, __shfl_down_sync(0xffffffffu, lo, d));
        hi = fmax(hi, __shfl_down_sync(0xffffffffu, hi, d));
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
        sl[threadIdx.x >> 5] = lo;
        sh[threadIdx.x >> 5] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int w = 1; w < kNqzThreads / 32; ++w) {
            lo = fmin(lo, sl[w]);
            hi = fmax(hi, sh[w]);
        }
}

// Everything Algorithm 1 does with one S^3TTVc result z (biased: zt) of the iterate x:
//  * unless `first`: the ratios zt_v / m_v^(N-1) (= z_v / x_v^(N-1), m_v = x_v 2^-e_v) and
//    their min and max -- lambda_min, lambda_max of this pass -- and the stopping test;
//  * the next iterate before normalisation, u_v = zt_v^(1/(N-1)) 2^e_v (= z_v^(1/(N-1))),
//    and its 1-norm, whose inverse goes to scal[0] for nqz_normalize_kernel.
// Each block stores partial sums / minima / maxima; the last block to finish (a counter in
// flags) reduces them in a fixed order with all its threads, so the results do not depend
// on which block is last.
template <typename T>
__global__ void __launch_bounds__(kNqzThreads) nqz_after_kernel(const T *__restrict__ zt, const T *__restrict__ xin,
                                                                int64_t n, int k, int first, double *__restrict__ u,
                                                                double *__restrict__ part_sum,
                                                                double *__restrict__ part_mm, double *__restrict__ scal,
                                                                double tol, int max_iter, double *__restrict__ hist,
                                                                int hist_cap, int32_t *flags) {
    if (flags[F_DONE]) return;
    __shared__ double sa[kNqzThreads / 32], sb[kNqzThreads / 32];
    __shared__ int last;
    double acc = 0.0, lo = INFINITY, hi = -INFINITY;
    DFE rlo{DF{1.f, 0.f}, INT_MAX}, rhi{DF{0.5f, 0.f}, INT_MIN};
    bool bad = false;
    for (int64_t v = (int64_t)blockIdx.x * kNqzThreads + threadIdx.x; v < n; v += (int64_t)gridDim.x * kNqzThreads) {
        const T zv = zt[v], xv = xin[v];
        if (!pos_normal(zv) || !pos_normal(xv)) {
            bad = true;
            u[v] = 0.0;
            continue;
        }
        int ez, ex;
        const DF zm = mant_df(zv, ez), m = mant_df(xv, ex);
        // zt = b 2^(q k) with b = zm 2^rem in [0.5, 2^(k-1)); z^(1/k) = b^(1/k) 2^(q + ex)
        const int q = ez >= 0 ? ez / k : -((-ez + k - 1) / k);
        const float sb = pow2f(ez - q * k);
        const DF r = root_df(DF{zm.hi * sb, zm.lo * sb}, k);
        const double rv = ((double)r.hi + (double)r.lo) * Arith<double>::pow2(q + ex);
        u[v] = rv;
        acc += rv;
        if (!first) {
            const DFE ratio = ratio_df(zm, ez, m, k);
            if (dfe_less(ratio, rlo)) rlo = ratio;
            if (dfe_less(rhi, ratio)) rhi = ratio;
        }
    }
    if (!first && rlo.E != INT_MAX) {
        lo = dfe_to_double(rlo);
        hi = dfe_to_double(rhi);
    }
    const int any_bad = __syncthreads_or(bad);
    const double bsum = block_sum(acc, sa);
    if (!first) block_minmax(lo, hi, sa, sb);
    if (threadIdx.x == 0) {
        if (any_bad) flags[F_RANGE] = 1;
        part_sum[blockIdx.x] = bsum;
        if (!first) {
            part_mm[2 * blockIdx.x] = lo;
            part_mm[2 * blockIdx.x + 1] = hi;
        }
        __threadfence();
        last = atomicAdd(flags + F_COUNT, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // the last block: reduce the partials (L2 loads: other blocks wrote them)
    acc = 0.0;
    lo = INFINITY;
    hi = -INFINITY;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += kNqzThreads) {
        acc += __ldcg(part_sum + i);
        if (!first) {
            lo = fmin(lo, __ldcg(part_mm + 2 * i));
            hi = fmax(hi, __ldcg(part_mm + 2 * i + 1));
        }
    }
    const double tot = block_sum(acc, sa);
    if (!first) block_minmax(lo, hi, sa, sb);
    if (threadIdx.x == 0) {
        scal[0] = 1.0 / tot;
        flags[F_COUNT] = 0;
        if (!first) {
            const int it = __ldcg(flags + F_ITERS);
            if (it < hist_cap) {
                hist[2 * it] = lo;
                hist[2 * it + 1] = hi;
            }
            flags[F_ITERS] = it + 1;
            if ((hi - lo) / lo < tol) flags[F_DONE] = 1;
            if (it + 1 >= max_iter) {
                flags[F_DONE] = 1;
                flags[F_MAXED] = 1;
            }
        }
        if (__ldcg(flags + F_RANGE)) flags[F_DONE] = 1;
    }
}

// x = u / ||u||_1 (FP64) and its FP32 copy
__global__ void __launch_bounds__(kNqzThreads) nqz_normalize_kernel(const double *__restrict__ u, int64_t n,
                                                                    const double *__restrict__ scal,
                                                                    double *__restrict__ x64, float *__restrict__ x32,
                                                                    int32_t *flags) {
    if (flags[F_DONE]) return;
    const double inv = scal[0];
    for (int64_t v = (int64_t)blockIdx.x * kNqzThreads + threadIdx.x; v < n; v += (int64_t)gridDim.x * kNqzThreads) {
        const double xv = u[v] * inv;
        x64[v] = xv;
        x32[v] = (float)xv;
    }
}

template <typename T>
__global__ void fill_kernel(T *p, int64_t n, T v) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

template <typename T>
__global__ void copy_cast_kernel(const double *src, T *dst, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = (T)src[i];
}

s3_status ensure_nqz_scratch(s3_graph_s *g, int hist_cap) {
    s3_status st;
    if (!g->d_nqz) {
        if ((st = dev_alloc(g, &g->d_nqz, 4 * (size_t)g->n)) != S3_OK) return st;
        if ((st = dev_alloc(g, &g->d_x32, (size_t)g->n)) != S3_OK) return st;
        if ((st = dev_alloc(g, &g->d_z32, (size_t)g->n)) != S3_OK) return st;
        if ((st = dev_alloc(g, &g->d_red, 4 * (size_t)kNqzBlocks)) != S3_OK) return st;
        if ((st = dev_alloc(g, &g->d_flags, 8)) != S3_OK) return st;
    }
    if (g->hist_cap < hist_cap) {
        if ((st = dev_alloc(g, &g->d_hist, 2 * (size_t)hist_cap)) != S3_OK) return st;
        g->hist_cap = hist_cap;
    }
    return S3_OK;
}

struct NqzBufs {
    double *x64, *u, *z64;
    float *x32, *z32;
    double *part_sum, *part_mm, *scal;
    int32_t *flags;
};

// The kernel that takes the S^3TTVc result of type dt (see nqz_after_kernel).
s3_status nqz_after(s3_graph_s *g, const NqzBufs &b, s3_dtype dt, bool first, double tol, int max_iter,
                    cudaStream_t st) {
    const int k = g->N - 1;
    if (dt == S3_F32)
        nqz_after_kernel<float><<<kNqzBlocks, kNqzThreads, 0, st>>>(b.z32, b.x32, g->n, k, first ? 1 : 0, b.u,
                                                                     b.part_sum, b.part_mm, b.scal, tol, max_iter,
                                                                     g->d_hist, g->hist_cap, b.flags);
    else
        nqz_after_kernel<double><<<kNqzBlocks, kNqzThreads, 0, st>>>(b.z64, b.x64, g->n, k, first ? 1 : 0, b.u,
                                                                      b.part_sum, b.part_mm, b.scal, tol, max_iter,
                                                                      g->d_hist, g->hist_cap, b.flags);
    S3_CUDA(cudaGetLastError());
    return S3_OK;
}

// One repeat-body pass of Algorithm 1: normalise the pending root vector u into x, z =
// S^3TTVc(x) with series of type tc, then ratios, bracket, test and the next u.
s3_status nqz_step(s3_graph_s *g, const NqzBufs &b, s3_dtype tc, double tol, int max_iter, cudaStream_t st) {
    const int64_t n = g->n;
    nqz_normalize_kernel<<<kNqzBlocks, kNqzThreads, 0, st>>>(b.u, n, b.scal, b.x64, b.x32, b.flags);
    S3_CUDA(cudaGetLastError());
    s3_status s;
    if (tc == S3_F32)
        s = g->opt.layout == S3_LAYOUT_CCSS && g->has_ccss ? run_ccss(g, S3_F32, b.x32, b.z32, 1, b.flags, st)
                                                            : run_edges(g, S3_F32, b.x32, b.z32, 1, b.flags, st);
    else
        // tc: S3_F64 or S3_DF64 (FP64 vectors either way; the CCSS layout runs FP64)
        s = g->opt.layout == S3_LAYOUT_CCSS && g->has_ccss ? run_ccss(g, S3_F64, b.x64, b.z64, 1, b.flags, st)
                                                            : run_edges(g, tc, b.x64, b.z64, 1, b.flags, st);
    if (s != S3_OK) return s;
    return nqz_after(g, b, tc == S3_F32 ? S3_F32 : S3_F64, false, tol, max_iter, st);
}

// ------------------------------------------ one NQZ update from a whole z --
//
// For callers that assemble z = B xhat^(N-1) themselves (e.g. the sum of the
// partial results of edge shards on several GPUs): the bracket of Algorithm 1
// from z and xhat, and the next iterate r = z^(1/(N-1)) both with 1-norm 1 and
// rescaled to max 1 (the ratio z / xhat^(N-1) does not depend on the scale of
// xhat, so the S^3TTVc input can be kept at max 1 and z in range).

enum { US_LO = 0, US_HI = 1, US_SUM = 2, US_MAX = 3 };

__global__ void __launch_bounds__(kNqzThreads) nqz_update_kernel(const double *__restrict__ z,
                                                                 const double *__restrict__ xhat, int64_t n, int k,
                                                                 double *__restrict__ r, double *__restrict__ part,
                                                                 double *__restrict__ scal, int32_t *flags) {
    __shared__ double sa[kNqzThreads / 32], sb[kNqzThreads / 32];
    __shared__ int last;
    double acc = 0.0, mx = 0.0, lo = INFINITY, hi = -INFINITY;
    for (int64_t v = (int64_t)blockIdx.x * kNqzThreads + threadIdx.x; v < n; v += (int64_t)gridDim.x * kNqzThreads) {
        const double zv = z[v];
        double pk = 1.0, base = xhat[v];
        for (int q = k; q > 0; q >>= 1) {
            if (q & 1) pk *= base;
            base *= base;
        }
        const double ratio = zv / pk;
        lo = fmin(lo, ratio);
        hi = fmax(hi, ratio);
        const double rv = root_k(zv, k);
        r[v] = rv;
        acc += rv;
        mx = fmax(mx, rv);
    }
    const double bsum = block_sum(acc, sa);
    block_minmax(lo, hi, sa, sb);
    double dummy = 0.0;
    block_minmax(dummy, mx, sa, sb);
    if (threadIdx.x == 0) {
        part[4 * blockIdx.x] = bsum;
        part[4 * blockIdx.x + 1] = lo;
        part[4 * blockIdx.x + 2] = hi;
        part[4 * blockIdx.x + 3] = mx;
        __threadfence();
        last = atomicAdd(flags + F_COUNT, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    acc = 0.0;
    mx = 0.0;
    lo = INFINITY;
    hi = -INFINITY;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += kNqzThreads) {
        acc += __ldcg(part + 4 * i);
        lo = fmin(lo, __ldcg(part + 4 * i + 1));
        hi = fmax(hi, __ldcg(part + 4 * i + 2));
        mx = fmax(mx, __ldcg(part + 4 * i + 3));
    }
    const double tot = block_sum(acc, sa);
    block_minmax(lo, hi, sa, sb);
    dummy = 0.0;
    block_minmax(dummy, mx, sa, sb);
    if (threadIdx.x == 0) {
        scal[US_LO] = lo;
        scal[US_HI] = hi;
        scal[US_SUM] = tot;
        scal[US_MAX] = mx;
        flags[F_COUNT] = 0;
    }
}

__global__ void __launch_bounds__(kNqzThreads) nqz_update_scale_kernel(const double *__restrict__ r, int64_t n,
                                                                       const double *__restrict__ scal,
                                                                       double *__restrict__ x1,
                                                                       double *__restrict__ xmax) {
    const double inv_sum = 1.0 / scal[US_SUM], inv_max = 1.0 / scal[US_MAX];
    for (int64_t v = (int64_t)blockIdx.x * kNqzThreads + threadIdx.x; v < n; v += (int64_t)gridDim.x * kNqzThreads) {
        const double rv = r[v];
        x1[v] = rv * inv_sum;
        xmax[v] = rv * inv_max;
    }
}

// ------------------------------------------------ Z-eigenpairs (SS-HOPM) --
//
// The shifted power method for the order-N blowup tensor (Sec. I names it and
// symmetric CP as consumers of S^3TTVc): x <- (B x^(N-1) + alpha x)/||.||_2,
// lambda = x . B x^(N-1).  S^3TTVc runs on xhat = x / m (m = max |x|, so xhat
// has entries <= 1 at any rank); with zhat = B xhat^(N-1) = B x^(N-1) / m^(N-1)
//     w = zhat - sum_q c_q x_q + sigma x,   sigma = alpha m^-(N-1),
//     c_q = lambda_q (x_q . xhat)^(N-1)     (greedy CP: the deflated components),
//     lambda = m^(N-1) x . (zhat - sum_q c_q x_q),
// and w is a positive multiple of the true shifted product.

constexpr int kZeigMaxR = 32;
// scalars: sigma, ||w||_2, x . zd, max |w|, m; deflation coefficients c_q and lambda_q
enum { ZS_SIGMA = 1, ZS_NORM = 2, ZS_DOT = 3, ZS_MAX = 4, ZS_M = 5, ZS_C = 8, ZS_LAM = 8 + kZeigMaxR,
       ZS_LEN = 8 + 2 * kZeigMaxR };

// d_q = X_q . xhat for q < R (X: R rows of n), then c_q = lambda_q d_q^k in the last block.
__global__ void __launch_bounds__(kNqzThreads) zeig_dots_kernel(const double *__restrict__ X, int R,
                                                                const double *__restrict__ xhat, int64_t n, int k,
                                                                double *__restrict__ part, double *__restrict__ scal,
                                                                int32_t *flags) {
    __shared__ double sa[kNqzThreads / 32];
    __shared__ int last;
    for (int q = 0; q < R; ++q) {
        double acc = 0.0;
        for (int64_t v = (int64_t)blockIdx.x * kNqzThreads + threadIdx.x; v < n; v += (int64_t)gridDim.x * kNqzThreads)
            acc += X[(int64_t)q * n + v] * xhat[v];
        const double b = block_sum(acc, sa);
        if (threadIdx.x == 0) part[(int64_t)q * gridDim.x + blockIdx.x] = b;
    }
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(flags + F_COUNT, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int q = 0; q < R; ++q) {
        double acc = 0.0;
        for (int i = threadIdx.x; i < (int)gridDim.x; i += kNqzThreads) acc += __ldcg(part + (int64_t)q * gridDim.x + i);
        const double d = block_sum(acc, sa);
        if (threadIdx.x == 0) {
            double p = 1.0, base = d;
            for (int e = k; e > 0; e >>= 1) {
                if (e & 1) p *= base;
                base *= base;
            }
            scal[ZS_C + q] = scal[ZS_LAM + q] * p;
        }
    }
    if (threadIdx.x == 0) flags[F_COUNT] = 0;
}

// w = zhat - sum_q c_q X_q + sigma x; ||w||_2, x . (zhat - sum_q c_q X_q) and max |w| to scal.
__global__ void __launch_bounds__(kNqzThreads) zeig_update_kernel(const double *__restrict__ zhat,
                                                                  const double *__restrict__ x,
                                                                  const double *__restrict__ X, int R, int use_sigma,
                                                                  int64_t n, double *__restrict__ w,
                                                                  double *__restrict__ part, double *__restrict__ scal,
                                                                  int32_t *flags) {
    __shared__ double sa[kNqzThreads / 32], sb[kNqzThreads / 32];
    __shared__ double c[kZeigMaxR];
    __shared__ int last;
    if (threadIdx.x < R) c[threadIdx.x] = scal[ZS_C + threadIdx.x];
    __syncthreads();
    const double sigma = use_sigma ? scal[ZS_SIGMA] : 0.0;
    double s2 = 0.0, dot = 0.0, mx = 0.0;
    for (int64_t v = (int64_t)blockIdx.x * kNqzThreads + threadIdx.x; v < n; v += (int64_t)gridDim.x * kNqzThreads) {
        double zd = zhat[v];
        for (int q = 0; q < R; ++q) zd -= c[q] * X[(int64_t)q * n + v];
        const double xv = x[v];
        const double wv = fma(sigma, xv, zd);
        w[v] = wv;
        s2 = fma(wv, wv, s2);
        dot = fma(xv, zd, dot);
        mx = fmax(mx, fabs(wv));
    }
    const double b2 = block_sum(s2, sa);
    const double bd = block_sum(dot, sa);
    double lo = 0.0;
    block_minmax(lo, mx, sa, sb);
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x] = b2;
        part[3 * blockIdx.x + 1] = bd;
        part[3 * blockIdx.x + 2] = mx;
        __threadfence();
        last = atomicAdd(flags + F_COUNT, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    s2 = 0.0;
    dot = 0.0;
    mx = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += kNqzThreads) {
        s2 += __ldcg(part + 3 * i);
        dot += __ldcg(part + 3 * i + 1);
        mx = fmax(mx, __ldcg(part + 3 * i + 2));
    }
    const double t2 = block_sum(s2, sa);
    const double td = block_sum(dot, sa);
    lo = 0.0;
    block_minmax(lo, mx, sa, sb);
    if (threadIdx.x == 0) {
        scal[ZS_NORM] = sqrt(t2);
        scal[ZS_DOT] = td;
        scal[ZS_MAX] = mx;
        flags[F_COUNT] = 0;
    }
}

// x = w / ||w||_2, xhat = w / max |w|; m = max |x| and sigma = alpha m^-k for the next step.
__global__ void __launch_bounds__(kNqzThreads) zeig_normalize_kernel(const double *__restrict__ w, int64_t n,
                                                                     double *__restrict__ x, double *__restrict__ xhat,
                                                                     double *__restrict__ scal, double alpha, int k) {
    const double inv_norm = 1.0 / scal[ZS_NORM], inv_max = 1.0 / scal[ZS_MAX];
    for (int64_t v = (int64_t)blockIdx.x * kNqzThreads + threadIdx.x; v < n; v += (int64_t)gridDim.x * kNqzThreads) {
        x[v] = w[v] * inv_norm;
        xhat[v] = w[v] * inv_max;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const double m = scal[ZS_MAX] * inv_norm;
        double p = 1.0, base = 1.0 / m;
        for (int e = k; e > 0; e >>= 1) {
            if (e & 1) p *= base;
            base *= base;
        }
        scal[ZS_M] = m;
        scal[ZS_SIGMA] = fmin(alpha * p, 1e300);
    }
}

s3_status ensure_zeig_scratch(s3_graph_s *g) {
    s3_status st = ensure_nqz_scratch(g, 2);
    if (st != S3_OK) return st;
    if (!g->d_zeig) {
        if ((st = dev_alloc(g, &g->d_zeig, (size_t)(kZeigMaxR + 3) * kNqzBlocks + ZS_LEN)) != S3_OK) return st;
    }
    return S3_OK;
}

// One SS-HOPM run on B minus the R components in X (device rows) with eigenvalues lam[R]
// (host); x0 (device) or NULL = uniform start; result in x_out (device).
s3_status zeig_run(s3_graph_s *g, const s3_zeig_options &opt, const double *x0, const double *X, int R,
                   const double *lam, double *x_out, s3_zeig_result *res, cudaStream_t st) {
    s3_status s = ensure_zeig_scratch(g);
    if (s != S3_OK) return s;
    const int64_t n = g->n;
    const int k = g->N - 1;
    double *x = g->d_nqz, *w = g->d_nqz + n, *zhat = g->d_nqz + 2 * n, *xhat = g->d_nqz + 3 * n;
    double *part = g->d_zeig, *scal = g->d_zeig + (size_t)(kZeigMaxR + 3) * kNqzBlocks;
    int32_t *flags = g->d_flags;
    const unsigned gb = (unsigned)((n + 255) / 256);
    S3_CUDA(cudaMemsetAsync(flags, 0, 8 * sizeof(int32_t), st));
    S3_CUDA(cudaMemsetAsync(scal, 0, sizeof(double) * ZS_LEN, st));
    if (R > 0) {
        double h[kZeigMaxR];
        for (int q = 0; q < R; ++q) h[q] = lam[q];
        S3_CUDA(cudaMemcpyAsync(scal + ZS_LAM, h, sizeof(double) * R, cudaMemcpyHostToDevice, st));
        S3_CUDA(cudaStreamSynchronize(st));   // h lives on this stack frame
    }
    // start: normalise x0 (or the all-ones vector) through the update/normalise pair
    if (x0) S3_CUDA(cudaMemcpyAsync(zhat, x0, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    else fill_kernel<double><<<gb, 256, 0, st>>>(zhat, n, 1.0);
    zeig_update_kernel<<<kNqzBlocks, kNqzThreads, 0, st>>>(zhat, zhat, X, 0, 0, n, w, part, scal, flags);
    zeig_normalize_kernel<<<kNqzBlocks, kNqzThreads, 0, st>>>(w, n, x, xhat, scal, opt.alpha, k);
    S3_CUDA(cudaGetLastError());
    double hs[8];
    double lam_prev = 0.0, lam_cur = 0.0;
    int it = 0;
    res->converged = 0;
    for (;; ++it) {
        if (R > 0) zeig_dots_kernel<<<kNqzBlocks, kNqzThreads, 0, st>>>(X, R, xhat, n, k, part + 3 * kNqzBlocks, scal, flags);
        S3_CUDA(cudaGetLastError());
        s = run_edges(g, S3_F64, xhat, zhat, 0, nullptr, st);
        if (s != S3_OK) return s;
        zeig_update_kernel<<<kNqzBlocks, kNqzThreads, 0, st>>>(zhat, x, X, R, 1, n, w, part, scal, flags);
        S3_CUDA(cudaGetLastError());
        S3_CUDA(cudaMemcpyAsync(hs, scal, sizeof(hs), cudaMemcpyDeviceToHost, st));
        S3_CUDA(cudaStreamSynchronize(st));
        lam_cur = std::pow(hs[ZS_M], (double)k) * hs[ZS_DOT];
        if (!std::isfinite(lam_cur) || !(hs[ZS_NORM] > 0.0)) return fail(S3_ERANGE, "Z-eigenvalue left the FP64 range");
        if (it > 0 && std::fabs(lam_cur - lam_prev) < opt.tol * std::max(1.0, std::fabs(lam_cur))) {
            res->converged = 1;
            break;
        }
        if (it >= opt.max_iter) break;
        zeig_normalize_kernel<<<kNqzBlocks, kNqzThreads, 0, st>>>(w, n, x, xhat, scal, opt.alpha, k);
        S3_CUDA(cudaGetLastError());
        lam_prev = lam_cur;
    }
    res->lambda = lam_cur;
    res->iters = it;
    S3_CUDA(cudaMemcpyAsync(x_out, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    return S3_OK;
}

}  // namespace
}  // namespace s3

using namespace s3;

extern "C" {

s3_status s3_nqz_options_init(s3_nqz_options *opt) {
    if (!opt) return fail(S3_EINVAL, "opt is NULL");
    std::memset(opt, 0, sizeof(*opt));
    opt->tol = 1e-8;
    opt->max_iter = 10000;
    opt->precision = 0;
    opt->switch_tol = 1e-5;
    opt->check_every = 8;
    return S3_OK;
}

s3_status s3_hcentrality(s3_graph_t g, const s3_nqz_options *opt_in, const double *x0, double *x_out,
                         s3_nqz_result *res, void *stream) {
    auto t0 = std::chrono::steady_clock::now();
    if (!g || !x_out || !res) return fail(S3_EINVAL, "NULL argument");
    s3_nqz_options opt;
    if (opt_in) opt = *opt_in;
    else s3_nqz_options_init(&opt);
    if (opt.max_iter <= 0) opt.max_iter = 10000;
    if (opt.check_every <= 0) opt.check_every = 8;
    if (opt.switch_tol <= 0) opt.switch_tol = 1e-5;
    if (!(opt.tol > 0)) return fail(S3_EINVAL, "tol must be > 0");
    if (opt.precision < 0 || opt.precision > 3) return fail(S3_EINVAL, "precision must be in 0..3");
    if (g->N < 2) return fail(S3_EINVAL, "NQZ needs rank >= 2");
    DeviceGuard guard(g->device);
    cudaStream_t st = (cudaStream_t)stream;
    // graphs cannot be captured on the legacy default stream: use a blocking
    // stream of our own (it synchronises implicitly with the legacy stream)
    struct OwnStream {
        cudaStream_t s = nullptr;
        ~OwnStream() {
            if (s) cudaStreamDestroy(s);
        }
    } own;
    if (st == nullptr) {
        S3_CUDA(cudaStreamCreate(&own.s));
        st = own.s;
    }
    std::memset(res, 0, sizeof(*res));
    // isolated nodes (found when the handle was built) make the ratio 0/0
    if (g->first_isolated >= 0)
        return fail(S3_EINVAL, "node " + std::to_string(g->first_isolated) + " belongs to no edge");
    s3_status s = ensure_nqz_scratch(g, opt.max_iter + 2);
    if (s != S3_OK) return s;
    NqzBufs b;
    b.x64 = g->d_nqz;
    b.u = g->d_nqz + g->n;
    b.z64 = g->d_nqz + 2 * g->n;
    b.x32 = g->d_x32;
    b.z32 = g->d_z32;
    b.part_sum = g->d_red;
    b.part_mm = g->d_red + kNqzBlocks;
    b.scal = g->d_red + 3 * kNqzBlocks;
    b.flags = g->d_flags;
    const int64_t n = g->n;
    const unsigned gb = (unsigned)((n + 255) / 256);

    S3_CUDA(cudaMemsetAsync(b.flags, 0, 8 * sizeof(int32_t), st));
    // start vector y (Algorithm 1: 1/n) and z = TTSV1(y)
    const bool fp32 = opt.precision == 1 || opt.precision == 2;
    const s3_dtype hi = opt.precision >= 2 ? S3_DF64 : S3_F64;  // series after the FP32 phase
    s3_dtype phase = fp32 ? S3_F32 : hi;
    if (x0) {
        if (fp32) copy_cast_kernel<float><<<gb, 256, 0, st>>>(x0, b.x32, n);
        else copy_cast_kernel<double><<<gb, 256, 0, st>>>(x0, b.x64, n);
    } else {
        if (fp32) fill_kernel<float><<<gb, 256, 0, st>>>(b.x32, n, 1.0f / (float)n);
        else fill_kernel<double><<<gb, 256, 0, st>>>(b.x64, n, 1.0 / (double)n);
    }
    S3_CUDA(cudaGetLastError());
    const bool ccss = g->opt.layout == S3_LAYOUT_CCSS && g->has_ccss;
    auto ttsv = [&](s3_dtype dt) -> s3_status {
        if (dt == S3_F32)
            return ccss ? run_ccss(g, S3_F32, b.x32, b.z32, 1, b.flags, st) : run_edges(g, S3_F32, b.x32, b.z32, 1, b.flags, st);
        return ccss ? run_ccss(g, S3_F64, b.x64, b.z64, 1, b.flags, st) : run_edges(g, dt, b.x64, b.z64, 1, b.flags, st);
    };
    s = ttsv(phase);
    if (s != S3_OK) return s;
    // the first root vector (no bracket yet: Algorithm 1 tests only after the loop's S^3TTVc)
    s = nqz_after(g, b, phase == S3_F32 ? S3_F32 : S3_F64, true, opt.tol, opt.max_iter, st);
    if (s != S3_OK) return s;

    int32_t flags[8] = {0};
    std::vector<double> hist;
    s3_dtype last_z = phase;
    bool switched = !fp32;
    int fp32_iters = 0;
    double best_prev = INFINITY, best_cur = INFINITY;
    while (true) {
        const double tol = phase == S3_F32 ? std::max(opt.switch_tol, opt.tol) : opt.tol;
        // a graph of check_every passes (the first pass after a precision change runs eagerly)
        if (last_z != phase) {
            s = nqz_step(g, b, phase, tol, opt.max_iter, st);
            if (s != S3_OK) return s;
            last_z = phase;
        } else {
            // captured passes are kept on the handle and reused while the settings match
            s3_graph_s::NqzExec &ce_ = g->nqz_exec[phase == S3_F32 ? 0 : phase == S3_F64 ? 1 : 2];
            if (ce_.exec && (ce_.tol != tol || ce_.max_iter != opt.max_iter || ce_.check_every != opt.check_every ||
                             ce_.hist != g->d_hist)) {
                cudaGraphExecDestroy(ce_.exec);
                ce_.exec = nullptr;
            }
            cudaGraphExec_t &exec = ce_.exec;
            if (!exec) {
                cudaGraph_t graph = nullptr;
                S3_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
                s3_status cs = S3_OK;
                for (int i = 0; i < opt.check_every && cs == S3_OK; ++i)
                    cs = nqz_step(g, b, phase, tol, opt.max_iter, st);
                cudaError_t ce = cudaStreamEndCapture(st, &graph);
                if (cs != S3_OK) {
                    if (graph) cudaGraphDestroy(graph);
                    return cs;
                }
                S3_CUDA(ce);
                ce = cudaGraphInstantiate(&exec, graph, 0);
                cudaGraphDestroy(graph);
                S3_CUDA(ce);
                ce_.tol = tol;
                ce_.max_iter = opt.max_iter;
                ce_.check_every = opt.check_every;
                ce_.hist = g->d_hist;
            }
            S3_CUDA(cudaGraphLaunch(exec, st));
        }
        S3_CUDA(cudaMemcpyAsync(flags, b.flags, 8 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        S3_CUDA(cudaStreamSynchronize(st));
        const int iters = flags[F_ITERS];
        hist.resize(2 * (size_t)iters);
        if (iters > 0)
            S3_CUDA(cudaMemcpy(hist.data(), g->d_hist, sizeof(double) * 2 * std::min(iters, g->hist_cap),
                               cudaMemcpyDeviceToHost));
        if (phase == S3_F32) fp32_iters = iters;
        const bool done = flags[F_DONE] != 0;
        if (phase == S3_F32) {
            // stagnation: the best gap of the last chunk is not clearly below the previous one
            best_prev = best_cur;
            best_cur = INFINITY;
            for (int i = std::max(0, iters - opt.check_every); i < iters; ++i) {
                double lo = hist[2 * i], hi = hist[2 * i + 1];
                best_cur = std::min(best_cur, (hi - lo) / lo);
            }
            const bool stalled = best_cur > 0.5 * best_prev;
            if (done || stalled || flags[F_RANGE]) {
                if (flags[F_MAXED]) break;
                // hand over to FP64: clear done/range, keep the iteration count
                int32_t zero = 0;
                S3_CUDA(cudaMemcpyAsync(b.flags + F_DONE, &zero, sizeof(int32_t), cudaMemcpyHostToDevice, st));
                S3_CUDA(cudaMemcpyAsync(b.flags + F_RANGE, &zero, sizeof(int32_t), cudaMemcpyHostToDevice, st));
                S3_CUDA(cudaStreamSynchronize(st));
                phase = hi;
                switched = true;
                if (flags[F_RANGE]) {
                    // the last FP32 z is unusable: redo z = TTSV1(x) in FP64 from the same x,
                    // and the root vector from it
                    s = ttsv(hi);
                    if (s != S3_OK) return s;
                    s = nqz_after(g, b, S3_F64, true, opt.tol, opt.max_iter, st);
                    if (s != S3_OK) return s;
                    last_z = hi;
                }
                continue;
            }
        } else if (done) {
            break;
        }
        if (iters >= opt.max_iter) break;
    }
    (void)switched;
    const int iters = flags[F_ITERS];
    res->iters = iters;
    res->iters_fp32 = fp32 ? fp32_iters : 0;
    if (iters > 0) {
        int i = std::min(iters, g->hist_cap) - 1;
        res->lambda_min = hist[2 * i];
        res->lambda_max = hist[2 * i + 1];
        res->converged = (res->lambda_max - res->lambda_min) / res->lambda_min < opt.tol;
    }
    S3_CUDA(cudaMemcpyAsync(x_out, b.x64, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    {
        s3_status ms = mark_done(g, st);
        if (ms != S3_OK) return ms;
    }
    S3_CUDA(cudaStreamSynchronize(st));
    res->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (flags[F_RANGE] && !res->converged) return fail(S3_ERANGE, "ratio z/x^(N-1) left the FP64 range");
    if (!res->converged) return fail(S3_ENOCONV, "NQZ did not reach the tolerance within max_iter");
    return S3_OK;
}

s3_status s3_nqz_update(s3_graph_t g, const double *z, const double *xhat, double *x_next, double *xhat_next,
                        double *lambda, void *stream) {
    if (!g || !z || !xhat || !x_next || !xhat_next || !lambda) return fail(S3_EINVAL, "NULL argument");
    if (g->N < 2) return fail(S3_EINVAL, "NQZ needs rank >= 2");
    if (x_next == xhat_next) return fail(S3_EINVAL, "x_next and xhat_next must differ");
    DeviceGuard guard(g->device);
    cudaStream_t st = (cudaStream_t)stream;
    s3_status s = ensure_zeig_scratch(g);
    if (s != S3_OK) return s;
    double *part = g->d_zeig, *scal = g->d_zeig + (size_t)(kZeigMaxR + 3) * kNqzBlocks;
    S3_CUDA(cudaMemsetAsync(g->d_flags + F_COUNT, 0, sizeof(int32_t), st));
    nqz_update_kernel<<<kNqzBlocks, kNqzThreads, 0, st>>>(z, xhat, g->n, g->N - 1, x_next, part, scal, g->d_flags);
    nqz_update_scale_kernel<<<kNqzBlocks, kNqzThreads, 0, st>>>(x_next, g->n, scal, x_next, xhat_next);
    S3_CUDA(cudaGetLastError());
    double h[4];
    S3_CUDA(cudaMemcpyAsync(h, scal, sizeof(h), cudaMemcpyDeviceToHost, st));
    s = mark_done(g, st);
    if (s != S3_OK) return s;
    S3_CUDA(cudaStreamSynchronize(st));
    lambda[0] = h[US_LO];
    lambda[1] = h[US_HI];
    if (!(h[US_LO] > 0.0) || !std::isfinite(h[US_HI]) || !(h[US_SUM] > 0.0))
        return fail(S3_ERANGE, "NQZ ratios or roots left the FP64 range (a node with z = 0 or x = 0?)");
    return S3_OK;
}

s3_status s3_zeig_options_init(s3_zeig_options *opt) {
    if (!opt) return fail(S3_EINVAL, "opt is NULL");
    std::memset(opt, 0, sizeof(*opt));
    opt->alpha = 0.0;
    opt->tol = 1e-12;
    opt->max_iter = 10000;
    return S3_OK;
}

namespace {
s3_status zeig_check(s3_graph_t g, const s3_zeig_options *opt_in, s3_zeig_options &opt) {
    if (!g) return fail(S3_EINVAL, "graph is NULL");
    if (opt_in) opt = *opt_in;
    else s3_zeig_options_init(&opt);
    if (opt.max_iter <= 0) opt.max_iter = 10000;
    if (!(opt.tol > 0)) return fail(S3_EINVAL, "tol must be > 0");
    if (!(opt.alpha >= 0)) return fail(S3_EINVAL, "alpha must be >= 0");
    if (g->N < 2) return fail(S3_EINVAL, "Z-eigenpairs need rank >= 2");
    return S3_OK;
}
}  // namespace

s3_status s3_zeigenpair(s3_graph_t g, const s3_zeig_options *opt_in, const double *x0, double *x_out,
                        s3_zeig_result *res, void *stream) {
    auto t0 = std::chrono::steady_clock::now();
    s3_zeig_options opt;
    s3_status s = zeig_check(g, opt_in, opt);
    if (s != S3_OK) return s;
    if (!x_out || !res) return fail(S3_EINVAL, "NULL argument");
    std::memset(res, 0, sizeof(*res));
    DeviceGuard guard(g->device);
    cudaStream_t st = (cudaStream_t)stream;
    s = zeig_run(g, opt, x0, nullptr, 0, nullptr, x_out, res, st);
    if (s != S3_OK) return s;
    s = mark_done(g, st);
    if (s != S3_OK) return s;
    S3_CUDA(cudaStreamSynchronize(st));
    res->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (!res->converged) return fail(S3_ENOCONV, "SS-HOPM did not reach the tolerance within max_iter");
    return S3_OK;
}

s3_status s3_symmetric_cp(s3_graph_t g, int32_t R, const s3_zeig_options *opt_in, const double *X0, double *X,
                          double *lambdas, int32_t *iters, void *stream) {
    s3_zeig_options opt;
    s3_status s = zeig_check(g, opt_in, opt);
    if (s != S3_OK) return s;
    if (R < 1 || R > kZeigMaxR) return fail(S3_EINVAL, "R must be in 1..32");
    if (!X || !lambdas) return fail(S3_EINVAL, "NULL argument");
    DeviceGuard guard(g->device);
    cudaStream_t st = (cudaStream_t)stream;
    bool all = true;
    for (int r = 0; r < R; ++r) {
        s3_zeig_result res{};
        s = zeig_run(g, opt, X0 ? X0 + (int64_t)r * g->n : nullptr, X, r, lambdas, X + (int64_t)r * g->n, &res, st);
        if (s != S3_OK) return s;
        lambdas[r] = res.lambda;
        if (iters) iters[r] = res.iters;
        all = all && res.converged;
    }
    s = mark_done(g, st);
    if (s != S3_OK) return s;
    S3_CUDA(cudaStreamSynchronize(st));
    if (!all) return fail(S3_ENOCONV, "a component did not reach the tolerance within max_iter");
    return S3_OK;
}

}  // extern "C"
