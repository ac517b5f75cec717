// Closed-form evaluation of small edges (inclusion-exclusion).
//
// Write n = N-1.  Expanding every factor Ebar(x_u) = e^(x_u t) - 1 in
// E(x_v) prod_{u in e, u != v} Ebar(x_u) turns the product into a signed sum
// of exponentials: one term e^(sigma_U t) for every subset U of e that
// contains v, with sigma_U = sum_{u in U} x_u and sign (-1)^(s-|U|).  The
// coefficient of t^n of e^(sigma t) is sigma^n / n!, so
//     c(e, v) = K(s,N) / n! * R_v,   R_v = sum_{U: v in U} (-1)^(s-|U|) sigma_U^n,
// the same value as the truncated series products (Sec. II-A, Algorithm 2).
// One pass over the 2^s - 1 nonempty subsets gives R_v for every v of the
// edge: about 2^s (log2 n + 12) instructions instead of the series' (2s-5)
// W(W+1)/2 multiply-adds (W = N-s+1), which pays for s <= 6 at ranks N of
// about 10 and more.
//
// The sum alternates in sign, so it is evaluated in a form whose error can be
// bounded edge by edge.  The x of the edge are scaled by a power of two so that
// sigma_e lies in [1, 2) (every term then lies in [0, 2^n), no overflow for
// n <= 127).  FP32 carries each subset sum as an unevaluated pair hi + lo (an
// error-free two-sum per subset) and adds the first-order term n lo / hi to
// hi^n, so each term is within about n u of sigma_U^n for unit roundoff u (the
// binary powering's rounding); FP64 sums the subsets plainly (error (s-1) n u,
// far below the FP64 tolerance).  The s accumulations of at most 2^(s-1) terms
// each add at most 2^(s-1) u sum|terms|.  So
//     |error of R_v| <= C u A,   A = sum_U |sigma_U^n|,
// with C = n + 2^(s-1) + 4 (FP32) or s n + 2^(s-1) + 4 (FP64).  An edge is
// accepted when every R_v > gate * A, gate = C u / tau, i.e. when its relative
// error bound is below tau (2^-17 for FP32, 2^-42 for FP64); members with x < 0
// are not accepted either.  Rejected edges (x of very different sizes inside
// one edge, zeros) are appended to a list that the series kernels then process
// in list mode (s3_series.cuh), so every result has the series path's accuracy
// or the bound above.
#pragma once

#include "s3_series.cuh"

namespace s3 {

// Edges per thread whose loads are in flight together (measured: four for size 2,
// two for sizes 3 and 4, one from size 5 on, where the subset sums need the registers).
template <int S> struct ClosedShape {
    static constexpr int E = S <= 2 ? 4 : S <= 4 ? 2 : 1;
};

// h^n for n = 2^NB + (lower NB bits): left-to-right binary powering, NB
// squarings and one multiply per set lower bit.
template <int NB, typename T>
__device__ __forceinline__ T closed_pow(T h, int n) {
    T r = h;
#pragma unroll
    for (int k = NB - 1; k >= 0; --k) {
        r = r * r;
        if ((n >> k) & 1) r = r * h;
    }
    return r;
}

template <typename T, int S, int NB, bool BUF>
__global__ void __launch_bounds__(256) edge_closed_kernel(EdgeBucketArgs b, const T *__restrict__ x, EdgeOutArgs o,
                                                          ClosedArgs c) {
    if (o.skip && *o.skip) return;
    constexpr int E = ClosedShape<S>::E;
    constexpr int NS = 1 << S;
    constexpr bool kComp = sizeof(T) == 4;  // FP32: compensated subset sums
    const int n = b.N - 1;
    const T gate = (T)c.gate;
    EdgeBucketArgs bk = b;  // output scaling by K(s,N)/n! instead of K(s,N)
    bk.K = c.Ki;
    bk.Km = c.Kim;
    bk.Ke = c.Kie;
    const int64_t span = (int64_t)blockDim.x * E;
    const int64_t stride = (int64_t)gridDim.x * span;
    int nbad = 0;
    for (int64_t e0 = (int64_t)blockIdx.x * span + threadIdx.x; e0 < b.m; e0 += stride) {
        int32_t id[E][S], tg[E][S];
        T X[E][S];
#pragma unroll
        for (int k = 0; k < E; ++k) {
            const int64_t e = e0 + (int64_t)k * blockDim.x;
            const bool in = e < b.m;
#pragma unroll
            for (int i = 0; i < S; ++i) {
                id[k][i] = in ? __ldg(b.ids + (int64_t)i * b.ld + e) : 0;
                tg[k][i] = BUF ? (in ? __ldg(b.slot + (int64_t)i * b.ld + e) : 0) : id[k][i];
            }
        }
#pragma unroll
        for (int k = 0; k < E; ++k)
#pragma unroll
            for (int i = 0; i < S; ++i) X[k][i] = __ldg(x + id[k][i]);
#pragma unroll
        for (int k = 0; k < E; ++k) {
            const int64_t e = e0 + (int64_t)k * blockDim.x;
            if (e >= b.m) break;
            T sum = T(0);
            bool ok = true;
#pragma unroll
            for (int i = 0; i < S; ++i) {
                sum += X[k][i];
                ok &= X[k][i] >= T(0);
            }
            // sum must be a normal number well inside the range (NaN fails too)
            ok &= sum > Arith<T>::tiny() * T(16777216.0) && sum < Arith<T>::huge() / T(16777216.0);
            const int p = 1 - Arith<T>::expo(sum);  // sigma_e 2^p in [1, 2)
            const T g = Arith<T>::pow2(p);
            T a[S];
#pragma unroll
            for (int i = 0; i < S; ++i) a[i] = X[k][i] * g;
            T hi[NS], lo[NS];
            T R[S];
#pragma unroll
            for (int i = 0; i < S; ++i) R[i] = T(0);
            T A = T(0);
#pragma unroll
            for (int mask = 1; mask < NS; ++mask) {
                const int low = mask & -mask;
                const int i = __ffs(low) - 1;  // the subset's lowest member, added last
                const int par = mask ^ low;
                if (par == 0) {
                    hi[mask] = a[i];
                    lo[mask] = T(0);
                } else if (kComp) {
                    const T sm = hi[par] + a[i];
                    const T bb = sm - hi[par];
                    const T err = (hi[par] - (sm - bb)) + (a[i] - bb);
                    hi[mask] = sm;
                    lo[mask] = lo[par] + err;
                } else {
                    hi[mask] = hi[par] + a[i];
                    lo[mask] = T(0);
                }
                T pw = closed_pow<NB>(hi[mask], n);
                if (kComp && par != 0) {  // a single member's sum is exact
                    // (hi + lo)^n = hi^n (1 + n lo / hi + O((lo/hi)^2)); hi >= 0, and lo = 0 when hi = 0
                    const float h = fmaxf((float)hi[mask], FLT_MIN);
                    pw = fmaf((float)pw, __fdividef((float)n * (float)lo[mask], h), (float)pw);
                }
                A += pw;
                const bool neg = ((S - __popc(mask)) & 1) != 0;
#pragma unroll
                for (int v = 0; v < S; ++v)
                    if ((mask >> v) & 1) R[v] = neg ? R[v] - pw : R[v] + pw;
            }
#pragma unroll
            for (int v = 0; v < S; ++v) ok &= R[v] > gate * A;
            if (ok) {
                const EdgeScale<T> sc = edge_scale(bk, o, p, T(0));
#pragma unroll
                for (int v = 0; v < S; ++v) {
                    if (sc.fast) emit_fast<T, BUF>(o, tg[k][v], R[v], sc.mult, nbad);
                    else emit_value<T, BUF>(bk, o, tg[k][v], tg[k][v], R[v], p, a[v]);
                }
            }
            // rejected edges go to the series kernels' list (one atomic per warp)
            const unsigned act = __activemask();
            const unsigned fm = __ballot_sync(act, !ok);
            if (fm) {
                const int lane = threadIdx.x & 31;
                const int leader = __ffs(fm) - 1;
                int base = 0;
                if (lane == leader) base = atomicAdd(c.fail_count, __popc(fm));
                base = __shfl_sync(act, base, leader);
                const int64_t at = (int64_t)base + __popc(fm & ((1u << lane) - 1u));
                if (!ok && at < b.m) c.fail_list[at] = (int32_t)e;  // at most m rejections per call
            }
        }
    }
    if (nbad && o.range_events) atomicAdd(o.range_events, (unsigned long long)nbad);
}

template <typename T, int S, int NB>
cudaError_t launch_closed_snb(const EdgeBucketArgs &b, const T *x, const EdgeOutArgs &o, const ClosedArgs &c,
                              cudaStream_t st) {
    constexpr int bs = 256;
    const int64_t need = (b.m + (int64_t)bs * ClosedShape<S>::E - 1) / ((int64_t)bs * ClosedShape<S>::E);
    if (o.mode == kOutBuffer) {
        const int64_t grid = std::min<int64_t>(need, full_grid<edge_closed_kernel<T, S, NB, true>, bs>());
        edge_closed_kernel<T, S, NB, true><<<(unsigned)grid, bs, 0, st>>>(b, x, o, c);
    } else {
        const int64_t grid = std::min<int64_t>(need, full_grid<edge_closed_kernel<T, S, NB, false>, bs>());
        edge_closed_kernel<T, S, NB, false><<<(unsigned)grid, bs, 0, st>>>(b, x, o, c);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_edge_closed_t(const EdgeBucketArgs &b, const T *x, const EdgeOutArgs &o, const ClosedArgs &c,
                                 cudaStream_t st) {
    const int n = b.N - 1;
    if (b.s < 2 || b.s > kClosedMaxS || n < 2 || n > 127 || !c.fail_list || !c.fail_count)
        return cudaErrorInvalidValue;
    if (b.m <= 0) return cudaSuccess;
    int nb = 0;
    while ((n >> (nb + 1)) != 0) ++nb;  // floor(log2 n), 1..6
    switch (b.s * 8 + nb) {
#define S3_CLOSED_CASE(S, NB) \
    case S * 8 + NB: return launch_closed_snb<T, S, NB>(b, x, o, c, st);
#define S3_CLOSED_NB(S) \
    S3_CLOSED_CASE(S, 1) S3_CLOSED_CASE(S, 2) S3_CLOSED_CASE(S, 3) S3_CLOSED_CASE(S, 4) S3_CLOSED_CASE(S, 5) \
    S3_CLOSED_CASE(S, 6)
        S3_CLOSED_NB(2) S3_CLOSED_NB(3) S3_CLOSED_NB(4) S3_CLOSED_NB(5) S3_CLOSED_NB(6)
#undef S3_CLOSED_NB
#undef S3_CLOSED_CASE
        default: break;
    }
    return cudaErrorInvalidValue;
}

}  // namespace s3
