// Leave-one-out through the Bernoulli series: all contributions of an edge from
// one product over its members.
//
// For an edge e = (v_1 .. v_s) at rank N (window W = N - s + 1) write
//     Ebar(x t) = e^(x t) - 1 = x t g_x(t),   g_x(t) = sum_k x^k t^k / (k+1)!,
// so F_e = prod_j Ebar(x_j t) = t^s (prod_j x_j) G(t) with G = prod_j g_{x_j}.
// Since E = e^(x t) and E(x t) / Ebar(x t) = 1 / (1 - e^(-x t)), which is
// (1 / (x t)) sum_k beta_k x^k t^k with beta_k = B_k^+ / k! (the Bernoulli
// numbers, B_1 = +1/2), the per-(edge, node) value of Algorithm 2 is
//     [t^(N-1)] E(x_i t) prod_{j != i} Ebar(x_j t)
//         = (prod_{j != i} x_j) * sum_{k=0}^{W-1} G[W-1-k] beta_k x_i^k.
// Every member then needs one short polynomial in x_i, and only the edge's x stay
// in shared memory (no stored prefix windows).  G is formed in one of two ways:
//   * FP32: the product of the members' series, each step W independent Horner
//     chains of W(W-1)/2 multiply-adds in all (about half of the prefix/suffix
//     scheme's (2s - 5) W^2 / 2 per edge, with the same parallelism);
//   * FP64: from the power sums p_k = sum_j x_j^k.  d/dt log g_x(t) =
//     sum_{k>=1} beta_k x^k t^(k-1), so G = exp(sum_k beta_k p_k t^k / k), i.e.
//     G_0 = 1, G_m = (1/m) sum_{k=1}^{m} beta_k p_k G_{m-k}: 2 (W-1) operations per
//     member and W(W-1)/2 multiply-adds once per edge -- fewer operations for the
//     FP64 pipe, less parallelism (the FP32 units measured faster with the product).
//
// beta_k alternates in sign for even k >= 4, so the final sum (and in FP64 the
// recurrence) can cancel.  FP32: with P the positive terms of the sum and Q the
// magnitude of the negative ones (G's coefficients are sums of positive terms, so
// P + Q bounds the error mass), an edge is accepted when every member has
// P + Q <= 4 (P - Q).  FP64: the recurrence runs a second time with |beta_k| (in FP32: all
// terms >= 0; its result A bounds the rounding error of G coefficient by
// coefficient) and an edge is accepted when every member has
// sum_k A[W-1-k] |beta_k| x_i^k <= 64 (P - Q).  Edges that fail, or hold an x <= 0,
// are recomputed by the warp with the prefix/suffix series (warp_edge_compute).
// For equal x at rank 25 the FP32 ratio is at most 1.15 for s >= 6 (2.1 with one
// member twice the others), the FP64 ratio at most 2.2.
#pragma once

#include <algorithm>

#include "s3_series.cuh"

namespace s3 {

// The Bernoulli sum of one member, split into its positive part P (k = 0, 1 and
// k = 2 mod 4) and the magnitude Q of its negative part (k = 0 mod 4, k >= 4):
// H[k] = G[W-1-k] beta_k, Horner in x^4 for each residue class.
template <typename T, int W>
__device__ __forceinline__ void bern_eval(const T (&H)[W], T xi, T &P, T &Q) {
    const T x2 = xi * xi, x4 = x2 * x2;
    T p2 = T(0);
    if constexpr (W > 2) {
#pragma unroll
        for (int k = 2 + 4 * ((W - 1 - 2) / 4); k >= 2; k -= 4) p2 = Arith<T>::fma_(p2, x4, H[k]);
    }
    T p = H[0];
    if constexpr (W > 1) p = Arith<T>::fma_(H[1], xi, p);
    P = Arith<T>::fma_(p2, x2, p);
    T q = T(0);
    if constexpr (W > 4) {
#pragma unroll
        for (int k = 4 + 4 * ((W - 1 - 4) / 4); k >= 4; k -= 4) q = Arith<T>::fma_(q, x4, -H[k]);
        q = q * x4;
    }
    Q = q;
}

// sum_k Ha[k] x^k for the nonnegative coefficients Ha (Ha[k] = 0 for odd k >= 3): Horner in x^2
// over the even k, plus the k = 1 term.
template <typename T, int W>
__device__ __forceinline__ T bern_majorant(const T (&Ha)[W], T xi) {
    const T x2 = xi * xi;
    T a = T(0);
#pragma unroll
    for (int k = 2 * ((W - 1) / 2); k >= 0; k -= 2) a = Arith<T>::fma_(a, x2, Ha[k]);
    if constexpr (W > 1) a = Arith<T>::fma_(Ha[1], xi, a);
    return a;
}

// prod / x for the scaled member values (x near 1, x > 0): FP32 multiplies by the hardware
// reciprocal (within 2 units in the last place; the division's IEEE sequence and its slow-path
// branch would sit in the per-member loop); FP64 refines an FP32 reciprocal seed by two Newton
// steps (relative error below 2^-52 before the product) instead of the FP64 division sequence.
__device__ __forceinline__ float others_product(float prod, float x) { return __fdividef(prod, x); }
__device__ __forceinline__ double others_product(double prod, double x) {
    double r = (double)__frcp_rn((float)x);
    r = fma(r, fma(-x, r, 1.0), r);
    r = fma(r, fma(-x, r, 1.0), r);
    return prod * r;
}

template <typename T> __device__ __forceinline__ T bern_beta(const BernArgs &c, int k);
template <> __device__ __forceinline__ float bern_beta<float>(const BernArgs &c, int k) { return c.beta32[k]; }
template <> __device__ __forceinline__ double bern_beta<double>(const BernArgs &c, int k) { return c.beta64[k]; }
template <typename T> __device__ __forceinline__ T bern_kmax(const BernArgs &c);
template <> __device__ __forceinline__ float bern_kmax<float>(const BernArgs &c) { return c.kmax32; }
template <> __device__ __forceinline__ double bern_kmax<double>(const BernArgs &c) { return c.kmax64; }

// The series fallback for an edge the gate rejected (kept out of line: it is rarely
// taken, and inlined into every window's code it would crowd the instruction cache).
template <typename T>
__device__ __noinline__ void bern_fallback(const EdgeBucketArgs &b, const T *__restrict__ x, const EdgeOutArgs &o,
                                           int64_t e, int W, T *fb) {
    warp_edge_compute<T>(b, x, o, e, W, fb);
}

// One edge per thread (e < b.m when valid).  lane_base: this warp's region, element i
// of lane l at i * kLS + l: the edge's x values, then (FP64 only) the member ids staged
// while x is gathered (FP32 stages each id in its own x slot, which the gather then
// overwrites).  Shared memory is kept to that -- the x gathers also use the L1 cache,
// which the rest of the shared-memory carve-out would take away.  fb: the warp's region
// for the series fallback.
template <typename T, int W, bool BUF, bool BIAS>
__device__ __forceinline__ void bern_edge(const EdgeBucketArgs &b, const T *__restrict__ x, const EdgeOutArgs &o,
                                          const BernArgs &c, int64_t e, bool valid, T *lane_base, T *fb) {
    const int lane = threadIdx.x & 31;
    const int s = b.s;
    T *xs = lane_base + lane;
    int32_t *idst = sizeof(T) == 4 ? reinterpret_cast<int32_t *>(lane_base) + lane
                                   : reinterpret_cast<int32_t *>(lane_base + s * kLS) + lane;
    bool ok = valid;
    int p = 0;
    if (valid) {
        for (int i = 0; i < s; ++i) cp_async<4>(idst + i * kLS, b.ids + (int64_t)i * b.ld + e);
        cp_async_commit();
        cp_async_wait_all();
        for (int i = 0; i < s; ++i) cp_async<(int)sizeof(T)>(xs + i * kLS, x + idst[i * kLS]);
        cp_async_commit();
        cp_async_wait_all();
        T S = T(0);
        bool pos = true;
        for (int i = 0; i < s; ++i) {
            const T v = xs[i * kLS];
            S += Arith<T>::absv(v);
            pos &= v > T(0);
        }
        p = scale_exponent<T>(S, b.target);
        const T g = Arith<T>::pow2(p);
        if constexpr (sizeof(T) == 4) {
            // G = g_{x_1} (its coefficients x^k / (k+1)!), then times g_{x_i}, i = 2..s, each product
            // in Horner form (W independent chains); P = the product of all (scaled) x
            T G[W];
            T prod;
            {
                const T x0 = xs[0] * g;
                xs[0] = x0;
                prod = x0;
                G[0] = T(1);
    #pragma unroll
                for (int k = 1; k < W; ++k) G[k] = G[k - 1] * (x0 * Num<T>::recip(k + 1));
            }
            for (int i = 1; i < s; ++i) {
                const T xi = xs[i * kLS] * g;
                xs[i * kLS] = xi;
                prod *= xi;
                T r[W];
    #pragma unroll
                for (int k = 1; k < W; ++k) r[k] = xi * Num<T>::recip(k + 1);
                // G[m] <- G[m] + r_1 (G[m-1] + r_2 (G[m-2] + ... + r_m G[0])), top down in place
    #pragma unroll
                for (int m = W - 1; m >= 1; --m) {
                    T t = G[0];
    #pragma unroll
                    for (int j = 1; j <= m; ++j) t = Arith<T>::fma_(r[m - j + 1], t, G[j]);
                    G[m] = t;
                }
            }
            T H[W];
    #pragma unroll
            for (int k = 0; k < W; ++k) H[k] = G[W - 1 - k] * bern_beta<T>(c, k);
            const T kmax = bern_kmax<T>(c);
            // every member: the Bernoulli sum (G's coefficients are exact sums of positive terms
            // up to rounding, so P + Q bounds the error mass), times prod_{j != i} x_j = P / x_i
            for (int i = 0; i < s; ++i) {
                const T xi = xs[i * kLS];
                T Pp, Q;
                bern_eval<T, W>(H, xi, Pp, Q);
                const T v = Pp - Q;
                ok &= (Pp + Q) <= kmax * v;
                if constexpr (BIAS) {
                    // the biased output of the centrality iteration: the scale of each result
                    // depends on its member's exponent, which is at hand here
                    xs[i * kLS] = scale_result<T>(v * others_product(prod, xi), b, p, Arith<T>::expo(xi) - p, nullptr);
                } else {
                    xs[i * kLS] = v * others_product(prod, xi);
                }
            }
        } else {
            // power sums p_k = sum_j x_j^k (k = 1..W-1, in q[k]) and P = prod_j x_j; each member's
            // powers by a binary tree (x^k = x^(k/2) x^(k - k/2)), so their dependency depth is log2 W
            T q[W];
    #pragma unroll
            for (int k = 0; k < W; ++k) q[k] = T(0);
            T prod = T(1);
            for (int i = 0; i < s; ++i) {
                const T xi = xs[i * kLS] * g;
                xs[i * kLS] = xi;
                prod *= xi;
                T pw[W];
                pw[0] = T(1);
                if constexpr (W > 1) pw[1] = xi;
    #pragma unroll
                for (int k = 2; k < W; ++k) pw[k] = pw[k / 2] * pw[k - k / 2];
    #pragma unroll
                for (int k = 1; k < W; ++k) q[k] += pw[k];
            }
            // G = exp(sum_k l_k p_k t^k) with k l_k = beta_k: G_0 = 1,
            // G_m = (1/m) sum_{k=1}^{m} beta_k p_k G_{m-k}; A the same recurrence with |beta_k|
            // (all terms >= 0), which bounds the rounding error of G.  A only has to bound, not to
            // be exact: it runs in FP32 (all its terms are positive, so its own relative error
            // stays below ~2^-18, which the gate's 1e-4 allowance covers), off the FP64 pipe.
    #pragma unroll
            for (int k = 1; k < W; ++k) q[k] *= bern_beta<T>(c, k);
            float qa[W];
    #pragma unroll
            for (int k = 1; k < W; ++k) qa[k] = fabsf((float)q[k]);
            T G[W];
            float A[W];
            G[0] = T(1);
            A[0] = 1.f;
    #pragma unroll
            for (int m = 1; m < W; ++m) {
                // from k = m down, so that G[m-1] (the value just formed) enters last
                T acc = T(0);
                float acca = 0.f;
    #pragma unroll
                for (int k = m; k >= 1; --k) {
                    acc = Arith<T>::fma_(q[k], G[m - k], acc);
                    acca = fmaf(qa[k], A[m - k], acca);
                }
                G[m] = acc * Num<T>::recip(m);
                A[m] = acca * (1.0f / (float)m);
            }
            T H[W];
            float Ha[W];
    #pragma unroll
            for (int k = 0; k < W; ++k) {
                H[k] = G[W - 1 - k] * bern_beta<T>(c, k);
                Ha[k] = A[W - 1 - k] * fabsf(c.beta32[k]);
            }
            const T kmax = bern_kmax<T>(c);
            // every member: the Bernoulli sum, its majorant (gate), times prod_{j != i} x_j = P / x_i
            for (int i = 0; i < s; ++i) {
                const T xi = xs[i * kLS];
                T Pp, Q;
                bern_eval<T, W>(H, xi, Pp, Q);
                const T v = Pp - Q;
                ok &= (T)bern_majorant<float, W>(Ha, (float)xi) * T(1.0001) <= kmax * v;
                if constexpr (BIAS) {
                    // the biased output of the centrality iteration: the scale of each result
                    // depends on its member's exponent, which is at hand here
                    xs[i * kLS] = scale_result<T>(v * others_product(prod, xi), b, p, Arith<T>::expo(xi) - p, nullptr);
                } else {
                    xs[i * kLS] = v * others_product(prod, xi);
                }
            }
        }
        ok &= pos;
    }
    const unsigned rej = __ballot_sync(0xffffffffu, valid && !ok);
    if (valid && ok) {
        const EdgeScale<T> sc = edge_scale(b, o, p, T(0));
        int nbad = 0;
        // the targets (incidence slots, or node ids in the atomic modes) in chunks of eight
        // independent loads, so that each store does not wait for its own round trip
        constexpr int kChunk = 8;
        for (int i0 = 0; i0 < s; i0 += kChunk) {
            int tv[kChunk];
#pragma unroll
            for (int j = 0; j < kChunk; ++j)
                tv[j] = i0 + j < s ? __ldg((BUF ? b.slot : b.ids) + (int64_t)(i0 + j) * b.ld + e) : 0;
#pragma unroll
            for (int j = 0; j < kChunk; ++j) {
                const int i = i0 + j;
                if (i >= s) break;
                const T val = xs[i * kLS];
                const int t = tv[j];
                if constexpr (BIAS) {
                    // scaled already (every x > 0, so every value is positive)
                    nbad += not_normal_pos(val);
                    if constexpr (BUF) reinterpret_cast<T *>(o.out)[t] = val;
                    else scatter_atomic<T>(o, t, val);
                } else if (sc.fast) {
                    emit_fast<T, BUF>(o, t, val, sc.mult, nbad);
                } else {
                    // scaled x of the member (its exponent sets the per-node bias of NQZ): reloaded
                    // here, off the common path
                    const T xhat = __ldg(x + __ldg(b.ids + (int64_t)i * b.ld + e)) * Arith<T>::pow2(p);
                    emit_value<T, BUF>(b, o, t, t, val, p, xhat);
                }
            }
        }
        if (nbad && o.range_events) atomicAdd(o.range_events, (unsigned long long)nbad);
    }
    // edges that failed the gate (or hold an x <= 0): the whole warp recomputes each with
    // the series
    if (rej && lane == 0 && c.rejected) atomicAdd(c.rejected, (unsigned long long)__popc(rej));
    for (unsigned r = rej; r; r &= r - 1) {
        const int64_t ee = __shfl_sync(0xffffffffu, e, __ffs(r) - 1);
        bern_fallback<T>(b, x, o, ee, W, fb);
    }
}

// All Bernoulli buckets of a call in one launch.  The buckets' edges form tiles of 128
// (one edge per thread; tab[k].block0 = the first tile of bucket k, ascending) and the
// blocks walk them (tile t, t + gridDim.x, ...); FP32 launches only as many blocks as are
// resident at once, so that blocks live long, the instruction caches stay warm and the
// bucket lookup only moves forward (2.5 % faster than a block per tile; FP64 was slower).  Per warp:
// lane_elems values per lane, then fb_elems values for the series fallback.
template <typename T, bool BUF, bool BIAS>
__global__ void __launch_bounds__(kBernThreads, sizeof(T) == 4 ? 7 : 3) edge_bern_kernel(const TailEntry *__restrict__ tab, int ntab,
                                                                 int64_t ntiles, int lane_elems, int fb_elems,
                                                                 const T *__restrict__ x, EdgeOutArgs o, BernArgs c) {
    if (o.skip && *o.skip) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const size_t warp_elems = (size_t)kLS * lane_elems + (size_t)fb_elems;
    T *base = reinterpret_cast<T *>(smem_raw) + (size_t)(threadIdx.x >> 5) * warp_elems;
    T *fb = base + (size_t)kLS * lane_elems;
    int k = 0;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        while (k + 1 < ntab && tab[k + 1].block0 <= t) ++k;
        const EdgeBucketArgs b = tab[k].b;
        const int64_t e = (t - tab[k].block0) * blockDim.x + threadIdx.x;
        const bool valid = e < b.m;
        if (__all_sync(0xffffffffu, !valid)) continue;
        switch (tab[k].W) {
#define S3_BERN_CASE(w) \
    case w: bern_edge<T, w, BUF, BIAS>(b, x, o, c, e, valid, base, fb); break;
            S3_W_CASES(S3_BERN_CASE)
#undef S3_BERN_CASE
            default: break;
        }
    }
}

// Launch for the output modes of one BIAS value (the biased centrality mode, or not): each
// value is instantiated in a translation unit of its own, to keep their compile times apart.
template <typename T, bool BIAS>
cudaError_t launch_edge_bern_t(const TailEntry *tab, int ntab, int64_t nblocks, int lane_elems, int fb_elems,
                               const T *x, const EdgeOutArgs &o, const BernArgs &c, cudaStream_t st) {
    if (ntab <= 0 || nblocks <= 0) return cudaSuccess;
    const size_t smem = bern_smem_bytes(lane_elems, fb_elems, sizeof(T));
    if (smem > kEdgeSmemCap || nblocks > INT32_MAX || (o.bias != 0) != BIAS) return cudaErrorInvalidConfiguration;
    // FP32: as many blocks as fit on the device at once (never more than there are tiles);
    // FP64 (3 blocks per SM): one block per tile, which measured faster there
    int64_t grid_blocks = nblocks;
    if (sizeof(T) == 4) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaError_t err = cudaGetDevice(&dev);
        if (err == cudaSuccess) err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (err == cudaSuccess)
            err = o.mode == kOutBuffer ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                             &per_sm, edge_bern_kernel<T, true, BIAS>, kBernThreads, smem)
                                       : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                             &per_sm, edge_bern_kernel<T, false, BIAS>, kBernThreads, smem);
        if (err != cudaSuccess) return err;
        const int64_t resident = (int64_t)std::max(sms, 1) * std::max(per_sm, 1);
        grid_blocks = std::min<int64_t>(nblocks, resident);
    }
    const dim3 grid((unsigned)grid_blocks), block(kBernThreads);
    if (o.mode == kOutBuffer)
        edge_bern_kernel<T, true, BIAS><<<grid, block, smem, st>>>(tab, ntab, nblocks, lane_elems, fb_elems, x, o, c);
    else
        edge_bern_kernel<T, false, BIAS><<<grid, block, smem, st>>>(tab, ntab, nblocks, lane_elems, fb_elems, x, o, c);
    return cudaGetLastError();
}

template <typename T, bool BIAS>
cudaError_t prepare_edge_bern_t() {
    const int cap = (int)kEdgeSmemCap;
    cudaError_t e = cudaFuncSetAttribute(edge_bern_kernel<T, true, BIAS>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(edge_bern_kernel<T, false, BIAS>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
    return e;
}

}  // namespace s3
