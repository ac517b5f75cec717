// Wide windows: eight lanes per edge, four edges per warp (instantiated in s3_group.cu).
//
// The algorithm is the one of edge_compute (prefix windows forward, suffix
// windows backward, one dot per leave-one-out value, Sec. III-A / Eq. 5), for
// windows W = N - s + 1 too wide for one thread's registers.  Lane c of an
// edge's group of eight owns the window coefficients [c C, c C + C) (C a
// multiple of 4 with 8 C >= W).  A window product out = P * Ebar(x),
//     out[j] = sum_{k >= 0} a_k P[j - k],   a_k = x^(k+1)/(k+1)!,
// runs with the lane's C accumulators and a C-register ring of P values that
// slides down by one coefficient per step: per step one broadcast table load,
// one ring load and C FMAs, so the lanes do arithmetic rather than
// shared-memory traffic.  Lane c needs the steps k < (c+1) C only; the prefix
// windows, the current suffix and the power table live in the edge's shared
// memory.

#pragma once

#include "s3_series.cuh"

namespace s3 {

constexpr int kGL = 8;              // lanes per edge
constexpr int kGEdges = 32 / kGL;   // edges per warp

// Per-edge shared memory (elements of T): Xs[s] | A[kGL C] | Pre[(s-1) W] | Qa[W] | Qb[W]
// (Pre slot i holds Pre_{i+2}; slot s-2 ends as Pre_s).
__host__ __device__ constexpr int64_t group_edge_elems(int s, int W, int C) {
    return (((int64_t)s + kGL * (int64_t)C + (int64_t)(s > 1 ? s - 1 : 1) * W + 2 * (int64_t)W) + 1) / 2 * 2;
}
// 1/k for k = 0..kGL C + 1 at the start of the block's shared memory (entry 0 unused)
__host__ __device__ constexpr int group_inv_elems(int C) { return (kGL * C + 2 + 1) / 2 * 2; }

// A[k] = x^(k+1)/(k+1)! for k < W, 0 for W <= k < kGL C.  Lane c forms its chunk as
// a running product and scales it by the product of the chunks before it (an
// exclusive scan over the group).
template <typename T, int C>
__device__ __forceinline__ void group_ptable(T x, T *A, int W, const T *inv, int c) {
    T loc[C];
    T run = T(1);
#pragma unroll
    for (int r = 0; r < C; ++r) {
        run = run * (x * inv[c * C + r + 1]);
        loc[r] = run;
    }
    T inc = run;  // inclusive product over lanes 0..c of the group
#pragma unroll
    for (int d = 1; d < kGL; d <<= 1) {
        const T t = __shfl_up_sync(0xffffffffu, inc, d, kGL);
        if (c >= d) inc = inc * t;
    }
    T pre = __shfl_up_sync(0xffffffffu, inc, 1, kGL);
    if (c == 0) pre = T(1);
#pragma unroll
    for (int r = 0; r < C; ++r) {
        const int k = c * C + r;
        A[k] = k < W ? pre * loc[r] : T(0);
    }
}

// out[j] = sum_{k=0}^{j} A[k] P[j - k] for this lane's j < W (P and out: W wide; A zero
// beyond W).  The ring holds P[j0 + r - k] at position (r - k) mod C at step k.
template <typename T, int C>
__device__ __forceinline__ void group_toeplitz(const T *P, const T *A, T *out, int W, int c) {
    const int j0 = c * C;
    T acc[C], ring[C];
#pragma unroll
    for (int r = 0; r < C; ++r) {
        acc[r] = T(0);
        ring[r] = j0 + r < W ? P[j0 + r] : T(0);
    }
    // steps k < j0 + C reach all of the lane's outputs; a lane whose chunk starts at or
    // past W has no outputs and skips the loop
    const int K = j0 < W ? j0 + C : 0;
    for (int k0 = 0; k0 < K; k0 += C) {
#pragma unroll
        for (int kk = 0; kk < C; ++kk) {
            const int k = k0 + kk;
            const T a = A[k];
#pragma unroll
            for (int r = 0; r < C; ++r) acc[r] = Arith<T>::fma_(a, ring[(r - kk + C) % C], acc[r]);
            const int idx = j0 - k - 1;  // enters for r = 0 at step k + 1; 0 <= idx < j0 < W
            ring[(C - 1 - kk + C) % C] = idx >= 0 ? P[idx] : T(0);
        }
    }
#pragma unroll
    for (int r = 0; r < C; ++r)
        if (j0 + r < W) out[j0 + r] = acc[r];
}

// sum_{j < n} U[j] V[off - j] over the group (every lane gets the total).
template <typename T, int C>
__device__ __forceinline__ T group_dot(const T *U, const T *V, int n, int off, int c) {
    T s0 = T(0), s1 = T(0);
#pragma unroll
    for (int r = 0; r < C; r += 2) {
        const int j = c * C + r;
        if (j < n) s0 = Arith<T>::fma_(U[j], V[off - j], s0);
        if (j + 1 < n) s1 = Arith<T>::fma_(U[j + 1], V[off - j - 1], s1);
    }
    T t = s0 + s1;
#pragma unroll
    for (int d = 1; d < kGL; d <<= 1) t += __shfl_xor_sync(0xffffffffu, t, d);
    return t;
}

template <typename T, int C>
__device__ __forceinline__ void group_copy(const T *src, T *dst, int W, int c) {
#pragma unroll
    for (int r = 0; r < C; ++r) {
        const int j = c * C + r;
        if (j < W) dst[j] = src[j];
    }
}

// One edge per group of eight lanes, grid-stride over warp-sized groups of edges.
// Control flow is uniform over the warp (every edge of a bucket has size s);
// groups past the end of the bucket compute on zeros and write nothing.
template <typename T, int C, bool BUF>
__global__ void __launch_bounds__(128) edge_group_kernel(EdgeBucketArgs b, const T *__restrict__ x, EdgeOutArgs o,
                                                         int W, int64_t edge_elems) {
    if (o.skip && *o.skip) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *inv = reinterpret_cast<T *>(smem_raw);
    const int ninv = group_inv_elems(C);
    for (int k = threadIdx.x; k < ninv; k += blockDim.x) inv[k] = k ? T(1) / T(k) : T(0);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const int c = lane & (kGL - 1), gi = lane / kGL;
    const int s = b.s;
    T *Xs = inv + ninv + ((int64_t)warp * kGEdges + gi) * edge_elems;
    T *A = Xs + s;
    T *Pre = A + kGL * C;
    T *Qa = Pre + (int64_t)(s > 1 ? s - 1 : 1) * W;
    T *Qb = Qa + W;
    const int64_t ngroups = (b.m + kGEdges - 1) / kGEdges;
    for (int64_t wg = (int64_t)blockIdx.x * wpb + warp; wg < ngroups; wg += (int64_t)gridDim.x * wpb) {
        const int64_t e = wg * kGEdges + gi;
        const bool has = e < b.m;
        T part = T(0);
        for (int i = c; i < s; i += kGL) {
            const T X = has ? __ldg(x + __ldg(b.ids + (int64_t)i * b.ld + e)) : T(0);
            Xs[i] = X;
            part += Arith<T>::absv(X);
        }
#pragma unroll
        for (int d = 1; d < kGL; d <<= 1) part += __shfl_xor_sync(0xffffffffu, part, d);
        const int p = scale_exponent<T>(part, b.target);
        const T g = Arith<T>::pow2(p);
        __syncwarp();
        for (int i = c; i < s; i += kGL) Xs[i] *= g;
        __syncwarp();
        const EdgeScale<T> sc = edge_scale(b, o, p, T(0));
        int nbad = 0;
        auto emit = [&](int q, T val) {
            if (!has || c != 0) return;
            const int t = BUF ? __ldg(b.slot + (int64_t)q * b.ld + e) : __ldg(b.ids + (int64_t)q * b.ld + e);
            if (sc.fast) emit_fast<T, BUF>(o, t, val, sc.mult, nbad);
            else emit_value<T, BUF>(b, o, t, t, val, p, Xs[q]);
        };

        // forward: slot 0 = Pre_2 = Ebar(x_{v_1}); slot i = slot i-1 * Ebar(x_{v_{i+1}})
        group_ptable<T, C>(Xs[0], A, W, inv, c);
        __syncwarp();
        group_copy<T, C>(A, Pre, W, c);
        __syncwarp();
        for (int i = 1; i <= s - 2; ++i) {
            group_ptable<T, C>(Xs[i], A, W, inv, c);
            __syncwarp();
            group_toeplitz<T, C>(Pre + (int64_t)(i - 1) * W, A, Pre + (int64_t)i * W, W, c);
            __syncwarp();
        }
        const T *Ps = Pre + (int64_t)(s - 2 > 0 ? s - 2 : 0) * W;   // Pre_s
        // backward: Q = Suf_{s-1} = Ebar(x_{v_s})
        group_ptable<T, C>(Xs[s - 1], A, W, inv, c);
        __syncwarp();
        group_copy<T, C>(A, Qa, W, c);
        __syncwarp();
        T *Q = Qa, *Qn = Qb;
        const T F = group_dot<T, C>(Ps, Q, W - 1, W - 2, c);
        emit(s - 1, F + Ps[W - 1]);
        T top = T(0);
        for (int q = s - 2; q >= 1; --q) {
            const T D = group_dot<T, C>(Pre + (int64_t)(q - 1) * W, Q, W, W - 1, c);
            emit(q, F + D);
            group_ptable<T, C>(Xs[q], A, W, inv, c);
            __syncwarp();
            if (q >= 2) {
                group_toeplitz<T, C>(Q, A, Qn, W, c);
                __syncwarp();
                T *t = Q;
                Q = Qn;
                Qn = t;
            } else {
                top = group_dot<T, C>(A, Q, W, W - 1, c);
            }
        }
        emit(0, F + (s == 2 ? Q[W - 1] : top));
        if (c == 0 && nbad && o.range_events) atomicAdd(o.range_events, (unsigned long long)nbad);
        __syncwarp();
    }
}

constexpr size_t kSmemCapGroup = 200 * 1024;   // per block

template <typename T, int C, bool BUF>
cudaError_t launch_group_cb(const EdgeBucketArgs &b, const T *x, const EdgeOutArgs &o, int W, int64_t ee, int wpb,
                            size_t smem, cudaStream_t st) {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 148;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, edge_group_kernel<T, C, BUF>, wpb * 32, smem) !=
            cudaSuccess || per_sm <= 0) {
        cudaGetLastError();
        per_sm = 1;
    }
    const int64_t ngroups = (b.m + kGEdges - 1) / kGEdges;
    const int64_t need = (ngroups + wpb - 1) / wpb;
    const int64_t full = (int64_t)sms * per_sm;
    const int64_t grid = need < full ? need : full;
    edge_group_kernel<T, C, BUF><<<(unsigned)grid, wpb * 32, smem, st>>>(b, x, o, W, ee);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_group_t(const EdgeBucketArgs &b, const T *x, const EdgeOutArgs &o, int W, cudaStream_t st,
                           int *launched) {
    *launched = 0;
    const int C = ((W + kGL - 1) / kGL + 3) / 4 * 4;
    if (C > 16) return cudaSuccess;
    const int64_t ee = group_edge_elems(b.s, W, C);
    auto bytes = [&](int w) { return ((size_t)group_inv_elems(C) + (size_t)w * kGEdges * (size_t)ee) * sizeof(T); };
    // warps per block: the most warps per SM (shared memory decides), then the larger block
    constexpr size_t kSmemSM = 227 * 1024;
    int wpb = 0, best = 0;
    for (int w = 4; w >= 1; w /= 2) {
        if (bytes(w) > kSmemCapGroup) continue;
        const int per_sm = (int)(kSmemSM / (bytes(w) + 1024)) * w;
        if (per_sm > best) {
            best = per_sm;
            wpb = w;
        }
    }
    if (wpb == 0) return cudaSuccess;
    *launched = 1;
    const bool buf = o.mode == kOutBuffer;
    switch (C) {
#define S3_GCASE(cc)                                                                                       \
    case cc:                                                                                               \
        return buf ? launch_group_cb<T, cc, true>(b, x, o, W, ee, wpb, bytes(wpb), st)                     \
                   : launch_group_cb<T, cc, false>(b, x, o, W, ee, wpb, bytes(wpb), st);
        S3_GCASE(4) S3_GCASE(8) S3_GCASE(12) S3_GCASE(16)
#undef S3_GCASE
        default: break;
    }
    *launched = 0;
    return cudaSuccess;
}

template <typename T>
cudaError_t prepare_group_t() {
    cudaError_t err = cudaSuccess;
#define S3_GPREP(cc)                                                                                       \
    if (err == cudaSuccess)                                                                                \
        err = cudaFuncSetAttribute(edge_group_kernel<T, cc, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                   (int)kSmemCapGroup);                                                    \
    if (err == cudaSuccess)                                                                                \
        err = cudaFuncSetAttribute(edge_group_kernel<T, cc, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                   (int)kSmemCapGroup);
    S3_GPREP(4) S3_GPREP(8) S3_GPREP(12) S3_GPREP(16)
#undef S3_GPREP
    return err;
}

}  // namespace s3
