// Per-edge truncated power-series kernels (the S^3TTVc hot path).
//
// For an edge e = (v_1 < ... < v_s) at rank N and a node v_i of e, the
// contribution c(e, v_i) of Algorithm 2 is
//     K(s,N) [t^(N-1)] E(x_{v_i}) prod_{j != i} Ebar(x_{v_j}),
// E(x) = e^(x t), Ebar(x) = e^(x t) - 1 (Sec. II-A).  Because E = Ebar + 1,
//     [t^(N-1)] E(x_{v_i}) F_{e,-i} = [t^(N-1)] F_e + [t^(N-1)] F_{e,-i},
// with F_e = prod_j Ebar(x_{v_j}) and F_{e,-i} = Pre_i Suf_i, the product of
// the factors before and after position i.  A product of k factors Ebar has
// no term below t^k, so Pre_i only matters on degrees i-1 .. i-1+w-1 and
// Suf_i on s-i .. s-i+w-1, with w = N-s+1: every series is kept as a window
// of w coefficients.  Multiplying a window by Ebar(x) is a lower-triangular
// Toeplitz product whose entries are a_k = x^k/k!, k >= 1.
//
// Per edge: prefix windows Pre_2..Pre_s forward (Pre_2 is the power table of
// x_{v_1}), then suffix windows backward; each leave-one-out value is a dot of
// Pre_i with the reversed Suf_i.  Before the products the edge's x values are
// multiplied by an exact power of two g chosen from sum_u |x_u| (target
// T(s,N), host side) so that all coefficients stay near 1; the result is
// multiplied back by K(s,N) g^-(N-1) (exact exponent arithmetic).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <cstdint>
#include <type_traits>

#include "s3_kernels.h"

namespace s3 {

// Window widths with a compile-time kernel instance (one thread per edge).
#define S3_W_CASES(M) \
    M(1) M(2) M(3) M(4) M(5) M(6) M(7) M(8) M(9) M(10) M(11) M(12) M(13) M(14) M(15) M(16) \
    M(17) M(18) M(19) M(20) M(21) M(22) M(23) M(24) M(25) M(26) M(27) M(28) M(29) M(30) M(31) M(32)

// ------------------------------------------------------------ arithmetic --

template <typename T> struct Arith;

template <> struct Arith<float> {
    // x = m 2^e with m in [0.5, 1) for normal x (0 -> 0, subnormal -> -126)
    __device__ __forceinline__ static int expo(float v) {
        int b = (__float_as_int(v) >> 23) & 0xff;
        return b == 0 ? -126 : b - 126;
    }
    // exact 2^p for p in [-126, 127]
    __device__ __forceinline__ static float pow2(int p) {
        p = max(-126, min(127, p));
        return __int_as_float((p + 127) << 23);
    }
    __device__ __forceinline__ static float absv(float v) { return fabsf(v); }
    __device__ __forceinline__ static float tiny() { return FLT_MIN; }
    __device__ __forceinline__ static float huge() { return FLT_MAX; }
    __device__ __forceinline__ static float scale2(float v, int e) { return ldexpf(v, e); }
    __device__ __forceinline__ static float fma_(float a, float b, float c) { return fmaf(a, b, c); }
};

template <> struct Arith<double> {
    __device__ __forceinline__ static int expo(double v) {
        int b = (int)((__double_as_longlong(v) >> 52) & 0x7ff);
        return b == 0 ? -1022 : b - 1022;
    }
    __device__ __forceinline__ static double pow2(int p) {
        p = max(-1022, min(1023, p));
        return __longlong_as_double((long long)(p + 1023) << 52);
    }
    __device__ __forceinline__ static double absv(double v) { return fabs(v); }
    __device__ __forceinline__ static double tiny() { return DBL_MIN; }
    __device__ __forceinline__ static double huge() { return DBL_MAX; }
    __device__ __forceinline__ static double scale2(double v, int e) { return ldexp(v, e); }
    __device__ __forceinline__ static double fma_(double a, double b, double c) { return fma(a, b, c); }
};

// --------------------------------------------------------- double-float --

// An unevaluated sum hi + lo of two FP32 numbers (|lo| <= ulp(hi)/2): about 44
// bits of significand from FP32 instructions, with the error-free sum of
// Knuth (TAOCP 4.2.2) and the FMA-based exact product (after Dekker, 1971).
// Every operation uses the _rn intrinsics, which the compiler never fuses, so
// the error-free transformations stay exact.  The series of an edge run in it
// when S^3TTVc is called with S3_DF64: GB300 executes FP32 at many times its
// FP64 rate, and the windows' values are all near 1 after the per-edge scaling.
struct DF {
    float hi, lo;
};

__device__ __forceinline__ DF df_fast_two_sum(float a, float b) {  // |a| >= |b| or a == 0
    const float s = __fadd_rn(a, b);
    return DF{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ DF df_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return DF{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ DF operator+(DF a, DF b) {
    const DF s = df_two_sum(a.hi, b.hi);
    return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ DF operator*(DF a, DF b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
    return df_fast_two_sum(p, e);
}
__device__ __forceinline__ DF df_from(double d) {
    const float h = __double2float_rn(d);
    return DF{h, __double2float_rn(d - (double)h)};
}
__device__ __forceinline__ double df_to(DF a) { return (double)a.hi + (double)a.lo; }

template <> struct Arith<DF> {
    // a b + c with one exact product error and one error-free sum; the result is left
    // unnormalised (its low part stays within a few units of the high part's last
    // place), which is all the accumulation chains of the window products need
    __device__ __forceinline__ static DF fma_(DF a, DF b, DF c) {
        const float p = __fmul_rn(a.hi, b.hi);
        const float ep = __fmaf_rn(a.hi, b.hi, -p);
        const float s = __fadd_rn(p, c.hi);
        const float bb = __fsub_rn(s, p);
        const float es = __fadd_rn(__fsub_rn(p, __fsub_rn(s, bb)), __fsub_rn(c.hi, bb));
        const float lo = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, __fadd_rn(__fadd_rn(ep, c.lo), es)));
        return DF{s, lo};
    }
};

// Value types of a kernel instance: T is the arithmetic of the series, In the
// type of x (and of the member values in shared memory and the scaling), Out
// the type of the results.
template <typename T> struct Num {
    using In = T;
    using Out = T;
    __device__ __forceinline__ static T cvt(In v) { return v; }
    __device__ __forceinline__ static Out out(T v) { return v; }
    __device__ __forceinline__ static T zero() { return T(0); }
    __device__ __forceinline__ static T add(T a, T b) { return a + b; }
    __device__ __forceinline__ static T recip(int k) { return T(1) / T(k); }
};
template <> struct Num<DF> {
    using In = double;
    using Out = double;
    __device__ __forceinline__ static DF cvt(double v) { return df_from(v); }
    __device__ __forceinline__ static double out(DF v) { return df_to(v); }
    __device__ __forceinline__ static DF zero() { return DF{0.f, 0.f}; }
    __device__ __forceinline__ static DF add(DF a, DF b) { return a + b; }
    __device__ __forceinline__ static DF recip(int k) { return df_from(1.0 / (double)k); }
};

// p such that 2^p * S is within a factor 2 of target (integer exponent arithmetic only).
template <typename T>
__device__ __forceinline__ int scale_exponent(T S, float target) {
    if (!(S > T(0)) || !(S <= T(3.0e38))) return 0;
    int es = Arith<T>::expo(S);
    int et = Arith<float>::expo(target);
    return et - es;
}

// ------------------------------------------------------ final scaling -----

template <typename T>
__device__ __forceinline__ T finalize_value(T val, const EdgeBucketArgs &b, int p, int bias_e,
                                            unsigned long long *range_events);

template <>
__device__ __forceinline__ float finalize_value<float>(float val, const EdgeBucketArgs &b, int p, int bias_e,
                                                       unsigned long long *range_events) {
    int ex = b.Ke - p * (b.N - 1) - bias_e * (b.N - 1);
    float c = ldexpf(val * b.Km, ex);
    if (val > 0.f && !(c >= FLT_MIN && c <= FLT_MAX) && range_events) atomicAdd(range_events, 1ull);
    return c;
}

template <>
__device__ __forceinline__ double finalize_value<double>(double val, const EdgeBucketArgs &b, int p, int bias_e,
                                                         unsigned long long *range_events) {
    int ex = -p * (b.N - 1) - bias_e * (b.N - 1);
    double c = ldexp(val * b.K, ex);
    if (val > 0.0 && !(c >= DBL_MIN && c <= DBL_MAX) && range_events) atomicAdd(range_events, 1ull);
    return c;
}

// -------------------------------------------------------------- scatter ---

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &err) {
    s = a + b;
    float bb = s - a;
    err = (a - (s - bb)) + (b - bb);
}

// Add c to out[v] (atomic modes) with aggregation over the lanes of the warp
// that target the same node.
template <typename T>
__device__ __forceinline__ void scatter_atomic(const EdgeOutArgs &o, int v, T c);

template <>
__device__ __forceinline__ void scatter_atomic<double>(const EdgeOutArgs &o, int v, double c) {
    unsigned act = __activemask();
    unsigned grp = __match_any_sync(act, v);
    int lane = threadIdx.x & 31;
    int leader = __ffs(grp) - 1;
    double acc = 0.0;
    for (unsigned mm = grp; mm; mm &= mm - 1) acc += __shfl_sync(grp, c, __ffs(mm) - 1);
    if (lane == leader) atomicAdd(reinterpret_cast<double *>(o.out) + v, acc);
}

template <>
__device__ __forceinline__ void scatter_atomic<float>(const EdgeOutArgs &o, int v, float c) {
    unsigned act = __activemask();
    unsigned grp = __match_any_sync(act, v);
    int lane = threadIdx.x & 31;
    int leader = __ffs(grp) - 1;
    float acc = 0.f, cmp = 0.f;
    for (unsigned mm = grp; mm; mm &= mm - 1) {
        float t = __shfl_sync(grp, c, __ffs(mm) - 1);
        float s, e;
        two_sum(acc, t, s, e);
        acc = s;
        cmp += e;
    }
    if (lane == leader) {
        float *y = reinterpret_cast<float *>(o.out);
        float old = atomicAdd(y + v, acc);
        if (o.mode == kOutAtomicComp) {
            float s, e;
            two_sum(old, acc, s, e);
            e += cmp;
            if (e != 0.f) atomicAdd(o.comp + v, e);
        }
    }
}

// ------------------------------------------------- thread-per-edge path ---

// a[k] = x^(k+1)/(k+1)!, k = 0..W-1
template <typename T, int W>
__device__ __forceinline__ void power_table(T X, T (&a)[W]) {
    a[0] = X;
#pragma unroll
    for (int k = 1; k < W; ++k) a[k] = a[k - 1] * (X * Num<T>::recip(k + 1));
}

// P <- P * Ebar(x) on the window (one degree up): P[j] = sum_{j' <= j} a[j-j'] P[j']
template <typename T, int W>
__device__ __forceinline__ void toeplitz_inplace(T (&P)[W], const T (&a)[W]) {
#pragma unroll
    for (int j = W - 1; j >= 0; --j) {
        T acc = a[j] * P[0];
#pragma unroll
        for (int jp = 1; jp <= j; ++jp) acc = Arith<T>::fma_(a[j - jp], P[jp], acc);
        P[j] = acc;
    }
}

// xk[k] = x/(k+1), k = 0..W-1: the ratios of consecutive coefficients of Ebar(x)
template <typename T, int W>
__device__ __forceinline__ void ratio_table(T X, T (&xk)[W]) {
#pragma unroll
    for (int k = 0; k < W; ++k) xk[k] = X * Num<T>::recip(k + 1);
}

// P <- P * Ebar(x) on the window, in Horner form: with xk[k] = x/(k+1),
//   P_new[j] = x (P[j] + x/2 (P[j-1] + x/3 (P[j-2] + ... + x/(j+1) P[0])))
// (j + 1 multiply-adds per coefficient, no power table).  Top-down, in place.
template <typename T, int W>
__device__ __forceinline__ void toeplitz_horner(T (&P)[W], const T (&xk)[W]) {
#pragma unroll
    for (int j = W - 1; j >= 0; --j) {
        T acc = P[0];
#pragma unroll
        for (int r = 1; r <= j; ++r) acc = Arith<T>::fma_(xk[j - r + 1], acc, P[r]);
        P[j] = xk[0] * acc;
    }
}

// [t^top] of Q * Ebar(x) where Q's window ends at degree top-1:
//   sum_{k=1}^{W} x^k/k! Q[W-k] = x (Q[W-1] + x/2 (Q[W-2] + ... + x/W Q[0]))
template <typename T, int W>
__device__ __forceinline__ T top_horner(const T (&Q)[W], const T (&xk)[W]) {
    T acc = Q[0];
#pragma unroll
    for (int r = 1; r < W; ++r) acc = Arith<T>::fma_(xk[W - r], acc, Q[r]);
    return xk[0] * acc;
}

// ---------------------------------------------------------- cp.async ---

__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// Asynchronous 4- or 8-byte copy global -> shared memory (completion tracked per thread).
template <int BYTES>
__device__ __forceinline__ void cp_async(void *smem_dst, const void *gmem_src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(smem_addr(smem_dst)), "l"(gmem_src),
                 "n"(BYTES));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Final scaling of one result: c = val * K * 2^(-p(N-1)) [* 2^(-(N-1) e_v) in biased mode]
// as one or two exact power-of-two multiplies (ldexp only when an exponent leaves the
// normal range).
template <typename T>
__device__ __forceinline__ T scale_result(T val, const EdgeBucketArgs &b, int p, int bias_e,
                                          unsigned long long *range_events);

template <>
__device__ __forceinline__ float scale_result<float>(float val, const EdgeBucketArgs &b, int p, int bias_e,
                                                     unsigned long long *range_events) {
    const int ex = b.Ke - (p + bias_e) * (b.N - 1);
    float c = (unsigned)(ex + 126) <= 253u ? (val * b.Km) * Arith<float>::pow2(ex) : ldexpf(val * b.Km, ex);
    // zero, subnormal or non-finite result of a positive value: exponent field 0 or 255
    const unsigned ef = (__float_as_uint(c) >> 23) & 0xffu;
    if ((ef == 0u || ef == 0xffu) && val > 0.f && range_events) atomicAdd(range_events, 1ull);
    return c;
}

template <>
__device__ __forceinline__ double scale_result<double>(double val, const EdgeBucketArgs &b, int p, int bias_e,
                                                       unsigned long long *range_events) {
    const int ex = -(p + bias_e) * (b.N - 1);
    double c = (unsigned)(ex + 1022) <= 2045u ? (val * b.K) * Arith<double>::pow2(ex) : ldexp(val * b.K, ex);
    const unsigned ef = (unsigned)((__double_as_longlong(c) >> 52) & 0x7ff);
    if ((ef == 0u || ef == 0x7ffu) && val > 0.0 && range_events) atomicAdd(range_events, 1ull);
    return c;
}

// BUF: results go to the node-sorted buffer at slot sl; otherwise atomically to y[v].
template <typename T, bool BUF>
__device__ __forceinline__ void emit_value(const EdgeBucketArgs &b, const EdgeOutArgs &o, int v, int sl, T val,
                                           int p, T xhat) {
    int bias_e = o.bias ? (Arith<T>::expo(xhat) - p) : 0;
    T c = scale_result<T>(val, b, p, bias_e, o.range_events);
    if constexpr (BUF) {
        reinterpret_cast<T *>(o.out)[sl] = c;
    } else {
        scatter_atomic<T>(o, v, c);
    }
}

// Output scaling of one edge.  Without the per-node bias every result of the
// edge is multiplied by the same K 2^(-p(N-1)); when that factor is a normal
// number it is formed once (exactly: a power-of-two scaling) and each result
// costs one multiply, the same rounding as scale_result.  Otherwise (and in
// biased mode) each result goes through scale_result.
template <typename T> struct EdgeScale {
    T mult;
    bool fast;
};

__device__ __forceinline__ EdgeScale<float> edge_scale(const EdgeBucketArgs &b, const EdgeOutArgs &o, int p, float) {
    EdgeScale<float> r;
    const int ex = b.Ke - p * (b.N - 1);
    r.fast = !o.bias && ex >= -125 && ex <= 127;  // Km 2^ex normal (Km in [0.5, 1))
    r.mult = b.Km * Arith<float>::pow2(ex);
    return r;
}
__device__ __forceinline__ EdgeScale<double> edge_scale(const EdgeBucketArgs &b, const EdgeOutArgs &o, int p,
                                                        double) {
    EdgeScale<double> r;
    const int ex = -p * (b.N - 1);
    r.mult = (ex >= -1022 && ex <= 1023) ? b.K * Arith<double>::pow2(ex) : 0.0;
    r.fast = !o.bias && r.mult >= DBL_MIN && r.mult <= DBL_MAX;
    return r;
}

// 1 if c is not a positive normal number (zero, subnormal, infinite or NaN).
__device__ __forceinline__ int not_normal_pos(float c) {
    return (__float_as_uint(c) - 0x00800000u) >= 0x7f000000u;
}
__device__ __forceinline__ int not_normal_pos(double c) {
    return ((unsigned long long)__double_as_longlong(c) - 0x0010000000000000ull) >= 0x7fe0000000000000ull;
}

// Store (or add) one result on the fast path; nbad counts results of positive
// values that left the normal range (reported once per edge).
template <typename T, bool BUF>
__device__ __forceinline__ void emit_fast(const EdgeOutArgs &o, int t, T val, T mult, int &nbad) {
    const T c = val * mult;
    nbad += (val > T(0)) & not_normal_pos(c);
    if constexpr (BUF) {
        reinterpret_cast<T *>(o.out)[t] = c;
    } else {
        scatter_atomic<T>(o, t, c);
    }
}

// Shared-memory layout of the thread-per-edge kernels: every warp owns a
// region in which element k of lane l sits at k * kLS + l, so that a lane's
// elements are a compile-time stride apart (immediate offsets) and a warp's
// accesses to one k hit 32 consecutive words.
constexpr int kLS = 32;

// All contributions of one edge.  Xs[i*kLS]: the member values (type In); Pre:
// this lane's column for Pre_2..Pre_{s-1}; ib/sb: its member ids / incidence slots.
template <typename T, int W, bool BUF>
__device__ __forceinline__ void edge_compute(const EdgeBucketArgs &b, const EdgeOutArgs &o,
                                             const typename Num<T>::In *Xs, T *Pre, const int32_t *ib,
                                             const int32_t *sb, int s) {
    using In = typename Num<T>::In;
    using Out = typename Num<T>::Out;
    In S = In(0);
    for (int i = 0; i < s; ++i) S += Arith<In>::absv(Xs[i * kLS]);
    const int p = scale_exponent<In>(S, b.target);
    const In g = Arith<In>::pow2(p);
    const int32_t *ob = BUF ? sb : ib;  // where each member's result goes
    const EdgeScale<Out> sc = edge_scale(b, o, p, Out(0));
    int nbad = 0;
    auto emit = [&](int q, T val, In xhat) {
        const int t = ob[q * kLS];
        const Out v = Num<T>::out(val);
        if (sc.fast) emit_fast<Out, BUF>(o, t, v, sc.mult, nbad);
        else emit_value<Out, BUF>(b, o, t, t, v, p, xhat);
    };

    // forward: P = Pre_2, then Pre_3 .. Pre_s (windows Pre_2..Pre_{s-1} kept in shared memory)
    T P[W];
    power_table<T, W>(Num<T>::cvt(Xs[0] * g), P);
    for (int i = 1; i <= s - 2; ++i) {
        T *slot = Pre + (i - 1) * W * kLS;
#pragma unroll
        for (int j = 0; j < W; ++j) slot[j * kLS] = P[j];
        T xk[W];
        ratio_table<T, W>(Num<T>::cvt(Xs[i * kLS] * g), xk);
        toeplitz_horner<T, W>(P, xk);
    }
    // P = Pre_s.  backward: Q = Suf_{s-1} = Ebar(x_{v_s})
    T Q[W];
    const In xs_last = Xs[(s - 1) * kLS] * g;
    power_table<T, W>(Num<T>::cvt(xs_last), Q);
    T F = Num<T>::zero();
#pragma unroll
    for (int j = 0; j <= W - 2; ++j) F = Arith<T>::fma_(P[j], Q[W - 2 - j], F);
    emit(s - 1, Num<T>::add(F, P[W - 1]), xs_last);
    T top = Num<T>::zero();
    for (int q = s - 2; q >= 1; --q) {
        // Q = Suf_{q+1}; Pre_{q+1} sits in slot q-1
        const T *slot = Pre + (q - 1) * W * kLS;
        T D = Num<T>::zero();
#pragma unroll
        for (int j = 0; j < W; ++j) D = Arith<T>::fma_(slot[j * kLS], Q[W - 1 - j], D);
        const In xq = Xs[q * kLS] * g;
        emit(q, Num<T>::add(F, D), xq);
        T xk[W];
        ratio_table<T, W>(Num<T>::cvt(xq), xk);
        if (q >= 2) toeplitz_horner<T, W>(Q, xk);
        else top = top_horner<T, W>(Q, xk);
    }
    T D1 = (s == 2) ? Q[W - 1] : top;
    emit(0, Num<T>::add(F, D1), Xs[0] * g);
    if (nbad && o.range_events) atomicAdd(o.range_events, (unsigned long long)nbad);
}

// Edges a launch processes: all m of the bucket, or in list mode the count that
// the closed-form kernel left (read once per thread, after that kernel finished).
__device__ __forceinline__ int64_t list_length(const EdgeBucketArgs &b) {
    return b.list ? min((int64_t)__ldcg(b.count), b.m) : b.m;
}

// List mode: the first thread of the grid adds the list's length to a running
// total (count[2..3], 8-byte aligned).  The length itself is cleared before the
// next call's closed-form launch.
__device__ __forceinline__ void list_tally(const EdgeBucketArgs &b) {
    if (b.list && blockIdx.x == 0 && threadIdx.x == 0) {
        const int c = __ldcg(b.count);
        if (c > 0) atomicAdd(reinterpret_cast<unsigned long long *>(b.count + 2), (unsigned long long)c);
    }
}

// Shared memory per lane: Xb[2][s] and Pre[(s-2) W] of T, then Ib[3][s] member
// ids and Sb[3][s] incidence slots (int32); 4-byte words.
template <typename T>
__host__ __device__ constexpr size_t thread_smem_words(int s, int W) {
    return (size_t)(2 * s + (s > 2 ? (s - 2) * W : 0)) * sizeof(T) / 4 + (size_t)6 * s;
}

// One thread per edge, several edges per thread (grid-stride), software
// pipelined with cp.async: while edge k is computed, the x gathers of edge k+1
// and the id/slot loads of edge k+2 are in flight.  Ring buffers rotate by
// pointer; global addresses advance by the grid stride.
template <typename T, int W, bool BUF>
__global__ void __launch_bounds__(256) edge_thread_kernel(EdgeBucketArgs b, const typename Num<T>::In *__restrict__ x,
                                                          EdgeOutArgs o) {
    using In = typename Num<T>::In;
    static_assert(sizeof(In) == sizeof(T), "member values and series values share the element size");
    if (o.skip && *o.skip) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int BS = blockDim.x;
    const int tid = threadIdx.x, lane = tid & 31;
    const int s = b.s;
    const size_t words = thread_smem_words<T>(s, W);
    T *wb = reinterpret_cast<T *>(smem_raw + (size_t)(tid >> 5) * words * 4 * kLS);  // this warp's region
    In *xc = reinterpret_cast<In *>(wb) + lane;   // X of the edge being computed
    In *xn = xc + s * kLS;                        // X of the next edge (in flight)
    T *Pre = wb + 2 * s * kLS + lane;
    int32_t *ibase = reinterpret_cast<int32_t *>(wb + (2 * s + (s > 2 ? (s - 2) * W : 0)) * kLS) + lane;
    const int ring = s * kLS;
    // ring slots (ids; the slots array sits 3 rings further): current, next, after next
    int32_t *r0 = ibase, *r1 = ibase + ring, *r2 = ibase + 2 * ring;
    const int64_t stride = (int64_t)gridDim.x * BS;
    int64_t e = (int64_t)blockIdx.x * BS + tid;
    const int64_t m = list_length(b);
    list_tally(b);
    const int64_t ld = b.ld;
    // member i of bucket edge k sits at ids[i*ld + k]; in list mode the j-th edge is list[j]
    auto edge_of = [&](int64_t j) -> int64_t { return b.list ? (int64_t)__ldg(b.list + j) : j; };
    auto issue_ids = [&](int64_t k, int32_t *dst) {
        const int32_t *gi = b.ids + k, *gs = b.slot + k;
        int32_t *d = dst;
        for (int i = 0; i < s; ++i) {
            cp_async<4>(d, gi);
            if (BUF) cp_async<4>(d + 3 * ring, gs);
            d += kLS;
            gi += ld;
            gs += ld;
        }
    };
    auto issue_x = [&](const int32_t *src, In *xb) {
        for (int i = 0; i < s; ++i) cp_async<(int)sizeof(In)>(xb + i * kLS, x + src[i * kLS]);
    };

    if (e < m) {
        issue_ids(edge_of(e), r0);
        cp_async_commit();
        cp_async_wait_all();
        issue_x(r0, xc);
        if (e + stride < m) issue_ids(edge_of(e + stride), r1);
        cp_async_commit();
        for (; e < m; e += stride) {
            cp_async_wait_all();
            if (e + stride < m) issue_x(r1, xn);
            if (e + 2 * stride < m) issue_ids(edge_of(e + 2 * stride), r2);
            cp_async_commit();
            edge_compute<T, W, BUF>(b, o, xc, Pre, r0, r0 + 3 * ring, s);
            int32_t *t = r0;
            r0 = r1;
            r1 = r2;
            r2 = t;
            In *tx = xc;
            xc = xn;
            xn = tx;
        }
        cp_async_wait_all();
    }
}

// Size-2 edges.  With P = Ebar(x_{v_1}) and Q = Ebar(x_{v_2}) on degrees 1..W
// (W = N - 1), F = [t^(N-1)] P Q = sum_{j=0}^{W-2} P[j] Q[W-2-j], and the two
// contributions are K (F + P[W-1]) for v_2 and K (F + Q[W-1]) for v_1 -- the
// general kernel's arithmetic at s = 2, in the same order.  The bucket moves
// 32 bytes per edge for about 5 W flops, so this variant keeps only Q in
// registers (P runs as a scalar), reads ids, slots and x with plain coalesced
// or L2 loads and no shared memory, and keeps the loads of kPairEdges edges
// per thread in flight together.
constexpr int kPairEdges = 4;

template <typename T, int W, bool BUF>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2) edge_pair_kernel(EdgeBucketArgs b, const typename Num<T>::In *__restrict__ x,
                                                           EdgeOutArgs o) {
    using In = typename Num<T>::In;
    using Out = typename Num<T>::Out;
    if (o.skip && *o.skip) return;
    constexpr int E = kPairEdges;
    const int64_t span = (int64_t)blockDim.x * E;
    const int64_t stride = (int64_t)gridDim.x * span;
    const int64_t m = list_length(b);
    list_tally(b);
    int nbad = 0;
    for (int64_t e0 = (int64_t)blockIdx.x * span + threadIdx.x; e0 < m; e0 += stride) {
        int v0[E], v1[E], t0[E], t1[E];
        In X0[E], X1[E];
#pragma unroll
        for (int k = 0; k < E; ++k) {
            const int64_t j = e0 + (int64_t)k * blockDim.x;
            const bool in = j < m;
            const int64_t e = in && b.list ? (int64_t)__ldg(b.list + j) : j;
            v0[k] = in ? __ldg(b.ids + e) : 0;
            v1[k] = in ? __ldg(b.ids + b.ld + e) : 0;
            t0[k] = BUF ? (in ? __ldg(b.slot + e) : 0) : v0[k];
            t1[k] = BUF ? (in ? __ldg(b.slot + b.ld + e) : 0) : v1[k];
        }
#pragma unroll
        for (int k = 0; k < E; ++k) {
            X0[k] = __ldg(x + v0[k]);
            X1[k] = __ldg(x + v1[k]);
        }
#pragma unroll
        for (int k = 0; k < E; ++k) {
            if (e0 + (int64_t)k * blockDim.x >= m) break;
            const int p = scale_exponent<In>(Arith<In>::absv(X0[k]) + Arith<In>::absv(X1[k]), b.target);
            const In g = Arith<In>::pow2(p);
            const In a0x = X0[k] * g, a1x = X1[k] * g;
            const T a0 = Num<T>::cvt(a0x), a1 = Num<T>::cvt(a1x);
            T Q[W];
            power_table<T, W>(a1, Q);
            T P = a0, F = Num<T>::zero();
#pragma unroll
            for (int j = 0; j <= W - 2; ++j) {
                F = Arith<T>::fma_(P, Q[W - 2 - j], F);
                P = P * (a0 * Num<T>::recip(j + 2));
            }
            const Out c1 = Num<T>::out(Num<T>::add(F, P)), c0 = Num<T>::out(Num<T>::add(F, Q[W - 1]));
            const EdgeScale<Out> sc = edge_scale(b, o, p, Out(0));
            if (sc.fast) {
                emit_fast<Out, BUF>(o, t1[k], c1, sc.mult, nbad);
                emit_fast<Out, BUF>(o, t0[k], c0, sc.mult, nbad);
            } else {
                emit_value<Out, BUF>(b, o, t1[k], t1[k], c1, p, a1x);
                emit_value<Out, BUF>(b, o, t0[k], t0[k], c0, p, a0x);
            }
        }
    }
    if (nbad && o.range_events) atomicAdd(o.range_events, (unsigned long long)nbad);
}

// --------------------------------------------- fused launch of small buckets --

// Shared memory per lane of the one-edge-per-thread tail kernel: X[s] and
// Pre[(s-2) W] of T, then ids[s] and slots[s] (int32); edge_tail_smem_words in
// s3_kernels.h counts its 4-byte words.  Every warp's region holds lane_words
// words per lane (the largest need of the launch's buckets).
template <typename T, int W, bool BUF>
__device__ __forceinline__ void tail_edge(const EdgeBucketArgs &b, const typename Num<T>::In *__restrict__ x,
                                          const EdgeOutArgs &o, int64_t e, unsigned char *smem_raw, int lane_words) {
    using In = typename Num<T>::In;
    const int tid = threadIdx.x, lane = tid & 31, s = b.s;
    T *wb = reinterpret_cast<T *>(smem_raw + (size_t)(tid >> 5) * lane_words * 4 * kLS);
    In *xs = reinterpret_cast<In *>(wb) + lane;
    T *Pre = wb + s * kLS + lane;
    int32_t *ib = reinterpret_cast<int32_t *>(wb + (s + (s > 2 ? (s - 2) * W : 0)) * kLS) + lane;
    int32_t *sb = ib + s * kLS;
    for (int i = 0; i < s; ++i) {
        cp_async<4>(ib + i * kLS, b.ids + (int64_t)i * b.ld + e);
        if (BUF) cp_async<4>(sb + i * kLS, b.slot + (int64_t)i * b.ld + e);
    }
    cp_async_commit();
    cp_async_wait_all();
    for (int i = 0; i < s; ++i) cp_async<(int)sizeof(In)>(xs + i * kLS, x + ib[i * kLS]);
    cp_async_commit();
    cp_async_wait_all();
    edge_compute<T, W, BUF>(b, o, xs, Pre, ib, sb, s);
}

// All small buckets of a call in one launch: block ranges of the grid map to
// buckets (TailEntry::block0 ascending), one edge per thread.  Buckets with few
// edges are bound by the latency of one edge's load -> gather -> compute chain,
// so one launch for all of them pays that latency once instead of per bucket.
template <typename T, bool BUF>
__global__ void __launch_bounds__(128) edge_tail_kernel(const TailEntry *__restrict__ tab, int ntab, int lane_words,
                                                        const typename Num<T>::In *__restrict__ x, EdgeOutArgs o) {
    if (o.skip && *o.skip) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int k = 0;
    while (k + 1 < ntab && tab[k + 1].block0 <= (int64_t)blockIdx.x) ++k;
    const EdgeBucketArgs b = tab[k].b;
    const int64_t e = ((int64_t)blockIdx.x - tab[k].block0) * blockDim.x + threadIdx.x;
    if (e >= b.m) return;
    switch (tab[k].W) {
#define S3_TAIL_CASE(w) \
    case w: tail_edge<T, w, BUF>(b, x, o, e, smem_raw, lane_words); break;
        S3_W_CASES(S3_TAIL_CASE)
#undef S3_TAIL_CASE
        default: break;
    }
}

// Size-1 edges: c(e, v) = x_v^(N-1) (K(1,N) [t^(N-1)] e^(x t) with K(1,N) = (N-1)!).
template <typename T>
__global__ void edge_single_kernel(EdgeBucketArgs b, const T *__restrict__ x, EdgeOutArgs o) {
    if (o.skip && *o.skip) return;
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= b.m) return;
    int v = __ldg(b.ids + e);
    T X = __ldg(x + v);
    // X = m 2^ex, m in [0.5,1): X^(N-1) = m^(N-1) 2^((N-1) ex)
    int ex = Arith<T>::expo(X);
    T mm = X * Arith<T>::pow2(-ex);
    T r = T(1), base = mm;
    for (int k = b.N - 1; k > 0; k >>= 1) {
        if (k & 1) r *= base;
        base *= base;
    }
    int bias_e = o.bias ? ex : 0;
    T c = Arith<T>::scale2(r, (b.N - 1) * (ex - bias_e));
    if (r != T(0) && !(Arith<T>::absv(c) >= Arith<T>::tiny() && Arith<T>::absv(c) <= Arith<T>::huge()) &&
        o.range_events)
        atomicAdd(o.range_events, 1ull);
    if (o.mode == kOutBuffer) {
        reinterpret_cast<T *>(o.out)[__ldg(b.slot + e)] = c;
    } else {
        scatter_atomic<T>(o, v, c);
    }
}

// --------------------------------------------------- warp-per-edge path ---

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    return v;
}

// out[k] = x^(k+1)/(k+1)!, k < W, as a prefix product of x/(k+1) over the lanes.
template <typename T>
__device__ __forceinline__ void power_table_warp(T X, T *out, int W) {
    const int lane = threadIdx.x & 31;
    T carry = T(1);
    for (int base = 0; base < W; base += 32) {
        int k = base + lane;
        T c = k < W ? X / T(k + 1) : T(1);
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            T t = __shfl_up_sync(0xffffffffu, c, d);
            if (lane >= d) c *= t;
        }
        c *= carry;
        if (k < W) out[k] = c;
        carry = __shfl_sync(0xffffffffu, c, 31);
    }
}

// One edge computed by one warp.  Per warp shared memory (elements of T): Xs[s] | C[s] |
// Pre[(s-2) W] (Pre_2..Pre_{s-1}) | Pcur[W] | Q[W] | A[W] | R[W].
template <typename T>
__device__ __forceinline__ void warp_edge_compute(const EdgeBucketArgs &b, const T *__restrict__ x,
                                                  const EdgeOutArgs &o, int64_t e, int W, T *base) {
    const int lane = threadIdx.x & 31;
    const int s = b.s;
    T *Xs = base;
    T *C = Xs + s;
    T *Pre = C + s;
    T *Pc = Pre + (int64_t)(s > 2 ? s - 2 : 0) * W;
    T *Q = Pc + W;
    T *A = Q + W;
    T *R = A + W;
    T part = T(0);
    for (int i = lane; i < s; i += 32) {
        T X = __ldg(x + __ldg(b.ids + (int64_t)i * b.ld + e));
        Xs[i] = X;
        part += Arith<T>::absv(X);
    }
    T S = warp_sum(part);
    const int p = scale_exponent<T>(S, b.target);
    const T g = Arith<T>::pow2(p);
    __syncwarp();
    for (int i = lane; i < s; i += 32) Xs[i] *= g;
    __syncwarp();
    // forward
    power_table_warp<T>(Xs[0], Pc, W);
    __syncwarp();
    for (int i = 1; i <= s - 2; ++i) {
        T *slotp = Pre + (int64_t)(i - 1) * W;
        for (int j = lane; j < W; j += 32) slotp[j] = Pc[j];
        power_table_warp<T>(Xs[i], A, W);
        __syncwarp();
        for (int j = lane; j < W; j += 32) {
            T acc = T(0);
            for (int jp = 0; jp <= j; ++jp) acc = Arith<T>::fma_(A[j - jp], slotp[jp], acc);
            Pc[j] = acc;
        }
        __syncwarp();
    }
    // backward
    power_table_warp<T>(Xs[s - 1], Q, W);
    __syncwarp();
    T fp = T(0);
    for (int j = lane; j <= W - 2; j += 32) fp = Arith<T>::fma_(Pc[j], Q[W - 2 - j], fp);
    const T F = warp_sum(fp);
    if (lane == 0) C[s - 1] = F + Pc[W - 1];
    T top = T(0);
    for (int q = s - 2; q >= 1; --q) {
        const T *pre = Pre + (int64_t)(q - 1) * W;
        T dp = T(0);
        for (int j = lane; j < W; j += 32) dp = Arith<T>::fma_(pre[j], Q[W - 1 - j], dp);
        T D = warp_sum(dp);
        if (lane == 0) C[q] = F + D;
        power_table_warp<T>(Xs[q], A, W);
        __syncwarp();
        if (q >= 2) {
            for (int j = lane; j < W; j += 32) {
                T acc = T(0);
                for (int jp = 0; jp <= j; ++jp) acc = Arith<T>::fma_(A[j - jp], Q[jp], acc);
                R[j] = acc;
            }
            __syncwarp();
            T *t = Q;
            Q = R;
            R = t;
        } else {
            T tp = T(0);
            for (int jp = lane; jp < W; jp += 32) tp = Arith<T>::fma_(A[W - 1 - jp], Q[jp], tp);
            top = warp_sum(tp);
        }
    }
    if (lane == 0) C[0] = F + (s == 2 ? Q[W - 1] : top);
    __syncwarp();
    for (int q = lane; q < s; q += 32) {
        int bias_e = o.bias ? (Arith<T>::expo(Xs[q]) - p) : 0;
        T c = finalize_value<T>(C[q], b, p, bias_e, o.range_events);
        if (o.mode == kOutBuffer) {
            reinterpret_cast<T *>(o.out)[__ldg(b.slot + (int64_t)q * b.ld + e)] = c;
        } else {
            int v = __ldg(b.ids + (int64_t)q * b.ld + e);
            if constexpr (sizeof(T) == 8) {
                atomicAdd(reinterpret_cast<double *>(o.out) + v, (double)c);
            } else {
                float *y = reinterpret_cast<float *>(o.out);
                float old = atomicAdd(y + v, (float)c);
                if (o.mode == kOutAtomicComp) {
                    float sm, er;
                    two_sum(old, (float)c, sm, er);
                    if (er != 0.f) atomicAdd(o.comp + v, er);
                }
            }
        }
    }
    __syncwarp();
}


// One edge per warp, grid-stride over the bucket.
template <typename T>
__global__ void __launch_bounds__(128) edge_warp_kernel(EdgeBucketArgs b, const T *__restrict__ x, EdgeOutArgs o,
                                                        int W, int64_t per_warp) {
    if (o.skip && *o.skip) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int wib = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    T *base = reinterpret_cast<T *>(smem_raw) + (int64_t)wib * per_warp;
    for (int64_t e = (int64_t)blockIdx.x * wpb + wib; e < b.m; e += (int64_t)gridDim.x * wpb)
        warp_edge_compute<T>(b, x, o, e, W, base);
}

}  // namespace s3

// ------------------------------------------------------------- launchers --

namespace s3 {

constexpr size_t kSmemCap = kEdgeSmemCap;     // per block, thread-per-edge kernels
constexpr size_t kSmemCapWarp = 200 * 1024;   // per block, warp-per-edge kernel
constexpr int kMaxThreadW = 32;

template <typename T, int W, bool BUF>
cudaError_t launch_thread_wb(const EdgeBucketArgs &b, const typename Num<T>::In *x, const EdgeOutArgs &o, int bs,
                             cudaStream_t st) {
    size_t smem = thread_smem_words<T>(b.s, W) * 4 * (size_t)bs;
    // enough blocks to fill the GPU (several edges per thread beyond that)
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 148;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, edge_thread_kernel<T, W, BUF>, bs, smem) != cudaSuccess ||
        per_sm <= 0) {
        cudaGetLastError();
        per_sm = 1;
    }
    int64_t full = (int64_t)sms * per_sm;
    int64_t need = (b.m + bs - 1) / bs;
    int64_t grid = need < full ? need : full;
    edge_thread_kernel<T, W, BUF><<<(unsigned)grid, bs, smem, st>>>(b, x, o);
    return cudaGetLastError();
}

template <typename T, int W>
cudaError_t launch_thread_w(const EdgeBucketArgs &b, const typename Num<T>::In *x, const EdgeOutArgs &o, int bs,
                            cudaStream_t st) {
    return o.mode == kOutBuffer ? launch_thread_wb<T, W, true>(b, x, o, bs, st)
                                : launch_thread_wb<T, W, false>(b, x, o, bs, st);
}

template <typename T, int W>
cudaError_t prepare_thread_w() {
    cudaError_t e =
        cudaFuncSetAttribute(edge_thread_kernel<T, W, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(edge_thread_kernel<T, W, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kSmemCap);
}

template <typename T>
cudaError_t prepare_edge_kernels_t() {
    cudaError_t err = cudaSuccess;
#define S3_PREP(w) if (err == cudaSuccess) err = prepare_thread_w<T, w>();
    S3_W_CASES(S3_PREP)
#undef S3_PREP
    if (err == cudaSuccess)
        err = cudaFuncSetAttribute(edge_warp_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCapWarp);
    if (err == cudaSuccess) err = prepare_edge_group(T(0));
    if (err == cudaSuccess)
        err = cudaFuncSetAttribute(edge_tail_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap);
    if (err == cudaSuccess)
        err = cudaFuncSetAttribute(edge_tail_kernel<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap);
    return err;
}

// Blocks of a grid-stride kernel that fill the device once (occupancy x SMs) for a
// fixed block size and no dynamic shared memory, queried once per kernel.
template <auto Kernel, int BS>
int64_t full_grid() {
    static int sms = 0, per_sm = 0;
    if (sms == 0) {
        int dev = 0, n = 0, k = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k, Kernel, BS, 0) != cudaSuccess || k <= 0) {
            cudaGetLastError();
            k = 1;
        }
        per_sm = k;
        sms = n;
    }
    return (int64_t)sms * per_sm;
}

template <typename T, int W>
cudaError_t launch_pair_w(const EdgeBucketArgs &b, const typename Num<T>::In *x, const EdgeOutArgs &o,
                          cudaStream_t st) {
    constexpr int bs = 256;
    const int64_t need = (b.m + bs - 1) / bs;
    if (o.mode == kOutBuffer) {
        const int64_t grid = std::min<int64_t>(need, full_grid<edge_pair_kernel<T, W, true>, bs>());
        edge_pair_kernel<T, W, true><<<(unsigned)grid, bs, 0, st>>>(b, x, o);
    } else {
        const int64_t grid = std::min<int64_t>(need, full_grid<edge_pair_kernel<T, W, false>, bs>());
        edge_pair_kernel<T, W, false><<<(unsigned)grid, bs, 0, st>>>(b, x, o);
    }
    return cudaGetLastError();
}

// The fused launch of the small buckets listed in tab (device memory, ntab entries,
// nblocks blocks of bs threads in total, smem bytes of dynamic shared memory).
template <typename T>
cudaError_t launch_edge_tail_t(const TailEntry *tab, int ntab, int64_t nblocks, int bs, size_t smem,
                               const typename Num<T>::In *x, const EdgeOutArgs &o, cudaStream_t st) {
    if (ntab <= 0 || nblocks <= 0) return cudaSuccess;
    if (smem > kSmemCap || nblocks > INT32_MAX) return cudaErrorInvalidConfiguration;
    const int lane_words = (int)(smem / 4 / (size_t)bs);
    if (o.mode == kOutBuffer)
        edge_tail_kernel<T, true><<<(unsigned)nblocks, bs, smem, st>>>(tab, ntab, lane_words, x, o);
    else
        edge_tail_kernel<T, false><<<(unsigned)nblocks, bs, smem, st>>>(tab, ntab, lane_words, x, o);
    return cudaGetLastError();
}

// Threads per block for the thread-per-edge kernel so that the block's shared
// memory stays under kSmemCap; 0 if not even one warp fits.
template <typename T>
int thread_block_size(int s, int W, int want) {
    size_t per_thread = thread_smem_words<T>(s, W) * 4;
    int bs = want;
    while (bs > 32 && per_thread * (size_t)bs > kSmemCap) bs -= 32;
    return per_thread * (size_t)bs > kSmemCap ? 0 : bs;
}

template <typename T>
cudaError_t launch_edge_bucket_t(const EdgeBucketArgs &b, const typename Num<T>::In *x, const EdgeOutArgs &o,
                                 int thread_max_w, int block_threads, cudaStream_t st) {
    if (b.m <= 0) return cudaSuccess;
    {
        if (b.s == 1) {
            int bs = 256;
            edge_single_kernel<T><<<(unsigned)((b.m + bs - 1) / bs), bs, 0, st>>>(b, x, o);
            return cudaGetLastError();
        }
    }
    const int W = b.N - b.s + 1;
    if (thread_max_w <= 0 || thread_max_w > kMaxThreadW) thread_max_w = kMaxThreadW;
    if (block_threads <= 0) block_threads = 128;
    if (b.s == 2 && W <= thread_max_w) {
        switch (W) {
#define S3_CASE(w) \
    case w: return launch_pair_w<T, w>(b, x, o, st);
            S3_W_CASES(S3_CASE)
#undef S3_CASE
            default: break;
        }
    }
    if (W <= thread_max_w) {
        int bs = thread_block_size<T>(b.s, W, block_threads);
        if (bs > 0) {
            switch (W) {
#define S3_CASE(w) \
    case w: return launch_thread_w<T, w>(b, x, o, bs, st);
                S3_W_CASES(S3_CASE)
#undef S3_CASE
                default: break;
            }
        }
    }
    {
        // wide windows: eight lanes per edge (s3_group.cuh) when four edges fit a warp's shared memory
        {
            int launched = 0;
            cudaError_t e = launch_edge_group(b, x, o, W, st, &launched);
            if (e != cudaSuccess || launched) return e;
        }
        // one warp per edge
        int64_t per_warp = warp_smem_elems(b.s, W);
        int wpb = 4;
        while (wpb > 1 && (size_t)wpb * per_warp * sizeof(T) > kSmemCapWarp) wpb /= 2;
        size_t smem = (size_t)wpb * per_warp * sizeof(T);
        if (smem > kSmemCapWarp) return cudaErrorInvalidConfiguration;
        int64_t grid = (b.m + wpb - 1) / wpb;
        if (grid > (1 << 22)) grid = 1 << 22;
        edge_warp_kernel<T><<<(unsigned)grid, wpb * 32, smem, st>>>(b, x, o, W, per_warp);
        return cudaGetLastError();
    }
}

}  // namespace s3
