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
// ranks push anything out of range.  Roots, the 1-norm, the ratios and their
// min/max are FP64; the series products are FP64, or FP32 until the gap stops
// shrinking or drops below switch_tol and then FP64 or double-float (pairs of
// FP32, S3_DF64), or double-float throughout (the precision option).
// Iterations run in captured CUDA graphs of `check_every` steps; a device flag
// turns the remaining launches of a graph into no-ops once the test passes.  The
// instantiated graphs stay on the handle and are replayed by later calls with
// the same tolerance, iteration cap and graph length.
#include <cuda_runtime.h>

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

// flags: [0] done, [1] iterations, [2] hit max_iter, [3] range trouble
enum { F_DONE = 0, F_ITERS = 1, F_MAXED = 2, F_RANGE = 3 };

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
    r = r - (rk1 * r - b) / ((double)k * rk1);
    return r * Arith<double>::pow2(q);
}

template <typename T>
__device__ __forceinline__ void block_sum_store(double v, double *out) {
    __shared__ double sh[kNqzThreads / 32];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kNqzThreads / 32; ++w) t += sh[w];
        *out = t;
    }
}

// u_v = zt_v^(1/(N-1)) 2^(e_v); partial 1-norms per block
template <typename TZ, typename TX>
__global__ void __launch_bounds__(kNqzThreads) nqz_root_kernel(const TZ *__restrict__ zt, const TX *__restrict__ xin,
                                                               int64_t n, int k, double *__restrict__ u,
                                                               double *__restrict__ partial, int32_t *flags) {
    if (flags[F_DONE]) return;
    double acc = 0.0;
    for (int64_t v = (int64_t)blockIdx.x * kNqzThreads + threadIdx.x; v < n; v += (int64_t)gridDim.x * kNqzThreads) {
        double z = (double)zt[v];
        int e = Arith<TX>::expo(xin[v]);
        double r = root_k(z, k) * Arith<double>::pow2(e);
        if (!(z > 0.0) || !isfinite(z)) flags[F_RANGE] = 1;
        u[v] = r;
        acc += r;
    }
    block_sum_store<double>(acc, partial + blockIdx.x);
}

// x = u / ||u||_1 (FP64) and its FP32 copy
__global__ void __launch_bounds__(kNqzThreads) nqz_normalize_kernel(const double *__restrict__ u, int64_t n,
                                                                    const double *__restrict__ partial, int nparts,
                                                                    double *__restrict__ x64, float *__restrict__ x32,
                                                                    int32_t *flags) {
    if (flags[F_DONE]) return;
    __shared__ double inv;
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < nparts; ++i) t += partial[i];
        inv = 1.0 / t;
    }
    __syncthreads();
    for (int64_t v = (int64_t)blockIdx.x * kNqzThreads + threadIdx.x; v < n; v += (int64_t)gridDim.x * kNqzThreads) {
        double xv = u[v] * inv;
        x64[v] = xv;
        x32[v] = (float)xv;
    }
}

// ratios zt_v / m_v^(N-1) (m_v = x_v 2^-e_v of the vector the TTSV1 call used); partial min/max
template <typename T>
__global__ void __launch_bounds__(kNqzThreads) nqz_ratio_kernel(const T *__restrict__ zt, const T *__restrict__ xin,
                                                                int64_t n, int k, double *__restrict__ partial,
                                                                int32_t *flags) {
    if (flags[F_DONE]) return;
    double lo = INFINITY, hi = -INFINITY;
    for (int64_t v = (int64_t)blockIdx.x * kNqzThreads + threadIdx.x; v < n; v += (int64_t)gridDim.x * kNqzThreads) {
        double xv = (double)xin[v];
        int e = Arith<double>::expo(xv);
        double m = xv * Arith<double>::pow2(-e);
        double pk = 1.0, base = m;
        for (int q = k; q > 0; q >>= 1) {
            if (q & 1) pk *= base;
            base *= base;
        }
        double r = (double)zt[v] / pk;
        if (!isfinite(r) || !(r > 0.0)) flags[F_RANGE] = 1;
        lo = fmin(lo, r);
        hi = fmax(hi, r);
    }
    __shared__ double sl[kNqzThreads / 32], sh[kNqzThreads / 32];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        lo = fmin(lo, __shfl_down_sync(0xffffffffu, lo, d));
        hi = fmax(hi, __shfl_down_sync(0xffffffffu, hi, d));
    }
    if ((threadIdx.x & 31) == 0) {
        sl[threadIdx.x >> 5] = lo;
        sh[threadIdx.x >> 5] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kNqzThreads / 32; ++w) {
            lo = fmin(lo, sl[w]);
            hi = fmax(hi, sh[w]);
        }
        partial[2 * blockIdx.x] = lo;
        partial[2 * blockIdx.x + 1] = hi;
    }
}

// convergence test of Algorithm 1; records (lambda_min, lambda_max) per iteration
__global__ void nqz_check_kernel(const double *__restrict__ partial, int nparts, double tol, int max_iter,
                                 double *__restrict__ hist, int hist_cap, int32_t *flags) {
    if (flags[F_DONE]) return;
    if (threadIdx.x != 0) return;
    double lo = INFINITY, hi = -INFINITY;
    for (int i = 0; i < nparts; ++i) {
        lo = fmin(lo, partial[2 * i]);
        hi = fmax(hi, partial[2 * i + 1]);
    }
    int it = flags[F_ITERS];
    if (it < hist_cap) {
        hist[2 * it] = lo;
        hist[2 * it + 1] = hi;
    }
    flags[F_ITERS] = it + 1;
    if ((hi - lo) / lo < tol) flags[F_DONE] = 1;
    if (flags[F_RANGE]) flags[F_DONE] = 1;
    if (it + 1 >= max_iter) {
        flags[F_DONE] = 1;
        flags[F_MAXED] = 1;
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
    double *part_sum, *part_mm;
    int32_t *flags;
};

// One repeat-body pass.  tz: type of the z from the previous pass; tc: type of this pass's TTSV1.
s3_status nqz_step(s3_graph_s *g, const NqzBufs &b, s3_dtype tz, s3_dtype tc, double tol, int max_iter,
                   cudaStream_t st) {
    const int k = g->N - 1;
    const int64_t n = g->n;
    if (tz == S3_F32)
        nqz_root_kernel<float, float><<<kNqzBlocks, kNqzThreads, 0, st>>>(b.z32, b.x32, n, k, b.u, b.part_sum, b.flags);
    else
        nqz_root_kernel<double, double><<<kNqzBlocks, kNqzThreads, 0, st>>>(b.z64, b.x64, n, k, b.u, b.part_sum,
                                                                             b.flags);
    S3_CUDA(cudaGetLastError());
    nqz_normalize_kernel<<<kNqzBlocks, kNqzThreads, 0, st>>>(b.u, n, b.part_sum, kNqzBlocks, b.x64, b.x32, b.flags);
    S3_CUDA(cudaGetLastError());
    s3_status s;
    if (tc == S3_F32) {
        s = g->opt.layout == S3_LAYOUT_CCSS && g->has_ccss ? run_ccss(g, S3_F32, b.x32, b.z32, 1, b.flags, st)
                                                            : run_edges(g, S3_F32, b.x32, b.z32, 1, b.flags, st);
        if (s != S3_OK) return s;
        nqz_ratio_kernel<float><<<kNqzBlocks, kNqzThreads, 0, st>>>(b.z32, b.x32, n, k, b.part_mm, b.flags);
    } else {
        // tc: S3_F64 or S3_DF64 (FP64 vectors either way; the CCSS layout runs FP64)
        s = g->opt.layout == S3_LAYOUT_CCSS && g->has_ccss ? run_ccss(g, S3_F64, b.x64, b.z64, 1, b.flags, st)
                                                            : run_edges(g, tc, b.x64, b.z64, 1, b.flags, st);
        if (s != S3_OK) return s;
        nqz_ratio_kernel<double><<<kNqzBlocks, kNqzThreads, 0, st>>>(b.z64, b.x64, n, k, b.part_mm, b.flags);
    }
    S3_CUDA(cudaGetLastError());
    nqz_check_kernel<<<1, 32, 0, st>>>(b.part_mm, kNqzBlocks, tol, max_iter, g->d_hist, g->hist_cap, b.flags);
    S3_CUDA(cudaGetLastError());
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
            s = nqz_step(g, b, last_z, phase, tol, opt.max_iter, st);
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
                    cs = nqz_step(g, b, phase, phase, tol, opt.max_iter, st);
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
                    // the last FP32 z is unusable: redo z = TTSV1(x) in FP64 from the same x
                    s = ttsv(hi);
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

}  // extern "C"
