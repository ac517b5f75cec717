// C ABI entry points: handles, format upload, S^3TTVc orchestration.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "s3_graph.h"

namespace s3 {

namespace {
thread_local std::string g_last_error;
}

void set_error(const std::string &msg) { g_last_error = msg; }

s3_status fail(s3_status st, const std::string &msg) {
    g_last_error = msg;
    return st;
}

s3_status cuda_fail(cudaError_t e, const char *what) {
    cudaGetLastError();
    return fail(S3_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

s3_status mark_done(s3_graph_s *g, cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    S3_CUDA(cudaStreamIsCapturing(st, &cs));
    if (cs == cudaStreamCaptureStatusNone) S3_CUDA(cudaEventRecord(g->ev_done, st));
    return S3_OK;
}

s3_status prepare_device(int dev) {
    static std::mutex mu;
    static std::vector<char> done;
    std::lock_guard<std::mutex> lock(mu);
    if ((int)done.size() <= dev) done.resize(dev + 1, 0);
    if (done[dev]) return S3_OK;
    S3_CUDA(prepare_edge_kernels_f32());
    S3_CUDA(prepare_edge_kernels_f64());
    S3_CUDA(prepare_edge_kernels_df());
    S3_CUDA(prepare_edge_bern_f32());
    S3_CUDA(prepare_edge_bern_f64());
    done[dev] = 1;
    return S3_OK;
}

namespace {

template <typename T>
s3_status upload(s3_graph_s *g, T **dst, const std::vector<T> &src) {
    s3_status st = dev_alloc(g, dst, src.size());
    if (st != S3_OK) return st;
    if (!src.empty()) S3_CUDA(cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
    return S3_OK;
}

void free_all(s3_graph_s *g) {
    for (auto &x : g->nqz_exec)
        if (x.exec) {
            cudaGraphExecDestroy(x.exec);
            x.exec = nullptr;
        }
    for (void *p : g->allocations) cudaFree(p);
    g->allocations.clear();
    for (int i = 0; i < 8; ++i) {
        if (g->aux[i]) cudaStreamDestroy(g->aux[i]);
        if (g->ev_join[i]) cudaEventDestroy(g->ev_join[i]);
        g->aux[i] = nullptr;
        g->ev_join[i] = nullptr;
    }
    if (g->ev_fork) cudaEventDestroy(g->ev_fork);
    g->ev_fork = nullptr;
    if (g->ev_done) cudaEventDestroy(g->ev_done);
    g->ev_done = nullptr;
    if (g->qstream) cudaStreamDestroy(g->qstream);
    g->qstream = nullptr;
    for (auto &ex : g->host_exec) {
        if (ex) cudaGraphExecDestroy(ex);
        ex = nullptr;
    }
    if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
    g->cap_stream = nullptr;
    if (g->h_range) cudaFreeHost(g->h_range);
    g->h_range = nullptr;
}

// Wait for the handle's last call (its completion event), not for the whole device.
s3_status wait_done(s3_graph_s *g) {
    S3_CUDA(cudaEventSynchronize(g->ev_done));
    return S3_OK;
}

}  // namespace

// Closed-form evaluation of small buckets (s3_closed.cuh): which call types may use
// it for bucket k (bit 1 = FP32, 2 = FP64), apart from the rule that it needs a launch
// of its own.  2 <= s <= closed_form_max_s, 2 <= N-1 <= 127, the bucket's series
// kernel takes lists (one thread per edge: W <= thread_max_w), the closed form needs
// fewer operations than the series, and edges with equal x pass the error gate with a
// margin of 2 (so that near-uniform inputs are not sent back).
int closed_form_mask(const s3_graph_s *g, size_t k) {
    const int max_s = g->opt.closed_form_max_s == 0 ? kClosedMaxS : std::min(g->opt.closed_form_max_s, kClosedMaxS);
    const int tmw = (g->opt.thread_max_w <= 0 || g->opt.thread_max_w > 32) ? 32 : g->opt.thread_max_w;
    const int n = g->N - 1;
    const HostBucket &hb = g->buckets[k];
    const int s = hb.s, W = g->N - s + 1;
    if (max_s < 2 || s < 2 || s > max_s || n < 2 || n > 127 || hb.m <= 0 || W > tmw) return 0;
    int lg = 0;
    while ((n >> (lg + 1)) != 0) ++lg;
    // instructions per edge.  FP32: per subset a two-sum, the powering, its correction and
    // the accumulations (~11 + 2 log2 n), per edge loads, scaling and stores (~40 + 20 s);
    // the series kernels: their multiply-adds plus ~3 s W (the size-2 kernel has no products
    // and little else).  FP64: the FP64 operations alone (the FP64 pipe is the bound).
    const double subsets = std::ldexp(1.0, s) - 1.0, half = std::ldexp(1.0, s - 1);
    const double series = s == 2 ? 5.0 * W : (2.0 * s - 5.0) * W * (W + 1) / 2.0 + 3.0 * s * W;
    const double closed32 = subsets * (11.0 + 2.0 * lg) + s * half + 40.0 + 20.0 * s;
    const double closed64 = subsets * (2.0 + 2.0 * lg) + s * half + 4.0;
    // equal x: sum of |terms| over the signed sum, sum_j C(s-1,j) (j+1)^n
    double pos = 0.0, sgn = 0.0, binom = 1.0;
    for (int j = 0; j < s; ++j) {
        const double t = binom * std::pow((double)(j + 1), (double)n);
        pos += t;
        sgn += ((s - 1 - j) & 1) ? -t : t;
        binom = binom * (double)(s - 1 - j) / (double)(j + 1);
    }
    const double kappa = sgn > 0.0 ? pos / sgn : 1e300;
    const double gate32 = ((double)n + half + 4.0) / 128.0;            // C 2^-24 / 2^-17
    const double gate64 = ((double)s * n + half + 4.0) / 2048.0;       // C 2^-53 / 2^-42
    // FP64 from size 6 on: the Bernoulli form's power sums cost fewer FP64 operations (its error
    // majorant runs on the FP32 units): per member 2W, the recurrence W(W-1)/2, per member its
    // sum, quotient and gate (~W/2 + 14), plus O(W)
    const double bern64 = s >= 6 ? s * (2.0 * W - 1.0) + 3.0 * (W - 1) + W * (W - 1) / 2.0 + W + s * (W / 2.0 + 14.0)
                                 : 1e300;
    int mask = 0;
    if (closed32 < 0.8 * series && gate32 * kappa <= 0.5) mask |= 1;
    if (closed64 < 0.8 * series && closed64 < bern64 && gate64 * kappa <= 0.5) mask |= 2;
    return mask;
}

// beta_k = B_k^+ / k!, the coefficients of z / (1 - e^(-z)), k < 32: the inverse of the
// series (1 - e^(-z)) / z = sum_k (-1)^k z^k / (k+1)!; beta_k = 0 for odd k >= 3.
void bernoulli_beta(double beta[32]) {
    double f[32];
    double fact = 1.0;
    for (int k = 0; k < 32; ++k) {
        fact *= (double)(k + 1);
        f[k] = ((k & 1) ? -1.0 : 1.0) / fact;
    }
    beta[0] = 1.0;
    for (int m = 1; m < 32; ++m) {
        double acc = 0.0;
        for (int k = 1; k <= m; ++k) acc -= f[k] * beta[m - k];
        beta[m] = (m >= 3 && (m & 1)) ? 0.0 : acc;
    }
}

namespace {
constexpr double kBernKmax32 = 4.0, kBernKmax64 = 64.0;
}

// Which call types evaluate bucket k in the Bernoulli form (bit 1 = FP32, 2 = FP64):
// 6 <= s <= 64, W <= thread_max_w, not in closed form for that type, fewer operations
// than the prefix/suffix series, and equal x with a gate ratio of at most kmax / 2 (so that
// x of somewhat different sizes still pass).  FP32 forms G as a product of the members'
// series, FP64 from their power sums (s3_bern.cuh); each has its own gate ratio and count.
int bernoulli_mask(const s3_graph_s *g, size_t k, const double beta[32]) {
    if (g->opt.bernoulli < 0) return 0;
    const int tmw = (g->opt.thread_max_w <= 0 || g->opt.thread_max_w > 32) ? 32 : g->opt.thread_max_w;
    const HostBucket &hb = g->buckets[k];
    const int s = hb.s, W = g->N - s + 1;
    if (s < 6 || s > 64 || hb.m <= 0 || W < 1 || W > tmw) return 0;
    // operations per edge: the series' products and dots; the product form's products and
    // per-member sums; the power-sum form's power sums, both recurrences and per-member sums
    const double series = (2.0 * s - 5.0) * W * (W + 1) / 2.0 + 2.0 * s * W;
    const double prod_form = (double)s * W * (W - 1) / 2.0 + 3.0 * s * W;
    const double sum_form = 2.0 * s * (W - 1) + (double)W * (W - 1) + 2.0 * s * W;
    // equal x (= 1).  Product form: G = ((e^z - 1)/z)^s on W coefficients; gate ratio
    // sum_k |G[W-1-k] beta_k| / sum_k G[W-1-k] beta_k.  Power-sum form: the recurrence
    // G_m = (1/m) sum_j beta_j p_j G_{m-j} with p_j = s, its majorant A (|beta_j|), and the
    // ratio sum_k A[W-1-k] |beta_k| / sum_k G[W-1-k] beta_k.
    std::vector<double> c(W), G(W, 0.0), Gn(W), R(W, 0.0), A(W, 0.0);
    double fact = 1.0;
    for (int i = 0; i < W; ++i) {
        fact *= (double)(i + 1);
        c[i] = 1.0 / fact;
    }
    G[0] = 1.0;
    for (int r = 0; r < s; ++r) {
        for (int m = 0; m < W; ++m) {
            double acc = 0.0;
            for (int i = 0; i <= m; ++i) acc += c[i] * G[m - i];
            Gn[m] = acc;
        }
        G.swap(Gn);
    }
    R[0] = A[0] = 1.0;
    for (int m = 1; m < W; ++m) {
        double acc = 0.0, acca = 0.0;
        for (int i = 1; i <= m; ++i) {
            acc += beta[i] * s * R[m - i];
            acca += std::fabs(beta[i]) * s * A[m - i];
        }
        R[m] = acc / m;
        A[m] = acca / m;
    }
    double sum = 0.0, abs_sum = 0.0, rsum = 0.0, maj = 0.0;
    for (int i = 0; i < W; ++i) {
        sum += G[W - 1 - i] * beta[i];
        abs_sum += std::fabs(G[W - 1 - i] * beta[i]);
        rsum += R[W - 1 - i] * beta[i];
        maj += A[W - 1 - i] * std::fabs(beta[i]);
    }
    const double kappa32 = sum > 0.0 ? abs_sum / sum : 1e300;
    const double kappa64 = rsum > 0.0 ? maj / rsum : 1e300;
    const int cm = closed_form_mask(g, k);
    int mask = 0;
    if (!(cm & 1) && prod_form < 0.9 * series && kappa32 <= kBernKmax32 / 2) mask |= 1;
    if (!(cm & 2) && sum_form < 0.9 * series && kappa64 <= kBernKmax64 / 2) mask |= 2;
    return mask;
}

// The device tables of the Bernoulli launch, one per call type (FP32, FP64).
s3_status plan_bernoulli(s3_graph_s *g) {
    for (int d = 0; d < 2; ++d) {
        std::vector<size_t> ks;
        for (size_t k = 0; k < g->buckets.size(); ++k)
            if (g->bern_mask[k] & (1 << d)) ks.push_back(k);
        if (ks.empty()) continue;
        std::stable_sort(ks.begin(), ks.end(), [&](size_t a, size_t b) { return g->bucket_cost[a] > g->bucket_cost[b]; });
        std::vector<TailEntry> tab;
        int64_t blocks = 0;
        int lane = 0, fb = 0;
        for (size_t k : ks) {
            const HostBucket &hb = g->buckets[k];
            TailEntry t{};
            t.b.ids = g->d_ids + hb.offset;
            t.b.slot = g->d_slot + hb.offset;
            t.b.m = hb.m;
            t.b.ld = hb.ld;
            t.b.s = hb.s;
            t.b.N = g->N;
            t.b.target = g->target[k];
            t.b.K = g->K[k];
            t.b.Km = g->Km[k];
            t.b.Ke = g->Ke[k];
            t.W = g->N - hb.s + 1;
            t.block0 = blocks;
            blocks += (hb.m + kBernThreads - 1) / kBernThreads;
            // per lane: the x values, plus (FP64) the member ids staged during the gather
            lane = std::max(lane, d ? hb.s + (hb.s + 1) / 2 : hb.s);
            fb = std::max(fb, (int)warp_smem_elems(hb.s, t.W));
            g->bern_cost[d] += (double)hb.m * ((d ? 2.0 * hb.s * (t.W - 1) + (double)t.W * (t.W - 1)
                                                  : (double)hb.s * t.W * (t.W - 1) / 2.0) + 60.0 * hb.s);
            tab.push_back(t);
        }
        if (bern_smem_bytes(lane, fb, d ? 8 : 4) > kEdgeSmemCap) {
            // too large for one launch's shared memory: these buckets keep their series kernels
            for (size_t k : ks) g->bern_mask[k] &= ~(1 << d);
            g->bern_cost[d] = 0.0;
            continue;
        }
        s3_status st = upload(g, &g->d_bern[d], tab);
        if (st != S3_OK) return st;
        g->n_bern[d] = (int32_t)tab.size();
        g->bern_blocks[d] = blocks;
        g->bern_lane[d] = lane;
        g->bern_fb[d] = fb;
    }
    double beta[32];
    bernoulli_beta(beta);
    for (int k = 0; k < 32; ++k) {
        g->bern_args.beta64[k] = beta[k];
        g->bern_args.beta32[k] = (float)beta[k];
    }
    g->bern_args.kmax32 = (float)kBernKmax32;
    g->bern_args.kmax64 = kBernKmax64;
    if (g->n_bern[0] + g->n_bern[1] > 0) {
        s3_status st = dev_alloc(g, &g->d_bern_rejected, 1);
        if (st != S3_OK) return st;
        if (cudaMemset(g->d_bern_rejected, 0, sizeof(unsigned long long)) != cudaSuccess)
            return cuda_fail(cudaGetLastError(), "memset");
        g->bern_args.rejected = g->d_bern_rejected;
    }
    return S3_OK;
}

// Closed-form plan of the handle: buckets with a launch of their own (not in the fused
// small-bucket launch) that closed_form_mask admits, their constants and rejected-edge lists.
s3_status plan_closed_form(s3_graph_s *g) {
    const size_t nb = g->buckets.size();
    g->closed_mask.assign(nb, 0);
    g->closed_args.assign(nb, ClosedArgs{});
    const int n = g->N - 1;
    int64_t list_len = 0;
    std::vector<int64_t> list_off(nb, 0);
    for (size_t k = 0; k < nb; ++k) {
        const HostBucket &hb = g->buckets[k];
        if (g->in_tail[k]) continue;
        const int mask = closed_form_mask(g, k);
        if (!mask) continue;
        g->closed_mask[k] = mask;
        ClosedArgs &c = g->closed_args[k];
        double fact = 1.0;  // (N-1)!
        for (int i = 2; i <= n; ++i) fact *= (double)i;
        c.Ki = g->K[k] / fact;
        int e = 0;
        c.Kim = (float)std::frexp(c.Ki, &e);
        c.Kie = e;
        list_off[k] = list_len;
        list_len += hb.m;
    }
    if (list_len == 0) return S3_OK;
    s3_status st;
    if ((st = dev_alloc(g, &g->d_closed_list, (size_t)list_len)) != S3_OK) return st;
    if ((st = dev_alloc(g, &g->d_closed_count, 4 * nb)) != S3_OK) return st;
    if (cudaMemset(g->d_closed_count, 0, sizeof(int32_t) * 4 * nb) != cudaSuccess)
        return cuda_fail(cudaGetLastError(), "memset");
    for (size_t k = 0; k < nb; ++k) {
        if (!g->closed_mask[k]) continue;
        g->closed_args[k].fail_list = g->d_closed_list + list_off[k];
        g->closed_args[k].fail_count = g->d_closed_count + 4 * k;
        // the scheduler's cost of a closed-form bucket (FP32 estimate)
        const double s = g->buckets[k].s;
        g->bucket_cost[k] = (double)g->buckets[k].m * ((std::ldexp(1.0, (int)s) - 1.0) * 20.0 + 60.0 * s);
    }
    std::stable_sort(g->bucket_order.begin(), g->bucket_order.end(),
                     [&](size_t a, size_t b) { return g->bucket_cost[a] > g->bucket_cost[b]; });
    return S3_OK;
}

// Launch the per-bucket edge kernels and the reduce for one call.
s3_status run_edges(s3_graph_s *g, s3_dtype dt, const void *x, void *y, int bias, const int32_t *skip,
                    cudaStream_t st, cudaEvent_t mid, cudaEvent_t *bern_ev) {
    int launches = 0;
    const bool seg = g->opt.reduce == S3_REDUCE_SEGMENTED;
    const size_t esz = dt == S3_F32 ? 4 : 8;
    EdgeOutArgs o{};
    o.bias = bias;
    o.range_events = g->d_range;
    o.skip = skip;
    if (seg) {
        o.out = g->d_buf;
        o.mode = kOutBuffer;
    } else {
        o.out = y;
        o.mode = dt == S3_F32 ? kOutAtomicComp : kOutAtomic;
        o.comp = g->d_comp;
        S3_CUDA(cudaMemsetAsync(y, 0, esz * (size_t)g->n, st));
        if (dt == S3_F32) S3_CUDA(cudaMemsetAsync(g->d_comp, 0, sizeof(float) * (size_t)g->n, st));
    }
    // the closed-form kernels append to lists that start empty: clear their lengths
    // (one strided memset: the first counter of every bucket, running totals untouched)
    if (g->d_closed_count && (dt == S3_F32 || dt == S3_F64))
        S3_CUDA(cudaMemset2DAsync(g->d_closed_count, 4 * sizeof(int32_t), 0, sizeof(int32_t), g->buckets.size(), st));
    // fork: buckets run concurrently on the handle's streams (heaviest first, greedy balance)
    const int ns = g->n_streams;
    if (ns > 1) {
        S3_CUDA(cudaEventRecord(g->ev_fork, st));
        for (int i = 0; i < ns; ++i) S3_CUDA(cudaStreamWaitEvent(g->aux[i], g->ev_fork, 0));
    }
    double load[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    auto pick = [&](double cost) {
        if (ns <= 1) return st;
        int best = 0;
        for (int i = 1; i < ns; ++i)
            if (load[i] < load[best]) best = i;
        load[best] += cost;
        return g->aux[best];
    };
    // Bernoulli-form buckets: one launch for all of them (FP32, FP64)
    const int bd = dt == S3_F32 ? 0 : dt == S3_F64 ? 1 : -1;
    const bool bern = bd >= 0 && g->n_bern[bd] > 0;
    bool bern_done = !bern;
    auto launch_bern = [&]() -> s3_status {
        bern_done = true;
        cudaStream_t bs = pick(g->bern_cost[bd]);
        if (bern_ev) S3_CUDA(cudaEventRecord(bern_ev[0], bs));
        cudaError_t e = dt == S3_F32 ? launch_edge_bern_f32(g->d_bern[0], g->n_bern[0], g->bern_blocks[0],
                                                            g->bern_lane[0], g->bern_fb[0], (const float *)x, o,
                                                            g->bern_args, bs)
                                     : launch_edge_bern_f64(g->d_bern[1], g->n_bern[1], g->bern_blocks[1],
                                                            g->bern_lane[1], g->bern_fb[1], (const double *)x, o,
                                                            g->bern_args, bs);
        if (e != cudaSuccess) return cuda_fail(e, "Bernoulli launch");
        if (bern_ev) S3_CUDA(cudaEventRecord(bern_ev[1], bs));
        ++launches;
        return S3_OK;
    };
    // small buckets share one launch (FP32, FP64); the double-float kernels launch per bucket
    const bool fuse = dt != S3_DF64;
    bool tail_done = !fuse || g->n_tail == 0;
    auto launch_tail = [&]() -> s3_status {
        tail_done = true;
        cudaStream_t ts = pick(g->tail_cost);
        cudaError_t e = dt == S3_F32 ? launch_edge_tail_f32(g->d_tail, g->n_tail, g->tail_blocks, g->tail_bs,
                                                            g->tail_smem[0], (const float *)x, o, ts)
                                     : launch_edge_tail_f64(g->d_tail, g->n_tail, g->tail_blocks, g->tail_bs,
                                                            g->tail_smem[1], (const double *)x, o, ts);
        if (e != cudaSuccess) return cuda_fail(e, "small-bucket launch");
        ++launches;
        return S3_OK;
    };
    for (size_t r = 0; r < g->bucket_order.size(); ++r) {
        const size_t k = g->bucket_order[r];
        const HostBucket &hb = g->buckets[k];
        if (hb.m <= 0 || (fuse && g->in_tail[k]) || (bern && (g->bern_mask[k] >> bd & 1))) continue;
        if (!bern_done && g->bern_cost[bd] >= g->bucket_cost[k]) {
            s3_status bs = launch_bern();
            if (bs != S3_OK) return bs;
        }
        if (!tail_done && g->tail_cost >= g->bucket_cost[k]) {
            s3_status ts = launch_tail();
            if (ts != S3_OK) return ts;
        }
        EdgeBucketArgs b{};
        b.ids = g->d_ids + hb.offset;
        b.slot = g->d_slot + hb.offset;
        b.m = hb.m;
        b.ld = hb.ld;
        b.s = hb.s;
        b.N = g->N;
        b.target = g->target[k];
        b.K = g->K[k];
        b.Km = g->Km[k];
        b.Ke = g->Ke[k];
        cudaStream_t bs = pick(g->bucket_cost[k]);
        const int tmw = g->opt.thread_max_w, bth = g->opt.block_threads;
        const int closed_bit = dt == S3_F32 ? 1 : dt == S3_F64 ? 2 : 0;
        if (g->closed_mask[k] & closed_bit) {
            // closed form first; the series kernel then takes only the edges it rejected
            ClosedArgs c = g->closed_args[k];
            const HostBucket &cb = g->buckets[k];
            const double half = std::ldexp(1.0, cb.s - 1);
            c.gate = dt == S3_F32 ? ((double)(g->N - 1) + half + 4.0) / 128.0
                                  : ((double)cb.s * (g->N - 1) + half + 4.0) / 2048.0;
            cudaError_t ce = dt == S3_F32 ? launch_edge_closed_f32(b, (const float *)x, o, c, bs)
                                          : launch_edge_closed_f64(b, (const double *)x, o, c, bs);
            if (ce != cudaSuccess) return cuda_fail(ce, "closed-form launch");
            ++launches;
            b.list = c.fail_list;
            b.count = c.fail_count;
        }
        cudaError_t e = dt == S3_F32   ? launch_edge_bucket_f32(b, (const float *)x, o, tmw, bth, bs)
                        : dt == S3_F64 ? launch_edge_bucket_f64(b, (const double *)x, o, tmw, bth, bs)
                                       : launch_edge_bucket_df(b, (const double *)x, o, tmw, bth, bs);
        if (e != cudaSuccess) return cuda_fail(e, "edge kernel launch");
        ++launches;
    }
    if (!bern_done) {
        s3_status bs = launch_bern();
        if (bs != S3_OK) return bs;
    }
    if (!tail_done) {
        s3_status ts = launch_tail();
        if (ts != S3_OK) return ts;
    }
    if (ns > 1) {
        for (int i = 0; i < ns; ++i) {
            S3_CUDA(cudaEventRecord(g->ev_join[i], g->aux[i]));
            S3_CUDA(cudaStreamWaitEvent(st, g->ev_join[i], 0));
        }
    }
    if (mid) S3_CUDA(cudaEventRecord(mid, st));
    if (seg) {
        const ReduceArgs r = reduce_args(g, skip);
        cudaError_t e = dt == S3_F32 ? launch_reduce_f32(r, (const float *)g->d_buf, (float *)y, st)
                                     : launch_reduce_f64(r, (const double *)g->d_buf, (double *)y, st);
        if (e != cudaSuccess) return cuda_fail(e, "reduce launch");
        ++launches;
    } else if (dt == S3_F32) {
        cudaError_t e = launch_add_comp((float *)y, g->d_comp, g->n, skip, st);
        if (e != cudaSuccess) return cuda_fail(e, "compensation launch");
        ++launches;
    }
    g->last_launches = launches;
    return S3_OK;
}

}  // namespace s3

using namespace s3;

extern "C" {

s3_status s3_options_init(s3_options *opt) {
    if (!opt) return fail(S3_EINVAL, "opt is NULL");
    std::memset(opt, 0, sizeof(*opt));
    opt->rank = 0;
    opt->reduce = S3_REDUCE_SEGMENTED;
    opt->layout = S3_LAYOUT_EDGE;
    opt->build_ccss = 0;
    opt->device = -1;
    opt->thread_max_w = 0;
    opt->block_threads = 0;
    opt->order = S3_ORDER_DEGREE;
    opt->streams = 0;
    return S3_OK;
}

s3_status s3_format_inspect(int64_t n, int64_t m, const int64_t *edge_ptr, const int32_t *members,
                            const s3_options *opt, s3_format_info *info) {
    if (!info) return fail(S3_EINVAL, "info is NULL");
    s3_options o;
    if (opt) o = *opt;
    else s3_options_init(&o);
    try {
        HostFormat f;
        s3_status st = build_host_format(n, m, edge_ptr, members, o, f);
        if (st != S3_OK) return st;
        fill_info(f, info);
        return S3_OK;
    } catch (const std::bad_alloc &) {
        return fail(S3_ENOMEM, "host allocation failed");
    }
}

s3_status s3_build_format(int64_t n, int64_t m, const int64_t *edge_ptr, const int32_t *members,
                          const s3_options *opt, s3_graph_t *out) {
    if (!out) return fail(S3_EINVAL, "out is NULL");
    *out = nullptr;
    s3_options o;
    if (opt) o = *opt;
    else s3_options_init(&o);
    if (o.reduce != S3_REDUCE_SEGMENTED && o.reduce != S3_REDUCE_ATOMIC) return fail(S3_EINVAL, "bad reduce mode");
    if (o.layout != S3_LAYOUT_EDGE && o.layout != S3_LAYOUT_CCSS) return fail(S3_EINVAL, "bad layout");
    if (o.thread_max_w < 0 || o.thread_max_w > 32) return fail(S3_EINVAL, "thread_max_w must be in 0..32");
    if (o.block_threads < 0 || o.block_threads > 256 || o.block_threads % 32) return fail(S3_EINVAL, "block_threads must be a multiple of 32 up to 256");
    if (o.streams < 0 || o.streams > 8) return fail(S3_EINVAL, "streams must be in 0..8");
    if (o.closed_form_max_s < -1 || o.closed_form_max_s > kClosedMaxS)
        return fail(S3_EINVAL, "closed_form_max_s must be in -1..6");
    if (o.order != S3_ORDER_DEGREE && o.order != S3_ORDER_INDEX) return fail(S3_EINVAL, "bad order");
    if (o.range_check != 0 && o.range_check != 1) return fail(S3_EINVAL, "range_check must be 0 or 1");
    HostFormat f;
    try {
        s3_status st = build_host_format(n, m, edge_ptr, members, o, f);
        if (st != S3_OK) return st;
    } catch (const std::bad_alloc &) {
        return fail(S3_ENOMEM, "host allocation failed");
    }
    int dev = o.device;
    if (dev < 0) S3_CUDA(cudaGetDevice(&dev));
    DeviceGuard guard(dev);
    s3_status st = prepare_device(dev);
    if (st != S3_OK) return st;

    s3_graph_s *g = new (std::nothrow) s3_graph_s();
    if (!g) return fail(S3_ENOMEM, "host allocation failed");
    g->device = dev;
    g->opt = o;
    g->n = f.n;
    g->m = f.m;
    g->nnz = f.nnz;
    g->N = f.N;
    fill_info(f, &g->info);
    g->buckets = f.buckets;
    for (const HostBucket &b : f.buckets) {
        double K = scale_K(b.s, f.N);
        g->K.push_back(K);
        int e = 0;
        double mant = std::frexp(K, &e);
        g->Km.push_back((float)mant);
        g->Ke.push_back(e);
        g->target.push_back(scale_target(b.s, f.N));
    }
    auto bail = [&](s3_status s) {
        free_all(g);
        delete g;
        return s;
    };
    if ((st = upload(g, &g->d_ids, f.ids)) != S3_OK) return bail(st);
    if ((st = upload(g, &g->d_slot, f.slot)) != S3_OK) return bail(st);
    if ((st = upload(g, &g->d_inc_ptr, f.inc_ptr)) != S3_OK) return bail(st);
    if ((st = upload(g, &g->d_grp_off, f.grp_off)) != S3_OK) return bail(st);
    if ((st = upload(g, &g->d_grp_node, f.grp_node)) != S3_OK) return bail(st);
    if ((st = upload(g, &g->d_grp_deg, f.grp_deg)) != S3_OK) return bail(st);
    if ((st = upload(g, &g->d_med8, f.med8_node)) != S3_OK) return bail(st);
    if ((st = upload(g, &g->d_med8_off, f.med8_off)) != S3_OK) return bail(st);
    if ((st = upload(g, &g->d_med8_len, f.med8_len)) != S3_OK) return bail(st);
    if ((st = upload(g, &g->d_med, f.med_node)) != S3_OK) return bail(st);
    if ((st = upload(g, &g->d_med_off, f.med_off)) != S3_OK) return bail(st);
    if ((st = upload(g, &g->d_med_len, f.med_len)) != S3_OK) return bail(st);
    if ((st = upload(g, &g->d_big_nodes, f.big_node)) != S3_OK) return bail(st);
    if ((st = upload(g, &g->d_big_piece_ptr, f.big_piece_ptr)) != S3_OK) return bail(st);
    if ((st = upload(g, &g->d_piece_big, f.piece_big)) != S3_OK) return bail(st);
    if ((st = dev_alloc(g, &g->d_big_count, f.big_node.size())) != S3_OK) return bail(st);
    if (!f.big_node.empty() && cudaMemset(g->d_big_count, 0, sizeof(int32_t) * f.big_node.size()) != cudaSuccess)
        return bail(cuda_fail(cudaGetLastError(), "memset"));
    if ((st = upload(g, &g->d_piece_start, f.piece_start)) != S3_OK) return bail(st);
    if ((st = upload(g, &g->d_piece_len, f.piece_len)) != S3_OK) return bail(st);
    for (int64_t v = 0; v < f.n; ++v)
        if (f.inc_ptr[v + 1] == f.inc_ptr[v]) {
            g->first_isolated = v;
            break;
        }
    g->n_grp = (int64_t)f.grp_off.size();
    g->n_med8 = (int64_t)f.med8_node.size();
    g->n_med = (int64_t)f.med_node.size();
    g->n_big = (int64_t)f.big_node.size();
    g->n_pieces = (int64_t)f.piece_start.size();
    double *dd = nullptr;
    g->buf_len = f.buf_len;
    if ((st = dev_alloc(g, &dd, (size_t)f.buf_len)) != S3_OK) return bail(st);
    g->d_buf = dd;
    if ((st = dev_alloc(g, &dd, (size_t)g->n_pieces)) != S3_OK) return bail(st);
    g->d_partial = dd;
    if ((st = dev_alloc(g, &g->d_comp, (size_t)f.n)) != S3_OK) return bail(st);
    if ((st = dev_alloc(g, &g->d_range, 1)) != S3_OK) return bail(st);
    if (cudaMemset(g->d_range, 0, sizeof(unsigned long long)) != cudaSuccess) return bail(cuda_fail(cudaGetLastError(), "memset"));
    if ((st = dev_alloc(g, &dd, (size_t)f.n)) != S3_OK) return bail(st);
    g->d_xh = dd;
    if ((st = dev_alloc(g, &dd, (size_t)f.n)) != S3_OK) return bail(st);
    g->d_yh = dd;
    if (f.has_ccss) {
        if ((st = upload_ccss(g, f)) != S3_OK) return bail(st);
    }
    // completion event of the last call, query stream, pinned words of the range check
    if (cudaEventCreateWithFlags(&g->ev_done, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&g->qstream, cudaStreamNonBlocking) != cudaSuccess)
        return bail(cuda_fail(cudaGetLastError(), "cudaEventCreate"));
    if (cudaHostAlloc((void **)&g->h_range, 2 * sizeof(unsigned long long), cudaHostAllocDefault) != cudaSuccess) {
        g->h_range = nullptr;
        return bail(cuda_fail(cudaGetLastError(), "cudaHostAlloc"));
    }
    // concurrent size buckets: streams, events, and a cost estimate per bucket
    g->n_streams = o.streams > 0 ? std::min(o.streams, 8) : 4;
    if (g->n_streams > 1) {
        if (cudaEventCreateWithFlags(&g->ev_fork, cudaEventDisableTiming) != cudaSuccess)
            return bail(cuda_fail(cudaGetLastError(), "cudaEventCreate"));
        for (int i = 0; i < g->n_streams; ++i) {
            if (cudaStreamCreateWithFlags(&g->aux[i], cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&g->ev_join[i], cudaEventDisableTiming) != cudaSuccess)
                return bail(cuda_fail(cudaGetLastError(), "cudaStreamCreate"));
        }
    }
    for (size_t k = 0; k < g->buckets.size(); ++k) {
        const HostBucket &b = g->buckets[k];
        double W = (double)(g->N - b.s + 1);
        double fma = b.s >= 3 ? (2.0 * b.s - 5.0) * W * (W + 1) / 2 + b.s * W : 2 * W;
        g->bucket_cost.push_back((double)b.m * (fma + 60.0 * b.s));
        g->bucket_order.push_back(k);
    }
    std::stable_sort(g->bucket_order.begin(), g->bucket_order.end(),
                     [&](size_t a, size_t b) { return g->bucket_cost[a] > g->bucket_cost[b]; });
    // Bernoulli-form buckets (decided before the fused small-bucket launch, which they leave)
    {
        double beta[32];
        bernoulli_beta(beta);
        g->bern_mask.assign(g->buckets.size(), 0);
        for (size_t k = 0; k < g->buckets.size(); ++k) g->bern_mask[k] = bernoulli_mask(g, k, beta);
    }
    // small thread-per-edge buckets: one fused launch.  A bucket of a few thousand
    // edges costs about as much as one edge's latency chain; fused, that latency is
    // paid once per call instead of once per bucket.
    {
        const int64_t lim = o.small_bucket_edges == 0 ? 40000 : o.small_bucket_edges;
        const int wmax = (o.thread_max_w <= 0 || o.thread_max_w > 32) ? 32 : o.thread_max_w;
        g->in_tail.assign(g->buckets.size(), 0);
        std::vector<TailEntry> tab;
        for (size_t k = 0; k < g->buckets.size(); ++k) {
            const HostBucket &hb = g->buckets[k];
            const int W = g->N - hb.s + 1;
            if (hb.s < 2 || hb.m <= 0 || hb.m > lim || W > wmax || g->bern_mask[k]) continue;
            if (edge_tail_smem_words(hb.s, W, 8) * 4 * (size_t)g->tail_bs > kEdgeSmemCap) continue;
            TailEntry t{};
            t.b.ids = g->d_ids + hb.offset;
            t.b.slot = g->d_slot + hb.offset;
            t.b.m = hb.m;
            t.b.ld = hb.ld;
            t.b.s = hb.s;
            t.b.N = g->N;
            t.b.target = g->target[k];
            t.b.K = g->K[k];
            t.b.Km = g->Km[k];
            t.b.Ke = g->Ke[k];
            t.W = W;
            t.block0 = g->tail_blocks;
            g->tail_blocks += (hb.m + g->tail_bs - 1) / g->tail_bs;
            for (int d = 0; d < 2; ++d)
                g->tail_smem[d] = std::max(g->tail_smem[d], edge_tail_smem_words(hb.s, W, d ? 8 : 4) * 4 * (size_t)g->tail_bs);
            g->tail_cost += g->bucket_cost[k];
            g->in_tail[k] = 1;
            tab.push_back(t);
        }
        if (tab.size() == 1) {  // a lone small bucket keeps its own kernel
            g->in_tail.assign(g->buckets.size(), 0);
            tab.clear();
            g->tail_blocks = 0;
            g->tail_cost = 0.0;
        }
        if (!tab.empty()) {
            if ((st = upload(g, &g->d_tail, tab)) != S3_OK) return bail(st);
            g->n_tail = (int32_t)tab.size();
        }
    }
    if ((st = plan_closed_form(g)) != S3_OK) return bail(st);
    if ((st = plan_bernoulli(g)) != S3_OK) return bail(st);
    g->info.device_bytes = g->device_bytes;
    *out = g;
    return S3_OK;
}

s3_status s3_graph_query(s3_graph_t g, s3_format_info *info) {
    if (!g || !info) return fail(S3_EINVAL, "NULL argument");
    *info = g->info;
    info->device_bytes = g->device_bytes;
    return S3_OK;
}

}  // extern "C"

namespace s3 {
namespace {

// One S^3TTVc call on an already validated handle and arguments.
s3_status sttsvc_dispatch(s3_graph_s *g, s3_dtype dt, int32_t layout, const void *x, void *y, cudaStream_t st) {
    if (layout == S3_LAYOUT_EDGE) return run_edges(g, dt, x, y, 0, nullptr, st);
    if (layout == S3_LAYOUT_CCSS) {
        if (!g->has_ccss) return fail(S3_EINVAL, "handle was built without the CCSS forest");
        return run_ccss(g, dt == S3_DF64 ? S3_F64 : dt, x, y, 0, nullptr, st);
    }
    return fail(S3_EINVAL, "bad layout");
}

// The call between two stream-ordered reads of the range counter; synchronises st and
// returns S3_ERANGE when the counter moved (y is written either way).
s3_status sttsvc_checked(s3_graph_s *g, s3_dtype dt, int32_t layout, const void *x, void *y, cudaStream_t st,
                         void *y_host, size_t y_bytes, cudaGraphExec_t exec = nullptr) {
    S3_CUDA(cudaMemcpyAsync(&g->h_range[0], g->d_range, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    if (exec) {
        S3_CUDA(cudaGraphLaunch(exec, st));
    } else {
        s3_status s = sttsvc_dispatch(g, dt, layout, x, y, st);
        if (s != S3_OK) return s;
    }
    s3_status s;
    if (y_host) S3_CUDA(cudaMemcpyAsync(y_host, y, y_bytes, cudaMemcpyDeviceToHost, st));
    S3_CUDA(cudaMemcpyAsync(&g->h_range[1], g->d_range, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    s = mark_done(g, st);
    if (s != S3_OK) return s;
    S3_CUDA(cudaStreamSynchronize(st));
    const unsigned long long d = g->h_range[1] - g->h_range[0];
    if (d != 0)
        return fail(S3_ERANGE, std::to_string(d) + " per-(edge, node) results of this call left the normal range of " +
                                   (dt == S3_F32 ? "FP32" : "FP64"));
    return S3_OK;
}

}  // namespace
}  // namespace s3

extern "C" {

s3_status s3_sttsvc_layout(s3_graph_t g, s3_dtype dt, int32_t layout, const void *x, void *y, void *stream) {
    if (!g) return fail(S3_EINVAL, "graph is NULL");
    if (dt != S3_F32 && dt != S3_F64 && dt != S3_DF64) return fail(S3_EINVAL, "bad dtype");
    if (!x || !y) return fail(S3_EINVAL, "x or y is NULL");
    const size_t esz = dt == S3_F32 ? 4 : 8;
    const char *xb = (const char *)x, *yb = (const char *)y;
    if (xb < yb + esz * g->n && yb < xb + esz * g->n) return fail(S3_EINVAL, "x and y overlap");
    DeviceGuard guard(g->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (g->opt.range_check) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        S3_CUDA(cudaStreamIsCapturing(st, &cs));
        if (cs != cudaStreamCaptureStatusNone)
            return fail(S3_ENOTSUP, "range_check synchronises the stream: not allowed during stream capture");
        return sttsvc_checked(g, dt, layout, x, y, st, nullptr, 0);
    }
    s3_status s = sttsvc_dispatch(g, dt, layout, x, y, st);
    if (s != S3_OK) return s;
    return mark_done(g, st);
}

s3_status s3_sttsvc(s3_graph_t g, s3_dtype dt, const void *x, void *y, void *stream) {
    if (!g) return fail(S3_EINVAL, "graph is NULL");
    return s3_sttsvc_layout(g, dt, g->opt.layout, x, y, stream);
}

s3_status s3_sttsvc_host(s3_graph_t g, s3_dtype dt, const void *x_host, void *y_host, void *stream) {
    if (!g) return fail(S3_EINVAL, "graph is NULL");
    if (!x_host || !y_host) return fail(S3_EINVAL, "x or y is NULL");
    if (dt != S3_F32 && dt != S3_F64 && dt != S3_DF64) return fail(S3_EINVAL, "bad dtype");
    DeviceGuard guard(g->device);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = (dt == S3_F32 ? 4 : 8) * (size_t)g->n;
    S3_CUDA(cudaMemcpyAsync(g->d_xh, x_host, bytes, cudaMemcpyHostToDevice, st));
    // the call on the staging buffers is the same every time: launch it as one captured graph
    // (captured on the handle's own stream at the first call of each type), which keeps the
    // dozen launches of a call off the host's critical path between the two copies
    cudaGraphExec_t &ex = g->host_exec[dt];
    if (!ex) {
        if (!g->cap_stream) S3_CUDA(cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking));
        cudaGraph_t graph = nullptr;
        S3_CUDA(cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeThreadLocal));
        s3_status s = sttsvc_dispatch(g, dt, g->opt.layout, g->d_xh, g->d_yh, g->cap_stream);
        cudaError_t ce = cudaStreamEndCapture(g->cap_stream, &graph);
        if (s != S3_OK) {
            if (graph) cudaGraphDestroy(graph);
            return s;
        }
        S3_CUDA(ce);
        ce = cudaGraphInstantiate(&ex, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) {
            ex = nullptr;
            return cuda_fail(ce, "graph instantiation");
        }
    }
    return sttsvc_checked(g, dt, g->opt.layout, g->d_xh, g->d_yh, st, y_host, bytes, ex);
}

s3_status s3_sttsvc_profile(s3_graph_t g, s3_dtype dt, const void *x, void *y, s3_profile *prof, void *stream) {
    if (!g || !prof) return fail(S3_EINVAL, "NULL argument");
    if (dt != S3_F32 && dt != S3_F64 && dt != S3_DF64) return fail(S3_EINVAL, "bad dtype");
    if (!x || !y) return fail(S3_EINVAL, "x or y is NULL");
    if (g->opt.layout != S3_LAYOUT_EDGE) return fail(S3_ENOTSUP, "profiling covers the edge layout");
    DeviceGuard guard(g->device);
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t ev[5];
    for (auto &e : ev) S3_CUDA(cudaEventCreate(&e));
    struct Cleanup {
        cudaEvent_t *e;
        ~Cleanup() {
            for (int i = 0; i < 5; ++i) cudaEventDestroy(e[i]);
        }
    } cleanup{ev};
    S3_CUDA(cudaEventRecord(ev[0], st));
    // the Bernoulli launch's events are recorded only when it runs (both stay unrecorded otherwise)
    const int bd = dt == S3_F32 ? 0 : dt == S3_F64 ? 1 : -1;
    const bool has_bern = bd >= 0 && g->n_bern[bd] > 0;
    s3_status s = run_edges(g, dt, x, y, 0, nullptr, st, ev[1], has_bern ? ev + 3 : nullptr);
    if (s != S3_OK) return s;
    S3_CUDA(cudaEventRecord(ev[2], st));
    s = mark_done(g, st);
    if (s != S3_OK) return s;
    S3_CUDA(cudaEventSynchronize(ev[2]));
    std::memset(prof, 0, sizeof(*prof));
    S3_CUDA(cudaEventElapsedTime(&prof->edge_ms, ev[0], ev[1]));
    S3_CUDA(cudaEventElapsedTime(&prof->reduce_ms, ev[1], ev[2]));
    S3_CUDA(cudaEventElapsedTime(&prof->total_ms, ev[0], ev[2]));
    if (has_bern) S3_CUDA(cudaEventElapsedTime(&prof->bern_ms, ev[3], ev[4]));
    prof->launches = g->last_launches;
    return S3_OK;
}

s3_status s3_range_events(s3_graph_t g, int64_t *count, int32_t reset) {
    if (!g || !count) return fail(S3_EINVAL, "NULL argument");
    DeviceGuard guard(g->device);
    s3_status s = wait_done(g);
    if (s != S3_OK) return s;
    S3_CUDA(cudaMemcpyAsync(&g->h_range[0], g->d_range, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                            g->qstream));
    if (reset) S3_CUDA(cudaMemsetAsync(g->d_range, 0, sizeof(unsigned long long), g->qstream));
    S3_CUDA(cudaStreamSynchronize(g->qstream));
    *count = (int64_t)g->h_range[0];
    return S3_OK;
}

s3_status s3_closed_form_query(s3_graph_t g, uint64_t *sizes_f32, uint64_t *sizes_f64, int64_t *rejected) {
    if (!g) return fail(S3_EINVAL, "graph is NULL");
    uint64_t m32 = 0, m64 = 0;
    for (size_t k = 0; k < g->closed_mask.size(); ++k) {
        if (!g->closed_mask[k]) continue;
        const uint64_t bit = 1ull << g->buckets[k].s;  // s <= kClosedMaxS for these buckets
        if (g->closed_mask[k] & 1) m32 |= bit;
        if (g->closed_mask[k] & 2) m64 |= bit;
    }
    if (sizes_f32) *sizes_f32 = m32;
    if (sizes_f64) *sizes_f64 = m64;
    if (rejected) {
        *rejected = 0;
        if (g->d_closed_count) {
            DeviceGuard guard(g->device);
            s3_status s = wait_done(g);
            if (s != S3_OK) return s;
            std::vector<int32_t> cnt(4 * g->buckets.size());
            S3_CUDA(cudaMemcpyAsync(cnt.data(), g->d_closed_count, sizeof(int32_t) * cnt.size(), cudaMemcpyDeviceToHost,
                                    g->qstream));
            S3_CUDA(cudaStreamSynchronize(g->qstream));
            for (size_t k = 0; k < g->buckets.size(); ++k) {
                unsigned long long t = 0;
                std::memcpy(&t, &cnt[4 * k + 2], sizeof(t));
                *rejected += (int64_t)t;
            }
        }
    }
    return S3_OK;
}

s3_status s3_bernoulli_query(s3_graph_t g, uint64_t *sizes_f32, uint64_t *sizes_f64, int64_t *rejected) {
    if (!g) return fail(S3_EINVAL, "graph is NULL");
    uint64_t m32 = 0, m64 = 0;
    for (size_t k = 0; k < g->bern_mask.size(); ++k) {
        const int s = g->buckets[k].s;  // <= 64 for these buckets
        if (g->bern_mask[k] & 1) m32 |= 1ull << (s - 1);
        if (g->bern_mask[k] & 2) m64 |= 1ull << (s - 1);
    }
    if (sizes_f32) *sizes_f32 = m32;
    if (sizes_f64) *sizes_f64 = m64;
    if (rejected) {
        *rejected = 0;
        if (g->d_bern_rejected) {
            DeviceGuard guard(g->device);
            s3_status s = wait_done(g);
            if (s != S3_OK) return s;
            unsigned long long c = 0;
            S3_CUDA(cudaMemcpyAsync(&c, g->d_bern_rejected, sizeof(c), cudaMemcpyDeviceToHost, g->qstream));
            S3_CUDA(cudaStreamSynchronize(g->qstream));
            *rejected = (int64_t)c;
        }
    }
    return S3_OK;
}

s3_status s3_destroy(s3_graph_t g) {
    if (!g) return S3_OK;
    {
        DeviceGuard guard(g->device);
        cudaDeviceSynchronize();
        free_all(g);
    }
    delete g;
    return S3_OK;
}

const char *s3_last_error(void) { return g_last_error.c_str(); }

const char *s3_status_string(s3_status st) {
    switch (st) {
        case S3_OK: return "S3_OK";
        case S3_EINVAL: return "S3_EINVAL";
        case S3_ENOMEM: return "S3_ENOMEM";
        case S3_ECUDA: return "S3_ECUDA";
        case S3_ENOCONV: return "S3_ENOCONV";
        case S3_ETIMEOUT: return "S3_ETIMEOUT";
        case S3_ERANGE: return "S3_ERANGE";
        case S3_ENOTSUP: return "S3_ENOTSUP";
    }
    return "S3_UNKNOWN";
}

int32_t s3_version(void) { return S3_VERSION; }

}  // extern "C"
