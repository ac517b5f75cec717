// Learned warm start for the NQZ iteration: per-node features, a 12-64-64-1
// MLP (BF16 weights, FP32 accumulation) and its training kernels.
//
// Features of node v (all log1p-scaled): degree; mean and max size of the
// edges containing v; an 8-bin histogram of those sizes (bins log-spaced on
// [2, N]); the sum over v's edges of the other members' degrees.  They are
// gathered edge by edge with integer atomics (exact, so the result does not
// depend on scheduling).  The network predicts log x*_v minus its mean over the
// graph; the warm start is exp(prediction), normalised to 1-norm 1.
//
// Training keeps FP32 master weights and their BF16 copies; the forward pass
// of training and of inference uses the BF16 copies with FP32 accumulation.
// One training step = fused forward/backward per block of nodes (activations
// in shared memory, per-block weight-gradient partials), an ordered reduction
// of the partials (deterministic) and an Adam update that refreshes the BF16
// copies.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "s3_graph.h"

namespace s3 {
namespace {

constexpr int F = S3_MLP_FEATURES;  // 12
constexpr int H = S3_MLP_HIDDEN;    // 64
// parameter layout (floats): W1[H][F] b1[H] W2[H][H] b2[H] W3[H] b3
constexpr int OW1 = 0, OB1 = OW1 + H * F, OW2 = OB1 + H, OB2 = OW2 + H * H, OW3 = OB2 + H, OB3 = OW3 + H;
constexpr int NP = OB3 + 1;
static_assert(NP == S3_MLP_PARAMS, "parameter count");

constexpr int kTrainNodes = 64;  // nodes per block in the training kernel
constexpr size_t kTrainSmem = sizeof(double) * kTrainNodes +
                              sizeof(float) * (NP + kTrainNodes * F + 4 * kTrainNodes * (H + 1) + kTrainNodes);

// ----------------------------------------------------------- features ---

// histogram bin of edge size s at rank N: floor(8 log(s/2) / log(N/2)) clamped to 0..7 (host, FP64)
int size_bin(int s, int N) {
    if (N <= 2 || s <= 2) return 0;
    double t = std::log((double)s / 2.0) / std::log((double)N / 2.0);
    int b = (int)std::floor(8.0 * t);
    return b < 0 ? 0 : (b > 7 ? 7 : b);
}

// One thread per edge of one bucket.  Members of neighbouring edges are often the
// same node (edges are sorted, hubs first), so the lanes of a warp that target one
// node combine their updates and one lane issues the atomics (the integer sums are
// exact in any order).
__global__ void feature_edge_kernel(EdgeBucketArgs b, int bin, const int64_t *__restrict__ inc_ptr,
                                    unsigned long long *__restrict__ nbr, unsigned int *__restrict__ size_sum,
                                    int *__restrict__ size_max, unsigned int *__restrict__ hist) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= b.m) return;
    const int s = b.s;
    unsigned long long D = 0;
    for (int i = 0; i < s; ++i) {
        int v = b.ids[(int64_t)i * b.ld + e];
        D += (unsigned long long)(inc_ptr[v + 1] - inc_ptr[v]);
    }
    const unsigned act = __activemask();
    const int lane = threadIdx.x & 31;
    for (int i = 0; i < s; ++i) {
        const int v = b.ids[(int64_t)i * b.ld + e];
        const unsigned long long dv = (unsigned long long)(inc_ptr[v + 1] - inc_ptr[v]);
        const unsigned grp = __match_any_sync(act, v);
        unsigned long long acc = 0;
        for (unsigned mm = grp; mm; mm &= mm - 1) acc += __shfl_sync(grp, D - dv, __ffs(mm) - 1);
        if (lane == __ffs(grp) - 1) {
            const unsigned cnt = (unsigned)__popc(grp);
            atomicAdd(nbr + v, acc);
            atomicAdd(size_sum + v, cnt * (unsigned int)s);
            atomicMax(size_max + v, s);
            atomicAdd(hist + (int64_t)v * 8 + bin, cnt);
        }
    }
}

__global__ void feature_finalize_kernel(int64_t n, const int64_t *__restrict__ inc_ptr,
                                        const unsigned long long *__restrict__ nbr,
                                        const unsigned int *__restrict__ size_sum, const int *__restrict__ size_max,
                                        const unsigned int *__restrict__ hist, float *__restrict__ feat) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const double d = (double)(inc_ptr[v + 1] - inc_ptr[v]);
    float *f = feat + v * F;
    f[0] = (float)log1p(d);
    f[1] = (float)log1p(d > 0 ? (double)size_sum[v] / d : 0.0);
    f[2] = (float)log1p((double)size_max[v]);
    for (int k = 0; k < 8; ++k) f[3 + k] = (float)log1p((double)hist[v * 8 + k]);
    f[11] = (float)log1p((double)nbr[v]);
}

// ---------------------------------------------------------- inference ---

// out[v] = W3 relu(W2 relu(W1 f_v + b1) + b2) + b3, BF16 weights, FP32 accumulation
__global__ void __launch_bounds__(128) mlp_forward_kernel(const __nv_bfloat16 *__restrict__ wbf,
                                                          const float *__restrict__ feat, int64_t n,
                                                          float *__restrict__ out) {
    __shared__ float w[NP];
    for (int i = threadIdx.x; i < NP; i += blockDim.x) w[i] = __bfloat162float(wbf[i]);
    __syncthreads();
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    float f[F];
#pragma unroll
    for (int i = 0; i < F; ++i) f[i] = feat[v * F + i];
    float h1[H];
#pragma unroll
    for (int j = 0; j < H; ++j) {
        float acc = w[OB1 + j];
#pragma unroll
        for (int i = 0; i < F; ++i) acc = fmaf(w[OW1 + j * F + i], f[i], acc);
        h1[j] = fmaxf(acc, 0.f);
    }
    float y = w[OB3];
    for (int j = 0; j < H; ++j) {
        float acc = w[OB2 + j];
#pragma unroll
        for (int k = 0; k < H; ++k) acc = fmaf(w[OW2 + j * H + k], h1[k], acc);
        y = fmaf(w[OW3 + j], fmaxf(acc, 0.f), y);
    }
    out[v] = y;
}

// ----------------------------------------------------------- training ---

// Fused forward + backward for kNodes nodes per block (blockDim = kNodes); loss
// = sum over the batch of (y - target)^2 / count.  Writes this block's gradient
// partial (NP floats) and loss partial.
__global__ void __launch_bounds__(kTrainNodes) mlp_train_kernel(const __nv_bfloat16 *__restrict__ wbf,
                                                                const float *__restrict__ feat,
                                                                const float *__restrict__ target, int64_t n,
                                                                float inv_count, float *__restrict__ gpart,
                                                                double *__restrict__ lpart) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *sL = reinterpret_cast<double *>(smem_raw);                       // [kTrainNodes]
    float *w = reinterpret_cast<float *>(sL + kTrainNodes);                  // [NP]
    float(*sF)[F] = reinterpret_cast<float(*)[F]>(w + NP);                   // [kTrainNodes][F]
    float(*sH1)[H + 1] = reinterpret_cast<float(*)[H + 1]>(&sF[kTrainNodes][0]);
    float(*sH2)[H + 1] = sH1 + kTrainNodes;
    float(*sD2)[H + 1] = sH2 + kTrainNodes;
    float(*sD1)[H + 1] = sD2 + kTrainNodes;
    float *sDy = &sD1[kTrainNodes][0];                                       // [kTrainNodes]
    const int t = threadIdx.x;
    for (int i = t; i < NP; i += blockDim.x) w[i] = __bfloat162float(wbf[i]);
    __syncthreads();
    const int64_t v = (int64_t)blockIdx.x * kTrainNodes + t;
    const bool live = v < n;
    // forward
    for (int i = 0; i < F; ++i) sF[t][i] = live ? feat[v * F + i] : 0.f;
    for (int j = 0; j < H; ++j) {
        float acc = w[OB1 + j];
        for (int i = 0; i < F; ++i) acc = fmaf(w[OW1 + j * F + i], sF[t][i], acc);
        sH1[t][j] = fmaxf(acc, 0.f);
    }
    float y = w[OB3];
    for (int j = 0; j < H; ++j) {
        float acc = w[OB2 + j];
        for (int k = 0; k < H; ++k) acc = fmaf(w[OW2 + j * H + k], sH1[t][k], acc);
        float h2 = fmaxf(acc, 0.f);
        sH2[t][j] = h2;
        y = fmaf(w[OW3 + j], h2, y);
    }
    const float d = live ? y - target[v] : 0.f;
    sL[t] = (double)d * (double)d * (double)inv_count;
    const float dy = 2.f * d * inv_count;
    sDy[t] = dy;
    // backward through layer 3 and the second ReLU
    for (int j = 0; j < H; ++j) sD2[t][j] = sH2[t][j] > 0.f ? dy * w[OW3 + j] : 0.f;
    // through layer 2 and the first ReLU
    for (int k = 0; k < H; ++k) {
        float acc = 0.f;
        for (int j = 0; j < H; ++j) acc = fmaf(w[OW2 + j * H + k], sD2[t][j], acc);
        sD1[t][k] = sH1[t][k] > 0.f ? acc : 0.f;
    }
    __syncthreads();
    // weight gradients: each thread owns some parameters and sums over the block's nodes in order
    float *gp = gpart + (int64_t)blockIdx.x * NP;
    for (int p = t; p < NP; p += blockDim.x) {
        float acc = 0.f;
        if (p < OB1) {
            int j = p / F, i = p % F;
            for (int q = 0; q < kTrainNodes; ++q) acc = fmaf(sD1[q][j], sF[q][i], acc);
        } else if (p < OW2) {
            int j = p - OB1;
            for (int q = 0; q < kTrainNodes; ++q) acc += sD1[q][j];
        } else if (p < OB2) {
            int j = (p - OW2) / H, k = (p - OW2) % H;
            for (int q = 0; q < kTrainNodes; ++q) acc = fmaf(sD2[q][j], sH1[q][k], acc);
        } else if (p < OW3) {
            int j = p - OB2;
            for (int q = 0; q < kTrainNodes; ++q) acc += sD2[q][j];
        } else if (p < OB3) {
            int j = p - OW3;
            for (int q = 0; q < kTrainNodes; ++q) acc = fmaf(sDy[q], sH2[q][j], acc);
        } else {
            for (int q = 0; q < kTrainNodes; ++q) acc += sDy[q];
        }
        gp[p] = acc;
    }
    if (t == 0) {
        double l = 0.0;
        for (int q = 0; q < kTrainNodes; ++q) l += sL[q];
        lpart[blockIdx.x] = l;
    }
}

// grad[p] = sum over blocks (in order) of the partials; loss likewise
__global__ void mlp_grad_reduce_kernel(const float *__restrict__ gpart, const double *__restrict__ lpart, int nblocks,
                                       float *__restrict__ grad, double *__restrict__ loss) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < NP) {
        double acc = 0.0;
        for (int b = 0; b < nblocks; ++b) acc += (double)gpart[(int64_t)b * NP + p];
        grad[p] = (float)acc;
    }
    if (p == 0) {
        double l = 0.0;
        for (int b = 0; b < nblocks; ++b) l += lpart[b];
        *loss = l;
    }
}

// Adam (bias-corrected) on the FP32 master weights; refreshes the BF16 copies
__global__ void mlp_adam_kernel(float *__restrict__ wf, __nv_bfloat16 *__restrict__ wbf, const float *__restrict__ grad,
                                float *__restrict__ m1, float *__restrict__ m2, float lr, float beta1, float beta2,
                                float eps, float c1, float c2) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NP) return;
    float g = grad[p];
    float a = beta1 * m1[p] + (1.f - beta1) * g;
    float b = beta2 * m2[p] + (1.f - beta2) * g * g;
    m1[p] = a;
    m2[p] = b;
    float wv = wf[p] - lr * (a / c1) / (sqrtf(b / c2) + eps);
    wf[p] = wv;
    wbf[p] = __float2bfloat16_rn(wv);
}

__global__ void to_bf16_kernel(const float *__restrict__ wf, __nv_bfloat16 *__restrict__ wbf) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < NP) wbf[p] = __float2bfloat16_rn(wf[p]);
}

// x0_v = exp(out_v - max out) / sum (two passes: max, then sum; then scale)
__global__ void warm_exp_kernel(const float *__restrict__ out, int64_t n, double shift, double *__restrict__ x0,
                                double *__restrict__ partial) {
    __shared__ double sh[256 / 32];
    double acc = 0.0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        double e = exp((double)out[v] - shift);
        x0[v] = e;
        acc += e;
    }
    for (int d = 16; d > 0; d >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, d);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 256 / 32; ++w) t += sh[w];
        partial[blockIdx.x] = t;
    }
}

__global__ void warm_scale_kernel(double *__restrict__ x0, int64_t n, const double *__restrict__ partial, int np) {
    __shared__ double inv;
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < np; ++i) t += partial[i];
        inv = 1.0 / t;
    }
    __syncthreads();
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        x0[v] *= inv;
}

__global__ void max_reduce_kernel(const float *__restrict__ out, int64_t n, float *__restrict__ res) {
    __shared__ float sh[256 / 32];
    float m = -INFINITY;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, out[v]);
    for (int d = 16; d > 0; d >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, d));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 256 / 32; ++w) m = fmaxf(m, sh[w]);
        res[blockIdx.x] = m;
    }
}

// target_v = log x_v - mean_v log x_v: per-block partial sums of log x, then subtract
__global__ void log_partial_kernel(const double *__restrict__ x, int64_t n, float *__restrict__ t,
                                   double *__restrict__ partial) {
    __shared__ double sh[256 / 32];
    double acc = 0.0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        double l = log(x[v]);
        t[v] = (float)l;
        acc += l;
    }
    for (int d = 16; d > 0; d >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, d);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < 256 / 32; ++w) tot += sh[w];
        partial[blockIdx.x] = tot;
    }
}

__global__ void center_kernel(const double *__restrict__ x, int64_t n, float *__restrict__ t,
                              const double *__restrict__ partial, int np) {
    __shared__ double mean;
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int i = 0; i < np; ++i) tot += partial[i];
        mean = tot / (double)n;
    }
    __syncthreads();
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        t[v] = (float)(log(x[v]) - mean);
}

}  // namespace
}  // namespace s3

using namespace s3;

struct s3_mlp_s {
    int device = 0;
    float *wf = nullptr;           // FP32 master weights
    __nv_bfloat16 *wbf = nullptr;  // BF16 copies
    float *m1 = nullptr, *m2 = nullptr, *grad = nullptr;
    double *loss = nullptr;
    float *gpart = nullptr;
    double *lpart = nullptr;
    int64_t part_cap = 0;          // blocks the partial arrays hold
    int64_t step = 0;
    std::vector<void *> allocations;
};

namespace {

s3_status mlp_alloc(s3_mlp_s *m, void **p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(S3_ENOMEM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
    }
    m->allocations.push_back(*p);
    return S3_OK;
}

s3_status ensure_parts(s3_mlp_s *m, int64_t blocks) {
    if (blocks <= m->part_cap) return S3_OK;
    void *p = nullptr;
    s3_status s = mlp_alloc(m, &p, sizeof(float) * (size_t)blocks * NP);
    if (s != S3_OK) return s;
    m->gpart = reinterpret_cast<float *>(p);
    if ((s = mlp_alloc(m, &p, sizeof(double) * (size_t)blocks)) != S3_OK) return s;
    m->lpart = reinterpret_cast<double *>(p);
    m->part_cap = blocks;
    return S3_OK;
}

// He-style initialisation from a counter-based hash of (seed, index): deterministic.
float init_value(uint64_t seed, int p) {
    uint64_t z = seed * 0x9E3779B97F4A7C15ull + (uint64_t)p * 0xBF58476D1CE4E5B9ull + 0x94D049BB133111EBull;
    z ^= z >> 31;
    z *= 0xD6E8FEB86659FD93ull;
    z ^= z >> 29;
    double u = ((z >> 11) + 0.5) / 9007199254740992.0;  // (0,1)
    double r = 2.0 * u - 1.0;                            // uniform in (-1, 1)
    if (p < OB1) return (float)(r * std::sqrt(6.0 / F));
    if (p < OW2) return 0.0f;
    if (p < OB2) return (float)(r * std::sqrt(6.0 / H));
    if (p < OW3) return 0.0f;
    if (p < OB3) return (float)(r * std::sqrt(3.0 / H));
    return 0.0f;
}

}  // namespace

extern "C" {

s3_status s3_features(s3_graph_t g, float *feat, void *stream) {
    if (!g || !feat) return fail(S3_EINVAL, "NULL argument");
    DeviceGuard guard(g->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (!g->d_feat_scratch) {
        // nbr (u64), size_sum (u32), size_max (i32), hist (8 x u32): 48 bytes per node
        s3_status s = dev_alloc(g, &g->d_feat_scratch, (size_t)g->n * 12 + 8);
        if (s != S3_OK) return s;
    }
    char *base = reinterpret_cast<char *>(g->d_feat_scratch);
    auto *nbr = reinterpret_cast<unsigned long long *>(base);
    auto *ssum = reinterpret_cast<unsigned int *>(base + 8 * (size_t)g->n);
    auto *smax = reinterpret_cast<int *>(base + 12 * (size_t)g->n);
    auto *hist = reinterpret_cast<unsigned int *>(base + 16 * (size_t)g->n);
    S3_CUDA(cudaMemsetAsync(base, 0, 48 * (size_t)g->n, st));
    for (size_t k = 0; k < g->buckets.size(); ++k) {
        const HostBucket &hb = g->buckets[k];
        if (hb.m <= 0) continue;
        EdgeBucketArgs b{};
        b.ids = g->d_ids + hb.offset;
        b.m = hb.m;
        b.ld = hb.ld;
        b.s = hb.s;
        b.N = g->N;
        feature_edge_kernel<<<(unsigned)((hb.m + 255) / 256), 256, 0, st>>>(b, size_bin(hb.s, g->N), g->d_inc_ptr, nbr,
                                                                           ssum, smax, hist);
        S3_CUDA(cudaGetLastError());
    }
    feature_finalize_kernel<<<(unsigned)((g->n + 255) / 256), 256, 0, st>>>(g->n, g->d_inc_ptr, nbr, ssum, smax, hist,
                                                                           feat);
    S3_CUDA(cudaGetLastError());
    return S3_OK;
}

s3_status s3_mlp_create(const float *params, uint64_t seed, s3_mlp_t *out) {
    if (!out) return fail(S3_EINVAL, "out is NULL");
    *out = nullptr;
    s3_mlp_s *m = new (std::nothrow) s3_mlp_s();
    if (!m) return fail(S3_ENOMEM, "host allocation failed");
    S3_CUDA(cudaGetDevice(&m->device));
    auto bail = [&](s3_status s) {
        for (void *p : m->allocations) cudaFree(p);
        delete m;
        return s;
    };
    void *p = nullptr;
    s3_status s;
    if ((s = mlp_alloc(m, &p, sizeof(float) * NP)) != S3_OK) return bail(s);
    m->wf = reinterpret_cast<float *>(p);
    if ((s = mlp_alloc(m, &p, sizeof(__nv_bfloat16) * NP)) != S3_OK) return bail(s);
    m->wbf = reinterpret_cast<__nv_bfloat16 *>(p);
    if ((s = mlp_alloc(m, &p, sizeof(float) * NP)) != S3_OK) return bail(s);
    m->m1 = reinterpret_cast<float *>(p);
    if ((s = mlp_alloc(m, &p, sizeof(float) * NP)) != S3_OK) return bail(s);
    m->m2 = reinterpret_cast<float *>(p);
    if ((s = mlp_alloc(m, &p, sizeof(float) * NP)) != S3_OK) return bail(s);
    m->grad = reinterpret_cast<float *>(p);
    if ((s = mlp_alloc(m, &p, sizeof(double))) != S3_OK) return bail(s);
    m->loss = reinterpret_cast<double *>(p);
    std::vector<float> h(NP);
    for (int i = 0; i < NP; ++i) h[i] = params ? params[i] : init_value(seed, i);
    if (cudaMemcpy(m->wf, h.data(), sizeof(float) * NP, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(m->m1, 0, sizeof(float) * NP) != cudaSuccess ||
        cudaMemset(m->m2, 0, sizeof(float) * NP) != cudaSuccess)
        return bail(cuda_fail(cudaGetLastError(), "cudaMemcpy"));
    if (cudaFuncSetAttribute(mlp_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTrainSmem) !=
        cudaSuccess)
        return bail(cuda_fail(cudaGetLastError(), "cudaFuncSetAttribute"));
    to_bf16_kernel<<<(NP + 255) / 256, 256>>>(m->wf, m->wbf);
    if (cudaDeviceSynchronize() != cudaSuccess) return bail(cuda_fail(cudaGetLastError(), "to_bf16"));
    *out = m;
    return S3_OK;
}

s3_status s3_mlp_get_params(s3_mlp_t m, float *params, int32_t bf16) {
    if (!m || !params) return fail(S3_EINVAL, "NULL argument");
    DeviceGuard guard(m->device);
    S3_CUDA(cudaDeviceSynchronize());
    if (!bf16) {
        S3_CUDA(cudaMemcpy(params, m->wf, sizeof(float) * NP, cudaMemcpyDeviceToHost));
        return S3_OK;
    }
    std::vector<__nv_bfloat16> h(NP);
    S3_CUDA(cudaMemcpy(h.data(), m->wbf, sizeof(__nv_bfloat16) * NP, cudaMemcpyDeviceToHost));
    for (int i = 0; i < NP; ++i) params[i] = __bfloat162float(h[i]);
    return S3_OK;
}

s3_status s3_mlp_forward(s3_mlp_t m, const float *feat, int64_t n, float *out, void *stream) {
    if (!m || !feat || !out || n < 0) return fail(S3_EINVAL, "bad argument");
    if (n == 0) return S3_OK;
    DeviceGuard guard(m->device);
    mlp_forward_kernel<<<(unsigned)((n + 127) / 128), 128, 0, (cudaStream_t)stream>>>(m->wbf, feat, n, out);
    S3_CUDA(cudaGetLastError());
    return S3_OK;
}

s3_status s3_mlp_loss_grad(s3_mlp_t m, const float *feat, const float *target, int64_t n, double *loss,
                           float *grad, void *stream) {
    if (!m || !feat || !target || n <= 0) return fail(S3_EINVAL, "bad argument");
    DeviceGuard guard(m->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t blocks = (n + kTrainNodes - 1) / kTrainNodes;
    s3_status s = ensure_parts(m, blocks);
    if (s != S3_OK) return s;
    mlp_train_kernel<<<(unsigned)blocks, kTrainNodes, kTrainSmem, st>>>(m->wbf, feat, target, n, 1.0f / (float)n,
                                                                        m->gpart, m->lpart);
    S3_CUDA(cudaGetLastError());
    mlp_grad_reduce_kernel<<<(NP + 255) / 256, 256, 0, st>>>(m->gpart, m->lpart, (int)blocks, m->grad, m->loss);
    S3_CUDA(cudaGetLastError());
    if (loss) S3_CUDA(cudaMemcpyAsync(loss, m->loss, sizeof(double), cudaMemcpyDeviceToHost, st));
    if (grad) S3_CUDA(cudaMemcpyAsync(grad, m->grad, sizeof(float) * NP, cudaMemcpyDeviceToHost, st));
    if (loss || grad) S3_CUDA(cudaStreamSynchronize(st));
    return S3_OK;
}

s3_status s3_mlp_adam_step(s3_mlp_t m, float lr, float beta1, float beta2, float eps, void *stream) {
    if (!m) return fail(S3_EINVAL, "NULL argument");
    DeviceGuard guard(m->device);
    m->step += 1;
    float c1 = 1.f - std::pow(beta1, (float)m->step), c2 = 1.f - std::pow(beta2, (float)m->step);
    mlp_adam_kernel<<<(NP + 255) / 256, 256, 0, (cudaStream_t)stream>>>(m->wf, m->wbf, m->grad, m->m1, m->m2, lr,
                                                                        beta1, beta2, eps, c1, c2);
    S3_CUDA(cudaGetLastError());
    return S3_OK;
}

s3_status s3_warmstart(s3_graph_t g, s3_mlp_t m, double *x0, void *stream) {
    if (!g || !m || !x0) return fail(S3_EINVAL, "NULL argument");
    DeviceGuard guard(g->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (!g->d_ws) {
        // features (12 floats per node), prediction (1 float per node), then max and sum partials
        s3_status s = dev_alloc(g, &g->d_ws, (size_t)g->n * 13 + 4096);
        if (s != S3_OK) return s;
    }
    float *feat = g->d_ws;
    float *out = g->d_ws + (size_t)g->n * 12;
    float *mx = out + g->n;
    double *part = reinterpret_cast<double *>(g->d_ws + (((size_t)g->n * 13 + 1024 + 1) & ~(size_t)1));
    s3_status s = s3_features(g, feat, stream);
    if (s != S3_OK) return s;
    s = s3_mlp_forward(m, feat, g->n, out, stream);
    if (s != S3_OK) return s;
    const int nb = 256;
    max_reduce_kernel<<<nb, 256, 0, st>>>(out, g->n, mx);
    S3_CUDA(cudaGetLastError());
    float hmx[256];
    S3_CUDA(cudaMemcpyAsync(hmx, mx, sizeof(float) * nb, cudaMemcpyDeviceToHost, st));
    S3_CUDA(cudaStreamSynchronize(st));
    float shift = -INFINITY;
    for (int i = 0; i < nb; ++i) shift = std::max(shift, hmx[i]);
    if (!std::isfinite(shift)) return fail(S3_ERANGE, "warm-start prediction is not finite");
    warm_exp_kernel<<<nb, 256, 0, st>>>(out, g->n, (double)shift, x0, part);
    S3_CUDA(cudaGetLastError());
    warm_scale_kernel<<<nb, 256, 0, st>>>(x0, g->n, part, nb);
    S3_CUDA(cudaGetLastError());
    return S3_OK;
}

s3_status s3_mlp_target(s3_graph_t g, const double *x, float *target, void *stream) {
    if (!g || !x || !target) return fail(S3_EINVAL, "NULL argument");
    DeviceGuard guard(g->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (!g->d_ws) {
        s3_status s = dev_alloc(g, &g->d_ws, (size_t)g->n * 13 + 4096);
        if (s != S3_OK) return s;
    }
    double *part = reinterpret_cast<double *>(g->d_ws + (((size_t)g->n * 13 + 1024 + 1) & ~(size_t)1));
    const int nb = 256;
    log_partial_kernel<<<nb, 256, 0, st>>>(x, g->n, target, part);
    S3_CUDA(cudaGetLastError());
    center_kernel<<<nb, 256, 0, st>>>(x, g->n, target, part, nb);
    S3_CUDA(cudaGetLastError());
    return S3_OK;
}

s3_status s3_mlp_destroy(s3_mlp_t m) {
    if (!m) return S3_OK;
    {
        DeviceGuard guard(m->device);
        cudaDeviceSynchronize();
        for (void *p : m->allocations) cudaFree(p);
    }
    delete m;
    return S3_OK;
}

}  // extern "C"
