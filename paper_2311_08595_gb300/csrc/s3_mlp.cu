// Learned warm start for the NQZ iteration: per-node features, a 12-64-64-1
// MLP (BF16 weights, FP32 accumulation) and its training kernels.
//
// Features of node v (all log1p-scaled): degree; mean and max size of the
// edges containing v; an 8-bin histogram of those sizes (bins log-spaced on
// [2, N]); the sum over v's edges of the other members' degrees.  Each edge writes
// one integer record per member into the member's slot of the reduce buffer, and the
// segmented reduce (s3_reduce.cu) folds each node's records without atomics (exact
// integer sums, so the result does not depend on scheduling).  The network predicts
// log x*_v minus its mean over the graph; the warm start is exp(prediction),
// normalised to 1-norm 1.
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

// Per-(edge, node) records for the features, one thread per edge, all buckets in one
// launch (block ranges map to buckets, tab[k].block0 ascending; the size-bin of bucket k's
// edges in tab[k].W): the record of member v of edge e goes to v's slot of the reduce
// buffer, holding |e| (bits 0-7), its bin (bits 8-10) and D_e - deg v (bits 16-63), D_e the
// degree sum of e's members.  The segmented reduce then folds each node's records.
__global__ void feature_record_kernel(const TailEntry *__restrict__ tab, int ntab, const int64_t *__restrict__ inc_ptr,
                                      unsigned long long *__restrict__ rec) {
    int k = 0;
    while (k + 1 < ntab && tab[k + 1].block0 <= (int64_t)blockIdx.x) ++k;
    const EdgeBucketArgs &b = tab[k].b;
    const unsigned long long tag = ((unsigned long long)tab[k].W << 8) | (unsigned long long)b.s;
    int64_t e = ((int64_t)blockIdx.x - tab[k].block0) * blockDim.x + threadIdx.x;
    if (e >= b.m) return;
    const int s = b.s;
    unsigned long long D = 0;
    for (int i = 0; i < s; ++i) {
        const int v = __ldg(b.ids + (int64_t)i * b.ld + e);
        D += (unsigned long long)(__ldg(inc_ptr + v + 1) - __ldg(inc_ptr + v));
    }
    for (int i = 0; i < s; ++i) {
        const int v = __ldg(b.ids + (int64_t)i * b.ld + e);
        const unsigned long long dv = (unsigned long long)(__ldg(inc_ptr + v + 1) - __ldg(inc_ptr + v));
        rec[__ldg(b.slot + (int64_t)i * b.ld + e)] = ((D - dv) << 16) | tag;
    }
}

// ---------------------------------------------------------- inference ---

// out[v] = W3 relu(W2 relu(W1 f_v + b1) + b2) + b3 with the BF16 weights, one tile of
// 128 nodes per CTA (4 warps, one node per thread, 64 TMEM columns).  Both hidden layers
// run on the tensor cores as D[128 x 64] = A B^T (tcgen05.mma kind::f16, M = 128, N = 64,
// K = 16 per instruction, FP32 accumulators in TMEM): layer 1 with A = the features (K = 12,
// padded to 16 with zeros) and B = W1, layer 2 with A = h1 and B = W2.  Each A is split into
// two BF16 terms, hi = bf16(a) and lo = bf16(a - hi), so that the FP32 accumulation of
// hi B^T + lo B^T equals a B^T to about 2^-17 relative (the weights are exactly BF16).  The
// FP32 units add the biases, apply the ReLUs, split h1 for layer 2, and evaluate the output
// layer from the second accumulator (tcgen05.ld).
//
// Operands in shared memory use the 128-byte-swizzled K-major layout: one 128-byte row
// per matrix row (64 BF16; layer 1 uses the first 16), 8-row atoms of 1 KB, the 16-byte
// chunk c of row r stored at chunk c ^ (r % 8).  Descriptor: stride between 8-row groups
// 1024 B; each K step of 16 advances the start address by 32 B inside the atom.  The A
// tiles of layer 1 are overwritten by those of layer 2 once the first MMAs have completed.
constexpr int kTcRows = 128;                       // nodes per CTA (the MMA's M)
constexpr int kTcCols = 64;                        // TMEM columns (the MMA's N; FP32 accumulators)
constexpr uint32_t kTcIdesc = (1u << 4)            // D: FP32
                              | (1u << 7)          // A: BF16
                              | (1u << 10)         // B: BF16
                              | ((uint32_t)(H >> 3) << 17)        // N = 64
                              | ((uint32_t)(kTcRows >> 4) << 24); // M = 128 (A and B K-major)
// dynamic shared memory: A_hi, A_lo (16 KB each), B1 and B2 (8 KB each), then FP32 copies of
// b1, b2, W3, b3 and the mbarrier / TMEM address words
constexpr size_t kTcA = (size_t)kTcRows * 128, kTcB = (size_t)H * 128;
constexpr int kTcSmall = H + H + H + 1;
constexpr size_t kTcSmem = 1024 /* alignment slack */ + 2 * kTcA + 2 * kTcB + sizeof(float) * kTcSmall + 32;
static_assert(kTcSmem <= 227 * 1024, "forward kernel shared memory");
constexpr long long kTcWaitPolls = 1ll << 22;      // bound on each MMA-completion wait

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor: 128-byte swizzle, K-major, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4)   // start address
           | ((uint64_t)1 << 16)                 // leading-dimension offset (unused with this swizzle)
           | ((uint64_t)(1024 >> 4) << 32)       // stride-dimension offset
           | ((uint64_t)1 << 46)                 // descriptor version
           | ((uint64_t)2 << 61);                // 128-byte swizzle
}

// byte offset of 16-byte chunk c of row r in a 128-byte-swizzled K-major tile
__device__ __forceinline__ uint32_t sw128_off(int r, int c) {
    return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((c ^ (r & 7)) << 4));
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    const __nv_bfloat16 x = __float2bfloat16_rn(a), y = __float2bfloat16_rn(b);
    return (uint32_t)__bfloat16_as_ushort(x) | ((uint32_t)__bfloat16_as_ushort(y) << 16);
}

// eight values as one 16-byte chunk of BF16 hi terms and one of BF16 lo terms
__device__ __forceinline__ void split_chunk(const float (&h)[8], uint4 &hi, uint4 &lo) {
    uint32_t H4[4], L4[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float x0 = h[2 * q], x1 = h[2 * q + 1];
        H4[q] = pack_bf16(x0, x1);
        const float r0 = x0 - __bfloat162float(__ushort_as_bfloat16((unsigned short)(H4[q] & 0xffffu)));
        const float r1 = x1 - __bfloat162float(__ushort_as_bfloat16((unsigned short)(H4[q] >> 16)));
        L4[q] = pack_bf16(r0, r1);
    }
    hi = make_uint4(H4[0], H4[1], H4[2], H4[3]);
    lo = make_uint4(L4[0], L4[1], L4[2], L4[3]);
}

// one thread issues the MMAs of a layer (accumulating over the hi and lo A tiles and the K
// steps) and commits them to the mbarrier
__device__ __forceinline__ void tc_layer(uint32_t tmem, uint32_t a_hi, uint32_t a_lo, uint32_t b, int ksteps,
                                         uint32_t mbar) {
    const uint32_t sa[2] = {a_hi, a_lo};
#pragma unroll
    for (int part = 0; part < 2; ++part) {
        for (int k = 0; k < ksteps; ++k) {
            const uint64_t da = sw128_desc(sa[part] + 32u * k);
            const uint64_t db = sw128_desc(b + 32u * k);
            const uint32_t accum = (part | k) ? 1u : 0u;
            asm volatile(
                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                "l"(da), "l"(db), "r"(kTcIdesc), "r"(accum)
                : "memory");
        }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

// bounded wait for phase `parity` of the mbarrier; false if it ran out
__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t parity) {
    for (long long it = 0; it < kTcWaitPolls; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred P;\n\tmbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
            "selp.b32 %0, 1, 0, P;\n\t}"
            : "=r"(ok)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (ok) return true;
        if (it > 64) __nanosleep(64);
    }
    return false;
}

// 16 accumulator columns of this warp's 32 TMEM lanes (one row per thread)
__device__ __forceinline__ void tc_load16(uint32_t ta, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
        "%13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(ta)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__global__ void __launch_bounds__(kTcRows) mlp_forward_tc_kernel(const __nv_bfloat16 *__restrict__ wbf,
                                                                  const float *__restrict__ feat, int64_t n,
                                                                  float *__restrict__ out, int vec_feat,
                                                                  int *__restrict__ err) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    unsigned char *a_hi = base, *a_lo = base + kTcA, *b_w1 = base + 2 * kTcA, *b_w2 = b_w1 + kTcB;
    float *b1 = reinterpret_cast<float *>(b_w2 + kTcB);
    float *b2 = b1 + H, *w3 = b2 + H, *b3 = w3 + H;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(
        (reinterpret_cast<uintptr_t>(b3 + 1) + 7) & ~(uintptr_t)7);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mbar + 1);
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t mb = smem_u32(mbar);

    // TMEM: 64 columns, allocated by warp 0
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mb), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // B tiles: W1 (row n: its 12 weights and 4 zeros in chunks 0-1) and W2 (row n: 64 weights);
    // biases and W3 as FP32
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(wbf + OW2);
        for (int i = tid; i < H * 8; i += kTcRows) {
            const int r = i >> 3, c = i & 7;
            *reinterpret_cast<uint4 *>(b_w2 + sw128_off(r, c)) = __ldg(src + i);
        }
        for (int i = tid; i < H * 2; i += kTcRows) {
            const int r = i >> 1, c = i & 1;
            uint32_t w[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int k0 = 8 * c + 2 * q;
                const unsigned short lo16 = k0 < F ? __bfloat16_as_ushort(wbf[OW1 + r * F + k0]) : 0;
                const unsigned short hi16 = k0 + 1 < F ? __bfloat16_as_ushort(wbf[OW1 + r * F + k0 + 1]) : 0;
                w[q] = (uint32_t)lo16 | ((uint32_t)hi16 << 16);
            }
            *reinterpret_cast<uint4 *>(b_w1 + sw128_off(r, c)) = make_uint4(w[0], w[1], w[2], w[3]);
        }
        for (int i = tid; i < H; i += kTcRows) {
            b1[i] = __bfloat162float(wbf[OB1 + i]);
            b2[i] = __bfloat162float(wbf[OB2 + i]);
            w3[i] = __bfloat162float(wbf[OW3 + i]);
        }
        if (tid == 0) *b3 = __bfloat162float(wbf[OB3]);
    }
    // layer-1 A tiles: this thread's row = node v's features, split (chunks 0-1, zero padded)
    const int64_t v = (int64_t)blockIdx.x * kTcRows + tid;
    {
        float f[16];
        if (v < n && vec_feat) {
            const float4 *fp = reinterpret_cast<const float4 *>(feat + v * F);
#pragma unroll
            for (int q = 0; q < F / 4; ++q) {
                const float4 t = __ldg(fp + q);
                f[4 * q] = t.x;
                f[4 * q + 1] = t.y;
                f[4 * q + 2] = t.z;
                f[4 * q + 3] = t.w;
            }
        } else {
#pragma unroll
            for (int i = 0; i < F; ++i) f[i] = v < n ? __ldg(feat + v * F + i) : 0.f;
        }
#pragma unroll
        for (int i = F; i < 16; ++i) f[i] = 0.f;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            float h[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) h[j] = f[8 * c + j];
            uint4 hi, lo;
            split_chunk(h, hi, lo);
            const uint32_t off = sw128_off(tid, c);
            *reinterpret_cast<uint4 *>(a_hi + off) = hi;
            *reinterpret_cast<uint4 *>(a_lo + off) = lo;
        }
    }
    // the tiles (generic-proxy stores) become visible to the tensor cores (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const uint32_t ta = tmem + ((uint32_t)(32 * warp) << 16);   // this warp's lanes

    if (tid == 0) tc_layer(tmem, smem_u32(a_hi), smem_u32(a_lo), smem_u32(b_w1), 1, mb);
    bool done = tc_wait(mb, 0);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const bool ok1 = __all_sync(0xffffffffu, done);
    // layer-1 epilogue: h1 = relu(acc + b1), split into the layer-2 A tiles (the layer-1 tiles
    // are free: their MMAs have completed)
    if (ok1) {
#pragma unroll 1
        for (int c0 = 0; c0 < H; c0 += 16) {
            float acc[16];
            tc_load16(ta + (uint32_t)c0, acc);
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                float h[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) h[j] = fmaxf(acc[8 * half + j] + b1[c0 + 8 * half + j], 0.f);
                uint4 hi, lo;
                split_chunk(h, hi, lo);
                const uint32_t off = sw128_off(tid, (c0 >> 3) + half);
                *reinterpret_cast<uint4 *>(a_hi + off) = hi;
                *reinterpret_cast<uint4 *>(a_lo + off) = lo;
            }
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    const int all1 = __syncthreads_and(ok1);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    bool ok2 = false;
    if (all1) {
        if (tid == 0) tc_layer(tmem, smem_u32(a_hi), smem_u32(a_lo), smem_u32(b_w2), H / 16, mb);
        done = tc_wait(mb, 1);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        ok2 = __all_sync(0xffffffffu, done);
    }
    if (ok2) {
        // output layer from the layer-2 accumulators
        float y = *b3;
#pragma unroll 1
        for (int c0 = 0; c0 < H; c0 += 16) {
            float acc[16];
            tc_load16(ta + (uint32_t)c0, acc);
#pragma unroll
            for (int j = 0; j < 16; ++j) y = fmaf(w3[c0 + j], fmaxf(acc[j] + b2[c0 + j], 0.f), y);
        }
        if (v < n) out[v] = y;
    } else if ((tid & 31) == 0) {
        atomicExch(err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols) : "memory");
    }
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
        // FP32 exponential: x0 is a start vector, whose precision does not decide the result
        const double e = (double)expf(out[v] - (float)shift);
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

// (blockDim.x = 256) every block sums the partials with all its threads in one fixed order
// (strided per thread, then a tree), so all blocks scale by the same 1/sum
__global__ void warm_scale_kernel(double *__restrict__ x0, int64_t n, const double *__restrict__ partial, int np) {
    __shared__ double sh[256];
    __shared__ double inv;
    double t = 0.0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) t += partial[i];
    sh[threadIdx.x] = t;
    __syncthreads();
    for (int d = 128; d > 0; d >>= 1) {
        if ((int)threadIdx.x < d) sh[threadIdx.x] += sh[threadIdx.x + d];
        __syncthreads();
    }
    if (threadIdx.x == 0) inv = 1.0 / sh[0];
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
    int *d_err = nullptr;          // set by a tensor-core wait that ran out
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

// the flag a tensor-core wait sets when it runs out: read (synchronising `st`), cleared, reported
s3_status take_error(s3_mlp_s *m, cudaStream_t st) {
    int h = 0;
    S3_CUDA(cudaMemcpyAsync(&h, m->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    S3_CUDA(cudaStreamSynchronize(st));
    if (!h) return S3_OK;
    S3_CUDA(cudaMemsetAsync(m->d_err, 0, sizeof(int), st));
    return fail(S3_ETIMEOUT, "a tensor-core completion wait of the MLP forward pass ran out");
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
    if (!g->d_feat_scratch && g->n_pieces > 0) {
        // per-piece partial accumulators of the hub nodes (64 bytes each)
        s3_status s = dev_alloc(g, &g->d_feat_scratch, (size_t)g->n_pieces * 16);
        if (s != S3_OK) return s;
    }
    if (!g->d_feat_tab) {
        // one table of the buckets for the fused launch (built once per handle)
        std::vector<TailEntry> tab;
        int64_t blocks = 0;
        for (size_t k = 0; k < g->buckets.size(); ++k) {
            const HostBucket &hb = g->buckets[k];
            if (hb.m <= 0) continue;
            TailEntry t{};
            t.b.ids = g->d_ids + hb.offset;
            t.b.slot = g->d_slot + hb.offset;
            t.b.m = hb.m;
            t.b.ld = hb.ld;
            t.b.s = hb.s;
            t.b.N = g->N;
            t.W = size_bin(hb.s, g->N);
            t.block0 = blocks;
            blocks += (hb.m + 255) / 256;
            tab.push_back(t);
        }
        if (!tab.empty()) {
            TailEntry *d = nullptr;
            s3_status s = dev_alloc(g, &d, tab.size());
            if (s != S3_OK) return s;
            S3_CUDA(cudaMemcpy(d, tab.data(), sizeof(TailEntry) * tab.size(), cudaMemcpyHostToDevice));
            g->d_feat_tab = d;
        }
        g->n_feat_tab = (int32_t)tab.size();
        g->feat_blocks = blocks;
    }
    auto *rec = reinterpret_cast<unsigned long long *>(g->d_buf);
    if (g->n_feat_tab > 0) {
        feature_record_kernel<<<(unsigned)g->feat_blocks, 256, 0, st>>>(g->d_feat_tab, g->n_feat_tab, g->d_inc_ptr,
                                                                        rec);
        S3_CUDA(cudaGetLastError());
    }
    ReduceArgs r = reduce_args(g, nullptr);
    r.partial = g->d_feat_scratch;
    S3_CUDA(launch_feature_reduce(r, rec, feat, st));
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
    if ((s = mlp_alloc(m, &p, sizeof(int))) != S3_OK) return bail(s);
    m->d_err = reinterpret_cast<int *>(p);
    std::vector<float> h(NP);
    for (int i = 0; i < NP; ++i) h[i] = params ? params[i] : init_value(seed, i);
    if (cudaMemcpy(m->wf, h.data(), sizeof(float) * NP, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(m->m1, 0, sizeof(float) * NP) != cudaSuccess ||
        cudaMemset(m->m2, 0, sizeof(float) * NP) != cudaSuccess || cudaMemset(m->d_err, 0, sizeof(int)) != cudaSuccess)
        return bail(cuda_fail(cudaGetLastError(), "cudaMemcpy"));
    if (cudaFuncSetAttribute(mlp_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTrainSmem) !=
            cudaSuccess ||
        cudaFuncSetAttribute(mlp_forward_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem) !=
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
    s3_status es = take_error(m, nullptr);
    if (es != S3_OK) return es;
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
    const int64_t blocks = (n + kTcRows - 1) / kTcRows;
    if (blocks > INT32_MAX) return fail(S3_EINVAL, "too many nodes");
    const int vec = (reinterpret_cast<uintptr_t>(feat) & 15) == 0;
    mlp_forward_tc_kernel<<<(unsigned)blocks, kTcRows, kTcSmem, (cudaStream_t)stream>>>(m->wbf, feat, n, out, vec,
                                                                                          m->d_err);
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
    s = take_error(m, st);   // synchronises st
    if (s != S3_OK) return s;
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
