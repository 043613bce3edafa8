// Learned refinement proposal: a 5-layer MLP, 32 -> 256 -> 256 -> 256 -> 256 -> 256,
// GELU after the four hidden layers, that maps an integral's parameters
// (sin/cos of qx, qy; one-hot l and m; log10 T; mu; t'; one-hot kind) to a
// 16 x 16 map of predicted log10 cell errors.  It only decides where the
// initial partition is pre-split; the cubature's own error sums still decide
// convergence.  (Not part of the paper: the proposal of the workload
// specification.)
//
// Kernels: the forward pass of all five layers in one launch on the tcgen05
// tensor cores (TMEM accumulators, fused bias / GELU / BF16 epilogues); for
// training, BF16 GEMMs on mma.sync m16n8k16 for the backward products, the
// MSE loss gradient, GELU backward, bias gradients and AdamW on FP32 master
// weights.
//
// Parameter buffer (FP32 master weights), layer l = 0..4 with K_0 = 32,
// K_l = 256 otherwise, N = 256:  W_l [K_l][N] row-major, then b_l [N].
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/paid.h"

namespace {

constexpr int kIn = PAID_MLP_IN, kHid = PAID_MLP_HIDDEN;
constexpr int kLayers = PAID_MLP_LAYERS;
static_assert(PAID_MLP_OUT == PAID_MLP_HIDDEN, "the output layer has the hidden width");

__host__ __device__ inline int layer_k(int l) { return l == 0 ? kIn : kHid; }
__host__ __device__ inline int64_t layer_w_off(int l)
{
    int64_t o = 0;
    for (int i = 0; i < l; ++i) o += int64_t(layer_k(i)) * kHid + kHid;
    return o;
}
__host__ __device__ inline int64_t param_count()
{
    return layer_w_off(kLayers);
}

// ---------------------------------------------------------------------------
// GEMM  C[M][N] = sum_k A(m, k) B(k, n), A(m, k) = A[m sam + k sak],
// B(k, n) = B[k sbk + n sbn] (BF16), FP32 accumulation on the tensor cores.
// Tiles 64 x 64 x 32, 4 warps of 32 x 32 (2 x 4 mma tiles of 16 x 8).
// Epilogues (the backward products of training):
//   EPI_STORE : C = acc + bias (FP32)
//   EPI_ATOMIC: C += acc (FP32 atomics; split reduction over k = blockIdx.z)
enum { EPI_STORE = 0, EPI_ATOMIC = 1 };
constexpr int BM = 64, BN = 64, BK = 32, PAD = 8;

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x)
{
    const float cdf = 0.5f * (1.0f + erff(x * 0.70710678118654752f));
    const float pdf = 0.39894228040143268f * expf(-0.5f * x * x);
    return cdf + x * pdf;
}

__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, const uint32_t* b)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <int EPI>
__global__ void __launch_bounds__(128)
k_gemm(int M, int N, int K, const __nv_bfloat16* __restrict__ A, int64_t sam, int64_t sak,
       const __nv_bfloat16* __restrict__ B, int64_t sbk, int64_t sbn, const float* __restrict__ bias,
       float* __restrict__ C, int64_t ldc, int k_chunk)
{
    __shared__ __align__(16) __nv_bfloat16 As[BM][BK + PAD];
    __shared__ __align__(16) __nv_bfloat16 Bs[BN][BK + PAD];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp >> 1, wn = warp & 1;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int kbeg = blockIdx.z * k_chunk;
    const int kend = min(K, kbeg + k_chunk);
    float acc[2][4][4] = {};
    const __nv_bfloat16 zero = __float2bfloat16(0.0f);
    for (int k0 = kbeg; k0 < kend; k0 += BK) {
        for (int idx = tid; idx < BM * BK; idx += 128) {
            const int m = idx / BK, k = idx % BK;
            const int gm = m0 + m, gk = k0 + k;
            As[m][k] = (gm < M && gk < kend) ? A[int64_t(gm) * sam + int64_t(gk) * sak] : zero;
        }
        for (int idx = tid; idx < BN * BK; idx += 128) {
            const int n = idx / BK, k = idx % BK;
            const int gn = n0 + n, gk = k0 + k;
            Bs[n][k] = (gn < N && gk < kend) ? B[int64_t(gk) * sbk + int64_t(gn) * sbn] : zero;
        }
        __syncthreads();
        const int r = lane >> 2, c = (lane & 3) * 2;
#pragma unroll
        for (int ks = 0; ks < BK; ks += 16) {
            uint32_t af[2][4], bf[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int row = wm * 32 + i * 16 + r;
                af[i][0] = *reinterpret_cast<const uint32_t*>(&As[row][ks + c]);
                af[i][1] = *reinterpret_cast<const uint32_t*>(&As[row + 8][ks + c]);
                af[i][2] = *reinterpret_cast<const uint32_t*>(&As[row][ks + c + 8]);
                af[i][3] = *reinterpret_cast<const uint32_t*>(&As[row + 8][ks + c + 8]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int col = wn * 32 + j * 8 + r;
                bf[j][0] = *reinterpret_cast<const uint32_t*>(&Bs[col][ks + c]);
                bf[j][1] = *reinterpret_cast<const uint32_t*>(&Bs[col][ks + c + 8]);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bf[j]);
        }
        __syncthreads();
    }
    const int r = lane >> 2, c = (lane & 3) * 2;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int gm = m0 + wm * 32 + i * 16 + r + (h >= 2 ? 8 : 0);
                const int gn = n0 + wn * 32 + j * 8 + c + (h & 1);
                if (gm >= M || gn >= N) continue;
                const float v = acc[i][j][h];
                if (EPI == EPI_ATOMIC) {
                    atomicAdd(&C[int64_t(gm) * ldc + gn], v);
                } else {
                    C[int64_t(gm) * ldc + gn] = v + (bias ? bias[gn] : 0.0f);
                }
            }
}

template <int EPI>
cudaError_t gemm(int M, int N, int K, const __nv_bfloat16* A, int64_t sam, int64_t sak,
                 const __nv_bfloat16* B, int64_t sbk, int64_t sbn, const float* bias, float* C,
                 int64_t ldc, int splits, cudaStream_t s)
{
    if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
    int chunk = (K + splits - 1) / splits;
    chunk = (chunk + BK - 1) / BK * BK;
    const int z = (K + chunk - 1) / chunk;
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, z);
    k_gemm<EPI><<<grid, 128, 0, s>>>(M, N, K, A, sam, sak, B, sbk, sbn, bias, C, ldc, chunk);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP32 master weights -> BF16 copies W [K][N], its transpose [N][K], and the
// transpose in the byte order of the forward kernel's shared-memory operand
// (canonical K-major layout of 8-row x 16-byte core matrices: element (n, k)
// of layer l at byte ((n/8) (K/8) + k/8) 128 + (n%8) 16 + (k%8) 2 of the
// layer's block), so that one bulk copy stages a layer.
__global__ void k_cast_weights(const float* __restrict__ p, __nv_bfloat16* __restrict__ w,
                               __nv_bfloat16* __restrict__ wt, __nv_bfloat16* __restrict__ wc)
{
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    int64_t o = 0, ob = 0;
    for (int l = 0; l < kLayers; ++l) {
        const int K = layer_k(l);
        const int64_t kn = int64_t(K) * kHid;
        if (i >= ob && i < ob + kn) {
            const int64_t e = i - ob;
            const int k = int(e / kHid), n = int(e % kHid);
            const __nv_bfloat16 v = __float2bfloat16(p[o + e]);
            w[ob + e] = v;
            wt[ob + int64_t(n) * K + k] = v;
            wc[ob + (((n >> 3) * (K >> 3) + (k >> 3)) * 64 + (n & 7) * 8 + (k & 7))] = v;
            return;
        }
        o += kn + kHid;
        ob += kn;
    }
}

// dy = 2 (y - t) / (M * N) (BF16 for the backward GEMMs); loss += sum (y - t)^2 / (M N)
__global__ void k_mse(const float* __restrict__ y, const float* __restrict__ t, int64_t n, float scale,
                      __nv_bfloat16* __restrict__ dy, float* __restrict__ loss)
{
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    float l = 0.0f;
    if (i < n) {
        const float d = y[i] - t[i];
        dy[i] = __float2bfloat16(2.0f * d * scale);
        l = d * d * scale;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0 && l != 0.0f) atomicAdd(loss, l);
}

// da = dh * gelu'(pre) (BF16 out); dh given as FP32
__global__ void k_gelu_back(const float* __restrict__ dh, const float* __restrict__ pre, int64_t n,
                            __nv_bfloat16* __restrict__ da)
{
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) da[i] = __float2bfloat16(dh[i] * gelu_grad(pre[i]));
}

// db[n] += sum_m d[m][n], one thread per column summing the rows in order
// (no atomics: training is bitwise reproducible)
__global__ void k_bias_grad(const __nv_bfloat16* __restrict__ d, int M, int N, float* __restrict__ db)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.0f;
#pragma unroll 8
    for (int m = 0; m < M; ++m) s += __bfloat162float(d[int64_t(m) * N + n]);
    db[n] += s;
}

// AdamW on the FP32 master weights (biases not decayed).
__global__ void k_adamw(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                        float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps,
                        float wd, float c1, float c2)
{
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    // bias entries: the last kHid of every layer block
    bool is_bias = false;
    int64_t o = 0;
    for (int l = 0; l < kLayers; ++l) {
        const int64_t kn = int64_t(layer_k(l)) * kHid;
        if (i >= o + kn && i < o + kn + kHid) is_bias = true;
        o += kn + kHid;
    }
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float upd = (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] -= lr * (upd + (is_bias ? 0.0f : wd * p[i]));
}

// Seeded uniform(-a, a) initialisation (a = 1/sqrt(K), biases 0) from a
// counter-based hash (splitmix64) of (seed, index).
__global__ void k_init(float* __restrict__ p, uint64_t seed)
{
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    int64_t o = 0;
    for (int l = 0; l < kLayers; ++l) {
        const int64_t kn = int64_t(layer_k(l)) * kHid;
        if (i >= o && i < o + kn + kHid) {
            if (i >= o + kn) { p[i] = 0.0f; return; }
            uint64_t z = seed + 0x9e3779b97f4a7c15ull * uint64_t(i + 1);
            z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
            z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
            z ^= z >> 31;
            const float u = float(z >> 40) * (1.0f / 16777216.0f);   // [0, 1)
            const float a = rsqrtf(float(layer_k(l)));
            p[i] = (2.0f * u - 1.0f) * a;
            return;
        }
        o += kn + kHid;
    }
}

struct MlpWork {
    __nv_bfloat16 *w, *wt, *wc;            // BF16 weights, transposes, forward-operand order
    float* pre[kLayers];                    // pre-activations (FP32) [M][256]
    __nv_bfloat16* h[kLayers];              // activations (BF16) [M][256]; h[4] unused
    __nv_bfloat16 *dy, *da;                 // BF16 gradients [M][256]
    float* dh;                              // FP32 [M][256]
    float* grad;                            // FP32 [param_count]
    float* loss;                            // FP32 scalar
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

size_t mlp_work_bytes(int64_t M, MlpWork* w, char* base)
{
    size_t o = 0;
    auto take = [&](size_t b) { size_t at = o; o = align256(o + b); return base ? base + at : nullptr; };
    const int64_t nw = param_count() - int64_t(kLayers) * kHid;   // weights only
    char* p;
    p = take(sizeof(__nv_bfloat16) * nw); if (w) w->w = (__nv_bfloat16*)p;
    p = take(sizeof(__nv_bfloat16) * nw); if (w) w->wt = (__nv_bfloat16*)p;
    p = take(sizeof(__nv_bfloat16) * nw); if (w) w->wc = (__nv_bfloat16*)p;
    for (int l = 0; l < kLayers; ++l) {
        p = take(sizeof(float) * M * kHid); if (w) w->pre[l] = (float*)p;
        p = take(sizeof(__nv_bfloat16) * M * kHid); if (w) w->h[l] = (__nv_bfloat16*)p;
    }
    p = take(sizeof(__nv_bfloat16) * M * kHid); if (w) w->dy = (__nv_bfloat16*)p;
    p = take(sizeof(__nv_bfloat16) * M * kHid); if (w) w->da = (__nv_bfloat16*)p;
    p = take(sizeof(float) * M * kHid); if (w) w->dh = (float*)p;
    p = take(sizeof(float) * param_count()); if (w) w->grad = (float*)p;
    p = take(sizeof(float)); if (w) w->loss = (float*)p;
    return o;
}

int64_t wofs(int l)   // offset of W_l in the BF16 weight arrays
{
    int64_t o = 0;
    for (int i = 0; i < l; ++i) o += int64_t(layer_k(i)) * kHid;
    return o;
}

// ---------------------------------------------------------------------------
// Forward pass on the 5th-generation tensor cores (tcgen05): one CTA of 256
// threads per 128 rows runs all five layers.  Per layer one bulk copy
// (cp.async.bulk, completion on an mbarrier) stages the layer's BF16 weights
// W_l^T [256][K], already in the operand's byte order, in shared memory; one
// thread issues K/16 tcgen05.mma (M = 128, N = 256, K = 16, BF16 in, FP32
// out) into 256 TMEM columns and commits them to a second mbarrier; the next
// layer's weight copy then starts at once and overlaps the epilogue, in which
// the eight warps read the accumulators back with tcgen05.ld (warp w: TMEM
// lanes = rows 32 (w mod 4) ..., columns 128 (w / 4) ...): + bias, GELU, BF16
// into shared memory as the next layer's input, or FP32 rows of the output
// after the last layer.
//
// Shared-memory operands use the canonical K-major layout without swizzling:
// 8-row x 16-byte core matrices, core matrix (r/8, k/8) at ((r/8) (K/8) + k/8)
// x 128 bytes, so the descriptor's K step between core matrices (leading byte
// offset) is 128 B and its row-group step (stride byte offset) K/8 x 128 B.
namespace tc {

constexpr int kRows = 128;            // rows per CTA = MMA M = TMEM lanes
constexpr int kThreads = 256;
constexpr uint32_t kCols = 256;       // TMEM columns: one FP32 accumulator per output
// instruction descriptor of kind::f16: D FP32 (bits 4-5 = 1), A and B BF16
// (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bit 17,
// M >> 4 at bit 24
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t(kHid) >> 3) << 17) |
                            ((uint32_t(kRows) >> 4) << 24);
constexpr int kWaitLimit = 1 << 22;   // mbarrier polls before the CTA gives up

struct Smem {
    unsigned char a[kRows * kHid * 2];   // input rows, canonical layout
    unsigned char b[kHid * kHid * 2];    // W_l^T, canonical layout
    unsigned long long bar_mma, bar_w;
    uint32_t tmem;
};
constexpr size_t kSmemBytes = sizeof(Smem) + 1024;   // + alignment of the operands

struct Args {
    const float* params;
    const __nv_bfloat16* wc;              // BF16 W_l^T in operand order, layers back to back
    const __nv_bfloat16* x;               // [M][32]
    int M;
    float* out;                           // last layer's pre-activation [M][256]
    float* pre[kLayers - 1];              // hidden pre-activations [M][256], or null
    __nv_bfloat16* h[kLayers - 1];        // hidden activations [M][256], or null
};

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint32_t canon(int row, int kg, int KG)
{
    return uint32_t(((row >> 3) * KG + kg) * 128 + (row & 7) * 16);
}
// shared-memory descriptor: start, leading byte offset (K), stride byte offset
// (rows), bits 46-47 = 1 (tcgen05 descriptor version), no swizzle
__device__ __forceinline__ uint64_t desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return uint64_t((saddr >> 4) & 0x3FFFu) | (uint64_t((lbo >> 4) & 0x3FFFu) << 16) |
           (uint64_t((sbo >> 4) & 0x3FFFu) << 32) | (uint64_t(1) << 46);
}
__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t parity)
{
    for (int it = 0; it < kWaitLimit; ++it) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done) : "r"(bar), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}
// layer l's weights (bytes, 16-byte aligned at both ends) into b, completing on bar
__device__ __forceinline__ void copy_weights(uint32_t sb, const __nv_bfloat16* src, uint32_t bytes,
                                             uint32_t bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 :: "r"(bar), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(sb), "l"(src), "r"(bytes), "r"(bar) : "memory");
}
__device__ __forceinline__ void ld16(uint32_t taddr, uint32_t* r)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                 "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                   "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                   "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

}  // namespace tc

__global__ void __launch_bounds__(tc::kThreads, 1) k_mlp_forward_tc(tc::Args g)
{
    extern __shared__ unsigned char smem_raw[];
    tc::Smem& S = *reinterpret_cast<tc::Smem*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quarter = warp & 3, half = warp >> 2;
    const int m0 = blockIdx.x * tc::kRows;
    const uint32_t bar_mma = tc::smem_u32(&S.bar_mma), bar_w = tc::smem_u32(&S.bar_w);
    const uint32_t sa = tc::smem_u32(S.a), sb = tc::smem_u32(S.b);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bar_mma) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bar_w) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(tc::smem_u32(&S.tmem)), "r"(tc::kCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = S.tmem;
    // layer 0's weights in flight while the input rows are staged
    if (tid == 0) tc::copy_weights(sb, g.wc, uint32_t(kIn * kHid * 2), bar_w);
    for (int c = tid; c < tc::kRows * kIn; c += tc::kThreads) {
        const int r = c / kIn, k = c - r * kIn;
        const __nv_bfloat16 v = m0 + r < g.M ? g.x[int64_t(m0 + r) * kIn + k]
                                             : __float2bfloat16(0.0f);
        *reinterpret_cast<__nv_bfloat16*>(S.a + tc::canon(r, k >> 3, kIn / 8) + (k & 7) * 2) = v;
    }
    const int row = quarter * 32 + lane, grow = m0 + row;   // this thread's TMEM lane and row
    bool ok = true;
    uint32_t phase = 0;            // completions seen on each barrier (one per layer)
    bool copy_pending = true;      // a weight copy issued and not yet waited for
    bool mma_pending = false;      // MMAs committed and not yet waited for
    int64_t wo = 0;                // offset of W_l^T in wc
    for (int l = 0; l < kLayers && ok; ++l) {
        const int K = layer_k(l), KG = K / 8;
        // generic-proxy writes of the input rows, visible to the tensor core
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            ok = tc::wait_bar(bar_w, phase & 1);       // this layer's weights
            if (ok) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                for (int kk = 0; kk < K / 16; ++kk) {
                    const uint64_t ad = tc::desc(sa + kk * 256, 128, KG * 128);
                    const uint64_t bd = tc::desc(sb + kk * 256, 128, KG * 128);
                    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                                 :: "r"(tmem), "l"(ad), "l"(bd), "r"(tc::kIdesc), "r"(kk)
                                 : "memory");
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                             :: "r"(bar_mma) : "memory");
            }
        }
        ok = __syncthreads_and(ok);
        if (!ok) break;
        copy_pending = false;
        mma_pending = true;
        ok = __syncthreads_and(tc::wait_bar(bar_mma, phase & 1));
        if (!ok) break;
        mma_pending = false;
        ++phase;
        wo += int64_t(K) * kHid;
        // the MMAs are done with b: the next layer's weights stream in during the epilogue
        if (tid == 0 && l + 1 < kLayers)
            tc::copy_weights(sb, g.wc + wo, uint32_t(kHid * kHid * 2), bar_w);
        copy_pending = l + 1 < kLayers;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const float* bias = g.params + layer_w_off(l) + int64_t(K) * kHid;
        const bool last = l == kLayers - 1;
        for (int c0 = half * 128; c0 < half * 128 + 128; c0 += 16) {
            uint32_t r[16];
            tc::ld16(tmem + (uint32_t(quarter * 32) << 16) + uint32_t(c0), r);
            float y[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) y[j] = __uint_as_float(r[j]) + __ldg(bias + c0 + j);
            if (last) {
                if (grow < g.M) {
#pragma unroll
                    for (int j = 0; j < 16; j += 4)
                        *reinterpret_cast<float4*>(g.out + int64_t(grow) * kHid + c0 + j) =
                            make_float4(y[j], y[j + 1], y[j + 2], y[j + 3]);
                }
            } else {
                __align__(16) __nv_bfloat16 hb[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) hb[j] = __float2bfloat16(gelu(y[j]));
                *reinterpret_cast<uint4*>(S.a + tc::canon(row, c0 >> 3, kHid / 8)) =
                    *reinterpret_cast<const uint4*>(hb);
                *reinterpret_cast<uint4*>(S.a + tc::canon(row, (c0 >> 3) + 1, kHid / 8)) =
                    *reinterpret_cast<const uint4*>(hb + 8);
                if (g.pre[l] && grow < g.M) {
#pragma unroll
                    for (int j = 0; j < 16; j += 4)
                        *reinterpret_cast<float4*>(g.pre[l] + int64_t(grow) * kHid + c0 + j) =
                            make_float4(y[j], y[j + 1], y[j + 2], y[j + 3]);
                    *reinterpret_cast<uint4*>(g.h[l] + int64_t(grow) * kHid + c0) =
                        *reinterpret_cast<const uint4*>(hb);
                    *reinterpret_cast<uint4*>(g.h[l] + int64_t(grow) * kHid + c0 + 8) =
                        *reinterpret_cast<const uint4*>(hb + 8);
                }
            }
        }
        // every TMEM read done before the next layer's MMAs overwrite the columns
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    }
    if (!ok) {
        // a copy or an MMA that never signalled: wait once more (bounded) so
        // that nothing is in flight when the CTA exits, and mark its rows
        if (copy_pending) tc::wait_bar(bar_w, phase & 1);
        if (mma_pending) tc::wait_bar(bar_mma, phase & 1);
        if (grow < g.M)
            for (int c = half * 128; c < half * 128 + 128; ++c)
                g.out[int64_t(grow) * kHid + c] = __int_as_float(0x7fc00000);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                     :: "r"(tmem), "r"(tc::kCols) : "memory");
    }
}

// forward of M rows: x [M][32] BF16 -> out [M][256] FP32 (the last layer's
// pre-activation); without out (training) the result goes to w.pre[4] and the
// hidden layers' pre-activations and activations are kept for the backward
cudaError_t forward(const float* params, const __nv_bfloat16* x, int64_t M, float* out,
                    MlpWork& w, cudaStream_t s)
{
    cudaError_t e;
    const int64_t nw = param_count() - int64_t(kLayers) * kHid;
    k_cast_weights<<<int((nw + 255) / 256), 256, 0, s>>>(params, w.w, w.wt, w.wc);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_mlp_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  int(tc::kSmemBytes))) != cudaSuccess)
        return e;
    tc::Args g{};
    g.params = params;
    g.wc = w.wc;
    g.x = x;
    g.M = int(M);
    g.out = out ? out : w.pre[kLayers - 1];
    for (int l = 0; l < kLayers - 1; ++l) {
        g.pre[l] = out ? nullptr : w.pre[l];
        g.h[l] = out ? nullptr : w.h[l];
    }
    k_mlp_forward_tc<<<int((M + tc::kRows - 1) / tc::kRows), tc::kThreads, tc::kSmemBytes, s>>>(g);
    return cudaGetLastError();
}

// MSE gradient of M rows into grad (zeroed first) and loss (zeroed first).
cudaError_t grad_rows(const float* params, const __nv_bfloat16* xb, const float* target, int64_t M,
                      float* grad, float* loss, MlpWork& w, cudaStream_t s)
{
    if (forward(params, xb, M, nullptr, w, s) != cudaSuccess) return cudaErrorLaunchFailure;
    const int64_t nout = M * kHid;
    const int tb = 256;
    cudaError_t e;
    if ((e = cudaMemsetAsync(grad, 0, sizeof(float) * param_count(), s)) != cudaSuccess ||
        (e = cudaMemsetAsync(loss, 0, sizeof(float), s)) != cudaSuccess)
        return e;
    k_mse<<<int((nout + tb - 1) / tb), tb, 0, s>>>(w.pre[kLayers - 1], target, nout,
                                                   1.0f / float(nout), w.dy, loss);
    const __nv_bfloat16* d = w.dy;   // gradient w.r.t. the current layer's pre-activation
    const int splits = int(std::min<int64_t>(64, (M + 1023) / 1024));
    for (int l = kLayers - 1; l >= 0; --l) {
        const int K = layer_k(l);
        const __nv_bfloat16* in = l == 0 ? xb : w.h[l - 1];
        float* gW = grad + layer_w_off(l);
        float* gb = gW + int64_t(K) * kHid;
        // dW[k][n] = sum_m in[m][k] d[m][n]:  A(k, m) = in[m K + k], B(m, n) = d[m 256 + n]
        if ((e = gemm<EPI_ATOMIC>(K, kHid, int(M), in, 1, K, d, kHid, 1, nullptr, gW, kHid,
                                  splits, s)) != cudaSuccess)
            return e;
        k_bias_grad<<<(kHid + 63) / 64, 64, 0, s>>>(d, int(M), kHid, gb);
        if (l == 0) break;
        // dh[m][k] = sum_n d[m][n] W_l[k][n]:  B(n, k) = W_l[k][n] = w[k 256 + n]
        if ((e = gemm<EPI_STORE>(int(M), K, kHid, d, kHid, 1, w.w + wofs(l), 1, kHid, nullptr,
                                 w.dh, K, 1, s)) != cudaSuccess)
            return e;
        k_gelu_back<<<int((M * K + tb - 1) / tb), tb, 0, s>>>(w.dh, w.pre[l - 1], M * K, w.da);
        // the next step reads da while this one's d may alias it: swap buffers
        d = w.da;
        if (l - 1 > 0) {
            // keep d in da, use dy as the next gradient buffer
            __nv_bfloat16* t = w.dy;
            w.dy = w.da;
            w.da = t;
        }
    }
    return cudaGetLastError();
}

// rows perm[r0 .. r0 + n) of x and target into xb, tb
__global__ void k_gather_rows(const __nv_bfloat16* __restrict__ x, const float* __restrict__ t,
                              const int32_t* __restrict__ perm, int64_t r0, int64_t n,
                              __nv_bfloat16* __restrict__ xb, float* __restrict__ tb)
{
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n * kHid) return;
    const int64_t r = i / kHid, c = i % kHid;
    const int64_t src = perm[r0 + r];
    tb[i] = t[src * kHid + c];
    if (c < kIn) xb[r * kIn + c] = x[src * kIn + c];
}

// AdamW with bias corrections for step k (counting from 1)
cudaError_t adamw_step(float* params, const float* grad, float* m, float* v, int step, float lr,
                       float weight_decay, cudaStream_t s)
{
    const int64_t n = param_count();
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - powf(b1, float(step)), c2 = 1.0f - powf(b2, float(step));
    k_adamw<<<int((n + 255) / 256), 256, 0, s>>>(params, grad, m, v, n, lr, b1, b2, 1e-8f,
                                                 weight_decay, c1, c2);
    return cudaGetLastError();
}

// Workspace of paid_proposal_train: the permutation, one minibatch of inputs
// and targets, the per-step losses of an epoch, the gradient and the forward /
// backward buffers of one minibatch.
struct TrainWork {
    int32_t* perm;
    __nv_bfloat16* xb;
    float* tb;
    float* losses;
    float* grad;
    char* mlp;
};

size_t train_work_bytes(int64_t M, int64_t batch, TrainWork* t, char* base)
{
    size_t o = 0;
    auto take = [&](size_t b) { size_t at = o; o = align256(o + b); return base ? base + at : nullptr; };
    const int64_t steps = (M + batch - 1) / batch;
    char* p;
    p = take(sizeof(int32_t) * M); if (t) t->perm = (int32_t*)p;
    p = take(sizeof(__nv_bfloat16) * batch * kIn); if (t) t->xb = (__nv_bfloat16*)p;
    p = take(sizeof(float) * batch * kHid); if (t) t->tb = (float*)p;
    p = take(sizeof(float) * steps); if (t) t->losses = (float*)p;
    p = take(sizeof(float) * param_count()); if (t) t->grad = (float*)p;
    p = take(mlp_work_bytes(batch, nullptr, nullptr)); if (t) t->mlp = p;
    return o;
}

// splitmix64 (Steele, Lea and Flood), the seeded source of the minibatch order
uint64_t splitmix64(uint64_t& z)
{
    uint64_t r = (z += 0x9e3779b97f4a7c15ull);
    r = (r ^ (r >> 30)) * 0xbf58476d1ce4e5b9ull;
    r = (r ^ (r >> 27)) * 0x94d049bb133111ebull;
    return r ^ (r >> 31);
}

constexpr char kMagic[8] = {'P', 'A', 'I', 'D', 'M', 'L', 'P', '1'};

bool aligned(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

}  // namespace

extern "C" {

int paid_mlp_param_count(int64_t* n)
{
    if (!n) return PAID_ERR_ARG;
    *n = param_count();
    return PAID_OK;
}

int paid_mlp_workspace_size(int64_t M, size_t* bytes)
{
    if (!bytes || M < 0) return PAID_ERR_ARG;
    *bytes = mlp_work_bytes(M, nullptr, nullptr);
    return PAID_OK;
}

int paid_mlp_init(float* params, uint64_t seed, void* stream)
{
    if (!params) return PAID_ERR_ARG;
    const int64_t n = param_count();
    k_init<<<int((n + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(params, seed);
    return cudaGetLastError() == cudaSuccess ? PAID_OK : PAID_ERR_CUDA;
}

int paid_mlp_forward(const float* params, const uint16_t* x, int64_t M, float* out, void* workspace,
                     size_t ws_bytes, void* stream)
{
    if (!params || (M > 0 && (!x || !out)) || M < 0) return PAID_ERR_ARG;
    if (M == 0) return PAID_OK;
    // the forward kernel stores output rows as 16-byte vectors and stages
    // weights with bulk copies from the workspace (16-byte aligned blocks)
    if (!aligned(out, 16) || !aligned(workspace, 256)) return PAID_ERR_ARG;
    if (M > int64_t(0x7fffffff)) return PAID_ERR_ARG;
    if (!workspace || ws_bytes < mlp_work_bytes(M, nullptr, nullptr)) return PAID_ERR_OOM;
    MlpWork w;
    mlp_work_bytes(M, &w, static_cast<char*>(workspace));
    return forward(params, reinterpret_cast<const __nv_bfloat16*>(x), M, out, w,
                   static_cast<cudaStream_t>(stream)) == cudaSuccess ? PAID_OK : PAID_ERR_CUDA;
}

int paid_mlp_grad(const float* params, const uint16_t* x, const float* target, int64_t M,
                  float* grad, float* loss, void* workspace, size_t ws_bytes, void* stream)
{
    if (!params || !x || !target || !grad || !loss || M <= 0) return PAID_ERR_ARG;
    if (M > int64_t(0x7fffffff)) return PAID_ERR_ARG;
    if (!aligned(workspace, 256)) return PAID_ERR_ARG;
    if (!workspace || ws_bytes < mlp_work_bytes(M, nullptr, nullptr)) return PAID_ERR_OOM;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    MlpWork w;
    mlp_work_bytes(M, &w, static_cast<char*>(workspace));
    return grad_rows(params, reinterpret_cast<const __nv_bfloat16*>(x), target, M, grad, loss, w,
                     s) == cudaSuccess ? PAID_OK : PAID_ERR_CUDA;
}

int paid_mlp_adamw(float* params, const float* grad, float* m, float* v, int step, float lr,
                   float weight_decay, void* stream)
{
    if (!params || !grad || !m || !v || step < 1) return PAID_ERR_ARG;
    return adamw_step(params, grad, m, v, step, lr, weight_decay,
                      static_cast<cudaStream_t>(stream)) == cudaSuccess ? PAID_OK : PAID_ERR_CUDA;
}

int paid_proposal_train_workspace_size(int64_t M, int64_t batch, size_t* bytes)
{
    if (!bytes || M <= 0 || batch <= 0 || M > int64_t(0x7fffffff)) return PAID_ERR_ARG;
    *bytes = train_work_bytes(M, std::min(M, batch), nullptr, nullptr);
    return PAID_OK;
}

int paid_proposal_train(float* params, float* m, float* v, const uint16_t* x, const float* target,
                        int64_t M, int epochs, int64_t batch, float lr, float weight_decay,
                        uint64_t seed, int* step, float* epoch_loss, void* workspace,
                        size_t ws_bytes, void* stream)
{
    if (!params || !m || !v || !x || !target || !step || *step < 0 || M <= 0 || epochs < 0 ||
        batch <= 0 || M > int64_t(0x7fffffff) || !(lr >= 0.0f) || !(weight_decay >= 0.0f))
        return PAID_ERR_ARG;
    batch = std::min(M, batch);
    if (!aligned(workspace, 256)) return PAID_ERR_ARG;
    if (!workspace || ws_bytes < train_work_bytes(M, batch, nullptr, nullptr)) return PAID_ERR_OOM;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    TrainWork t;
    train_work_bytes(M, batch, &t, static_cast<char*>(workspace));
    MlpWork w;
    mlp_work_bytes(batch, &w, t.mlp);
    const __nv_bfloat16* xb = reinterpret_cast<const __nv_bfloat16*>(x);
    const int64_t steps = (M + batch - 1) / batch;
    const int64_t total = steps * int64_t(epochs);
    std::vector<int32_t> perm(static_cast<size_t>(M));
    std::vector<float> losses(static_cast<size_t>(steps));
    uint64_t z = seed;
    int64_t k = 0;
    for (int ep = 0; ep < epochs; ++ep) {
        // a fresh Fisher-Yates order of the rows for every epoch
        for (int64_t i = 0; i < M; ++i) perm[size_t(i)] = int32_t(i);
        for (int64_t i = M - 1; i > 0; --i) {
            const int64_t j = int64_t(splitmix64(z) % uint64_t(i + 1));
            std::swap(perm[size_t(i)], perm[size_t(j)]);
        }
        // the host order is copied before this call returns control (pageable
        // source), so the vector may be refilled for the next epoch
        if (cudaMemcpyAsync(t.perm, perm.data(), sizeof(int32_t) * M, cudaMemcpyHostToDevice, s) !=
            cudaSuccess)
            return PAID_ERR_CUDA;
        for (int64_t b = 0; b < steps; ++b, ++k) {
            const int64_t r0 = b * batch, n = std::min(batch, M - r0);
            k_gather_rows<<<int((n * kHid + 255) / 256), 256, 0, s>>>(xb, target, t.perm, r0, n,
                                                                     t.xb, t.tb);
            // cosine decay of the learning rate over all steps of the call
            const float a = lr * 0.5f * (1.0f + cosf(3.14159265358979f * float(k) /
                                                     float(std::max<int64_t>(1, total))));
            if (grad_rows(params, t.xb, t.tb, n, t.grad, t.losses + b, w, s) != cudaSuccess ||
                adamw_step(params, t.grad, m, v, *step + 1, a, weight_decay, s) != cudaSuccess)
                return PAID_ERR_CUDA;
            ++*step;
        }
        if (epoch_loss) {
            if (cudaMemcpyAsync(losses.data(), t.losses, sizeof(float) * steps,
                                cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess)
                return PAID_ERR_CUDA;
            double sum = 0.0;
            for (float l : losses) sum += l;
            epoch_loss[ep] = float(sum / double(steps));
        }
    }
    return cudaGetLastError() == cudaSuccess ? PAID_OK : PAID_ERR_CUDA;
}

int paid_proposal_save(const float* params, const char* path, void* stream)
{
    if (!params || !path) return PAID_ERR_ARG;
    const int64_t n = param_count();
    std::vector<float> h(static_cast<size_t>(n));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(h.data(), params, sizeof(float) * n, cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return PAID_ERR_CUDA;
    FILE* f = std::fopen(path, "wb");
    if (!f) return PAID_ERR_ARG;
    const bool ok = std::fwrite(kMagic, 1, 8, f) == 8 && std::fwrite(&n, sizeof(n), 1, f) == 1 &&
                    std::fwrite(h.data(), sizeof(float), size_t(n), f) == size_t(n);
    return (std::fclose(f) == 0 && ok) ? PAID_OK : PAID_ERR_ARG;
}

int paid_proposal_load(float* params, const char* path, void* stream)
{
    if (!params || !path) return PAID_ERR_ARG;
    FILE* f = std::fopen(path, "rb");
    if (!f) return PAID_ERR_ARG;
    char magic[8] = {};
    int64_t n = 0;
    const int64_t want = param_count();
    std::vector<float> h(static_cast<size_t>(want));
    const bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kMagic, 8) == 0 &&
                    std::fread(&n, sizeof(n), 1, f) == 1 && n == want &&
                    std::fread(h.data(), sizeof(float), size_t(n), f) == size_t(n) &&
                    std::fgetc(f) == EOF;
    std::fclose(f);
    if (!ok) return PAID_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the host copy lives on this call's stack: wait for the upload
    if (cudaMemcpyAsync(params, h.data(), sizeof(float) * n, cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return PAID_ERR_CUDA;
    return PAID_OK;
}

}  // extern "C"
