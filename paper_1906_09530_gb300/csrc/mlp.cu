// mlp.cu -- the surrogate network of the warm start (lbm_mlp_* of
// include/cplbm.h): a 3-256-256-256-256 multilayer perceptron with tanh hidden
// layers that maps (T_r, kappa-hat, k) to a 256-point equilibrium interface
// profile, trained and evaluated by the kernels of this file.
//
// Arithmetic: every matrix product runs on the tensor cores in BF16 with FP32
// accumulation; master weights, Adam moments, biases, activations kept for the
// backward pass, and the loss are FP32 (the loss sum FP64).  The products:
//   forward            Z_l   = A_{l-1} W_l          [B x fan_in] [fan_in x fan_out]
//   weight gradient    dW_l  = A_{l-1}^T D_l        [fan_in x B] [B x fan_out]
//   input gradient     D_{l-1} = (D_l W_l^T) (1 - A_{l-1}^2)
// with fused epilogues (bias + tanh, tanh derivative).  The forward and
// input-gradient products have 256 output columns and a batch of rows: they run
// as tcgen05 MMAs of 128 x 256 x 16 with the accumulator in tensor memory and
// the operands brought in by tensor copies (k_gemm_umma).  The weight gradient,
// whose K is the batch, and any product whose tensor map cannot be made, use the
// strided mma.sync tile kernel (k_gemm), which stages its operands in shared
// memory with the K index contiguous.
#include <cuda.h>  // CUtensorMap and its encoder's types (the encoder is fetched at run time)
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <new>
#include <utility>
#include <vector>

#include "cplbm_internal.cuh"

namespace cplbm {
namespace {

constexpr int kIn = 3, kW = 256, kOut = 256, kLayers = 4;
constexpr int kInPad = 16;  // the first product's K, padded to one mma k-step
constexpr int kFanIn[kLayers] = {kIn, kW, kW, kW};
constexpr int kFanOut[kLayers] = {kW, kW, kW, kOut};

// offset of W_l in the parameter vector (W_l then b_l, layer after layer);
// closed form on scalar constants, so device code can evaluate it too
__host__ __device__ constexpr long long param_offset(int l) {
    static_assert(kOut == kW, "the output layer has the hidden width");
    return l == 0 ? 0 : (long long)(kIn * kW + kW) + (long long)(l - 1) * (kW * kW + kW);
}
constexpr long long kParams = param_offset(kLayers);

// ---------------------------------------------------------------------------
// GEMM: C[m][n] = sum_k A(m, k) B(k, n), A(m, k) = A[m sam + k sak],
// B(k, n) = B[k sbk + n sbn], BF16 operands, FP32 accumulation.  Block tile
// 64 x 64 x 16, four warps of 32 x 32 (2 x 4 mma tiles of 16 x 8).
// ---------------------------------------------------------------------------
constexpr int BM = 64, BN = 64, BK = 16, KP = BK + 8;  // KP: padded shared row

enum Epi : int {
    EPI_STORE = 0,      // out32[m][n] = acc
    EPI_BIAS_TANH = 1,  // a = tanh(acc + bias[n]): out32 = a, out16 = bf16(a)
    EPI_BIAS = 2,       // out32 = acc + bias[n]
    EPI_TANH_BACK = 3,  // d = acc (1 - aprev[m][n]^2): out32 = d, out16 = bf16(d)
};

struct GemmArgs {
    const __nv_bfloat16* A;
    long long sam, sak;
    const __nv_bfloat16* B;
    long long sbk, sbn;
    int M, N, K;
    int epi;
    const float* bias;   // [N]
    const float* aprev;  // [M][N] (EPI_TANH_BACK)
    float* out32;        // [M][N], row-major, leading dimension N
    __nv_bfloat16* out16;
    int ld16;            // leading dimension of out16
};

__device__ __forceinline__ void mma_bf16(float c[4], const unsigned a[4], const unsigned b[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__global__ void __launch_bounds__(128) k_gemm(GemmArgs g) {
    __shared__ __align__(16) __nv_bfloat16 As[BM][KP];  // [m][k]
    __shared__ __align__(16) __nv_bfloat16 Bs[BN][KP];  // [n][k]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp >> 1, wn = warp & 1;
    const int gq = lane >> 2, tq = lane & 3;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.0f;
    const __nv_bfloat16 zero = __float2bfloat16_rn(0.0f);
    for (int k0 = 0; k0 < g.K; k0 += BK) {
        // stage: 64 x 16 of A and of B, element by element (out of range: 0)
        for (int e = tid; e < BM * BK; e += 128) {
            const int r = e / BK, k = e - r * BK;
            const int m = m0 + r, kk = k0 + k;
            As[r][k] = (m < g.M && kk < g.K) ? g.A[m * g.sam + kk * g.sak] : zero;
            const int n = n0 + r;
            Bs[r][k] = (n < g.N && kk < g.K) ? g.B[kk * g.sbk + n * g.sbn] : zero;
        }
        __syncthreads();
        unsigned a[2][4], b[4][2];
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int r = wm * 32 + i * 16 + gq;
            a[i][0] = *reinterpret_cast<const unsigned*>(&As[r][2 * tq]);
            a[i][1] = *reinterpret_cast<const unsigned*>(&As[r + 8][2 * tq]);
            a[i][2] = *reinterpret_cast<const unsigned*>(&As[r][2 * tq + 8]);
            a[i][3] = *reinterpret_cast<const unsigned*>(&As[r + 8][2 * tq + 8]);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = wn * 32 + j * 8 + gq;
            b[j][0] = *reinterpret_cast<const unsigned*>(&Bs[n][2 * tq]);
            b[j][1] = *reinterpret_cast<const unsigned*>(&Bs[n][2 * tq + 8]);
        }
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], a[i], b[j]);
        __syncthreads();
    }
    // epilogue: accumulator (i, j, q) is row m0 + wm 32 + i 16 + gq (+8 for
    // q >= 2), column n0 + wn 32 + j 8 + 2 tq (+1 for odd q)
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int m = m0 + wm * 32 + i * 16 + gq + (q >= 2 ? 8 : 0);
                const int n = n0 + wn * 32 + j * 8 + 2 * tq + (q & 1);
                if (m >= g.M || n >= g.N) continue;
                float v = acc[i][j][q];
                const long long o = (long long)m * g.N + n;
                if (g.epi == EPI_BIAS_TANH) {
                    v = tanhf(v + g.bias[n]);
                    g.out16[(long long)m * g.ld16 + n] = __float2bfloat16_rn(v);
                } else if (g.epi == EPI_BIAS) {
                    v += g.bias[n];
                } else if (g.epi == EPI_TANH_BACK) {
                    const float ap = g.aprev[o];
                    v *= 1.0f - ap * ap;
                    g.out16[(long long)m * g.ld16 + n] = __float2bfloat16_rn(v);
                }
                g.out32[o] = v;
            }
}

// ---------------------------------------------------------------------------
// Tensor-core products on tcgen05 (5th-generation tensor cores, accumulator in
// tensor memory): D[M x 256] = A[M x K] Bt[256 x K]^T, K = 16 or 256, BF16
// operands, FP32 accumulation, with the epilogues of k_gemm.  They serve the
// forward products (A = the layer input, Bt = the transposed weights) and the
// input gradients (A = the backward signal, Bt = the weights as stored).
//
// A CTA of 4 warps owns 128 rows and all 256 columns.  Both operands are moved
// into shared memory by tensor copies (TMA) in the K-major, unswizzled layout of
// the tensor cores: core matrices of 8 rows x 8 elements (128 bytes), K-adjacent
// core matrices 128 bytes apart, row-adjacent ones K/8 x 128 bytes apart.  A
// 4-D tensor map (8 elements, 8 rows, K/8, rows/8) writes exactly that order.
// One thread issues the K/16 MMAs of shape 128 x 256 x 16 into a 256-column
// accumulator and commits them to an mbarrier; after a bounded wait each warp
// reads its 32 rows back with tcgen05.ld and applies the epilogue.  A wait that
// runs out sets the error word and the CTA frees its tensor memory and leaves.
// ---------------------------------------------------------------------------
constexpr int UM = 128, UN = 256;
constexpr unsigned kUmmaSpins = 1u << 22;

struct UmmaArgs {
    int M, K;
    int epi;
    const float* bias;   // [256]
    const float* aprev;  // [M][256] (EPI_TANH_BACK)
    float* out32;        // [M][256]
    __nv_bfloat16* out16;
    int ld16;
    int* err;            // set to 1 when a wait runs out
};

__device__ __forceinline__ unsigned su32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ bool umma_try_wait(uint64_t* bar) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(su32(bar))
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool umma_wait(uint64_t* bar) {
    for (unsigned i = 0; i < kUmmaSpins; ++i)
        if (umma_try_wait(bar)) return true;
    return false;
}
// shared-memory matrix descriptor: start address, leading (K-adjacent) and
// stride (row-adjacent) byte offsets, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t umma_desc(unsigned addr, unsigned lbo, unsigned sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

__global__ void __launch_bounds__(128, 1)
    k_gemm_umma(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb,
                UmmaArgs g) {
    extern __shared__ __align__(1024) unsigned char usm[];
    unsigned char* As = usm;                          // UM x K bf16
    unsigned char* Bs = usm + (size_t)UM * g.K * 2;   // UN x K bf16
    __shared__ __align__(8) uint64_t bar[2];          // [0] operands arrived, [1] MMAs done
    __shared__ uint32_t tbase;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * UM;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         su32(&tbase)),
                     "r"(UN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(su32(&bar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(su32(&bar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tbase;
    const int KG = g.K / 8;
    if (tid == 0) {
        const unsigned bytes = (unsigned)((UM + UN) * g.K * 2);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(
                         su32(&bar[0])),
                     "r"(bytes)
                     : "memory");
        asm volatile(
            "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
            " [%0], [%1, {%2, %3, %4, %5}], [%6];\n" ::"r"(su32(As)),
            "l"(reinterpret_cast<uint64_t>(&ta)), "r"(0), "r"(0), "r"(0), "r"(m0 / 8),
            "r"(su32(&bar[0]))
            : "memory");
        asm volatile(
            "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
            " [%0], [%1, {%2, %3, %4, %5}], [%6];\n" ::"r"(su32(Bs)),
            "l"(reinterpret_cast<uint64_t>(&tb)), "r"(0), "r"(0), "r"(0), "r"(0),
            "r"(su32(&bar[0]))
            : "memory");
    }
    bool ok = umma_wait(&bar[0]);
    ok = __syncthreads_and(ok) != 0;
    bool mma_issued = false;
    if (ok) {
        // D f32 (bits 4-5), A and B bf16 (7-9, 10-12), both K-major, N >> 3 at bit 17,
        // M >> 4 at bit 24
        const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) |
                               ((uint32_t)(UN >> 3) << 17) | ((uint32_t)(UM >> 4) << 24);
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            for (int ks = 0; ks < g.K / 16; ++ks) {
                const uint64_t da = umma_desc(su32(As) + ks * 256, 128, KG * 128);
                const uint64_t db = umma_desc(su32(Bs) + ks * 256, 128, KG * 128);
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(da), "l"(db), "r"(idesc), "r"(ks > 0 ? 1u : 0u)
                    : "memory");
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::
                    "r"(su32(&bar[1]))
                : "memory");
        }
        mma_issued = true;
        ok = umma_wait(&bar[1]);
        ok = __syncthreads_and(ok) != 0;
    }
    if (!ok) {
        // a copy or the MMAs never completed: report, give what is in flight one
        // more bounded wait, free the tensor memory and leave
        if (tid == 0) atomicExch(g.err, 1);
        umma_wait(&bar[0]);
        if (mma_issued) umma_wait(&bar[1]);
    }
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (ok) {
        const int row = m0 + warp * 32 + lane;
        const bool live = row < g.M;
        for (int c = 0; c < UN; c += 8) {
            uint32_t v[8];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                  "=r"(v[6]), "=r"(v[7])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
            if (!live) continue;
            float o[8];
            __nv_bfloat16 h[8];
            const long long base = (long long)row * UN + c;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                float x = __uint_as_float(v[j]);
                if (g.epi == EPI_BIAS_TANH) {
                    x = tanhf(x + g.bias[c + j]);
                } else if (g.epi == EPI_BIAS) {
                    x += g.bias[c + j];
                } else if (g.epi == EPI_TANH_BACK) {
                    const float ap = g.aprev[base + j];
                    x *= 1.0f - ap * ap;
                }
                o[j] = x;
                h[j] = __float2bfloat16_rn(x);
            }
            float4* o4 = reinterpret_cast<float4*>(g.out32 + base);
            o4[0] = make_float4(o[0], o[1], o[2], o[3]);
            o4[1] = make_float4(o[4], o[5], o[6], o[7]);
            if (g.out16 && (g.epi == EPI_BIAS_TANH || g.epi == EPI_TANH_BACK))
                *reinterpret_cast<uint4*>(g.out16 + (long long)row * g.ld16 + c) =
                    *reinterpret_cast<const uint4*>(h);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                     "r"(UN)
                     : "memory");
}

// x [B][3] FP32 -> BF16 [B][16], zero-padded
__global__ void k_input(const float* __restrict__ x, __nv_bfloat16* __restrict__ x16, int B) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * kInPad) return;
    const int b = i / kInPad, k = i - b * kInPad;
    x16[i] = __float2bfloat16_rn(k < kIn ? x[b * kIn + k] : 0.0f);
}

// FP32 master weights -> BF16 copies ([fan_in padded][fan_out] for layer 0),
// and the same transposed ([fan_out][fan_in padded]) for the tensor-core
// products, whose second operand is K-major
__global__ void k_weights16(const float* __restrict__ p, __nv_bfloat16* __restrict__ w16,
                            __nv_bfloat16* __restrict__ w16t) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long n16 = (long long)kInPad * kW + 3LL * kW * kW;
    if (i >= n16) return;
    if (i < (long long)kInPad * kW) {
        const int k = (int)(i / kW), n = (int)(i - (long long)k * kW);
        const __nv_bfloat16 v = __float2bfloat16_rn(k < kIn ? p[k * kW + n] : 0.0f);
        w16[i] = v;
        w16t[(long long)n * kInPad + k] = v;
        return;
    }
    const long long j = i - (long long)kInPad * kW;  // layers 1..3
    const int l = 1 + (int)(j / (kW * kW));
    const long long r = j - (long long)(l - 1) * kW * kW;
    const int k = (int)(r / kW), n = (int)(r - (long long)k * kW);
    const __nv_bfloat16 v = __float2bfloat16_rn(p[param_offset(l) + r]);
    w16[i] = v;
    w16t[(long long)kInPad * kW + (long long)(l - 1) * kW * kW + (long long)n * kW + k] = v;
}

// dL/dy = 2 (y - t) / (B N) (FP32 and BF16), and the squared-error sum
__global__ void k_loss_grad(const float* __restrict__ y, const float* __restrict__ t, int total,
                            float scale, float* __restrict__ d32, __nv_bfloat16* __restrict__ d16,
                            double* __restrict__ sse) {
    __shared__ double red[256];
    double s = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const float e = y[i] - t[i];
        const float d = 2.0f * e * scale;
        d32[i] = d;
        d16[i] = __float2bfloat16_rn(d);
        s += (double)e * e;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(sse, red[0]);
}

// column sums: db[n] = sum_b d[b][n]
__global__ void k_bias_grad(const float* __restrict__ d, int B, int N, float* __restrict__ db) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.0f;
    for (int b = 0; b < B; ++b) s += d[(long long)b * N + n];
    db[n] = s;
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, long long n, float lr, float c1, float c2) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

}  // namespace
}  // namespace cplbm

using namespace cplbm;

struct lbm_mlp {
    int dev, max_batch;
    cudaStream_t stream;
    float *p, *g, *m, *v;        // FP32 parameters, gradient, Adam moments
    __nv_bfloat16* w16;          // BF16 weight copies, layer by layer ([fan_in][fan_out])
    __nv_bfloat16* w16t;         // the same transposed ([fan_out][fan_in]; fan_in 16 for layer 0)
    int* err;                    // device word: a tensor-core product's wait ran out
    int* h_err;                  // pinned mirror
    __nv_bfloat16* x16;          // [max_batch][16]
    float* a32[kLayers];         // layer outputs, FP32 [B][256]
    __nv_bfloat16* a16[kLayers - 1];  // hidden outputs, BF16 (inputs of the next product)
    float* d32;                  // backward signal, FP32 [B][256]
    __nv_bfloat16* d16;          // its BF16 copy
    float* e32;                  // the previous layer's signal
    __nv_bfloat16* e16;
    double* sse;                 // device scalar
    double* h_sse;               // pinned mirror
    long long step;
    bool tensor_cores;           // forward and input-gradient products by tcgen05
};

namespace {

size_t al(size_t v) { return (v + 255) / 256 * 256; }

struct MlpLayout {
    size_t p, g, m, v, w16, w16t, x16, a32, a16, d32, d16, e32, e16, sse, err, total;
};

// Rows of the batch-sized buffers: a multiple of 8, so that the tensor copies of
// 8-row core matrices stay inside the buffers.
int rows_of(int B) { return (B + 7) / 8 * 8; }

MlpLayout mlp_layout(int B0) {
    const int B = rows_of(B0);
    MlpLayout L;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o += al(bytes);
        return at;
    };
    L.p = take(kParams * 4);
    L.g = take(kParams * 4);
    L.m = take(kParams * 4);
    L.v = take(kParams * 4);
    L.w16 = take(((size_t)kInPad * kW + 3ull * kW * kW) * 2);
    L.w16t = take(((size_t)kInPad * kW + 3ull * kW * kW) * 2);
    L.x16 = take((size_t)B * kInPad * 2);
    L.a32 = take((size_t)kLayers * B * kW * 4);
    L.a16 = take((size_t)(kLayers - 1) * B * kW * 2);
    L.d32 = take((size_t)B * kW * 4);
    L.d16 = take((size_t)B * kW * 2);
    L.e32 = take((size_t)B * kW * 4);
    L.e16 = take((size_t)B * kW * 2);
    L.sse = take(8);
    L.err = take(4);
    L.total = o;
    return L;
}

#define CK(call)                                  \
    do {                                          \
        cudaError_t e_ = (call);                  \
        if (e_ != cudaSuccess) return LBM_ECUDA;  \
    } while (0)

cudaError_t gemm(const GemmArgs& g, cudaStream_t s) {
    dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM);
    k_gemm<<<grid, 128, 0, s>>>(g);
    return cudaGetLastError();
}

const __nv_bfloat16* w16_of(const lbm_mlp* n, int l) {
    return l == 0 ? n->w16 : n->w16 + (size_t)kInPad * kW + (size_t)(l - 1) * kW * kW;
}
const __nv_bfloat16* w16t_of(const lbm_mlp* n, int l) {
    return l == 0 ? n->w16t : n->w16t + (size_t)kInPad * kW + (size_t)(l - 1) * kW * kW;
}

// Drain the stream; a tensor-core product whose bounded wait ran out since the
// last check makes this LBM_ETIMEOUT (and the word is cleared).
lbm_status sync(lbm_mlp* n) {
    if (cudaMemcpyAsync(n->h_err, n->err, sizeof(int), cudaMemcpyDeviceToHost, n->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(n->stream) != cudaSuccess)
        return LBM_ECUDA;
    if (*n->h_err) {
        *n->h_err = 0;
        if (cudaMemsetAsync(n->err, 0, sizeof(int), n->stream) != cudaSuccess) return LBM_ECUDA;
        return LBM_ETIMEOUT;
    }
    return LBM_OK;
}

// ---- tensor-core products: host side ----
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encoder() {
    static EncodeTiledFn fn = nullptr;
    static bool looked = false;
    if (!looked) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        looked = true;
    }
    return fn;
}

// Tensor map of a BF16 matrix [rows][K] (row stride K) that a box of `box_rows`
// rows lands in shared memory as K-major core matrices: the 4-D view (8
// elements, 8 rows, K/8, rows/8) with strides (2, 2K, 16, 16K) bytes.  The
// matrix's allocation must hold rows rounded up to 8.
bool core_matrix_map(const __nv_bfloat16* A, int rows, int K, int box_rows, CUtensorMap* m) {
    const EncodeTiledFn enc = encoder();
    if (!enc) return false;
    const cuuint64_t dims[4] = {8, 8, (cuuint64_t)(K / 8), (cuuint64_t)((rows + 7) / 8)};
    const cuuint64_t strides[3] = {(cuuint64_t)K * 2, 16, (cuuint64_t)K * 16};
    const cuuint32_t box[4] = {8, 8, (cuuint32_t)(K / 8), (cuuint32_t)(box_rows / 8)};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<__nv_bfloat16*>(A), dims,
               strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

// D[M x 256] = A[M x K] Bt[256 x K]^T on the tensor cores, with the epilogue of g;
// false when no tensor map can be made (the caller then uses k_gemm)
bool gemm_tc(const __nv_bfloat16* A, const __nv_bfloat16* Bt, UmmaArgs g, cudaStream_t s,
             cudaError_t* e) {
    CUtensorMap ta, tb;
    if (!core_matrix_map(A, g.M, g.K, UM, &ta) || !core_matrix_map(Bt, UN, g.K, UN, &tb))
        return false;
    const size_t smem = (size_t)(UM + UN) * g.K * 2;
    static unsigned long long attr_set = 0;  // one bit per device
    int dev = 0;
    *e = cudaGetDevice(&dev);
    if (*e != cudaSuccess) return true;
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(attr_set & bit)) {
        *e = cudaFuncSetAttribute(k_gemm_umma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)((UM + UN) * kW * 2));
        if (*e != cudaSuccess) return true;
        attr_set |= bit;
    }
    k_gemm_umma<<<(g.M + UM - 1) / UM, 128, smem, s>>>(ta, tb, g);
    *e = cudaGetLastError();
    return true;
}

// forward pass of a batch whose inputs are in x (device FP32 [B][3]); the
// output is a32[3]
lbm_status forward(lbm_mlp* n, const float* x, int B) {
    cudaStream_t s = n->stream;
    k_input<<<(B * kInPad + 255) / 256, 256, 0, s>>>(x, n->x16, B);
    CK(cudaGetLastError());
    for (int l = 0; l < kLayers; ++l) {
        if (n->tensor_cores) {
            UmmaArgs u{};
            u.M = B;
            u.K = l == 0 ? kInPad : kW;
            u.epi = l < kLayers - 1 ? EPI_BIAS_TANH : EPI_BIAS;
            u.bias = n->p + param_offset(l) + (long long)kFanIn[l] * kFanOut[l];
            u.out32 = n->a32[l];
            u.out16 = l < kLayers - 1 ? n->a16[l] : nullptr;
            u.ld16 = kW;
            u.err = n->err;
            cudaError_t e = cudaSuccess;
            if (gemm_tc(l == 0 ? n->x16 : n->a16[l - 1], w16t_of(n, l), u, s, &e)) {
                CK(e);
                continue;
            }
            n->tensor_cores = false;  // no tensor map: the mma.sync kernel from here on
        }
        GemmArgs g{};
        g.A = l == 0 ? n->x16 : n->a16[l - 1];
        g.sam = l == 0 ? kInPad : kW;
        g.sak = 1;
        g.B = w16_of(n, l);
        g.sbk = kFanOut[l];
        g.sbn = 1;
        g.M = B;
        g.N = kFanOut[l];
        g.K = l == 0 ? kInPad : kW;
        g.epi = l < kLayers - 1 ? EPI_BIAS_TANH : EPI_BIAS;
        g.bias = n->p + param_offset(l) + (long long)kFanIn[l] * kFanOut[l];
        g.out32 = n->a32[l];
        g.out16 = l < kLayers - 1 ? n->a16[l] : nullptr;
        g.ld16 = kW;
        CK(gemm(g, s));
    }
    return LBM_OK;
}

// loss and gradient into n->g (device), after forward()
lbm_status backward(lbm_mlp* n, const float* x, const float* t, int B) {
    cudaStream_t s = n->stream;
    CK(cudaMemsetAsync(n->sse, 0, sizeof(double), s));
    const int total = B * kOut;
    k_loss_grad<<<(total + 255) / 256 < 1024 ? (total + 255) / 256 : 1024, 256, 0, s>>>(
        n->a32[kLayers - 1], t, total, 1.0f / (float)total, n->d32, n->d16, n->sse);
    CK(cudaGetLastError());
    float* d32 = n->d32;
    __nv_bfloat16* d16 = n->d16;
    float* e32 = n->e32;
    __nv_bfloat16* e16 = n->e16;
    for (int l = kLayers - 1; l >= 0; --l) {
        const int fi = kFanIn[l], fo = kFanOut[l];
        float* gw = n->g + param_offset(l);
        float* gb = gw + (long long)fi * fo;
        // dW = A_{l-1}^T D (the input layer's padded columns are not kept)
        GemmArgs g{};
        g.A = l == 0 ? n->x16 : n->a16[l - 1];
        g.sam = 1;
        g.sak = l == 0 ? kInPad : kW;
        g.B = d16;
        g.sbk = fo;
        g.sbn = 1;
        g.M = fi;
        g.N = fo;
        g.K = B;
        g.epi = EPI_STORE;
        g.out32 = gw;
        CK(gemm(g, s));
        k_bias_grad<<<(fo + 127) / 128, 128, 0, s>>>(d32, B, fo, gb);
        CK(cudaGetLastError());
        if (l == 0) break;
        // D_{l-1} = (D W_l^T) (1 - A_{l-1}^2): K-major operands are D [B][fo] and
        // W_l itself ([fi][fo])
        bool done = false;
        if (n->tensor_cores) {
            UmmaArgs u{};
            u.M = B;
            u.K = fo;
            u.epi = EPI_TANH_BACK;
            u.aprev = n->a32[l - 1];
            u.out32 = e32;
            u.out16 = e16;
            u.ld16 = fi;
            u.err = n->err;
            cudaError_t e = cudaSuccess;
            done = gemm_tc(d16, w16_of(n, l), u, s, &e);
            if (done) CK(e);
            else n->tensor_cores = false;
        }
        if (done) {
            std::swap(d32, e32);
            std::swap(d16, e16);
            continue;
        }
        GemmArgs h{};
        h.A = d16;
        h.sam = fo;
        h.sak = 1;
        h.B = w16_of(n, l);
        h.sbk = 1;
        h.sbn = fo;
        h.M = B;
        h.N = fi;
        h.K = fo;
        h.epi = EPI_TANH_BACK;
        h.aprev = n->a32[l - 1];
        h.out32 = e32;
        h.out16 = e16;
        h.ld16 = fi;
        CK(gemm(h, s));
        std::swap(d32, e32);
        std::swap(d16, e16);
    }
    (void)x;
    return LBM_OK;
}

lbm_status refresh_w16(lbm_mlp* n) {
    const long long n16 = (long long)kInPad * kW + 3LL * kW * kW;
    k_weights16<<<(unsigned)((n16 + 255) / 256), 256, 0, n->stream>>>(n->p, n->w16, n->w16t);
    CK(cudaGetLastError());
    return LBM_OK;
}

}  // namespace

extern "C" {

int64_t lbm_mlp_param_count(void) { return kParams; }

size_t lbm_mlp_workspace_bytes(int32_t max_batch) {
    if (max_batch < 1 || max_batch > (1 << 20)) return 0;
    return mlp_layout(max_batch).total;
}

lbm_status lbm_mlp_init(lbm_mlp** out, int32_t max_batch, void* d_ws, size_t bytes,
                        void* stream) {
    if (!out) return LBM_EINVAL;
    *out = nullptr;
    if (max_batch < 1 || max_batch > (1 << 20) || !d_ws || ((uintptr_t)d_ws % 256))
        return LBM_EINVAL;
    const MlpLayout L = mlp_layout(max_batch);
    if (bytes < L.total) return LBM_ENOMEM;
    lbm_mlp* n = new (std::nothrow) lbm_mlp();
    if (!n) return LBM_ENOMEM;
    if (cudaGetDevice(&n->dev) != cudaSuccess) {
        delete n;
        return LBM_ECUDA;
    }
    char* w = (char*)d_ws;
    n->max_batch = max_batch;
    n->stream = (cudaStream_t)stream;
    n->p = (float*)(w + L.p);
    n->g = (float*)(w + L.g);
    n->m = (float*)(w + L.m);
    n->v = (float*)(w + L.v);
    n->w16 = (__nv_bfloat16*)(w + L.w16);
    n->x16 = (__nv_bfloat16*)(w + L.x16);
    const size_t R = (size_t)rows_of(max_batch);
    for (int l = 0; l < kLayers; ++l) n->a32[l] = (float*)(w + L.a32) + (size_t)l * R * kW;
    for (int l = 0; l < kLayers - 1; ++l)
        n->a16[l] = (__nv_bfloat16*)(w + L.a16) + (size_t)l * R * kW;
    n->w16t = (__nv_bfloat16*)(w + L.w16t);
    n->err = (int*)(w + L.err);
    n->d32 = (float*)(w + L.d32);
    n->d16 = (__nv_bfloat16*)(w + L.d16);
    n->e32 = (float*)(w + L.e32);
    n->e16 = (__nv_bfloat16*)(w + L.e16);
    n->sse = (double*)(w + L.sse);
    n->step = 0;
    n->tensor_cores = true;
    if (cudaMallocHost((void**)&n->h_sse, sizeof(double)) != cudaSuccess) {
        delete n;
        return LBM_ECUDA;
    }
    if (cudaMallocHost((void**)&n->h_err, sizeof(int)) != cudaSuccess) {
        cudaFreeHost(n->h_sse);
        delete n;
        return LBM_ECUDA;
    }
    if (cudaMemsetAsync(w, 0, L.total, n->stream) != cudaSuccess) {
        lbm_mlp_free(n);
        return LBM_ECUDA;
    }
    *out = n;
    return LBM_OK;
}

lbm_status lbm_mlp_set_tcgen05(lbm_mlp* n, int32_t on) {
    if (!n || (on != 0 && on != 1)) return LBM_EINVAL;
    n->tensor_cores = on == 1;
    return LBM_OK;
}

int32_t lbm_mlp_tcgen05(const lbm_mlp* n) { return n ? (n->tensor_cores ? 1 : 0) : -1; }

void lbm_mlp_free(lbm_mlp* n) {
    if (!n) return;
    cudaSetDevice(n->dev);
    if (n->h_sse) cudaFreeHost(n->h_sse);
    if (n->h_err) cudaFreeHost(n->h_err);
    delete n;
}

lbm_status lbm_mlp_set_params(lbm_mlp* n, const float* h_params) {
    if (!n || !h_params) return LBM_EINVAL;
    CK(cudaSetDevice(n->dev));
    CK(cudaMemcpyAsync(n->p, h_params, kParams * 4, cudaMemcpyHostToDevice, n->stream));
    CK(cudaMemsetAsync(n->m, 0, kParams * 4, n->stream));
    CK(cudaMemsetAsync(n->v, 0, kParams * 4, n->stream));
    n->step = 0;
    lbm_status st = refresh_w16(n);
    if (st) return st;
    return sync(n);
}

lbm_status lbm_mlp_get_params(lbm_mlp* n, float* h_params) {
    if (!n || !h_params) return LBM_EINVAL;
    CK(cudaSetDevice(n->dev));
    CK(cudaMemcpyAsync(h_params, n->p, kParams * 4, cudaMemcpyDeviceToHost, n->stream));
    return sync(n);
}

lbm_status lbm_mlp_forward(lbm_mlp* n, const float* d_x, int32_t batch, float* d_y) {
    if (!n || !d_x || !d_y || batch < 1 || batch > n->max_batch) return LBM_EINVAL;
    CK(cudaSetDevice(n->dev));
    lbm_status st = forward(n, d_x, batch);
    if (st) return st;
    CK(cudaMemcpyAsync(d_y, n->a32[kLayers - 1], (size_t)batch * kOut * 4,
                       cudaMemcpyDeviceToDevice, n->stream));
    return LBM_OK;
}

lbm_status lbm_mlp_loss_grad(lbm_mlp* n, const float* d_x, const float* d_t, int32_t batch,
                             double* h_loss, float* d_grad) {
    if (!n || !d_x || !d_t || batch < 1 || batch > n->max_batch) return LBM_EINVAL;
    CK(cudaSetDevice(n->dev));
    lbm_status st = forward(n, d_x, batch);
    if (!st) st = backward(n, d_x, d_t, batch);
    if (st) return st;
    if (d_grad)
        CK(cudaMemcpyAsync(d_grad, n->g, kParams * 4, cudaMemcpyDeviceToDevice, n->stream));
    if (h_loss) {
        CK(cudaMemcpyAsync(n->h_sse, n->sse, 8, cudaMemcpyDeviceToHost, n->stream));
        st = sync(n);
        if (st) return st;
        *h_loss = *n->h_sse / ((double)batch * kOut);
    }
    return LBM_OK;
}

lbm_status lbm_mlp_train_step(lbm_mlp* n, const float* d_x, const float* d_t, int32_t batch,
                              float lr, double* h_loss) {
    if (!n || !(lr > 0)) return LBM_EINVAL;
    lbm_status st = lbm_mlp_loss_grad(n, d_x, d_t, batch, h_loss, nullptr);
    if (st) return st;
    n->step += 1;
    const float c1 = (float)(1.0 - std::pow(0.9, (double)n->step));
    const float c2 = (float)(1.0 - std::pow(0.999, (double)n->step));
    k_adam<<<592, 256, 0, n->stream>>>(n->p, n->g, n->m, n->v, kParams, lr, c1, c2);
    CK(cudaGetLastError());
    return refresh_w16(n);
}

}  // extern "C"
