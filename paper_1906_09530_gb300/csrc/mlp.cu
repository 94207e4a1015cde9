// mlp.cu -- the surrogate network of the warm start (lbm_mlp_* of
// include/cplbm.h): a 4-256-256-256-256 multilayer perceptron with tanh hidden
// layers that maps (T_r, kappa-hat, k, 1/R) to a 256-point equilibrium interface
// profile (R the radius of a drop; 0 for flat interfaces), trained and evaluated
// by the kernels of this file.
//
// Arithmetic: every matrix product runs on the tensor cores in BF16 with FP32
// accumulation; master weights, Adam moments, biases, activations kept for the
// backward pass, and the loss are FP32 (the loss sum FP64).  The products:
//   forward            Z_l   = A_{l-1} W_l          [B x fan_in] [fan_in x fan_out]
//   weight gradient    dW_l  = A_{l-1}^T D_l        [fan_in x B] [B x fan_out]
//   input gradient     D_{l-1} = (D_l W_l^T) (1 - A_{l-1}^2)
// with fused epilogues (bias + tanh, tanh derivative).  All of them run as
// tcgen05 MMAs with the accumulator in tensor memory and the operands brought in
// by tensor copies: the forward and input-gradient products (256 output columns,
// a batch of rows) in the persistent k_umma_rows, the weight gradient (K = the
// batch) split over K in k_umma_wgrad.  The strided mma.sync tile kernel
// (k_gemm) is kept as the comparison point, selected by lbm_mlp_set_tcgen05, and
// runs a call whose tensor maps cannot be made.
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

constexpr int kIn = 4, kW = 256, kOut = 256, kLayers = 4;
constexpr int kInPad = 16;  // the first product's K on mma.sync, padded to one k-step
constexpr int kK0 = 64;     // row stride of the BF16 input and K of its tcgen05 product
                            // (zero-padded to one 128-byte swizzle row)
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
    EPI_LOSS = 4,       // y = acc + bias[n], e = y - target[m][n]: d = e scale, sum e^2
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

// tanh(x) = 1 - 2 / (1 + exp(2x)) with the fast exponential and division
// intrinsics: six instructions, exact limits at +-inf, NaN in NaN out.  Its
// absolute error stays below about 3e-7 at every x (relative error grows only
// where |tanh x| < 1e-3, where the BF16 rounding that every activation gets,
// 2^-9 relative, is still larger in absolute terms above |x| ~ 1.5e-4).
__device__ __forceinline__ float tanh_act(float x) {
    return 1.0f - __fdividef(2.0f, 1.0f + __expf(2.0f * x));
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
                    v = tanh_act(v + g.bias[n]);
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
// tensor memory), BF16 operands, FP32 accumulation.  Operands move in K chunks
// of 64 elements: a tensor copy (TMA) of a box of 64 x rows with 128-byte
// swizzling writes each row's 128 bytes with its 16-byte pieces permuted by the
// row index mod 8, which is the tensor cores' K-major 128-byte-swizzle layout
// (8-row groups 1024 bytes apart); the MMA of the k-th 16-wide step starts
// 32 k bytes into the chunk.  Every wait on an mbarrier is
// bounded: one that runs out sets the error word and a shared abort flag, the
// other roles see the flag and leave their loops, and the CTA waits (bounded)
// for its copies and MMAs in flight before it frees its tensor memory.
//
// k_umma_rows: D[M x 256] = A[M x K] Bt[256 x K]^T, K = 64 or 256: the forward
// products (A = the layer input, Bt = the transposed weights) and the input
// gradients (A = the backward signal, Bt = the weights as stored).  Persistent:
// one CTA per SM walks 128-row tiles of A.  Warp 8 (one thread) streams the
// 64-wide K chunks of A and Bt (Bt is re-read from L2 for every tile) through a
// three-stage ring; warp 9 (one thread) issues the MMAs (128 x 256 x 16 each)
// into one of two 256-column accumulators; warps 0-7 drain the other
// accumulator (the previous tile) meanwhile, two warps per quarter of the
// tensor-memory lanes, one per half of the columns.  The epilogue stages each
// 32-row x 16-column block in shared memory so that its global loads and stores
// are row pieces of 64 (FP32) or 32 (BF16) bytes.
//
// k_umma_wgrad: the weight gradient dW[fi x 256] = A^T D over the batch, as
// At[fi x K] Dt[256 x K]^T with K the batch: the epilogues above also write the
// transposed BF16 copies At and Dt.  K is split into slices (grid.y) so that the
// product fills the GPU; each CTA streams its slice through a four-stage ring
// of 64-wide K chunks (warp 4 loads, warp 5 issues the MMAs) and writes an FP32
// partial; k_wgrad_reduce adds the partials in a fixed order (deterministic).
// ---------------------------------------------------------------------------
constexpr int UM = 128, UN = 256;
constexpr unsigned kUmmaSpins = 1u << 22;
constexpr int kS32 = 20, kS16 = 24;  // padded rows of the epilogue's staging blocks
constexpr int kKC = 64;              // K chunk of the streamed operands
// k_umma_rows: 8 epilogue warps (two per tensor-memory lane quarter, one per
// half of the 256 columns), a loader warp and an MMA warp; 3-stage ring
constexpr int kRowEpi = 8, kRowStages = 3;
constexpr int kRowsThreads = 32 * (kRowEpi + 2);
// k_umma_wgrad: 4 epilogue warps, a loader warp and an MMA warp; 4-stage ring
constexpr int kWgEpi = 4, kStages = 4;
constexpr int kWgThreads = 32 * (kWgEpi + 2);
constexpr int kRowGridCap = 256;  // most CTAs of a k_umma_rows launch
constexpr size_t kChunkBytes = (size_t)(UM + UN) * kKC * 2;
// (+1024: the stages are aligned to 1024 bytes inside the dynamic allocation)
constexpr size_t kRowsSmem = 1024 + kRowStages * kChunkBytes +
                             (size_t)kRowEpi * 32 * (kS32 * 4 + kS16 * 2) + UN * 4 +
                             (size_t)kRowEpi * (UN / 2) * 4;
constexpr size_t kWgSmem = 1024 + kStages * kChunkBytes + (size_t)kWgEpi * 32 * kS32 * 4;
static_assert(kRowsSmem <= 227 * 1024 - 1024, "row kernel shared memory");
static_assert(kWgSmem <= 227 * 1024 - 1024, "weight-gradient kernel shared memory");

struct RowArgs {
    int M, K;
    int epi;
    const float* bias;   // [256] (EPI_BIAS_TANH, EPI_BIAS, EPI_LOSS)
    const float* aprev;  // [M][256]: the activations (EPI_TANH_BACK) or targets (EPI_LOSS)
    float scale;         // EPI_LOSS: dL/dy = scale (y - target)
    double* sse;         // EPI_LOSS: sum of (y - target)^2 (added to)
    float* bpart;        // or null: column sums of the result, [grid][4][256] (see below)
    float* out32;        // [M][ld32] or null
    int ld32;
    __nv_bfloat16* out16;   // [M][ld16] or null
    int ld16;
    __nv_bfloat16* out16t;  // [256][ldt] (column c of D at row c) or null
    int ldt, rows_t;        // transposed copy: entries m < rows_t written, zero for m >= M
    int* err;
};

struct WgArgs {
    int mtiles;       // 128-row tiles of At (fi rows)
    int chunks;       // K chunks (64 wide) in all
    int per_slice;    // K chunks per slice
    float* part;      // [slices][mtiles * 128][256]
    int* err;
};

__device__ __forceinline__ unsigned su32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ bool mb_try(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(su32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait for the phase of the given parity; gives up early when another
// role has raised the abort flag (null: no early exit)
__device__ __forceinline__ bool mb_wait(uint64_t* bar, unsigned parity,
                                        const volatile int* abort_flag) {
    for (unsigned i = 0; i < kUmmaSpins; ++i) {
        if (mb_try(bar, parity)) return true;
        if (abort_flag && *abort_flag) return false;
    }
    return false;
}
__device__ __forceinline__ void mb_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(su32(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void mb_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(su32(bar)) : "memory");
}
__device__ __forceinline__ void mb_expect(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(su32(bar)),
                 "r"(bytes)
                 : "memory");
}
// 2-D tensor copy global -> shared of the box at (k, row), completing on bar
__device__ __forceinline__ void tma2(void* dst, const CUtensorMap* map, int k, int row,
                                     uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];\n" ::"r"(su32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(k), "r"(row), "r"(su32(bar))
        : "memory");
}
// shared-memory matrix descriptor of a K-major operand in the 128-byte swizzle
// layout: start address, leading byte offset 16 (unused by this layout), stride
// byte offset 1024 (one 8-row group), descriptor version 1, layout type 2
__device__ __forceinline__ uint64_t umma_desc(unsigned addr) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// instruction descriptor: D f32 (bits 4-5), A and B bf16 (7-9, 10-12), both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(UN >> 3) << 17) |
                            ((uint32_t)(UM >> 4) << 24);
__device__ __forceinline__ void umma(uint32_t tmem, uint64_t da, uint64_t db, bool acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(da), "l"(db), "r"(kIdesc), "r"(acc ? 1u : 0u)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
            su32(bar))
        : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}
// kNC consecutive accumulator columns of this warp's 32 lanes (one row a thread)
constexpr int kNC = 16;
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* x) {
    uint32_t v[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
        "%13,%14,%15}, [%16];\n"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
          "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int j = 0; j < kNC; ++j) x[j] = __uint_as_float(v[j]);
}

// this warp's 32 rows [r0, r0 + 32) x kNC columns [c, c + kNC) of a row-major
// FP32 matrix (row stride ld): thread `lane` holds row r0 + lane in x.  Stores
// and loads go through the warp's staging block s (32 rows of kS32 floats), so
// that the global accesses are 64-byte row pieces, eight rows an instruction.
__device__ __forceinline__ void rows_store32(float* s, const float* x, float* out, long long ld,
                                             int r0, int c, int M, int lane) {
#pragma unroll
    for (int j = 0; j < kNC / 4; ++j)
        *reinterpret_cast<float4*>(s + lane * kS32 + 4 * j) =
            make_float4(x[4 * j], x[4 * j + 1], x[4 * j + 2], x[4 * j + 3]);
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int rr = 8 * j + (lane >> 2), q = lane & 3;
        if (r0 + rr < M)
            *reinterpret_cast<float4*>(out + (long long)(r0 + rr) * ld + c + 4 * q) =
                *reinterpret_cast<const float4*>(s + rr * kS32 + 4 * q);
    }
    __syncwarp();
}

// coalesced loads of this warp's 32 rows x kNC columns of a row-major FP32
// matrix [M][256], issued ahead of use (rows >= M read as zero): piece j holds
// row 8 j + lane / 4, columns 4 (lane % 4) .. + 3
__device__ __forceinline__ void aux_fetch(float4* pf, const float* in, int r0, int c, int M,
                                          int lane) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int rr = 8 * j + (lane >> 2), q = lane & 3;
        pf[j] = r0 + rr < M
                    ? __ldg(reinterpret_cast<const float4*>(in + (long long)(r0 + rr) * UN + c +
                                                            4 * q))
                    : make_float4(0.f, 0.f, 0.f, 0.f);
    }
}
// the fetched pieces -> row r0 + lane in aux, through the staging block s
__device__ __forceinline__ void aux_rows(const float4* pf, float* s, float* aux, int lane) {
#pragma unroll
    for (int j = 0; j < 4; ++j)
        *reinterpret_cast<float4*>(s + (8 * j + (lane >> 2)) * kS32 + 4 * (lane & 3)) = pf[j];
    __syncwarp();
#pragma unroll
    for (int j = 0; j < kNC / 4; ++j) {
        const float4 a = *reinterpret_cast<const float4*>(s + lane * kS32 + 4 * j);
        aux[4 * j] = a.x;
        aux[4 * j + 1] = a.y;
        aux[4 * j + 2] = a.z;
        aux[4 * j + 3] = a.w;
    }
    __syncwarp();
}

// The epilogue of one kNC-column chunk [c, c + kNC) of a warp's 32 rows (x: row
// r0 + lane; aux: the same entries of aprev, for EPI_TANH_BACK and EPI_LOSS).
// Column sums of the result over the warp's rows are added to bsum[0..kNC).
__device__ __forceinline__ void rows_epilogue(const RowArgs& g, float* x, const float* aux,
                                              const float* bias_s, float* s32,
                                              __nv_bfloat16* s16, int r0, int c, int lane,
                                              float* bsum, double& sse) {
    const bool live = r0 + lane < g.M;
    if (g.epi == EPI_TANH_BACK) {
#pragma unroll
        for (int j = 0; j < kNC; ++j) x[j] *= 1.0f - aux[j] * aux[j];
    } else if (g.epi == EPI_BIAS_TANH) {
#pragma unroll
        for (int j = 0; j < kNC; ++j) x[j] = tanh_act(x[j] + bias_s[c + j]);
    } else if (g.epi == EPI_BIAS) {
#pragma unroll
        for (int j = 0; j < kNC; ++j) x[j] += bias_s[c + j];
    } else if (g.epi == EPI_LOSS) {
        float e2 = 0.0f;
#pragma unroll
        for (int j = 0; j < kNC; ++j) {
            const float e = live ? x[j] + bias_s[c + j] - aux[j] : 0.0f;
            e2 = fmaf(e, e, e2);
            x[j] = 2.0f * e * g.scale;
        }
        sse += (double)e2;
    }
    if (!live) {
#pragma unroll
        for (int j = 0; j < kNC; ++j) x[j] = 0.0f;  // rows past M add nothing to the sums
    }
    if (g.out32 || g.bpart) {
#pragma unroll
        for (int j = 0; j < kNC / 4; ++j)
            *reinterpret_cast<float4*>(s32 + lane * kS32 + 4 * j) =
                make_float4(x[4 * j], x[4 * j + 1], x[4 * j + 2], x[4 * j + 3]);
        __syncwarp();
        if (g.out32) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int rr = 8 * j + (lane >> 2), q = lane & 3;
                if (r0 + rr < g.M)
                    *reinterpret_cast<float4*>(g.out32 + (long long)(r0 + rr) * g.ld32 + c +
                                               4 * q) =
                        *reinterpret_cast<const float4*>(s32 + rr * kS32 + 4 * q);
            }
        }
        if (g.bpart) {
            // lane l adds column l % 16 over rows 16 (l / 16) .. + 15, then the halves
            const int col = lane & (kNC - 1), h = lane >> 4;
            float cs = 0.0f;
#pragma unroll
            for (int r = 0; r < 16; ++r) cs += s32[(16 * h + r) * kS32 + col];
            cs += __shfl_down_sync(0xffffffffu, cs, 16);
            if (lane < kNC) bsum[lane] += cs;
        }
        __syncwarp();
    }
    if (!g.out16 && !g.out16t) return;
    __nv_bfloat16 hv[kNC];
#pragma unroll
    for (int j = 0; j < kNC; ++j) hv[j] = __float2bfloat16_rn(x[j]);
    if (g.out16) {
#pragma unroll
        for (int j = 0; j < kNC / 8; ++j)
            *reinterpret_cast<uint4*>(s16 + lane * kS16 + 8 * j) =
                *reinterpret_cast<const uint4*>(hv + 8 * j);
        __syncwarp();
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int rr = 16 * j + (lane >> 1), q = lane & 1;
            if (r0 + rr < g.M)
                *reinterpret_cast<uint4*>(g.out16 + (long long)(r0 + rr) * g.ld16 + c + 8 * q) =
                    *reinterpret_cast<const uint4*>(s16 + rr * kS16 + 8 * q);
        }
        __syncwarp();
    }
    if (g.out16t) {
        // column c + j of D is row c + j of the copy: the warp writes 64 bytes a
        // column (zeros, set above, for rows in [M, rows_t))
        const int m = r0 + lane;
        if (m < g.rows_t) {
#pragma unroll
            for (int j = 0; j < kNC; ++j) g.out16t[(long long)(c + j) * g.ldt + m] = hv[j];
        }
    }
}

__global__ void __launch_bounds__(kRowsThreads, 1)
    k_umma_rows(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb,
                RowArgs g) {
    extern __shared__ __align__(1024) unsigned char usm_raw[];
    // the swizzle pattern repeats every 1024 bytes: stages start on such a boundary
    unsigned char* usm = usm_raw + ((1024u - (su32(usm_raw) & 1023u)) & 1023u);
    const int nkc = g.K / kKC;  // 64-wide chunks: K = 64 or 256
    constexpr unsigned abytes = UM * kKC * 2;
    // stage s: A chunk (UM x kc) then Bt chunk (UN x kc), kChunkBytes apart
    float* st32 = reinterpret_cast<float*>(usm + kRowStages * kChunkBytes);
    __nv_bfloat16* st16 = reinterpret_cast<__nv_bfloat16*>(st32 + kRowEpi * 32 * kS32);
    float* bias_s = reinterpret_cast<float*>(st16 + kRowEpi * 32 * kS16);
    float* bsum_s = bias_s + UN;  // [kRowEpi][128]: column sums of each warp's half
    // [0..2] stage full, [3..5] stage free, [6..7] accumulator 0/1 full,
    // [8..9] accumulator 0/1 drained
    constexpr int F0 = 0, E0 = kRowStages, AF = 2 * kRowStages, AE = AF + 2;
    __shared__ __align__(8) uint64_t bar[2 * kRowStages + 4];
    __shared__ uint32_t tbase;
    __shared__ int abort_s;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntiles = (g.M + UM - 1) / UM;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         su32(&tbase)),
                     "r"(2 * UN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        for (int q = 0; q < AE; ++q) mb_init(&bar[q], 1);
        mb_init(&bar[AE], kRowEpi);
        mb_init(&bar[AE + 1], kRowEpi);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        abort_s = 0;
    }
    for (int i = tid; i < UN; i += blockDim.x) bias_s[i] = g.bias ? g.bias[i] : 0.0f;
    for (int i = tid; i < kRowEpi * (UN / 2); i += blockDim.x) bsum_s[i] = 0.0f;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tbase;
    volatile int* abort_v = &abort_s;
    if (warp == kRowEpi) {
        if (lane == 0) {
            // loader: every chunk of every tile through the ring
            int q = 0;  // chunks issued
            bool ok = true;
            for (int t = blockIdx.x; ok && t < ntiles; t += gridDim.x)
                for (int j = 0; j < nkc; ++j, ++q) {
                    const int st = q % kRowStages;
                    if (q >= kRowStages)
                        ok = mb_wait(&bar[E0 + st], ((q / kRowStages) - 1) & 1, abort_v);
                    if (!ok) break;
                    unsigned char* A = usm + st * kChunkBytes;
                    mb_expect(&bar[F0 + st], (unsigned)kChunkBytes);
                    tma2(A, &ta, j * kKC, t * UM, &bar[F0 + st]);
                    tma2(A + abytes, &tb, j * kKC, 0, &bar[F0 + st]);
                }
            if (!ok) {
                atomicExch(g.err, 1);
                *abort_v = 1;
            }
            // the copies issued last complete before the CTA leaves (bounded)
            for (int r = (q > kRowStages ? q - kRowStages : 0); r < q; ++r)
                mb_wait(&bar[F0 + r % kRowStages], (r / kRowStages) & 1, nullptr);
        }
    } else if (warp == kRowEpi + 1) {
        if (lane == 0) {
            // MMA issuer: one accumulator per tile, alternating
            int q = 0, i = 0, committed = -1;
            bool ok = true;
            for (int t = blockIdx.x; ok && t < ntiles; t += gridDim.x, ++i) {
                if (i >= 2) ok = mb_wait(&bar[AE + (i & 1)], ((i - 2) >> 1) & 1, abort_v);
                if (!ok) break;
                const uint32_t acc = tmem + (uint32_t)((i & 1) * UN);
                for (int j = 0; j < nkc; ++j, ++q) {
                    const int st = q % kRowStages;
                    ok = mb_wait(&bar[F0 + st], (q / kRowStages) & 1, abort_v);
                    if (!ok) break;
                    tc_fence_after();
                    const unsigned A = su32(usm + st * kChunkBytes);
                    for (int kk = 0; kk < kKC / 16; ++kk)
                        umma(acc, umma_desc(A + kk * 32), umma_desc(A + abytes + kk * 32),
                             j > 0 || kk > 0);
                    umma_commit(&bar[E0 + st]);
                    committed = q;
                }
                if (!ok) break;
                umma_commit(&bar[AF + (i & 1)]);
            }
            if (!ok) {
                atomicExch(g.err, 1);
                *abort_v = 1;
                if (committed >= 0)
                    mb_wait(&bar[E0 + committed % kRowStages], (committed / kRowStages) & 1,
                            nullptr);
            }
        }
    } else {
        float* s32 = st32 + warp * 32 * kS32;
        __nv_bfloat16* s16 = st16 + warp * 32 * kS16;
        float* bsum = bsum_s + warp * (UN / 2);
        const int quarter = warp & 3, c0 = (warp >> 2) * (UN / 2);
        const bool need_aux = g.epi == EPI_TANH_BACK || g.epi == EPI_LOSS;
        double sse = 0.0;
        int i = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
            bool ok = mb_wait(&bar[AF + (i & 1)], (i >> 1) & 1, abort_v);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) {
                if (lane == 0) {
                    atomicExch(g.err, 1);
                    *abort_v = 1;
                }
                break;
            }
            tc_fence_after();
            const uint32_t acc =
                tmem + (uint32_t)((i & 1) * UN) + ((uint32_t)(quarter * 32) << 16);
            const int r0 = t * UM + quarter * 32;
            float4 pf[4];
            if (need_aux) aux_fetch(pf, g.aprev, r0, c0, g.M, lane);
            for (int c = c0; c < c0 + UN / 2; c += kNC) {
                float x[kNC], aux[kNC];
                tmem_ld16(acc + (uint32_t)c, x);
                if (need_aux) {
                    aux_rows(pf, s32, aux, lane);
                    // the next chunk's operand is on its way while this one is worked
                    if (c + kNC < c0 + UN / 2) aux_fetch(pf, g.aprev, r0, c + kNC, g.M, lane);
                }
                rows_epilogue(g, x, aux, bias_s, s32, s16, r0, c, lane, bsum + (c - c0), sse);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mb_arrive(&bar[AE + (i & 1)]);
        }
        __syncwarp();
        if (g.bpart)
            for (int j = lane; j < UN / 2; j += 32)
                g.bpart[((long long)blockIdx.x * 4 + quarter) * UN + c0 + j] = bsum[j];
        if (g.sse) {
            for (int o = 16; o > 0; o >>= 1) sse += __shfl_down_sync(0xffffffffu, sse, o);
            if (lane == 0) atomicAdd(g.sse, sse);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                     "r"(2 * UN)
                     : "memory");
}

__global__ void __launch_bounds__(kWgThreads, 1)
    k_umma_wgrad(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb,
                 WgArgs g) {
    extern __shared__ __align__(1024) unsigned char usm_raw[];
    unsigned char* usm = usm_raw + ((1024u - (su32(usm_raw) & 1023u)) & 1023u);
    // stage s: A chunk (UM x kKC) then B chunk (UN x kKC)
    constexpr unsigned kAbytes = UM * kKC * 2, kBbytes = UN * kKC * 2;
    static_assert(kAbytes + kBbytes == kChunkBytes, "chunk layout");
    float* st32 = reinterpret_cast<float*>(usm + (size_t)kStages * (kAbytes + kBbytes));
    // [0..3] stage full, [4..7] stage free, [8] all MMAs done
    __shared__ __align__(8) uint64_t bar[2 * kStages + 1];
    __shared__ uint32_t tbase;
    __shared__ int abort_s;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int mt = blockIdx.x, slice = blockIdx.y;
    const int j0 = slice * g.per_slice;
    const int nk = min(g.per_slice, g.chunks - j0);  // >= 1 by the host's choice of slices
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         su32(&tbase)),
                     "r"(UN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        for (int s = 0; s < 2 * kStages + 1; ++s) mb_init(&bar[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        abort_s = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tbase;
    volatile int* abort_v = &abort_s;
    if (warp == kWgEpi) {
        if (lane == 0) {
            // loader
            int loaded = 0;  // chunks whose copies were issued
            bool ok = true;
            for (int j = 0; j < nk; ++j) {
                const int s = j % kStages;
                if (j >= kStages) ok = mb_wait(&bar[kStages + s], ((j / kStages) - 1) & 1, abort_v);
                if (!ok) break;
                unsigned char* A = usm + (size_t)s * (kAbytes + kBbytes);
                mb_expect(&bar[s], kAbytes + kBbytes);
                tma2(A, &ta, (j0 + j) * kKC, mt * UM, &bar[s]);
                tma2(A + kAbytes, &tb, (j0 + j) * kKC, 0, &bar[s]);
                loaded = j + 1;
            }
            if (!ok) {
                atomicExch(g.err, 1);
                *abort_v = 1;
            }
            // every issued copy completes before the CTA leaves (bounded)
            for (int j = (loaded > kStages ? loaded - kStages : 0); j < loaded; ++j)
                mb_wait(&bar[j % kStages], (j / kStages) & 1, nullptr);
        }
    } else if (warp == kWgEpi + 1) {
        if (lane == 0) {
            // MMA issuer
            bool ok = true;
            int issued = 0;
            for (int j = 0; j < nk; ++j) {
                const int s = j % kStages;
                ok = mb_wait(&bar[s], (j / kStages) & 1, abort_v);
                if (!ok) break;
                tc_fence_after();
                const unsigned A = su32(usm + (size_t)s * (kAbytes + kBbytes));
                for (int kk = 0; kk < kKC / 16; ++kk)
                    umma(tmem, umma_desc(A + kk * 32), umma_desc(A + kAbytes + kk * 32),
                         j > 0 || kk > 0);
                umma_commit(&bar[kStages + s]);
                issued = j + 1;
            }
            if (ok) {
                umma_commit(&bar[2 * kStages]);
            } else {
                atomicExch(g.err, 1);
                *abort_v = 1;
                if (issued > 0)
                    mb_wait(&bar[kStages + (issued - 1) % kStages], ((issued - 1) / kStages) & 1,
                            nullptr);
            }
        }
    } else {
        bool ok = mb_wait(&bar[2 * kStages], 0, abort_v);
        ok = __all_sync(0xffffffffu, ok);
        if (ok) {
            tc_fence_after();
            float* s32 = st32 + warp * 32 * kS32;
            const uint32_t acc = tmem + ((uint32_t)(warp * 32) << 16);
            const int r0 = mt * UM + warp * 32;
            float* out = g.part + (long long)slice * g.mtiles * UM * UN;
            for (int c = 0; c < UN; c += kNC) {
                float x[kNC];
                tmem_ld16(acc + (uint32_t)c, x);
                rows_store32(s32, x, out, UN, r0, c, g.mtiles * UM, lane);
            }
        } else if (lane == 0) {
            atomicExch(g.err, 1);
            *abort_v = 1;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                     "r"(UN)
                     : "memory");
}

// dW[k][n] = sum over slices of part[s][k][n] (k < fi), and db[n] = sum of
// the nb column-sum rows bpart[p][n] the row kernel left.  A block takes 32
// outputs with 8 threads each: thread phase y adds rows y, y + 8, ..., and the
// eight phase sums are added in phase order, so the result does not depend on
// timing.
__global__ void __launch_bounds__(256) k_wgrad_reduce(const float* __restrict__ part, int slices,
                                                      int rows, int fi, float* __restrict__ gw,
                                                      const float* __restrict__ bpart, int nb,
                                                      float* __restrict__ gb) {
    __shared__ float acc[8][33];
    const int o = blockIdx.x * 32 + threadIdx.x, y = threadIdx.y;
    float s = 0.0f;
    if (o < fi * UN) {
        for (int q = y; q < slices; q += 8) s += part[(long long)q * rows * UN + o];
    } else if (o < fi * UN + UN) {
        const int n = o - fi * UN;
        for (int q = y; q < nb; q += 8) s += bpart[(long long)q * UN + n];
    }
    acc[y][threadIdx.x] = s;
    __syncthreads();
    if (y == 0 && o < fi * UN + UN) {
        float t = acc[0][threadIdx.x];
        for (int p = 1; p < 8; ++p) t += acc[p][threadIdx.x];
        if (o < fi * UN) gw[o] = t;
        else gb[o - fi * UN] = t;
    }
}

// x [B][4] FP32 -> BF16 [B][kK0], zero-padded, and (x16t not null) its transpose
// [16][ldt] with zeros for b in [B, rows_t)
__global__ void k_input(const float* __restrict__ x, __nv_bfloat16* __restrict__ x16, int B,
                        __nv_bfloat16* __restrict__ x16t, int ldt, int rows_t) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < B * kK0) {
        const int b = i / kK0, k = i - b * kK0;
        x16[i] = __float2bfloat16_rn(k < kIn ? x[b * kIn + k] : 0.0f);
    }
    if (x16t && i < kInPad * rows_t) {
        const int k = i / rows_t, b = i - k * rows_t;
        x16t[(long long)k * ldt + b] =
            __float2bfloat16_rn(k < kIn && b < B ? x[b * kIn + k] : 0.0f);
    }
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
        w16t[(long long)n * kK0 + k] = v;  // columns 16..63 stay zero
        return;
    }
    const long long j = i - (long long)kInPad * kW;  // layers 1..3
    const int l = 1 + (int)(j / (kW * kW));
    const long long r = j - (long long)(l - 1) * kW * kW;
    const int k = (int)(r / kW), n = (int)(r - (long long)k * kW);
    const __nv_bfloat16 v = __float2bfloat16_rn(p[param_offset(l) + r]);
    w16[i] = v;
    w16t[(long long)kK0 * kW + (long long)(l - 1) * kW * kW + (long long)n * kW + k] = v;
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

struct lbm_mlp;

namespace {

// tensor maps of the tcgen05 products for one batch size (they depend on the
// batch through the row and K extents)
struct TcMaps {
    int B = -1;
    CUtensorMap fwdA[kLayers];    // x16, a16[0..2]: [B][K], boxes 128 rows x 64
    CUtensorMap fwdB[kLayers];    // w16t of each layer: [256][K], boxes 256 x 64
    CUtensorMap sigA[2];          // d16, e16 (the backward signal as the A operand)
    CUtensorMap sigB[kLayers];    // w16 of layers 1..3 ([fi][fo] = [256][K = fo])
    CUtensorMap wgA[kLayers];     // x16t, a16t[0..2]: [fi rows][K = batch], 64-wide K boxes
    CUtensorMap wgB[2];           // d16t, e16t
};

}  // namespace

struct lbm_mlp {
    int dev, max_batch, R, nsm;  // R: rows of the batch-sized buffers (max_batch rounded to 8)
    cudaStream_t stream;
    float *p, *g, *m, *v;        // FP32 parameters, gradient, Adam moments
    __nv_bfloat16* w16;          // BF16 weight copies, layer by layer ([fan_in][fan_out])
    __nv_bfloat16* w16t;         // the same transposed ([fan_out][fan_in]; fan_in kK0 for layer 0)
    int* err;                    // device word: a tensor-core product's wait ran out
    int* h_err;                  // pinned mirror
    __nv_bfloat16* x16;          // [R][kK0]
    __nv_bfloat16* x16t;         // [16][R]
    float* a32[kLayers];         // layer outputs, FP32 [R][256]
    __nv_bfloat16* a16[kLayers - 1];   // hidden outputs, BF16 (inputs of the next product)
    __nv_bfloat16* a16t[kLayers - 1];  // the same transposed, [256][R]
    float* d32;                  // backward signal, FP32 [R][256]
    __nv_bfloat16* d16;          // its BF16 copy
    __nv_bfloat16* d16t;         // transposed, [256][R]
    float* e32;                  // the previous layer's signal
    __nv_bfloat16* e16;
    __nv_bfloat16* e16t;
    float* part;                 // weight-gradient partials [slices][256][256]
    float* bpart;                // bias-gradient partials [slices][256]
    double* sse;                 // device scalar
    double* h_sse;               // pinned mirror
    long long step;
    bool tensor_cores;           // forward and input-gradient products by tcgen05
    TcMaps maps;
};

namespace {

size_t al(size_t v) { return (v + 255) / 256 * 256; }

struct MlpLayout {
    size_t p, g, m, v, w16, w16t, x16, x16t, a32, a16, a16t, d32, d16, d16t, e32, e16, e16t,
        part, bpart, sse, err, total;
};

// Rows of the batch-sized buffers: a multiple of 8, so that the tensor copies of
// 8-row core matrices stay inside the buffers and the transposed copies' rows
// are whole 16-byte pieces.
int rows_of(int B) { return (B + 7) / 8 * 8; }

// K slices of the weight gradient for a batch of B: 64-wide chunks, at most
// kWgSlices slices of equal whole-chunk length
constexpr int kWgSlices = 74;
struct Slicing {
    int chunks, per_slice, slices;
};
Slicing slicing(int B) {
    Slicing s;
    s.chunks = (rows_of(B) + kKC - 1) / kKC;
    s.per_slice = (s.chunks + kWgSlices - 1) / kWgSlices;
    s.slices = (s.chunks + s.per_slice - 1) / s.per_slice;
    return s;
}

MlpLayout mlp_layout(int B0) {
    const size_t B = (size_t)rows_of(B0);
    // slices of any batch up to B0: at most kWgSlices, and at most its chunks
    const int chunks = slicing(B0).chunks;
    const size_t S = (size_t)(chunks < kWgSlices ? chunks : kWgSlices);
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
    L.w16t = take(((size_t)kK0 * kW + 3ull * kW * kW) * 2);
    L.x16 = take(B * kK0 * 2);
    L.x16t = take(B * kInPad * 2);
    L.a32 = take((size_t)kLayers * B * kW * 4);
    L.a16 = take((size_t)(kLayers - 1) * B * kW * 2);
    L.a16t = take((size_t)(kLayers - 1) * B * kW * 2);
    L.d32 = take(B * kW * 4);
    L.d16 = take(B * kW * 2);
    L.d16t = take(B * kW * 2);
    L.e32 = take(B * kW * 4);
    L.e16 = take(B * kW * 2);
    L.e16t = take(B * kW * 2);
    L.part = take(S * kW * UN * 4);
    L.bpart = take((size_t)kRowGridCap * 4 * UN * 4);
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
    return l == 0 ? n->w16t : n->w16t + (size_t)kK0 * kW + (size_t)(l - 1) * kW * kW;
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

// Tensor map of a BF16 matrix [rows][kext] (row stride ld elements, a multiple
// of 8) whose boxes of 64 (K) x box_rows land in shared memory in the
// 128-byte-swizzle layout; parts of a box outside the matrix arrive as zeros.
bool sw128_map(const __nv_bfloat16* A, int rows, int kext, int ld, int box_rows, CUtensorMap* m) {
    const EncodeTiledFn enc = encoder();
    if (!enc) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)kext, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kKC, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(A), dims,
               strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

// every tensor map of the tcgen05 path for a batch of B; false if one cannot
// be made (the call then runs on the mma.sync kernel)
bool prepare_maps(lbm_mlp* n, int B) {
    TcMaps& t = n->maps;
    if (t.B == B) return true;
    t.B = -1;
    const int kB = rows_of(B);
    bool ok = true;
    for (int l = 0; l < kLayers; ++l) {
        const int K = l == 0 ? kK0 : kW;
        ok = ok && sw128_map(l == 0 ? n->x16 : n->a16[l - 1], B, K, K, UM, &t.fwdA[l]);
        ok = ok && sw128_map(w16t_of(n, l), UN, K, K, UN, &t.fwdB[l]);
        if (l > 0) ok = ok && sw128_map(w16_of(n, l), UN, kW, kW, UN, &t.sigB[l]);
        ok = ok && sw128_map(l == 0 ? n->x16t : n->a16t[l - 1], l == 0 ? kInPad : kW, kB, n->R,
                             UM, &t.wgA[l]);
    }
    ok = ok && sw128_map(n->d16, B, kW, kW, UM, &t.sigA[0]);
    ok = ok && sw128_map(n->e16, B, kW, kW, UM, &t.sigA[1]);
    ok = ok && sw128_map(n->d16t, UN, kB, n->R, UN, &t.wgB[0]);
    ok = ok && sw128_map(n->e16t, UN, kB, n->R, UN, &t.wgB[1]);
    if (ok) t.B = B;
    return ok;
}

cudaError_t set_smem_attrs(int dev) {
    static unsigned long long done = 0;  // one bit per device
    const unsigned long long bit = 1ull << (dev & 63);
    if (done & bit) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_umma_rows, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kRowsSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_umma_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kWgSmem);
    if (e == cudaSuccess) done |= bit;
    return e;
}

// CTAs of the persistent row kernel for M rows: one per SM at most, and at
// most kRowGridCap (the rows of column sums it leaves are sized by that)
int rows_grid(const lbm_mlp* n, int M) {
    const int tiles = (M + UM - 1) / UM;
    const int cap = n->nsm < kRowGridCap ? n->nsm : kRowGridCap;
    return tiles < cap ? tiles : cap;
}

// D[M x 256] = A Bt^T with the epilogue of g
cudaError_t rows_tc(lbm_mlp* n, const CUtensorMap& ta, const CUtensorMap& tb, const RowArgs& g) {
    k_umma_rows<<<rows_grid(n, g.M), kRowsThreads, kRowsSmem, n->stream>>>(ta, tb, g);
    return cudaGetLastError();
}

// gw [fi][256] = A^T D over a batch of B, and gb [256] from the nb column-sum
// rows that the kernel producing D left in n->bpart
cudaError_t wgrad_tc(lbm_mlp* n, const CUtensorMap& ta, const CUtensorMap& tb, int fi, int B,
                     float* gw, int nb, float* gb) {
    const Slicing sl = slicing(B);
    const int mtiles = (fi + UM - 1) / UM;
    WgArgs w;
    w.mtiles = mtiles;
    w.chunks = sl.chunks;
    w.per_slice = sl.per_slice;
    w.part = n->part;
    w.err = n->err;
    k_umma_wgrad<<<dim3(mtiles, sl.slices), kWgThreads, kWgSmem, n->stream>>>(ta, tb, w);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_wgrad_reduce<<<(fi * UN + UN + 31) / 32, dim3(32, 8), 0, n->stream>>>(
        n->part, sl.slices, mtiles * UM, fi, gw, n->bpart, nb, gb);
    return cudaGetLastError();
}

// forward pass on tcgen05.  t null: inference, only the output (written to y).
// t not null: training; the hidden layers keep what the backward pass needs
// (FP32 activations, transposed BF16 copies), and the last layer's epilogue
// turns its output straight into the loss signal dL/dy (BF16, transposed BF16,
// column sums) and the squared-error sum, without storing y.
lbm_status forward_tc(lbm_mlp* n, const float* x, int B, const float* t, float* y) {
    cudaStream_t s = n->stream;
    const bool train = t != nullptr;
    const int kB = rows_of(B);
    const int threads = kK0 * B > kInPad * kB ? kK0 * B : kInPad * kB;
    k_input<<<(threads + 255) / 256, 256, 0, s>>>(x, n->x16, B, train ? n->x16t : nullptr, n->R,
                                                  kB);
    CK(cudaGetLastError());
    if (train) CK(cudaMemsetAsync(n->sse, 0, sizeof(double), s));
    for (int l = 0; l < kLayers; ++l) {
        const bool hidden = l < kLayers - 1;
        RowArgs g{};
        g.M = B;
        g.K = l == 0 ? kK0 : kW;
        g.bias = n->p + param_offset(l) + (long long)kFanIn[l] * kFanOut[l];
        g.ld32 = kW;
        g.ld16 = kW;
        g.ldt = n->R;
        g.rows_t = kB;
        g.err = n->err;
        if (hidden) {
            g.epi = EPI_BIAS_TANH;
            g.out32 = train ? n->a32[l] : nullptr;
            g.out16 = n->a16[l];
            g.out16t = train ? n->a16t[l] : nullptr;
        } else if (train) {
            g.epi = EPI_LOSS;
            g.aprev = t;
            g.scale = 1.0f / ((float)B * kOut);
            g.sse = n->sse;
            g.out16 = n->d16;
            g.out16t = n->d16t;
            g.bpart = n->bpart;
        } else {
            g.epi = EPI_BIAS;
            g.out32 = y;
        }
        CK(rows_tc(n, n->maps.fwdA[l], n->maps.fwdB[l], g));
    }
    return LBM_OK;
}

// the gradient on tcgen05, after forward_tc with targets
lbm_status backward_tc(lbm_mlp* n, int B) {
    int sig = 0;  // which of (d, e) holds the current signal
    for (int l = kLayers - 1; l >= 0; --l) {
        const int fi = kFanIn[l], fo = kFanOut[l];
        float* gw = n->g + param_offset(l);
        float* gb = gw + (long long)fi * fo;
        // dW = A_{l-1}^T D from the transposed copies; db from the column sums
        CK(wgrad_tc(n, n->maps.wgA[l], n->maps.wgB[sig], fi, B, gw, 4 * rows_grid(n, B), gb));
        if (l == 0) break;
        // D_{l-1} = (D W_l^T) (1 - A_{l-1}^2): K-major operands are D [B][fo] and
        // W_l itself ([fi][fo])
        RowArgs g{};
        g.M = B;
        g.K = fo;
        g.epi = EPI_TANH_BACK;
        g.aprev = n->a32[l - 1];
        g.out16 = sig == 0 ? n->e16 : n->d16;
        g.ld16 = fi;
        g.out16t = sig == 0 ? n->e16t : n->d16t;
        g.ldt = n->R;
        g.rows_t = rows_of(B);
        g.bpart = n->bpart;
        g.err = n->err;
        CK(rows_tc(n, n->maps.sigA[sig], n->maps.sigB[l], g));
        sig ^= 1;
    }
    return LBM_OK;
}

// the mma.sync forward pass (every layer's FP32 output kept)
lbm_status forward_ms(lbm_mlp* n, const float* x, int B) {
    cudaStream_t s = n->stream;
    k_input<<<(B * kK0 + 255) / 256, 256, 0, s>>>(x, n->x16, B, nullptr, 0, 0);
    CK(cudaGetLastError());
    for (int l = 0; l < kLayers; ++l) {
        GemmArgs g{};
        g.A = l == 0 ? n->x16 : n->a16[l - 1];
        g.sam = l == 0 ? kK0 : kW;
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

// whether this call runs on tcgen05 (maps for batch B made, attributes set)
bool use_tc(lbm_mlp* n, int B, lbm_status* st) {
    *st = LBM_OK;
    if (!n->tensor_cores) return false;
    if (!prepare_maps(n, B)) {
        n->tensor_cores = false;  // no tensor map: the mma.sync kernel from here on
        return false;
    }
    if (set_smem_attrs(n->dev) != cudaSuccess) *st = LBM_ECUDA;
    return true;
}


// loss and gradient into n->g (device) on the mma.sync kernel, after forward_ms()
lbm_status backward_ms(lbm_mlp* n, const float* t, int B) {
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
        g.sak = l == 0 ? kK0 : kW;
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
        // D_{l-1} = (D W_l^T) (1 - A_{l-1}^2)
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
    n->w16t = (__nv_bfloat16*)(w + L.w16t);
    n->x16 = (__nv_bfloat16*)(w + L.x16);
    n->x16t = (__nv_bfloat16*)(w + L.x16t);
    n->R = rows_of(max_batch);
    const size_t R = (size_t)n->R;
    for (int l = 0; l < kLayers; ++l) n->a32[l] = (float*)(w + L.a32) + (size_t)l * R * kW;
    for (int l = 0; l < kLayers - 1; ++l) {
        n->a16[l] = (__nv_bfloat16*)(w + L.a16) + (size_t)l * R * kW;
        n->a16t[l] = (__nv_bfloat16*)(w + L.a16t) + (size_t)l * R * kW;
    }
    n->err = (int*)(w + L.err);
    n->d32 = (float*)(w + L.d32);
    n->d16 = (__nv_bfloat16*)(w + L.d16);
    n->d16t = (__nv_bfloat16*)(w + L.d16t);
    n->e32 = (float*)(w + L.e32);
    n->e16 = (__nv_bfloat16*)(w + L.e16);
    n->e16t = (__nv_bfloat16*)(w + L.e16t);
    n->part = (float*)(w + L.part);
    n->bpart = (float*)(w + L.bpart);
    n->sse = (double*)(w + L.sse);
    n->step = 0;
    n->tensor_cores = true;
    if (cudaDeviceGetAttribute(&n->nsm, cudaDevAttrMultiProcessorCount, n->dev) != cudaSuccess ||
        n->nsm < 1) {
        delete n;
        return LBM_ECUDA;
    }
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
    lbm_status st = LBM_OK;
    if (use_tc(n, batch, &st)) return st ? st : forward_tc(n, d_x, batch, nullptr, d_y);
    if (st) return st;
    st = forward_ms(n, d_x, batch);
    if (st) return st;
    CK(cudaMemcpyAsync(d_y, n->a32[kLayers - 1], (size_t)batch * kOut * 4,
                       cudaMemcpyDeviceToDevice, n->stream));
    return LBM_OK;
}

lbm_status lbm_mlp_loss_grad(lbm_mlp* n, const float* d_x, const float* d_t, int32_t batch,
                             double* h_loss, float* d_grad) {
    if (!n || !d_x || !d_t || batch < 1 || batch > n->max_batch) return LBM_EINVAL;
    CK(cudaSetDevice(n->dev));
    lbm_status st = LBM_OK;
    const bool tc = use_tc(n, batch, &st);
    if (st) return st;
    if (tc) {
        st = forward_tc(n, d_x, batch, d_t, nullptr);
        if (!st) st = backward_tc(n, batch);
    } else {
        st = forward_ms(n, d_x, batch);
        if (!st) st = backward_ms(n, d_t, batch);
    }
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
