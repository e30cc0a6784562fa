// BF16 tensor-core GEMM for the learned transfer function (sm_103a, mma.sync m16n8k16 with
// FP32 accumulation), with the epilogues the MLP needs fused in.
//
//   C[M, N] = A[M, K] * B[K, N]
//   A_T = false: A stored row-major M x K (lda = K);  A_T = true: A stored as K x M (lda = M)
//   B_T = false: B stored row-major K x N (ldb = N);  B_T = true: B stored as N x K (ldb = K)
// M, N multiples of 128, K a multiple of 32 (callers pad).  CTA tile 128 x 128 x 32, eight
// warps (2 x 4) of 64 x 32, operands staged in shared memory with cp.async double buffering
// and loaded into fragments with ldmatrix (transposed where the storage is K-major).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace odx {
namespace mlp {

constexpr int BM = 128, BN = 128, BK = 32, GEMM_THREADS = 256;

enum Epilogue : int {
    EPI_BIAS_SILU = 0,    // z = acc + bias[n]; Z = bf16(z) (if Z), H = bf16(silu(z))
    EPI_DSILU = 1,        // dZ = bf16(acc * silu'(Z))
    EPI_ATOMIC_F32 = 2,   // C32[m, n] += acc (split-K weight gradients)
};

struct EpiArgs {
    const float *bias;        // EPI_BIAS_SILU
    __nv_bfloat16 *Z;         // EPI_BIAS_SILU (may be null) / EPI_DSILU input
    __nv_bfloat16 *H;         // EPI_BIAS_SILU output / EPI_DSILU output (dZ)
    float *C32;               // EPI_ATOMIC_F32
    int ldc;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(smem)), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ void ldsm_x4(uint32_t r[4], const void *p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t r[4], const void *p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}

__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float silu(float z) { return z / (1.f + __expf(-z)); }
__device__ __forceinline__ float dsilu(float z)
{
    const float s = 1.f / (1.f + __expf(-z));
    return s * (1.f + z * (1.f - s));
}

// Shared-memory tile geometry (padded rows keep ldmatrix conflict-light and 16-byte aligned).
template <bool T_KMAJOR, int ROWS_MN>
struct TileGeom {
    // T_KMAJOR = false: stored [ROWS_MN][BK]; true: stored [BK][ROWS_MN]
    static constexpr int LD = T_KMAJOR ? ROWS_MN + 8 : BK + 8;
    static constexpr int ELEMS = T_KMAJOR ? BK * LD : ROWS_MN * LD;
};

template <bool A_T, bool B_T, int EPI>
__global__ void __launch_bounds__(GEMM_THREADS) gemm_bf16_kernel(
    const __nv_bfloat16 *__restrict__ A, const __nv_bfloat16 *__restrict__ B, int M, int N,
    int K, int lda, int ldb, int k_per_split, EpiArgs ep)
{
    using GA = TileGeom<A_T, BM>;
    using GB = TileGeom<!B_T, BN>;  // B stored K x N is "K-major" (rows = k)
    __shared__ __align__(16) __nv_bfloat16 sA[2][GA::ELEMS];
    __shared__ __align__(16) __nv_bfloat16 sB[2][GB::ELEMS];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp >> 2, wn = warp & 3;  // 2 x 4 warps
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int k_begin = blockIdx.z * k_per_split;
    const int k_end = min(K, k_begin + k_per_split);
    const int ktiles = (k_end - k_begin) / BK;

    auto load_tile = [&](int buf, int kt) {
        const int k0 = k_begin + kt * BK;
        // 512 16-byte chunks per operand tile, 2 per thread
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int chunk = tid + c * GEMM_THREADS;
            if (!A_T) {  // [BM][BK]: 4 chunks per row
                const int r = chunk >> 2, cc = (chunk & 3) * 8;
                cp_async16(&sA[buf][r * GA::LD + cc], A + (size_t)(m0 + r) * lda + k0 + cc);
            } else {     // [BK][BM]: 16 chunks per row
                const int r = chunk >> 4, cc = (chunk & 15) * 8;
                cp_async16(&sA[buf][r * GA::LD + cc], A + (size_t)(k0 + r) * lda + m0 + cc);
            }
            if (B_T) {   // stored [BN][BK]
                const int r = chunk >> 2, cc = (chunk & 3) * 8;
                cp_async16(&sB[buf][r * GB::LD + cc], B + (size_t)(n0 + r) * ldb + k0 + cc);
            } else {     // stored [BK][BN]
                const int r = chunk >> 4, cc = (chunk & 15) * 8;
                cp_async16(&sB[buf][r * GB::LD + cc], B + (size_t)(k0 + r) * ldb + n0 + cc);
            }
        }
        cp_async_commit();
    };

    float acc[4][4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[i][j][v] = 0.f;

    if (ktiles > 0) load_tile(0, 0);
    for (int kt = 0; kt < ktiles; ++kt) {
        const int buf = kt & 1;
        if (kt + 1 < ktiles) {
            load_tile(buf ^ 1, kt + 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const __nv_bfloat16 *a_s = sA[buf];
        const __nv_bfloat16 *b_s = sB[buf];
        const int j8 = lane >> 3, r8 = lane & 7;
#pragma unroll
        for (int ks = 0; ks < BK; ks += 16) {
            uint32_t af[4][4], bf[2][4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int mm = wm * 64 + i * 16;
                if (!A_T) {
                    ldsm_x4(af[i], a_s + (mm + (lane & 15)) * GA::LD + ks + (lane >> 4) * 8);
                } else {
                    ldsm_x4_t(af[i], a_s + (ks + r8 + (j8 >> 1) * 8) * GA::LD + mm + (j8 & 1) * 8);
                }
            }
#pragma unroll
            for (int jj = 0; jj < 2; ++jj) {  // two n16 groups = four n8 tiles
                const int nn = wn * 32 + jj * 16;
                if (B_T) {
                    ldsm_x4(bf[jj], b_s + (nn + r8 + (j8 >> 1) * 8) * GB::LD + ks + (j8 & 1) * 8);
                } else {
                    ldsm_x4_t(bf[jj], b_s + (ks + r8 + (j8 & 1) * 8) * GB::LD + nn + (j8 >> 1) * 8);
                }
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    mma_bf16(acc[i][j], af[i], bf[j >> 1][(j & 1) * 2], bf[j >> 1][(j & 1) * 2 + 1]);
        }
        __syncthreads();
    }

    // epilogue: fragment (i, j): rows g, g+8 and columns 2q, 2q+1 of the 16 x 8 tile
    const int g = lane >> 2, q = lane & 3;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int m = m0 + wm * 64 + i * 16 + g + h * 8;
                const int n = n0 + wn * 32 + j * 8 + 2 * q;
                const float v0 = acc[i][j][2 * h], v1 = acc[i][j][2 * h + 1];
                if constexpr (EPI == EPI_BIAS_SILU) {
                    const float z0 = v0 + ep.bias[n], z1 = v1 + ep.bias[n + 1];
                    const size_t o = (size_t)m * ep.ldc + n;
                    if (ep.Z)
                        *reinterpret_cast<__nv_bfloat162 *>(ep.Z + o) = __floats2bfloat162_rn(z0, z1);
                    *reinterpret_cast<__nv_bfloat162 *>(ep.H + o) =
                        __floats2bfloat162_rn(silu(z0), silu(z1));
                } else if constexpr (EPI == EPI_DSILU) {
                    const size_t o = (size_t)m * ep.ldc + n;
                    const __nv_bfloat162 z = *reinterpret_cast<const __nv_bfloat162 *>(ep.Z + o);
                    const float2 zf = __bfloat1622float2(z);
                    *reinterpret_cast<__nv_bfloat162 *>(ep.H + o) =
                        __floats2bfloat162_rn(v0 * dsilu(zf.x), v1 * dsilu(zf.y));
                } else {
                    float *c = ep.C32 + (size_t)m * ep.ldc + n;
                    atomicAdd(c, v0);
                    atomicAdd(c + 1, v1);
                }
            }
        }
    }
}

}  // namespace mlp
}  // namespace odx
