// Learned thin-disk transfer function (alpha, beta, a, cos i) -> (capture logit, log r_cross,
// phi_cross / pi, g): 4 -> 256 -> 256 -> 256 -> 256 -> 4 with SiLU, BF16 weights and
// activations, FP32 accumulation.  The 256 x 256 layers run on the tcgen05 tensor cores
// (accumulators in tensor memory): inference and the training forward pass as one fused
// chain per 128-row tile (mlp_chain_tc), the backward dL/dZ chain the same way, and the
// weight gradients as batch-reduction MMAs (mlp_dw_tc); the 4-wide input and output layers
// and Adam run on CUDA cores.  The surrogate render
// classifies each pixel and hands the uncertain ones (near the Bardeen critical curve or
// with an unsure capture probability) back to the ray tracer.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "f32x2.cuh"
#include "kerr_device.cuh"
#include "odx_internal.h"
#include "tcgen05.cuh"

namespace odx {
int32_t validate_scene_table(const odx_scene *scenes, int32_t n_scenes);
void fill_dev_scene(DevScene &d, const odx_scene &s, int64_t ray_begin, int64_t n_rays,
                    int64_t img_offset);
struct CtxView {
    int device, num_sms;
    odx_launch launch;
    unsigned long long *queue;
    DevStats *stats;
};
int32_t ctx_view(odx_ctx *ctx, CtxView *v);
}  // namespace odx

using namespace odx;
using bf16 = __nv_bfloat16;

namespace {

constexpr int HID = ODX_MLP_HIDDEN, NIN = 4, NOUT = 4, NLAYER_HIDDEN = ODX_MLP_DEPTH;
// flat FP32 parameter layout: W1[4][256] b1[256] (W[256][256] b[256]) x 3 W5[256][4] b5[4]
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NIN * HID;
constexpr int OFF_W2 = OFF_B1 + HID;
constexpr int LAYER_SZ = HID * HID + HID;
constexpr int OFF_W5 = OFF_W2 + (NLAYER_HIDDEN - 1) * LAYER_SZ;
constexpr int OFF_B5 = OFF_W5 + HID * NOUT;
constexpr int NPARAM = OFF_B5 + NOUT;
static_assert(NPARAM == ODX_MLP_PARAMS, "parameter count");

__host__ __device__ constexpr int off_w(int l) { return OFF_W2 + (l - 2) * LAYER_SZ; }  // l = 2..4
__host__ __device__ constexpr int off_b(int l) { return off_w(l) + HID * HID; }

// 16-byte global -> shared copies (cp.async groups), used to stage the weight-gradient operands
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(
                     static_cast<uint32_t>(__cvta_generic_to_shared(smem))),
                 "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

}  // namespace

struct odx_mlp {
    odx_ctx *ctx = nullptr;
    int device = 0;
    int64_t max_batch = 0;  // multiple of 128
    float *p = nullptr;      // FP32 master parameters
    bf16 *pb = nullptr;      // BF16 copy used by the kernels
    float *grad = nullptr, *m1 = nullptr, *m2 = nullptr;
    int64_t step = 0;
    bf16 *Z[5] = {}, *H[5] = {};  // layers 1..4
    bf16 *dZ[5] = {};             // dL/dZ_l, layers 1..4 (backward)
    float *dY = nullptr, *loss = nullptr;
    float *loss_part = nullptr, *col_part = nullptr;  // per-block loss and column partials
    float *xin = nullptr;   // padded input rows for inference
    bf16 *wpack = nullptr;   // hidden-layer weights as forward tensor-core operands (W^T)
    bf16 *wpackB = nullptr;  // ... and as backward operands (W)
    float *dw_part = nullptr;  // per-split weight-gradient partial sums
    int *tc_err = nullptr;  // set by a tensor-core kernel whose wait timed out
    uint32_t wait_limit = 0;  // polls of an in-loop tensor-core wait (0: TC_WAIT)
    int num_sms = 0;
    // surrogate render workspace
    int64_t surr_cap = 0;
    float *surr_x = nullptr, *surr_y = nullptr;
    double *fb_rays = nullptr;
    int64_t *fb_pix = nullptr;
    unsigned long long *fb_count = nullptr;
    float *bcrit = nullptr;  // critical-curve table
    DevScene *scene_tab = nullptr;
};

namespace {

#define MLP_CUDA(call)                                   \
    do {                                                 \
        if ((call) != cudaSuccess) return ODX_ERR_CUDA;  \
    } while (0)

__device__ __forceinline__ float bfv(const bf16 *p, int64_t i) { return __bfloat162float(p[i]); }

// Adam (Kingma & Ba 2015) on the FP32 master weights; refreshes the BF16 copy.
__global__ void adam_step(float *p, bf16 *pb, const float *g, float *m1, float *m2, int n,
                          float lr, float b1, float b2, float eps, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float a = b1 * m1[i] + (1.f - b1) * gi;
    const float v = b2 * m2[i] + (1.f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = v;
    const float w = p[i] - lr * (a / c1) / (sqrtf(v / c2) + eps);
    p[i] = w;
    pb[i] = __float2bfloat16_rn(w);
}

__global__ void to_bf16(const float *p, bf16 *pb, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) pb[i] = __float2bfloat16_rn(p[i]);
}

// Deterministic initialisation: counter-based hash -> uniform in [-s, s], s = 1/sqrt(fan_in).
__device__ __forceinline__ uint64_t mix64(uint64_t z)
{
    z += 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}
__global__ void init_params(float *p, bf16 *pb, uint64_t seed)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NPARAM) return;
    int fan_in;
    bool bias;
    if (i < OFF_B1) { fan_in = NIN; bias = false; }
    else if (i < OFF_W2) { fan_in = NIN; bias = true; }
    else if (i < OFF_W5) {
        const int r = (i - OFF_W2) % LAYER_SZ;
        fan_in = HID;
        bias = r >= HID * HID;
    } else { fan_in = HID; bias = i >= OFF_B5; }
    const double u = (double)(mix64(seed ^ (uint64_t)i * 0x2545f4914f6cdd1dULL) >> 11) * 0x1.0p-53;
    const float w = bias ? 0.f : (float)((2.0 * u - 1.0) / sqrt((double)fan_in));
    p[i] = w;
    pb[i] = __float2bfloat16_rn(w);
}

// ---- training targets from traced rays -----------------------------------------------------
// x = (alpha/20, beta/20, a, cos i); t = (captured, log r, phi/pi, g, mask_cross, mask_g, 0, 0)
// where (r, phi) is the disk hit for rays that stop on the disk, else the first crossing if
// r <= r_max; g is defined on disk hits.
__global__ void make_targets(const odx_ray_record *__restrict__ rec, const double *__restrict__ rays,
                             int64_t n, int64_t n_pad, double r_max, float *x, float *t)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_pad) return;
    float xv[4] = {0.f, 0.f, 0.f, 0.f}, tv[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (i < n) {
        const double *r4 = rays + 4 * i;
        xv[0] = (float)(r4[0] / 20.0);
        xv[1] = (float)(r4[1] / 20.0);
        xv[2] = (float)r4[2];
        xv[3] = (float)r4[3];
        const odx_ray_record &R = rec[i];
        tv[0] = (R.status == ODX_CAPTURED) ? 1.f : 0.f;
        if (R.status == ODX_DISK_HIT) {
            tv[1] = (float)log(R.r_hit);
            tv[2] = (float)(R.phi_hit / M_PI);
            tv[3] = (float)R.g;
            tv[4] = 1.f;
            tv[5] = 1.f;
        } else if (R.n_cross >= 1 && R.r_cross <= r_max && R.status != ODX_CAPTURED) {
            tv[1] = (float)log(R.r_cross);
            tv[2] = (float)(R.phi_cross / M_PI);
            tv[4] = 1.f;
        }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) x[i * 4 + k] = xv[k];
#pragma unroll
    for (int k = 0; k < 8; ++k) t[i * 8 + k] = tv[k];
}

// ---- surrogate render ---------------------------------------------------------------------
constexpr int BCRIT_N = 4096;

// Critical curve of Kerr (Bardeen 1973): spherical photon orbits at r in [r_pro, r_ret] with
// xi = L/E, eta = Q/E^2; image-plane point alpha = -xi / sin i, beta = +-sqrt(eta + a^2 cos^2 i
// - xi^2 cot^2 i).  Table: for BCRIT_N polar angles psi in [-pi, pi), the radius b_c(psi).
__global__ void bcrit_table(double a, double inc, double r_in_scene, float *tab)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j == 0) tab[BCRIT_N] = (float)(r_in_scene > 0.0 ? r_in_scene : isco_radius(a));
    if (j >= BCRIT_N) return;
    const double psi = -M_PI + (j + 0.5) * (2.0 * M_PI / BCRIT_N);
    if (fabs(a) < 1e-6) {
        tab[j] = (float)(3.0 * sqrt(3.0));
        return;
    }
    const double si = fmax(sin(inc), 1e-6), ci = cos(inc);
    const double r_pro = 2.0 * (1.0 + cos(2.0 / 3.0 * acos(-a)));
    const double r_ret = 2.0 * (1.0 + cos(2.0 / 3.0 * acos(a)));
    const double sgn = psi >= 0.0 ? 1.0 : -1.0;  // upper or lower half
    const double target = fabs(psi);             // angle from +alpha on that half, in [0, pi]
    // along r the upper-half angle decreases from ~pi (prograde side) to ~0 (retrograde side);
    // bisect on r over the part of the curve that is visible (beta^2 >= 0)
    auto point = [&](double r, double &al, double &be2) {
        const double xi = (r * r * (3.0 - r) - a * a * (r + 1.0)) / (a * (r - 1.0));
        const double eta = r * r * r * (4.0 * a * a - r * (r - 3.0) * (r - 3.0)) /
                           (a * a * (r - 1.0) * (r - 1.0));
        al = -xi / si;
        be2 = eta + a * a * ci * ci - xi * xi * ci * ci / (si * si);
    };
    double lo = r_pro, hi = r_ret;
    for (int it = 0; it < 80; ++it) {
        const double mid = 0.5 * (lo + hi);
        double al, be2;
        point(mid, al, be2);
        const double ang = atan2(sqrt(fmax(be2, 0.0)), al);
        if (ang > target) lo = mid; else hi = mid;
    }
    double al, be2;
    point(0.5 * (lo + hi), al, be2);
    (void)sgn;
    tab[j] = (float)sqrt(al * al + fmax(be2, 0.0));
}

__global__ void surrogate_inputs(const DevScene *S, int64_t n_pad, float *x)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_pad) return;
    const odx_scene &s = S->s;
    const int64_t n = (int64_t)s.n_alpha * s.n_beta;
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    if (p < n) {
        const int64_t i = p % s.n_alpha, j = p / s.n_alpha;
        const double al = s.alpha_min + (((double)i + 0.5) * (s.alpha_max - s.alpha_min)) / s.n_alpha;
        const double be = s.beta_min + (((double)j + 0.5) * (s.beta_max - s.beta_min)) / s.n_beta;
        v[0] = (float)(al / 20.0);
        v[1] = (float)(be / 20.0);
        v[2] = (float)s.a;
        v[3] = (float)cos(s.theta_obs);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) x[p * 4 + k] = v[k];
}

// Per pixel: fallback if |b - b_c(psi)| < band or the capture probability is in [p_lo, p_hi];
// otherwise the surrogate's thin-disk intensity.  Fallback pixels are compacted per warp
// (ballot, one atomicAdd per warp) into a ray list and a pixel list.
__global__ void surrogate_classify(const DevScene *S, const float *__restrict__ y,
                                   const float *__restrict__ tab, double band, float p_lo,
                                   float p_hi, double *image, double *fb_rays, int64_t *fb_pix,
                                   unsigned long long *fb_count)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const odx_scene &s = S->s;
    const int64_t n = (int64_t)s.n_alpha * s.n_beta;
    bool fb = false;
    double al = 0.0, be = 0.0;
    if (p < n) {
        const int64_t i = p % s.n_alpha, j = p / s.n_alpha;
        al = s.alpha_min + (((double)i + 0.5) * (s.alpha_max - s.alpha_min)) / s.n_alpha;
        be = s.beta_min + (((double)j + 0.5) * (s.beta_max - s.beta_min)) / s.n_beta;
        const float *yp = y + p * 4;
        const float prob = 1.f / (1.f + __expf(-yp[0]));
        const float alf = (float)al, bef = (float)be;
        const float psi = atan2f(bef, alf);
        int k = (int)floorf((psi + (float)M_PI) / (2.f * (float)M_PI) * BCRIT_N);
        k = min(max(k, 0), BCRIT_N - 1);
        const float b = sqrtf(alf * alf + bef * bef);
        fb = fabsf(b - tab[k]) < (float)band || (prob >= p_lo && prob <= p_hi);
        float I = 0.f;
        if (!fb && prob < 0.5f) {
            const float r = __expf(yp[1]);
            if (r >= tab[BCRIT_N] && r <= (float)s.r_out) {
                const float g = yp[3];
                I = g * g * g * g * __powf(r, -(float)s.q_emis);
            }
        }
        image[p] = fb ? 0.0 : (double)I;
    }
    const unsigned m = __ballot_sync(0xffffffffu, fb);
    if (m == 0u) return;
    const int lane = threadIdx.x & 31;
    unsigned long long base = 0;
    if (lane == __ffs(m) - 1) base = atomicAdd(fb_count, (unsigned long long)__popc(m));
    base = __shfl_sync(0xffffffffu, base, __ffs(m) - 1);
    if (fb) {
        const unsigned long long slot = base + __popc(m & ((1u << lane) - 1u));
        fb_rays[4 * slot + 0] = al;
        fb_rays[4 * slot + 1] = be;
        fb_rays[4 * slot + 2] = s.a;
        fb_rays[4 * slot + 3] = cos(s.theta_obs);
        fb_pix[slot] = p;
    }
}

__global__ void scatter_fallback(const odx_ray_record *__restrict__ rec,
                                 const int64_t *__restrict__ pix, int64_t m, double *image)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < m) image[pix[j]] = rec[j].intensity;
}

unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// ---- training passes on the fifth-generation tensor cores (tcgen05) ----------------------
// One CTA per SM walks 128-row tiles.  Per tile: layer 1 (4 -> 256) on CUDA cores (or dZ_4
// from HBM) into the activation tile A (shared memory, BF16, K-major core-matrix layout);
// for each 256 x 256 layer the weights W_l^T (packed once into the same layout, 128 KB)
// arrive by bulk copy, one thread issues 16 MMAs of 128 x 256 x 16 with the FP32 accumulator
// in tensor memory (256 of its 512 columns), the warps read the accumulator back (bias +
// SiLU, BF16; or SiLU' for the backward pass) into A and HBM.  The next layer's weights are
// loaded while the epilogue runs.  Every wait is bounded: on a time-out the kernel flags
// *err, waits (bounded) for its own copies and MMAs, frees its tensor memory and returns.
constexpr int TC_THREADS = 512, TC_ROWS = 128, TC_CG = TC_THREADS / TC_ROWS;  // column groups
constexpr int TC_COLS = HID / TC_CG;  // columns of one row per thread (64)
constexpr uint32_t TC_A_BYTES = TC_ROWS * HID * 2, TC_B_BYTES = HID * HID * 2;
constexpr uint32_t TC_TMEM_COLS = 256;
constexpr uint32_t TC_WAIT = 1u << 20;
// small operands staged in shared memory: W1^T as float4 per column, biases b1..b4 (and,
// for inference, W5 as float4 per input column and b5)
constexpr size_t TC_CONST_BYTES = (HID * 4 + 4 * HID) * sizeof(float);
constexpr size_t TC_SMEM = 1024 + TC_A_BYTES + TC_B_BYTES + TC_CONST_BYTES + 64;
static_assert(TC_SMEM <= 232448, "shared memory of one CTA");

// The training passes share one kernel shape (a 128-row tile through the three 256 x 256
// layers); inference has a kernel of its own (mlp_infer_ts).
enum TcMode : int {
    TC_TRAIN = 1,  // training forward: Z_l and H_l (l = 1..4) kept in HBM for the backward pass
    TC_BWD = 2,    // backward: dZ_4 -> dZ_3, dZ_2, dZ_1 through W_4^T, W_3^T, W_2^T and SiLU'
};

struct TcArgs {
    const float *x;     // forward: input rows [n][4]
    const bf16 *pb;     // BF16 parameters (W1, W5)
    const float *p;     // FP32 parameters (biases)
    const bf16 *wpack;  // the three packed B operands in the order of use, 128 KB each
    int64_t n_rows;
    float *y;           // inference: outputs [n][4]
    bf16 *Z[5], *H[5];  // TC_TRAIN: written (l = 1..4); TC_BWD: Z_1..Z_3 read
    const bf16 *dZ4;    // TC_BWD: input
    bf16 *dZ[5];        // TC_BWD: dZ_3, dZ_2, dZ_1 written
    int *err;
    uint32_t wait_limit;  // polls of a wait inside the tile loop (teardown waits use TC_WAIT)
};

// Forward operands: B[n][k] = W_l[k][n] (z = h W); backward operands: B[k][n] = W_l[k][n]
// (dh = dz W^T).  Either way the K-major core-matrix layout, one 128 KB block per layer,
// blocks in the order the pass uses them (forward l = 2, 3, 4; backward l = 4, 3, 2).
__global__ void pack_hidden_weights(const bf16 *__restrict__ pb, bf16 *__restrict__ wpack,
                                    int backward, float scale)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 3 * HID * HID) return;
    const int i = idx / (HID * HID), e = idx % (HID * HID);
    const int k = e / HID, n = e % HID;  // W_l[k][n]
    const int l = backward ? 4 - i : 2 + i;
    const uint32_t off = backward ? tc::kmajor_offset(k, n, HID) : tc::kmajor_offset(n, k, HID);
    wpack[(size_t)i * HID * HID + off / 2] =
        __float2bfloat16_rn(__bfloat162float(pb[off_w(l) + k * HID + n]) * scale);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&v);
}

__device__ __forceinline__ float tanh_fast(float x)
{
    float t;
    asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(x));
    return t;
}
// SiLU as z (1 + tanh(z / 2)) / 2 and its derivative s (1 + z (1 - s)), s = (1 + tanh(z/2)) / 2,
// with the hardware tanh (one SFU operation; relative error ~2^-11, under the BF16 rounding)
__device__ __forceinline__ float silu_fast(float z)
{
    const float hz = 0.5f * z;
    return fmaf(hz, tanh_fast(hz), hz);
}
__device__ __forceinline__ float dsilu_fast(float z)
{
    const float s = fmaf(0.5f, tanh_fast(0.5f * z), 0.5f);
    return s * fmaf(z, 1.f - s, 1.f);
}

__device__ __forceinline__ uint4 pack8(const float *h)
{
    return make_uint4(pack_bf16x2(h[0], h[1]), pack_bf16x2(h[2], h[3]), pack_bf16x2(h[4], h[5]),
                      pack_bf16x2(h[6], h[7]));
}
__device__ __forceinline__ void unpack8(uint4 u, float *f)
{
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const __nv_bfloat162 v = *reinterpret_cast<const __nv_bfloat162 *>(&w[i]);
        const float2 t = __bfloat1622float2(v);
        f[2 * i] = t.x;
        f[2 * i + 1] = t.y;
    }
}

template <int MODE>
__global__ void __launch_bounds__(TC_THREADS, 1) mlp_chain_tc(const __grid_constant__ TcArgs A)
{
    extern __shared__ __align__(16) unsigned char tc_raw[];
    unsigned char *sA = reinterpret_cast<unsigned char *>(
        ((uintptr_t)tc_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *sB = sA + TC_A_BYTES;
    float4 *sW1 = reinterpret_cast<float4 *>(sB + TC_B_BYTES);  // [256]
    float *sBias = reinterpret_cast<float *>(sW1 + HID);         // [4][256]: b1..b4
    uint64_t *bars = reinterpret_cast<uint64_t *>(
        ((uintptr_t)(sBias + 4 * HID) + 7) & ~(uintptr_t)7);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 2);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t wbar = tc::smem_u32(&bars[0]), mbar = tc::smem_u32(&bars[1]);
    const uint32_t a_base = tc::smem_u32(sA), b_base = tc::smem_u32(sB);
    const int64_t n_rows = A.n_rows;
    const int64_t n_tiles = (n_rows + TC_ROWS - 1) / TC_ROWS;
    if (tid == 0) {
        tc::mbar_init(wbar, 1);
        tc::mbar_init(mbar, 1);
        tc::mbar_fence_init();
    }
    if constexpr (MODE != TC_BWD) {
        for (int n = tid; n < HID; n += TC_THREADS) {
            sW1[n] = make_float4(bfv(A.pb, OFF_W1 + 0 * HID + n), bfv(A.pb, OFF_W1 + 1 * HID + n),
                                 bfv(A.pb, OFF_W1 + 2 * HID + n), bfv(A.pb, OFF_W1 + 3 * HID + n));
            sBias[n] = A.p[OFF_B1 + n];
            for (int l = 2; l <= 4; ++l) sBias[(l - 1) * HID + n] = A.p[off_b(l) + n];
        }
    }
    if (warp == 0) tc::tmem_alloc(tslot, TC_TMEM_COLS);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;

    // packed operand i (0..2) into sB (thread 0): one 128 KB image, four bulk copies
    auto load_weights = [&](int i) {
        tc::mbar_expect_tx(wbar, TC_B_BYTES);
#pragma unroll
        for (int c = 0; c < 4; ++c)
            tc::bulk_g2s(b_base + c * (TC_B_BYTES / 4),
                         A.wpack + (size_t)i * HID * HID + c * (HID * HID / 4), TC_B_BYTES / 4,
                         wbar);
    };
    uint32_t wphase = 0, mphase = 0;
    bool w_pending = false, m_pending = false, failed = false;
    if (tid == 0 && blockIdx.x < n_tiles) {
        load_weights(0);
        w_pending = true;
    }
    const uint32_t idesc = tc::idesc_bf16_f32(TC_ROWS, HID);
    const int row = tid & (TC_ROWS - 1), cg1 = tid >> 7;  // tile input: row, column group
    const int lg = warp & 3, cg = warp >> 2;               // epilogue: TMEM lanes, column group
    const int r = 32 * lg + lane;                          // epilogue row

    auto load_x = [&](int64_t tile) {
        const int64_t gr = tile * TC_ROWS + row;
        if constexpr (MODE == TC_BWD) {
            return make_float4(0.f, 0.f, 0.f, 0.f);
        } else {
            return (tile < n_tiles && gr < n_rows)
                       ? *reinterpret_cast<const float4 *>(A.x + gr * NIN)
                       : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };
    float4 x_next = load_x(blockIdx.x);
    for (int64_t tile = blockIdx.x; tile < n_tiles && !failed; tile += gridDim.x) {
        // ---- tile input: row `row`, columns cg1 * 64 .. +63 -------------------------------
        {
            const int64_t gr = tile * TC_ROWS + row;
            const bool in = gr < n_rows;
            if constexpr (MODE == TC_BWD) {  // dZ_4 from HBM
#pragma unroll 2
                for (int c = 0; c < TC_COLS / 8; ++c) {
                    const int n0 = cg1 * TC_COLS + c * 8;
                    const uint4 v = in ? *reinterpret_cast<const uint4 *>(A.dZ4 + gr * HID + n0)
                                       : make_uint4(0u, 0u, 0u, 0u);
                    *reinterpret_cast<uint4 *>(sA + tc::kmajor_offset(row, n0, HID)) = v;
                }
            } else {  // layer 1 (4 -> 256) on CUDA cores
                const float4 xi = x_next;
                x_next = load_x(tile + gridDim.x);  // in flight through this tile's layers
#pragma unroll 2
                for (int c = 0; c < TC_COLS / 8; ++c) {
                    const int n0 = cg1 * TC_COLS + c * 8;
                    float z[8], h[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const float4 w = sW1[n0 + j];
                        z[j] = sBias[n0 + j] + xi.x * w.x + xi.y * w.y + xi.z * w.z + xi.w * w.w;
                        h[j] = silu_fast(z[j]);
                    }
                    const uint4 hb = pack8(h);
                    *reinterpret_cast<uint4 *>(sA + tc::kmajor_offset(row, n0, HID)) = hb;
                    if constexpr (MODE == TC_TRAIN) {
                        if (in) {
                            *reinterpret_cast<uint4 *>(A.Z[1] + gr * HID + n0) = pack8(z);
                            *reinterpret_cast<uint4 *>(A.H[1] + gr * HID + n0) = hb;
                        }
                    }
                }
            }
        }
        tc::fence_proxy_async();
        for (int i = 0; i < 3; ++i) {
            // A tile written and previous accumulator reads done; weights present
            bool to = false;
            if (tid == 0 && w_pending) {
                to = !tc::mbar_wait(wbar, wphase, A.wait_limit);
                if (!to) {
                    wphase ^= 1u;
                    w_pending = false;
                }
            }
            tc::fence_before_sync();
            if (__syncthreads_or(to)) {
                failed = true;
                break;
            }
            tc::fence_after_sync();
            if (tid == 0) {
#pragma unroll 1
                for (int j = 0; j < HID / 16; ++j) {
                    const uint64_t ad = tc::smem_desc(a_base + j * 256, 128, (HID / 8) * 128);
                    const uint64_t bd = tc::smem_desc(b_base + j * 256, 128, (HID / 8) * 128);
                    tc::mma_bf16(tmem, ad, bd, idesc, j > 0 ? 1u : 0u);
                }
                tc::mma_commit(mbar);
                m_pending = true;
            }
            // accumulator complete: A and B free again (thread 0 polls, the rest sleep in the
            // block barrier instead of spinning on the mbarrier)
            if (tid == 0) {
                to = !tc::mbar_wait(mbar, mphase, A.wait_limit);
                if (!to) {
                    mphase ^= 1u;
                    m_pending = false;
                }
            }
            if (__syncthreads_or(to)) {
                failed = true;
                break;
            }
            tc::fence_after_sync();
            if (tid == 0) {  // next operand while the epilogue runs
                if (i < 2) {
                    load_weights(i + 1);
                    w_pending = true;
                } else if (tile + gridDim.x < n_tiles) {
                    load_weights(0);
                    w_pending = true;
                }
            }
            // ---- epilogue: row r (TMEM lane), columns cg * 64 .. +63 ----------------------
            const int64_t gr = tile * TC_ROWS + r;
            const bool in = gr < n_rows;
            const int l_out = MODE == TC_BWD ? 3 - i : 2 + i;  // layer whose Z/H/dZ this writes
            const float *bias = sBias + (l_out - 1) * HID;
            const uint32_t trow = tmem + ((uint32_t)(32 * lg) << 16);
#pragma unroll 1
            for (int c = 0; c < TC_COLS / 16; c += 2) {
                const int n0 = cg * TC_COLS + c * 16;
                uint32_t v[2][16];
                tc::tmem_ld16(trow + n0, v[0]);
                tc::tmem_ld16(trow + n0 + 16, v[1]);
                tc::tmem_ld_wait();
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int nb = n0 + 16 * u;
                    float h[16];
                    if constexpr (MODE == TC_BWD) {
                        // dZ_{l-1} = (dZ_l W_l^T) * SiLU'(Z_{l-1})
                        float zf[16];
#pragma unroll
                        for (int q = 0; q < 2; ++q) {
                            const uint4 zz = in ? *reinterpret_cast<const uint4 *>(
                                                      A.Z[l_out] + gr * HID + nb + 8 * q)
                                                : make_uint4(0u, 0u, 0u, 0u);
                            unpack8(zz, zf + 8 * q);
                        }
#pragma unroll
                        for (int j = 0; j < 16; ++j) h[j] = __uint_as_float(v[u][j]) * dsilu_fast(zf[j]);
                    } else {
                        float z[16];
#pragma unroll
                        for (int j4 = 0; j4 < 4; ++j4) {
                            const float4 b4 = *reinterpret_cast<const float4 *>(bias + nb + 4 * j4);
                            z[4 * j4 + 0] = __uint_as_float(v[u][4 * j4 + 0]) + b4.x;
                            z[4 * j4 + 1] = __uint_as_float(v[u][4 * j4 + 1]) + b4.y;
                            z[4 * j4 + 2] = __uint_as_float(v[u][4 * j4 + 2]) + b4.z;
                            z[4 * j4 + 3] = __uint_as_float(v[u][4 * j4 + 3]) + b4.w;
                        }
#pragma unroll
                        for (int j = 0; j < 16; ++j) h[j] = silu_fast(z[j]);
                        if constexpr (MODE == TC_TRAIN) {
                            if (in) {
#pragma unroll
                                for (int q = 0; q < 2; ++q) {
                                    *reinterpret_cast<uint4 *>(A.Z[l_out] + gr * HID + nb + 8 * q) =
                                        pack8(z + 8 * q);
                                    *reinterpret_cast<uint4 *>(A.H[l_out] + gr * HID + nb + 8 * q) =
                                        pack8(h + 8 * q);
                                }
                            }
                        }
                    }
                    if (i < 2) {  // next layer's operand
#pragma unroll
                        for (int q = 0; q < 2; ++q)
                            *reinterpret_cast<uint4 *>(sA + tc::kmajor_offset(r, nb + 8 * q, HID)) =
                                pack8(h + 8 * q);
                    }
                    if constexpr (MODE == TC_BWD) {
                        if (in) {
#pragma unroll
                            for (int q = 0; q < 2; ++q)
                                *reinterpret_cast<uint4 *>(A.dZ[l_out] + gr * HID + nb + 8 * q) =
                                    pack8(h + 8 * q);
                        }
                    }
                }
            }
            tc::fence_proxy_async();
            tc::fence_before_sync();
        }
        if (failed) break;
    }
    // ---- teardown: nothing of ours in flight, then free the tensor memory -------------------
    if (tid == 0) {
        if (failed) atomicExch(A.err, 1);
        // bounded waits for our own MMAs and copies still in flight
        if (m_pending) tc::mbar_wait(mbar, mphase, TC_WAIT);
        if (w_pending) tc::mbar_wait(wbar, wphase, TC_WAIT);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, TC_TMEM_COLS);
}

// ---- inference with the activations in tensor memory -------------------------------------
// One CTA per SM walks 128-row tiles.  Tensor memory (512 columns) holds two FP32
// accumulators of 128 x 128 (the two column halves of a 256-wide layer's output, columns
// 0-127 and 128-255) and two BF16 activation tiles of 128 x 256 (two values per 32-bit
// column, 128 columns each), so each 256 x 256 layer takes its A operand from tensor memory
// (tcgen05.mma with A in TMEM) and shared memory holds only weights: the two 64 KB column
// halves of one packed W^T.  One control thread issues the weight copies and the MMAs: per
// layer and column half, K = 0..127 once the epilogue has written that half of the input,
// K = 128..255 once it has written the other, then a commit; each weight half is refilled
// with the next layer's as soon as its MMAs are done.  Two groups of 8 epilogue warps, one
// per accumulator half, each read their half back into the other activation tile as soon as
// its MMAs are done, independently of the other half, and compute their half of layer 1
// (4 -> 256) of the next tile while the last 256 x 256 layer of this one runs.  The weights
// and biases of layers 1-4 come halved (exact), so the accumulators hold z / 2 and SiLU is
// z/2 (1 + tanh(z/2)): per pair of activations one packed add (bias), two tanh, one packed
// FMA and one BF16 pack.  Hand-offs go through mbarriers (each completes at most one phase
// ahead of its waiter); every wait is bounded, and on a time-out the CTA flags *err, drains
// its own MMAs and copies (bounded) and frees its tensor memory.
constexpr int TS_EPI = 512, TS_THREADS = TS_EPI + 32;  // 16 epilogue warps + the control warp
constexpr uint32_t TS_WH_BYTES = TC_B_BYTES / 2;        // a column half of a packed W^T: 64 KB
constexpr uint32_t TS_ABUF = 256;                        // activation tiles at columns 256, 384
constexpr size_t TS_RED_BYTES = 2 * (size_t)(TC_CG - 1) * TC_ROWS * NOUT * sizeof(float);
constexpr size_t TS_CONST_BYTES = TC_CONST_BYTES + (HID * 4 + 4) * sizeof(float);
constexpr size_t TS_SMEM = 1024 + 2 * TS_WH_BYTES + TS_CONST_BYTES + TS_RED_BYTES + 128;
static_assert(TS_SMEM <= 232448, "shared memory of one CTA");
// mbarriers: wfull[h] weight half present, accfull[h] accumulator half complete, afree[h]
// accumulator half read out, aready[h] / l1ready[h] K-half h of the next layer's input
// written by a hidden-layer epilogue / by layer 1, redfull the layer-5 partial sums of
// column quarters 1..3 written, l1go the tensor cores done with layer 3 (both halves; its
// input tile takes the next tile's layer 1), drain (teardown)
enum : int { TS_WFULL = 0, TS_ACCFULL = 2, TS_AFREE = 4, TS_AREADY = 6, TS_L1READY = 8,
             TS_REDFULL = 10, TS_L1GO = 11, TS_DRAIN = 12, TS_NBAR = 13 };
constexpr int TS_GROUP_WARPS = TS_EPI / 64;  // epilogue warps per accumulator half
// waits sleep up to TS_SLEEP_NS per try when the poll limit is at least TS_SLEEP_POLLS (a
// limit below that, a test's, polls without sleeping)
constexpr uint32_t TS_SLEEP_NS = 1000, TS_SLEEP_POLLS = 4096;

// Activation tile holding the input of layer i (0..2: layers 2..4) of a tile whose parity
// among this CTA's tiles is par; layer 1 writes the input of i = 0.
__device__ __forceinline__ uint32_t ts_in_col(uint32_t par, int i)
{
    return TS_ABUF + 128u * ((par + (i == 1 ? 1u : 0u)) & 1u);
}

__global__ void __launch_bounds__(TS_THREADS, 1) mlp_infer_ts(const __grid_constant__ TcArgs A)
{
    extern __shared__ __align__(16) unsigned char ts_raw[];
    unsigned char *sW = reinterpret_cast<unsigned char *>(
        ((uintptr_t)ts_raw + 1023) & ~(uintptr_t)1023);          // [2][64 KB]
    float4 *sW1 = reinterpret_cast<float4 *>(sW + 2 * TS_WH_BYTES);  // [128][2]: column pairs
    float *sBias = reinterpret_cast<float *>(sW1 + HID);             // [4][256]: b1..b4
    float4 *sW5 = reinterpret_cast<float4 *>(sBias + 4 * HID);      // [256]
    float *sB5 = reinterpret_cast<float *>(sW5 + HID);              // [4]
    float *red = sB5 + 4;                                            // [2][TC_CG-1][128][4]
    uint64_t *bars = reinterpret_cast<uint64_t *>(
        ((uintptr_t)(red + 2 * (TC_CG - 1) * TC_ROWS * NOUT) + 7) & ~(uintptr_t)7);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + TS_NBAR);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t n_rows = A.n_rows;
    const int64_t n_tiles = (n_rows + TC_ROWS - 1) / TC_ROWS;
    auto bar = [&](int k) { return tc::smem_u32(&bars[k]); };
    if (tid == 0) {
        for (int h = 0; h < 2; ++h) {
            tc::mbar_init(bar(TS_WFULL + h), 1);
            tc::mbar_init(bar(TS_ACCFULL + h), 1);
            tc::mbar_init(bar(TS_AFREE + h), TS_GROUP_WARPS);
            tc::mbar_init(bar(TS_AREADY + h), TS_GROUP_WARPS);
            tc::mbar_init(bar(TS_L1READY + h), TS_GROUP_WARPS);
        }
        tc::mbar_init(bar(TS_REDFULL), 3 * TS_GROUP_WARPS / 2);  // the warps of quarters 1..3
        tc::mbar_init(bar(TS_L1GO), 1);
        tc::mbar_init(bar(TS_DRAIN), 1);
        tc::mbar_fence_init();
    }
    // layers 1-4 halved (exactly), as the packed W^T: every pre-activation comes out as z / 2
    // W1 by column pairs (n, n + 1): {W1[0][n], W1[0][n+1], W1[1][n], W1[1][n+1]},
    // {W1[2][n], W1[2][n+1], W1[3][n], W1[3][n+1]}
    for (int q = tid; q < HID; q += TS_THREADS) {
        const int n = 2 * (q >> 1), k0 = 2 * (q & 1);
        auto w = [&](int k, int c) { return 0.5f * bfv(A.pb, OFF_W1 + k * HID + c); };
        sW1[q] = make_float4(w(k0, n), w(k0, n + 1), w(k0 + 1, n), w(k0 + 1, n + 1));
    }
    for (int n = tid; n < HID; n += TS_THREADS) {
        sBias[n] = 0.5f * A.p[OFF_B1 + n];
        for (int l = 2; l <= 4; ++l) sBias[(l - 1) * HID + n] = 0.5f * A.p[off_b(l) + n];
        sW5[n] = make_float4(bfv(A.pb, OFF_W5 + n * NOUT + 0), bfv(A.pb, OFF_W5 + n * NOUT + 1),
                             bfv(A.pb, OFF_W5 + n * NOUT + 2), bfv(A.pb, OFF_W5 + n * NOUT + 3));
    }
    if (tid < NOUT) sB5[tid] = A.p[OFF_B5 + tid];
    if (warp == 0) tc::tmem_alloc(tslot, 512);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    const int64_t first = blockIdx.x, stride = gridDim.x;
    bool failed = false;
    const uint32_t sleep_ns = A.wait_limit >= TS_SLEEP_POLLS ? TS_SLEEP_NS : 0u;
    auto mwait = [&](int k, uint32_t ph) {
        return sleep_ns ? tc::mbar_wait_sleep(bar(k), ph, A.wait_limit, sleep_ns)
                        : tc::mbar_wait(bar(k), ph, A.wait_limit);
    };

    if (warp == TS_EPI / 32) {
        // ---- control thread: weight copies and MMAs ---------------------------------------
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_bf16_f32(TC_ROWS, HID / 2);
            const uint32_t w_base = tc::smem_u32(sW);
            uint32_t ph_w[2] = {0u, 0u}, ph_acc[2] = {0u, 0u}, ph_af[2] = {0u, 0u},
                     ph_ar[2] = {0u, 0u}, ph_l1[2] = {0u, 0u};
            bool w_pend[2] = {false, false}, acc_used = false, ok = true;
            auto wait = [&](int k, uint32_t &ph) {
                if (!mwait(k, ph)) return false;
                ph ^= 1u;
                return true;
            };
            auto load_half = [&](int blk, int h) {  // packed block blk (layer blk + 2), half h
                tc::mbar_expect_tx(bar(TS_WFULL + h), TS_WH_BYTES);
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    tc::bulk_g2s(w_base + h * TS_WH_BYTES + c * (TS_WH_BYTES / 4),
                                 A.wpack + (size_t)blk * HID * HID + (size_t)h * (HID * HID / 2) +
                                     (size_t)c * (HID * HID / 8),
                                 TS_WH_BYTES / 4, bar(TS_WFULL + h));
                w_pend[h] = true;
            };
            // B descriptors of the two weight halves; K step j starts 256 bytes further
            // (the start-address field counts 16-byte units)
            const uint64_t bdesc[2] = {
                tc::smem_desc(w_base, 128, (HID / 8) * 128),
                tc::smem_desc(w_base + TS_WH_BYTES, 128, (HID / 8) * 128)};
            auto mmas8 = [&](uint32_t d, uint32_t a, uint64_t bd, int j0) {  // K steps j0..j0+7
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    tc::mma_bf16_ts(d, a + 8 * (j0 + j), bd + (uint64_t)(16 * (j0 + j)), idesc,
                                    (j0 + j) > 0 ? 1u : 0u);
            };
            if (first < n_tiles) {
                load_half(0, 0);
                load_half(0, 1);
            }
            for (int64_t tile = first; tile < n_tiles && ok; tile += stride) {
                const uint32_t par = (uint32_t)((tile - first) / stride) & 1u;
                for (int i = 0; i < 3 && ok; ++i) {
                    const uint32_t a_col = ts_in_col(par, i);
                    const int rdy = i == 0 ? TS_L1READY : TS_AREADY;
                    uint32_t *ph_rdy = i == 0 ? ph_l1 : ph_ar;
                    // column half 0: K 0..127 once its input half is written, then K 128..255
                    ok = wait(rdy, ph_rdy[0]) && (!acc_used || wait(TS_AFREE, ph_af[0])) &&
                         wait(TS_WFULL, ph_w[0]);
                    if (!ok) break;
                    w_pend[0] = false;
                    tc::fence_after_sync();
                    mmas8(tmem, tmem + a_col, bdesc[0], 0);
                    ok = wait(rdy + 1, ph_rdy[1]);
                    if (!ok) break;
                    tc::fence_after_sync();
                    mmas8(tmem, tmem + a_col, bdesc[0], 8);
                    tc::mma_commit(bar(TS_ACCFULL + 0));
                    // column half 1: the whole input is written by now
                    ok = (!acc_used || wait(TS_AFREE + 1, ph_af[1])) && wait(TS_WFULL + 1, ph_w[1]);
                    if (!ok) break;
                    w_pend[1] = false;
                    tc::fence_after_sync();
                    mmas8(tmem + 128, tmem + a_col, bdesc[1], 0);
                    mmas8(tmem + 128, tmem + a_col, bdesc[1], 8);
                    tc::mma_commit(bar(TS_ACCFULL + 1));
                    if (i == 1 && tile + stride < n_tiles) tc::mma_commit(bar(TS_L1GO));
                    acc_used = true;
                    // refill each weight half with the next layer's once its MMAs are done
                    const bool more = i < 2 || tile + stride < n_tiles;
                    for (int h = 0; h < 2 && ok; ++h) {
                        ok = wait(TS_ACCFULL + h, ph_acc[h]);
                        if (ok && more) load_half((i + 1) % 3, h);
                    }
                }
            }
            failed = !ok;
            // drain: every MMA issued here complete, every copy landed (bounded)
            tc::mma_commit(bar(TS_DRAIN));
            tc::mbar_wait(bar(TS_DRAIN), 0, TC_WAIT);
            for (int h = 0; h < 2; ++h)
                if (w_pend[h]) tc::mbar_wait(bar(TS_WFULL + h), ph_w[h], TC_WAIT);
        }
        __syncwarp();
    } else {
        // ---- epilogue warps: group g = accumulator half g, row r (TMEM lane), columns
        //      cq * 64 .. +63 of the half.  Each warp waits for its own hand-offs. -----------
        const int g = warp >> 3, lg = warp & 3, cq = (warp >> 2) & 1;
        const int r = 32 * lg + lane;
        const uint32_t lane_off = (uint32_t)(32 * lg) << 16;
        uint32_t ph_acc = 0u, ph_red = 0u, ph_go = 0u;
        auto warp_wait = [&](int k, uint32_t &ph) {  // bounded; lane 0 polls for the warp
            int ok = 1;
            if (lane == 0) ok = mwait(k, ph) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            __syncwarp();
            if (ok) ph ^= 1u;
            return ok != 0;
        };
        auto load_x = [&](int64_t tile) {
            const int64_t gr = tile * TC_ROWS + r;
            return (tile < n_tiles && gr < n_rows)
                       ? *reinterpret_cast<const float4 *>(A.x + gr * NIN)
                       : make_float4(0.f, 0.f, 0.f, 0.f);
        };
        auto arrive = [&](int k) {  // this warp's tensor- and shared-memory writes are done
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(bar(k));
        };
        // layer 1 (4 -> 256) of a tile, this warp's columns, into the activation tile at a_col
        auto layer1 = [&](float4 xi, uint32_t a_col) {
#pragma unroll 1
            for (int c = 0; c < 2; ++c) {
                uint32_t packed[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) {  // columns n, n + 1
                    const int n = g * 128 + cq * 64 + c * 32 + 2 * j;
                    const float4 w01 = sW1[n], w23 = sW1[n + 1];
                    float2 z = *reinterpret_cast<const float2 *>(sBias + n);
                    z = fma2(dup2(xi.x), make_float2(w01.x, w01.y), z);
                    z = fma2(dup2(xi.y), make_float2(w01.z, w01.w), z);
                    z = fma2(dup2(xi.z), make_float2(w23.x, w23.y), z);
                    z = fma2(dup2(xi.w), make_float2(w23.z, w23.w), z);
                    const float2 h = fma2(z, make_float2(tanh_fast(z.x), tanh_fast(z.y)), z);
                    packed[j] = pack_bf16x2(h.x, h.y);
                }
                tc::tmem_st16(tmem + lane_off + a_col + g * 64 + cq * 32 + c * 16, packed);
            }
            tc::tmem_st_wait();
            arrive(TS_L1READY + g);
        };
        if (first < n_tiles) layer1(load_x(first), ts_in_col(0, 0));
        for (int64_t tile = first; tile < n_tiles && !failed; tile += stride) {
            const uint32_t par = (uint32_t)((tile - first) / stride) & 1u;
            const float4 x_next = load_x(tile + stride);  // in flight through two layers
            float2 acc01 = make_float2(0.f, 0.f), acc23 = make_float2(0.f, 0.f);  // layer 5
            for (int i = 0; i < 3; ++i) {
                const float *bias = sBias + (i + 1) * HID;  // layer i + 2
                if (!warp_wait(TS_ACCFULL + g, ph_acc)) {
                    failed = true;
                    break;
                }
                tc::fence_after_sync();
                const uint32_t acc = tmem + lane_off + 128u * g + cq * 64;
                const uint32_t a_out = ts_in_col(par, i + 1) + g * 64 + cq * 32;
#pragma unroll 1
                for (int c = 0; c < 2; ++c) {  // 32 columns at a time
                    uint32_t v[2][16];
                    tc::tmem_ld16(acc + 32 * c, v[0]);
                    tc::tmem_ld16(acc + 32 * c + 16, v[1]);
                    tc::tmem_ld_wait();
                    if (c == 1) arrive(TS_AFREE + g);
                    const int nb = g * 128 + cq * 64 + 32 * c;  // output column of v[0][0]
                    if (i < 2) {
                        uint32_t packed[16];
#pragma unroll
                        for (int u = 0; u < 2; ++u) {
#pragma unroll
                            for (int j = 0; j < 8; ++j) {
                                const int n = nb + 16 * u + 2 * j;
                                const float2 hz = add2(make_float2(__uint_as_float(v[u][2 * j]),
                                                                   __uint_as_float(v[u][2 * j + 1])),
                                                       *reinterpret_cast<const float2 *>(bias + n));
                                const float2 h =
                                    fma2(hz, make_float2(tanh_fast(hz.x), tanh_fast(hz.y)), hz);
                                packed[8 * u + j] = pack_bf16x2(h.x, h.y);
                            }
                        }
                        tc::tmem_st16(tmem + lane_off + a_out + 16 * c, packed);
                    } else {  // layer 5 (256 -> 4) on the BF16-rounded activations
#pragma unroll
                        for (int u = 0; u < 2; ++u) {
#pragma unroll
                            for (int j = 0; j < 8; ++j) {
                                const int n = nb + 16 * u + 2 * j;
                                const float2 hz = add2(make_float2(__uint_as_float(v[u][2 * j]),
                                                                   __uint_as_float(v[u][2 * j + 1])),
                                                       *reinterpret_cast<const float2 *>(bias + n));
                                const float2 h =
                                    fma2(hz, make_float2(tanh_fast(hz.x), tanh_fast(hz.y)), hz);
                                const float2 hb = __bfloat1622float2(__floats2bfloat162_rn(h.x, h.y));
                                const float4 w0 = sW5[n], w1 = sW5[n + 1];
                                acc01 = fma2(dup2(hb.x), make_float2(w0.x, w0.y), acc01);
                                acc23 = fma2(dup2(hb.x), make_float2(w0.z, w0.w), acc23);
                                acc01 = fma2(dup2(hb.y), make_float2(w1.x, w1.y), acc01);
                                acc23 = fma2(dup2(hb.y), make_float2(w1.z, w1.w), acc23);
                            }
                        }
                    }
                }
                if (i < 2) {
                    tc::tmem_st_wait();
                    arrive(TS_AREADY + g);
                }
                // the next tile's layer 1 runs while this tile's last layer is on the tensor
                // cores, into the tile that layer 3 read: once both its halves are done
                if (i == 1 && tile + stride < n_tiles) {
                    if (!warp_wait(TS_L1GO, ph_go)) {
                        failed = true;
                        break;
                    }
                    tc::fence_after_sync();
                    layer1(x_next, ts_in_col(par ^ 1u, 0));
                }
            }
            if (failed) break;
            // ---- layer 5: the four column quarters of each row, added in quarter order ---------
            float *rb = red + (size_t)par * (TC_CG - 1) * TC_ROWS * NOUT;
            const int quarter = 2 * g + cq;
            if (quarter > 0) {
                *reinterpret_cast<float4 *>(rb + ((quarter - 1) * TC_ROWS + r) * NOUT) =
                    make_float4(acc01.x, acc01.y, acc23.x, acc23.y);
                arrive(TS_REDFULL);
            } else {
                if (!warp_wait(TS_REDFULL, ph_red)) {
                    failed = true;
                    break;
                }
                const int64_t gr = tile * TC_ROWS + r;
                if (gr < n_rows) {
                    const float acc5[NOUT] = {acc01.x, acc01.y, acc23.x, acc23.y};
                    float out[NOUT];
#pragma unroll
                    for (int o = 0; o < NOUT; ++o) {
                        out[o] = acc5[o] + sB5[o];
#pragma unroll
                        for (int q = 0; q < TC_CG - 1; ++q) out[o] += rb[(q * TC_ROWS + r) * NOUT + o];
                    }
                    *reinterpret_cast<float4 *>(A.y + gr * NOUT) =
                        make_float4(out[0], out[1], out[2], out[3]);
                }
            }
        }
    }
    if (failed) atomicExch(A.err, 1);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

// ---- layer 5 (256 -> 4), the loss and the column reductions on CUDA cores -----------------
// Weights from the BF16 copy, biases from the FP32 master.  One warp per sample row, lane l
// holding columns 8 l .. 8 l + 7 (one 16-byte load of H4 and of Z4 covers the row):
//   y = H4 W5 + b5; loss = softplus(y0) - c y0 + m_x (e1^2 + e2^2) + m_g e3^2 with
//   e_k = y_k - t_k (mean over the batch); dL/dy; dL/dZ4 = (dL/dy W5^T) silu'(Z4)
// (sigmoid and silu' in the tanh form the tensor-core chain uses).
// Each block writes its loss partial; grad_finish adds them in block order.
constexpr int L5_THREADS = 256, L5_BLOCKS = 1024;

__global__ void __launch_bounds__(L5_THREADS, 3) layer5_fused(
    const bf16 *__restrict__ H4, const bf16 *__restrict__ Z4, const bf16 *__restrict__ pb,
    const float *__restrict__ p, int64_t B, const float *__restrict__ t, float *__restrict__ dY,
    bf16 *__restrict__ dZ4, float *__restrict__ loss_part)
{
    __shared__ float sl[L5_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float w[8][NOUT], b5[NOUT];
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
        for (int o = 0; o < NOUT; ++o) w[j][o] = bfv(pb, OFF_W5 + (8 * lane + j) * NOUT + o);
#pragma unroll
    for (int o = 0; o < NOUT; ++o) b5[o] = p[OFF_B5 + o];
    const float inv = 1.f / (float)B;
    float lsum = 0.f;
    const int64_t wstride = (int64_t)gridDim.x * (L5_THREADS / 32);
    for (int64_t b = (int64_t)blockIdx.x * (L5_THREADS / 32) + warp; b < B; b += wstride) {
        float h[8], z[8];
        unpack8(*reinterpret_cast<const uint4 *>(H4 + b * HID + 8 * lane), h);
        unpack8(*reinterpret_cast<const uint4 *>(Z4 + b * HID + 8 * lane), z);
        float y[NOUT] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
            for (int o = 0; o < NOUT; ++o) y[o] = fmaf(h[j], w[j][o], y[o]);
#pragma unroll
        for (int o = 0; o < NOUT; ++o) {
#pragma unroll
            for (int s = 16; s > 0; s >>= 1) y[o] += __shfl_xor_sync(0xffffffffu, y[o], s);
            y[o] += b5[o];
        }
        const float4 t0 = *reinterpret_cast<const float4 *>(t + b * 8);
        const float4 t1 = *reinterpret_cast<const float4 *>(t + b * 8 + 4);
        const float c = t0.x, mx = t1.x, mg = t1.y;
        const float e1 = y[1] - t0.y, e2 = y[2] - t0.z, e3 = y[3] - t0.w;
        const float sg = fmaf(0.5f, tanh_fast(0.5f * y[0]), 0.5f);  // sigmoid(y0)
        const float d[NOUT] = {inv * (sg - c), inv * 2.f * mx * e1,
                               inv * 2.f * mx * e2, inv * 2.f * mg * e3};
        if (lane == 0) {
            const float sp = fmaxf(y[0], 0.f) - c * y[0] + log1pf(__expf(-fabsf(y[0])));
            lsum += inv * (sp + mx * (e1 * e1 + e2 * e2) + mg * e3 * e3);
            *reinterpret_cast<float4 *>(dY + b * NOUT) = make_float4(d[0], d[1], d[2], d[3]);
        }
        float dz[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            float v = 0.f;
#pragma unroll
            for (int o = 0; o < NOUT; ++o) v = fmaf(d[o], w[j][o], v);
            dz[j] = v * dsilu_fast(z[j]);
        }
        *reinterpret_cast<uint4 *>(dZ4 + b * HID + 8 * lane) = pack8(dz);
    }
    if (lane == 0) sl[warp] = lsum;
    __syncthreads();
    if (threadIdx.x == 0) {
        float v = 0.f;
        for (int i = 0; i < L5_THREADS / 32; ++i) v += sl[i];
        loss_part[blockIdx.x] = v;
    }
}

// Batch sums for the bias and the 4-wide weight gradients, one job per blockIdx.y:
//   jobs 0-2: gb_l[n] = sum_b dZ_l[b][n]                (l = 4, 3, 2)
//   job 3:    gb_1[n] = sum_b dZ_1[b][n], gW1[k][n] = sum_b x[b][k] dZ_1[b][n]
//   job 4:    gW5[n][o] = sum_b H4[b][n] dY[b][o],     gb5[o] = sum_b dY[b][o]
// A block takes a contiguous run of rows; thread (row phase r, column group g) adds every
// 8th row of columns 8 g .. 8 g + 7, the 8 phases are then added in order through shared
// memory, and the block writes part[job][block][k][n] (k: the CR_K weighted sums).
constexpr int CR_THREADS = 256, CR_BLOCKS = 128, CR_K = 5, CR_JOBS = 5;

struct ColArgs {
    const bf16 *A[CR_JOBS];  // dZ4, dZ3, dZ2, dZ1, H4
    const float *x, *dY;
    int64_t B;
    float *part;  // [CR_JOBS][CR_BLOCKS][CR_K][HID]
};

template <int JOB>
__device__ __forceinline__ void col_rows(const ColArgs &C, int64_t r0, int64_t r1, int rp, int g,
                                         float (&acc)[CR_K][8])
{
    const bf16 *A = C.A[JOB];
#pragma unroll 4
    for (int64_t b = r0 + rp; b < r1; b += 8) {
        float a[8];
        unpack8(*reinterpret_cast<const uint4 *>(A + b * HID + 8 * g), a);
        if constexpr (JOB < 3) {
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[0][j] += a[j];
        } else if constexpr (JOB == 3) {
            const float4 xv = *reinterpret_cast<const float4 *>(C.x + b * NIN);
            const float wk[NIN] = {xv.x, xv.y, xv.z, xv.w};
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                acc[0][j] += a[j];
#pragma unroll
                for (int k = 0; k < NIN; ++k) acc[1 + k][j] = fmaf(wk[k], a[j], acc[1 + k][j]);
            }
        } else {
            const float4 dv = *reinterpret_cast<const float4 *>(C.dY + b * NOUT);
            const float wk[NOUT] = {dv.x, dv.y, dv.z, dv.w};
#pragma unroll
            for (int j = 0; j < 8; ++j)
#pragma unroll
                for (int k = 0; k < NOUT; ++k) acc[k][j] = fmaf(wk[k], a[j], acc[k][j]);
            if (g == 0)
#pragma unroll
                for (int k = 0; k < NOUT; ++k) acc[4][k] += wk[k];  // gb5 in slot (4, k)
        }
    }
}

__global__ void __launch_bounds__(CR_THREADS) col_reduce(const __grid_constant__ ColArgs C)
{
    __shared__ float sh[8][HID];
    const int job = blockIdx.y, g = threadIdx.x & 31, rp = threadIdx.x >> 5;
    const int64_t r0 = C.B * blockIdx.x / gridDim.x, r1 = C.B * (blockIdx.x + 1) / gridDim.x;
    float acc[CR_K][8];
#pragma unroll
    for (int k = 0; k < CR_K; ++k)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[k][j] = 0.f;
    switch (job) {
    case 0: col_rows<0>(C, r0, r1, rp, g, acc); break;
    case 1: col_rows<1>(C, r0, r1, rp, g, acc); break;
    case 2: col_rows<2>(C, r0, r1, rp, g, acc); break;
    case 3: col_rows<3>(C, r0, r1, rp, g, acc); break;
    default: col_rows<4>(C, r0, r1, rp, g, acc); break;
    }
    float *out = C.part + ((size_t)job * gridDim.x + blockIdx.x) * CR_K * HID;
#pragma unroll
    for (int k = 0; k < CR_K; ++k) {
#pragma unroll
        for (int j = 0; j < 8; ++j) sh[rp][8 * g + j] = acc[k][j];
        __syncthreads();
        const int n = threadIdx.x;
        float v = 0.f;
#pragma unroll
        for (int q = 0; q < 8; ++q) v += sh[q][n];
        out[k * HID + n] = v;
        __syncthreads();
    }
}

// Gradients of the biases and the 4-wide layers, and the loss, one warp per output: lane l
// adds partials l, l + 32, ... in order, then a fixed shuffle tree.  Outputs, in warp order:
// gb_4, gb_3, gb_2 (3 x 256), gb_1 and gW1 (5 x 256), gW5 (4 x 256), gb5 (4), the loss.
constexpr int GF_OUTPUTS = 3 * HID + 5 * HID + 4 * HID + NOUT + 1;

__global__ void grad_finish(const float *__restrict__ part, const float *__restrict__ loss_part,
                            float *__restrict__ grad, float *__restrict__ loss)
{
    const int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (w >= GF_OUTPUTS) return;
    int job, k, n;
    const float *src;
    int count, stride;
    if (w == GF_OUTPUTS - 1) {
        src = loss_part, count = L5_BLOCKS, stride = 1;
        job = k = n = -1;
    } else {
        if (w < 3 * HID) job = w / HID, k = 0, n = w % HID;
        else if (w < 8 * HID) job = 3, k = (w - 3 * HID) / HID, n = w % HID;
        else if (w < 12 * HID) job = 4, k = (w - 8 * HID) / HID, n = w % HID;
        else job = 4, k = 4, n = w - 12 * HID;
        src = part + ((size_t)job * CR_BLOCKS * CR_K + k) * HID + n;
        count = CR_BLOCKS, stride = CR_K * HID;
    }
    float v = 0.f;
    for (int i = lane; i < count; i += 32) v += src[(size_t)i * stride];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane != 0) return;
    if (job < 0) *loss = v;
    else if (job < 3) grad[off_b(4 - job) + n] = v;
    else if (job == 3) grad[k == 0 ? OFF_B1 + n : OFF_W1 + (k - 1) * HID + n] = v;
    else if (k < NOUT) grad[OFF_W5 + n * NOUT + k] = v;
    else grad[OFF_B5 + n] = v;
}

// ---- weight gradients on tcgen05: dW_l = H_{l-1}^T dZ_l --------------------------------------
// The batch index is the reduction index and the row index of both operands in HBM, so both
// are MN-major for the tensor core: a 16-byte piece of one row (8 consecutive features) is one
// core-matrix row.  Grid (splits, 3 layers); each CTA reduces a contiguous run of 64-row
// chunks through a three-stage cp.async ring into two 128 x 256 FP32 accumulators (all 512
// tensor-memory columns: features 0-127 and 128-255 of H), then writes its partial sum; a
// second kernel adds the partials in split order (deterministic).
constexpr int DW_THREADS = 256, DW_KC = 64, DW_STAGES = 3, DW_MAX_SPLITS = 48;
constexpr uint32_t DW_OP_BYTES = HID * DW_KC * 2;                 // one operand chunk, 32 KB
constexpr uint32_t DW_LBO = (HID / 8) * 128;                      // K (batch) core stride
constexpr size_t DW_SMEM = 1024 + (size_t)DW_STAGES * 2 * DW_OP_BYTES + 64;
static_assert(DW_SMEM <= 232448, "shared memory of one CTA");

struct DwArgs {
    const bf16 *H[3], *dZ[3];  // per layer slot: H_{l-1}, dZ_l (row-major [B][256]) for l = 4, 3, 2
    int64_t n_chunks;          // B / 64
    float *part;               // [3][splits][256][256]
    int *err;
};

__global__ void __launch_bounds__(DW_THREADS, 1) mlp_dw_tc(const __grid_constant__ DwArgs A)
{
    extern __shared__ __align__(16) unsigned char dw_raw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(((uintptr_t)dw_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + (size_t)DW_STAGES * 2 * DW_OP_BYTES);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + DW_STAGES);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int layer = blockIdx.y, splits = gridDim.x, s = blockIdx.x;
    const bf16 *Hg = A.H[layer], *Zg = A.dZ[layer];
    const int64_t c0 = A.n_chunks * s / splits, c1 = A.n_chunks * (s + 1) / splits;
    const int nc = (int)(c1 - c0);
    uint32_t mbar[DW_STAGES];
#pragma unroll
    for (int i = 0; i < DW_STAGES; ++i) mbar[i] = tc::smem_u32(&bars[i]);
    if (tid == 0) {
        for (int i = 0; i < DW_STAGES; ++i) tc::mbar_init(mbar[i], 1);
        tc::mbar_fence_init();
    }
    if (warp == 0) tc::tmem_alloc(tslot, 512);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;

    // chunk c of this CTA into stage st: rows 64 c .. +63 of H and dZ, 2 x 2048 pieces of 16 B
    auto load_chunk = [&](int c, int st) {
        unsigned char *a = sm + (size_t)st * 2 * DW_OP_BYTES, *b = a + DW_OP_BYTES;
        const int64_t row0 = (c0 + c) * DW_KC;
#pragma unroll
        for (int q = 0; q < 2048 / DW_THREADS; ++q) {
            const int piece = tid + q * DW_THREADS;
            const int r = piece >> 5, g = piece & 31;  // row in chunk, feature group
            const uint32_t off = g * 128 + (r >> 3) * DW_LBO + (r & 7) * 16;
            cp_async16(a + off, Hg + (row0 + r) * HID + g * 8);
            cp_async16(b + off, Zg + (row0 + r) * HID + g * 8);
        }
    };
    uint32_t mph = 0;  // parity bits of the stage barriers (bit i: next completion of stage i)
    bool failed = false, pending = false;
    int last_st = 0;   // stage barrier of the most recent commit
#pragma unroll
    for (int i = 0; i < DW_STAGES - 1; ++i) {
        if (i < nc) load_chunk(i, i);
        cp_async_commit();
    }
    const uint32_t idesc = tc::idesc_bf16_f32(128, HID, true, true);
    for (int c = 0; c < nc; ++c) {
        const int st = c % DW_STAGES;
        cp_async_wait<DW_STAGES - 2>();  // chunk c landed (this thread's pieces)
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (tid == 0) {
            const uint32_t a = tc::smem_u32(sm + (size_t)st * 2 * DW_OP_BYTES), b = a + DW_OP_BYTES;
#pragma unroll
            for (int j = 0; j < DW_KC / 16; ++j)
#pragma unroll
                for (int h = 0; h < 2; ++h)
                    tc::mma_bf16(tmem + h * 256,
                                 tc::smem_desc(a + h * 16 * 128 + 2 * j * DW_LBO, DW_LBO, 128),
                                 tc::smem_desc(b + 2 * j * DW_LBO, DW_LBO, 128), idesc,
                                 (c > 0 || j > 0) ? 1u : 0u);
            tc::mma_commit(mbar[st]);
            pending = true;
            last_st = st;
        }
        // refill the stage chunk c - 1 used, once its MMAs are done
        const int cn = c + DW_STAGES - 1, sn = cn % DW_STAGES;
        bool to = false;
        if (tid == 0 && c >= 1 && cn < nc) {
            to = !tc::mbar_wait(mbar[sn], (mph >> sn) & 1u, TC_WAIT);
            if (!to) mph ^= 1u << sn;
        }
        if (__syncthreads_or(to)) {
            failed = true;
            break;
        }
        if (cn < nc) load_chunk(cn, sn);
        cp_async_commit();
    }
    cp_async_wait<0>();  // none of our copies outstanding
    // all MMAs complete: the last commit covers the earlier ones (earlier phases of its
    // barrier were waited for by the refills)
    bool to = false;
    if (tid == 0 && pending) {
        to = !tc::mbar_wait(mbar[last_st], (mph >> last_st) & 1u, TC_WAIT);
        pending = to;
    }
    if (__syncthreads_or(to) || failed) {
        if (tid == 0) {
            atomicExch(A.err, 1);
            if (pending) tc::mbar_wait(mbar[last_st], (mph >> last_st) & 1u, TC_WAIT);  // bounded
        }
        failed = true;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (!failed) {
        // rows k = 128 (warp / 4) + 32 (warp % 4) + lane of the partial, 256 columns
        const int h = warp >> 2, k = 128 * h + 32 * (warp & 3) + lane;
        float *out = A.part + (((size_t)layer * splits + s) * HID + k) * HID;
        const uint32_t trow = tmem + h * 256 + ((uint32_t)(32 * (warp & 3)) << 16);
        for (int c = 0; c < HID; c += 16) {
            uint32_t v[16];
            tc::tmem_ld16(trow + c, v);
            tc::tmem_ld_wait();
            if (nc == 0)
#pragma unroll
                for (int q = 0; q < 16; ++q) v[q] = 0u;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                *reinterpret_cast<float4 *>(out + c + 4 * q) =
                    make_float4(__uint_as_float(v[4 * q]), __uint_as_float(v[4 * q + 1]),
                                __uint_as_float(v[4 * q + 2]), __uint_as_float(v[4 * q + 3]));
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

// grad_W[l] = sum over splits of the partials, in split order
__global__ void dw_reduce(const float *__restrict__ part, int splits, float *__restrict__ grad)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 3 * HID * HID) return;
    const int slot = (int)(idx / (HID * HID)), e = (int)(idx % (HID * HID));
    const int l = 4 - slot;
    float sum = 0.f;
    for (int q = 0; q < splits; ++q) sum += part[((size_t)slot * splits + q) * HID * HID + e];
    grad[off_w(l) + e] = sum;
}

template <int MODE>
void launch_chain(odx_mlp *m, const TcArgs &a, int64_t n, cudaStream_t st)
{
    if (n <= 0) return;
    const int64_t tiles = (n + TC_ROWS - 1) / TC_ROWS;
    const unsigned grid = (unsigned)std::min<int64_t>(tiles, std::max(1, m->num_sms));
    mlp_chain_tc<MODE><<<grid, TC_THREADS, TC_SMEM, st>>>(a);
}

TcArgs chain_args(odx_mlp *m, const bf16 *wpack, int64_t n)
{
    TcArgs a{};
    a.pb = m->pb;
    a.p = m->p;
    a.wpack = wpack;
    a.n_rows = n;
    a.err = m->tc_err;
    a.wait_limit = m->wait_limit ? m->wait_limit : TC_WAIT;
    for (int l = 1; l <= 4; ++l) {
        a.Z[l] = m->Z[l];
        a.H[l] = m->H[l];
        a.dZ[l] = m->dZ[l];
    }
    return a;
}

// Training forward pass of B rows (B a multiple of 128, targets t[B][8]) on the tensor
// cores: Z_l, H_l kept for the backward pass, the loss partials, dL/dy and dL/dZ4.
void forward(odx_mlp *m, const float *x, int64_t B, const float *t, cudaStream_t st)
{
    pack_hidden_weights<<<blocks_for(3 * HID * HID, 256), 256, 0, st>>>(m->pb, m->wpack, 0, 1.f);
    TcArgs a = chain_args(m, m->wpack, B);
    a.x = x;
    launch_chain<TC_TRAIN>(m, a, B, st);
    layer5_fused<<<L5_BLOCKS, L5_THREADS, 0, st>>>(m->H[4], m->Z[4], m->pb, m->p, B, t, m->dY,
                                                   m->dZ[4], m->loss_part);
}

// Backward pass after forward(): every gradient into m->grad, the loss into m->loss.  dL/dZ
// through the three 256 x 256 layers on the tensor cores (one chain per row tile); the weight
// gradients dW_l = H_{l-1}^T dZ_l reduce over the batch on the tensor cores too (split over
// the batch, partials added in split order); bias and 4-wide-layer gradients as column sums.
void backward(odx_mlp *m, const float *x, int64_t B, cudaStream_t st)
{
    pack_hidden_weights<<<blocks_for(3 * HID * HID, 256), 256, 0, st>>>(m->pb, m->wpackB, 1, 1.f);
    TcArgs a = chain_args(m, m->wpackB, B);
    a.dZ4 = m->dZ[4];
    launch_chain<TC_BWD>(m, a, B, st);
    // dW_l = H_{l-1}^T dZ_l for l = 4, 3, 2 on the tensor cores, split over the batch
    DwArgs dw{};
    for (int slot = 0; slot < 3; ++slot) {
        dw.H[slot] = m->H[3 - slot];
        dw.dZ[slot] = m->dZ[4 - slot];
    }
    dw.n_chunks = B / DW_KC;
    dw.part = m->dw_part;
    dw.err = m->tc_err;
    const int splits = (int)std::min<int64_t>(DW_MAX_SPLITS, dw.n_chunks);
    mlp_dw_tc<<<dim3((unsigned)splits, 3), DW_THREADS, DW_SMEM, st>>>(dw);
    dw_reduce<<<blocks_for(3 * HID * HID, 256), 256, 0, st>>>(m->dw_part, splits, m->grad);
    ColArgs c{};
    for (int l = 4; l >= 1; --l) c.A[4 - l] = m->dZ[l];
    c.A[4] = m->H[4];
    c.x = x;
    c.dY = m->dY;
    c.B = B;
    c.part = m->col_part;
    col_reduce<<<dim3(CR_BLOCKS, CR_JOBS), CR_THREADS, 0, st>>>(c);
    grad_finish<<<blocks_for((int64_t)GF_OUTPUTS * 32, 256), 256, 0, st>>>(m->col_part, m->loss_part,
                                                                        m->grad, m->loss);
}

void free_mlp(odx_mlp *m)
{
    cudaSetDevice(m->device);
    for (void *q : {(void *)m->p, (void *)m->pb, (void *)m->grad, (void *)m->m1, (void *)m->m2,
                    (void *)m->dY, (void *)m->loss, (void *)m->loss_part, (void *)m->col_part, (void *)m->wpackB,
                    (void *)m->dw_part,
                    (void *)m->xin, (void *)m->surr_x, (void *)m->surr_y, (void *)m->fb_rays,
                    (void *)m->fb_pix, (void *)m->fb_count, (void *)m->bcrit,
                    (void *)m->scene_tab, (void *)m->wpack, (void *)m->tc_err})
        if (q) cudaFree(q);
    for (int l = 1; l <= 4; ++l) {
        if (m->Z[l]) cudaFree(m->Z[l]);
        if (m->H[l]) cudaFree(m->H[l]);
        if (m->dZ[l]) cudaFree(m->dZ[l]);
    }
    delete m;
}

int64_t round128(int64_t n) { return (n + 127) / 128 * 128; }

// Report and clear the tensor-core kernels' time-out flag (synchronous).
int32_t take_tc_flag(odx_mlp *m)
{
    int h = 0;
    if (cudaMemcpy(&h, m->tc_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return ODX_ERR_CUDA;
    if (h == 0) return ODX_OK;
    if (cudaMemset(m->tc_err, 0, sizeof(int)) != cudaSuccess) return ODX_ERR_CUDA;
    return ODX_ERR_DEVICE_FLAG;
}

// Inference of n rows on the tensor cores (weights packed from the current BF16 copy, halved:
// the kernel's accumulators then hold z / 2, the argument of SiLU's tanh form).
void infer_tc(odx_mlp *m, const float *x, int64_t n, float *y, cudaStream_t st)
{
    if (n <= 0) return;
    pack_hidden_weights<<<blocks_for(3 * HID * HID, 256), 256, 0, st>>>(m->pb, m->wpack, 0, 0.5f);
    TcArgs a = chain_args(m, m->wpack, n);
    a.x = x;
    a.y = y;
    const int64_t tiles = (n + TC_ROWS - 1) / TC_ROWS;
    const unsigned grid = (unsigned)std::min<int64_t>(tiles, std::max(1, m->num_sms));
    mlp_infer_ts<<<grid, TS_THREADS, TS_SMEM, st>>>(a);
}

}  // namespace

extern "C" {

int32_t odx_mlp_create(odx_ctx *ctx, int64_t max_batch, uint64_t seed, odx_mlp **out)
{
    if (!ctx || !out || max_batch < 1 || max_batch > (int64_t)1 << 22) return ODX_ERR_INVALID_ARG;
    *out = nullptr;
    CtxView v;
    if (ctx_view(ctx, &v) != ODX_OK) return ODX_ERR_INVALID_ARG;
    if (cudaSetDevice(v.device) != cudaSuccess) return ODX_ERR_CUDA;
    odx_mlp *m = new odx_mlp();
    m->ctx = ctx;
    m->device = v.device;
    m->max_batch = round128(max_batch);
    const size_t act = (size_t)m->max_batch * HID * sizeof(bf16);
    bool ok = cudaMalloc(&m->p, NPARAM * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&m->pb, NPARAM * sizeof(bf16)) == cudaSuccess &&
              cudaMalloc(&m->grad, NPARAM * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&m->m1, NPARAM * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&m->m2, NPARAM * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&m->wpackB, (size_t)3 * HID * HID * sizeof(bf16)) == cudaSuccess &&
              cudaMalloc(&m->dw_part, (size_t)3 * DW_MAX_SPLITS * HID * HID * sizeof(float)) ==
                  cudaSuccess &&
              cudaMalloc(&m->loss_part, L5_BLOCKS * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&m->col_part, (size_t)CR_JOBS * CR_BLOCKS * CR_K * HID * sizeof(float)) ==
                  cudaSuccess &&
              cudaMalloc(&m->dY, m->max_batch * NOUT * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&m->loss, sizeof(float)) == cudaSuccess &&
              cudaMalloc(&m->xin, m->max_batch * NIN * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&m->bcrit, (BCRIT_N + 1) * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&m->scene_tab, sizeof(DevScene)) == cudaSuccess &&
              cudaMalloc(&m->fb_count, sizeof(unsigned long long)) == cudaSuccess &&
              cudaMalloc(&m->wpack, (size_t)3 * HID * HID * sizeof(bf16)) == cudaSuccess &&
              cudaMalloc(&m->tc_err, sizeof(int)) == cudaSuccess;
    for (int l = 1; l <= 4 && ok; ++l)
        ok = cudaMalloc(&m->Z[l], act) == cudaSuccess && cudaMalloc(&m->H[l], act) == cudaSuccess &&
             cudaMalloc(&m->dZ[l], act) == cudaSuccess;
    if (!ok) {
        free_mlp(m);
        return ODX_ERR_CUDA;
    }
    cudaMemset(m->m1, 0, NPARAM * sizeof(float));
    cudaMemset(m->m2, 0, NPARAM * sizeof(float));
    if (cudaFuncSetAttribute(mlp_infer_ts, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)TS_SMEM) != cudaSuccess ||
        cudaFuncSetAttribute(mlp_chain_tc<TC_TRAIN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)TC_SMEM) != cudaSuccess ||
        cudaFuncSetAttribute(mlp_chain_tc<TC_BWD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)TC_SMEM) != cudaSuccess ||
        cudaFuncSetAttribute(mlp_dw_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)DW_SMEM) != cudaSuccess ||
        cudaDeviceGetAttribute(&m->num_sms, cudaDevAttrMultiProcessorCount, m->device) !=
            cudaSuccess ||
        cudaMemset(m->tc_err, 0, sizeof(int)) != cudaSuccess) {
        free_mlp(m);
        return ODX_ERR_CUDA;
    }
    init_params<<<blocks_for(NPARAM, 256), 256>>>(m->p, m->pb, seed);
    if (cudaDeviceSynchronize() != cudaSuccess) {
        free_mlp(m);
        return ODX_ERR_CUDA;
    }
    *out = m;
    return ODX_OK;
}

int32_t odx_mlp_destroy(odx_mlp *m)
{
    if (m) free_mlp(m);
    return ODX_OK;
}

int32_t odx_mlp_get_params(odx_mlp *m, float *host)
{
    if (!m || !host) return ODX_ERR_INVALID_ARG;
    MLP_CUDA(cudaSetDevice(m->device));
    MLP_CUDA(cudaMemcpy(host, m->p, NPARAM * sizeof(float), cudaMemcpyDeviceToHost));
    return take_tc_flag(m);
}

int32_t odx_mlp_set_params(odx_mlp *m, const float *host)
{
    if (!m || !host) return ODX_ERR_INVALID_ARG;
    MLP_CUDA(cudaSetDevice(m->device));
    MLP_CUDA(cudaMemcpy(m->p, host, NPARAM * sizeof(float), cudaMemcpyHostToDevice));
    to_bf16<<<blocks_for(NPARAM, 256), 256>>>(m->p, m->pb, NPARAM);
    MLP_CUDA(cudaMemset(m->m1, 0, NPARAM * sizeof(float)));
    MLP_CUDA(cudaMemset(m->m2, 0, NPARAM * sizeof(float)));
    m->step = 0;
    MLP_CUDA(cudaDeviceSynchronize());
    return ODX_OK;
}

int32_t odx_mlp_set_wait_limit(odx_mlp *m, uint32_t tries)
{
    if (!m) return ODX_ERR_INVALID_ARG;
    m->wait_limit = tries;
    return ODX_OK;
}

int32_t odx_mlp_forward(odx_mlp *m, const float *x, int64_t n, float *y, void *stream)
{
    if (!m || n < 0 || (n > 0 && (!x || !y))) return ODX_ERR_INVALID_ARG;
    if (((uintptr_t)x & 15u) || ((uintptr_t)y & 15u)) return ODX_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    MLP_CUDA(cudaSetDevice(m->device));
    infer_tc(m, x, n, y, st);
    MLP_CUDA(cudaGetLastError());
    return ODX_OK;
}

int32_t odx_mlp_gradients(odx_mlp *m, const float *x, const float *t, int64_t n, float *grad_host,
                          float *loss_host)
{
    if (!m || !x || !t || n < 1 || n > m->max_batch || n % 128 != 0 || ((uintptr_t)x & 15u) ||
        ((uintptr_t)t & 15u))
        return ODX_ERR_INVALID_ARG;
    MLP_CUDA(cudaSetDevice(m->device));
    forward(m, x, n, t, nullptr);
    backward(m, x, n, nullptr);
    MLP_CUDA(cudaDeviceSynchronize());
    if (grad_host)
        MLP_CUDA(cudaMemcpy(grad_host, m->grad, NPARAM * sizeof(float), cudaMemcpyDeviceToHost));
    if (loss_host) MLP_CUDA(cudaMemcpy(loss_host, m->loss, sizeof(float), cudaMemcpyDeviceToHost));
    return take_tc_flag(m);
}

int32_t odx_mlp_train_step(odx_mlp *m, const float *x, const float *t, int64_t n, float lr,
                           float *loss_dev, void *stream)
{
    if (!m || !x || !t || n < 1 || n > m->max_batch || n % 128 != 0 || !(lr > 0.f) ||
        ((uintptr_t)x & 15u) || ((uintptr_t)t & 15u))
        return ODX_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    MLP_CUDA(cudaSetDevice(m->device));
    forward(m, x, n, t, st);
    backward(m, x, n, st);
    m->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)m->step), c2 = 1.f - powf(b2, (float)m->step);
    adam_step<<<blocks_for(NPARAM, 256), 256, 0, st>>>(m->p, m->pb, m->grad, m->m1, m->m2, NPARAM,
                                                       lr, b1, b2, 1e-8f, c1, c2);
    if (loss_dev)
        MLP_CUDA(cudaMemcpyAsync(loss_dev, m->loss, sizeof(float), cudaMemcpyDeviceToDevice, st));
    MLP_CUDA(cudaGetLastError());
    return ODX_OK;
}

int32_t odx_mlp_targets(odx_ctx *ctx, const odx_ray_record *rec, const double *rays, int64_t n,
                        double r_max, float *x, float *t, void *stream)
{
    if (!ctx || n < 0 || (n > 0 && (!rec || !rays || !x || !t))) return ODX_ERR_INVALID_ARG;
    if (n == 0) return ODX_OK;
    const int64_t n_pad = round128(n);
    make_targets<<<blocks_for(n_pad, 256), 256, 0, (cudaStream_t)stream>>>(rec, rays, n, n_pad,
                                                                           r_max, x, t);
    MLP_CUDA(cudaGetLastError());
    return ODX_OK;
}

int32_t odx_surrogate_render(odx_mlp *m, const odx_scene *scene, double band, double p_lo,
                             double p_hi, odx_ray_record *fb_records, int64_t *fb_pixels,
                             double *image, int64_t *n_fallback, void *stream)
{
    if (!m || !scene || !fb_records || !image || !(band >= 0.0) || !(p_lo <= p_hi))
        return ODX_ERR_INVALID_ARG;
    if (validate_scene_table(scene, 1) != ODX_OK || scene->emitter != ODX_EMIT_THIN_DISK)
        return ODX_ERR_INVALID_ARG;
    if (((uintptr_t)fb_records & 15u) != 0) return ODX_ERR_INVALID_ARG;
    CtxView v;
    if (ctx_view(m->ctx, &v) != ODX_OK) return ODX_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    MLP_CUDA(cudaSetDevice(m->device));
    const int64_t n = (int64_t)scene->n_alpha * scene->n_beta;
    const int64_t n_pad = round128(n);
    if (m->surr_cap < n_pad) {
        for (void *q : {(void *)m->surr_x, (void *)m->surr_y, (void *)m->fb_rays, (void *)m->fb_pix})
            if (q) cudaFree(q);
        m->surr_x = m->surr_y = nullptr;
        m->fb_rays = nullptr;
        m->fb_pix = nullptr;
        m->surr_cap = 0;
        MLP_CUDA(cudaMalloc(&m->surr_x, n_pad * NIN * sizeof(float)));
        MLP_CUDA(cudaMalloc(&m->surr_y, n_pad * NOUT * sizeof(float)));
        MLP_CUDA(cudaMalloc(&m->fb_rays, n_pad * 4 * sizeof(double)));
        MLP_CUDA(cudaMalloc(&m->fb_pix, n_pad * sizeof(int64_t)));
        m->surr_cap = n_pad;
    }
    DevScene d;
    fill_dev_scene(d, *scene, 0, n, 0);
    MLP_CUDA(cudaMemcpyAsync(m->scene_tab, &d, sizeof(DevScene), cudaMemcpyHostToDevice, st));
    MLP_CUDA(cudaMemsetAsync(m->fb_count, 0, sizeof(unsigned long long), st));
    bcrit_table<<<blocks_for(BCRIT_N, 128), 128, 0, st>>>(scene->a, scene->theta_obs, scene->r_in,
                                                          m->bcrit);
    surrogate_inputs<<<blocks_for(n_pad, 256), 256, 0, st>>>(m->scene_tab, n_pad, m->surr_x);
    infer_tc(m, m->surr_x, n_pad, m->surr_y, st);
    surrogate_classify<<<blocks_for(n, 256), 256, 0, st>>>(m->scene_tab, m->surr_y, m->bcrit, band,
                                                          (float)p_lo, (float)p_hi, image,
                                                          m->fb_rays, m->fb_pix, m->fb_count);
    unsigned long long nfb = 0;
    MLP_CUDA(cudaMemcpyAsync(&nfb, m->fb_count, sizeof(nfb), cudaMemcpyDeviceToHost, st));
    MLP_CUDA(cudaStreamSynchronize(st));
    const int32_t flag = take_tc_flag(m);
    if (flag != ODX_OK) return flag;
    if (n_fallback) *n_fallback = (int64_t)nfb;
    if (nfb > 0) {
        // trace the fallback pixels (list mode, the scene's own precision) and scatter them
        fill_dev_scene(d, *scene, 0, (int64_t)nfb, 0);
        MLP_CUDA(cudaMemcpyAsync(m->scene_tab, &d, sizeof(DevScene), cudaMemcpyHostToDevice, st));
        MLP_CUDA(cudaMemsetAsync(v.queue, 0, sizeof(unsigned long long), st));
        TraceArgs a{};
        a.scenes = m->scene_tab;
        a.n_scenes = 1;
        a.list_mode = 1;
        a.rays = m->fb_rays;
        a.n_total = (int64_t)nfb;
        a.records = fb_records;
        a.image = nullptr;
        a.queue = v.queue;
        a.stats = v.stats;
        a.chunk = v.launch.chunk;
        a.persistent = v.launch.persistent;
        a.fp64_batch = v.launch.fp64_batch;
        set_launch_medium(a, d, true);
        const cudaError_t e = scene->precision == ODX_MIXED
                                  ? launch_trace_mixed(a, 0, v.launch, v.num_sms, st)
                                  : launch_trace_fp64(a, 0, v.launch, v.num_sms, st);
        if (e != cudaSuccess) return ODX_ERR_CUDA;
        scatter_fallback<<<blocks_for((int64_t)nfb, 256), 256, 0, st>>>(fb_records, m->fb_pix,
                                                                       (int64_t)nfb, image);
        if (fb_pixels)
            MLP_CUDA(cudaMemcpyAsync(fb_pixels, m->fb_pix, nfb * sizeof(int64_t),
                                     cudaMemcpyDeviceToDevice, st));
    }
    MLP_CUDA(cudaGetLastError());
    return ODX_OK;
}

}  // extern "C"
