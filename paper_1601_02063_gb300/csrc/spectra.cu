// Image-integrated flux (spectra) and its frequency integral (light curves), Section 4.4:
// the flux density of one image plane at the observer is the intensity summed over the
// image times the solid angle of a pixel, F_nu = sum I_nu dalpha dbeta / r_obs^2; a light
// curve point is F integrated over the frequency bins of the image.
//
// Deterministic: every plane is cut into fixed chunks, each summed by one block in a fixed
// order (strided thread sums, then a fixed shuffle and shared-memory tree), and a second
// kernel adds a plane's chunk sums in index order, so the result does not depend on the
// schedule.  HBM-bound: one read of the image.
#include <cuda_runtime.h>
#include <stdint.h>

#include "odx_internal.h"

namespace odx {

constexpr int FLUX_THREADS = 512;

// Plane p of the launch: scene s, plane j, pixel range [first, first + n).
struct PlaneRef {
    int64_t first, n;
    int32_t scene, j;
};

__device__ __forceinline__ double block_sum(double v, double *sh)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    v = 0.0;
    if (warp == 0) {
        v = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    return v;  // valid in thread 0
}

// grid (chunks, planes): partial[p * chunks + c] = sum of chunk c of plane p
__global__ void __launch_bounds__(FLUX_THREADS) flux_partial_kernel(
    const double *__restrict__ image, const PlaneRef *__restrict__ planes, int64_t chunk,
    double *__restrict__ partial)
{
    __shared__ double sh[FLUX_THREADS / 32];
    const PlaneRef P = planes[blockIdx.y];
    const int64_t lo = (int64_t)blockIdx.x * chunk;
    const int64_t hi = lo + chunk < P.n ? lo + chunk : P.n;
    double v = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += FLUX_THREADS) v += image[P.first + i];
    v = block_sum(v, sh);
    if (threadIdx.x == 0) partial[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = v;
}

// one thread per plane: F = (sum of chunk sums) * pixel solid angle
__global__ void flux_finish_kernel(const DevScene *__restrict__ scenes,
                                   const PlaneRef *__restrict__ planes, int32_t n_planes,
                                   int32_t chunks, const double *__restrict__ partial,
                                   double *__restrict__ flux)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_planes) return;
    const PlaneRef P = planes[p];
    const odx_scene &s = scenes[P.scene].s;
    double sum = 0.0;
    for (int c = 0; c < chunks; ++c) sum += partial[(int64_t)p * chunks + c];
    const double da = (s.alpha_max - s.alpha_min) / s.n_alpha;
    const double db = (s.beta_max - s.beta_min) / s.n_beta;
    flux[p] = sum * (da * db) / (s.r_obs * s.r_obs);
}

// one thread per scene: trapezoid rule of F over nu (a single plane: F itself)
__global__ void lum_kernel(const DevScene *__restrict__ scenes, int32_t n_scenes,
                           int32_t planes_per_scene, const double *__restrict__ flux,
                           double *__restrict__ lum)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_scenes) return;
    const odx_scene &s = scenes[k].s;
    const double *F = flux + (int64_t)k * planes_per_scene;
    if (planes_per_scene < 2) {
        lum[k] = F[0];
        return;
    }
    double L = 0.0;
    for (int j = 0; j + 1 < planes_per_scene; ++j)
        L += 0.5 * (F[j] + F[j + 1]) * (s.freqs[j + 1] - s.freqs[j]);
    lum[k] = L;
}

cudaError_t launch_image_flux(const DevScene *scenes_dev, const void *planes_dev,
                              int32_t n_scenes, int32_t planes_per_scene, int64_t max_plane,
                              const double *image, double *partial, int32_t chunks,
                              double *flux, double *lum, cudaStream_t st)
{
    const int32_t n_planes = n_scenes * planes_per_scene;
    const int64_t chunk = (max_plane + chunks - 1) / chunks;
    const PlaneRef *planes = static_cast<const PlaneRef *>(planes_dev);
    flux_partial_kernel<<<dim3((unsigned)chunks, (unsigned)n_planes), FLUX_THREADS, 0, st>>>(
        image, planes, chunk, partial);
    flux_finish_kernel<<<(n_planes + 127) / 128, 128, 0, st>>>(scenes_dev, planes, n_planes,
                                                               chunks, partial, flux);
    if (lum)
        lum_kernel<<<(n_scenes + 127) / 128, 128, 0, st>>>(scenes_dev, n_scenes,
                                                          planes_per_scene, flux, lum);
    return cudaGetLastError();
}

size_t plane_ref_bytes() { return sizeof(PlaneRef); }

void fill_plane_ref(void *dst, int64_t first, int64_t n, int32_t scene, int32_t j)
{
    PlaneRef *p = static_cast<PlaneRef *>(dst);
    p->first = first;
    p->n = n;
    p->scene = scene;
    p->j = j;
}

}  // namespace odx
