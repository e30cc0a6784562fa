// Internal declarations shared by the host API (odx_api.cu) and the kernel translation
// units.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/odyssey.h"

namespace odx {

// Image planes of a scene: one per observed frequency for the torus, the Novikov-Thorne disk,
// the synchrotron shell and the hot spot, otherwise one (thin-disk intensity, or zero for geodesics only).
__host__ __device__ inline int32_t scene_planes(const odx_scene &s)
{
    return (s.emitter == ODX_EMIT_TORUS || s.emitter == ODX_EMIT_NT_DISK ||
            s.emitter == ODX_EMIT_SYNCH || s.emitter == ODX_EMIT_SPOT)
               ? s.n_freq
               : 1;
}
// Emitters whose rays stop on the opaque equatorial disk r_in <= r <= r_out.
__host__ __device__ inline bool disk_emitter(int32_t e)
{
    return e == ODX_EMIT_THIN_DISK || e == ODX_EMIT_NT_DISK;
}

// A scene as the kernels read it: the caller's description plus where its rays sit in the
// launch-wide ray numbering and where its image planes start.
struct DevScene {
    odx_scene s;
    int64_t ray_begin;  // first global ray index of this scene
    int64_t n_rays;     // n_alpha * n_beta (list mode: n)
    int64_t img_offset; // offset of this scene's image planes, in doubles
    int64_t pad;
    // FP64 constants of the initial state (Section 2.2) shared by the scene's pixels:
    // sin, cos of theta_obs and phi_obs, sqrt(r_obs^2 + a^2), r_ISCO and the stop radius
    double o_sto, o_cto, o_spo, o_cpo, o_Ro, o_r_isco, o_r_stop;
    // error-scale floors of the transfer intensities (rt_floor, kerr_device.cuh), per
    // frequency slot, padded past n_freq with the last; infinite without transfer
    double rt_floor[ODX_MAX_FREQ];
    // FP32 constants of the FP32 stages (filled by fill_dev_scene)
    float f_r_out, f_hmax_frac, f_rtol32;
    float f_T_index;   // 1/T_e = exp(T_index ln r) / T0
    float f_inv_T0;
    float f_lr_pref;   // C n_e^2 T_e^-1/2 = f_pref0 exp(f_lr_pref ln r + f_c2_pref cos^2 theta)
    float f_c2_pref;
    float f_pref0;
    float f_nu[ODX_MAX_FREQ];       // observed frequencies, padded past n_freq with the last
                                    // (synchrotron shell: in GHz)
    float f_inv_nu3[ODX_MAX_FREQ];  // 1 / f_nu^3
    // synchrotron shell (f_synch = 1): n_e / n_e0 = exp(f_lr_pref ln r + f_c2_pref cos^2),
    // 1 / Theta_e from f_T_index, f_inv_T0 as for the torus; SynchK in FP32
    float f_inv_kc, f_ky, f_Atau;
    int32_t f_synch;
    float f_rt_floor[ODX_MAX_FREQ];  // rt_floor in FP32
    // hot spot: sqrt(r_s^2 + a^2), Omega, the centre's azimuth at emission time 0 for an
    // image at t_obs (spot_phase + Omega t_obs, reduced mod 2 pi), 4 r_spot
    float f_spot_Rs, f_spot_om, f_spot_ph, f_spot_R4;
};

// One scene-table entry for a scene whose rays start at ray_begin (all table builders).
void fill_dev_scene(DevScene &d, const odx_scene &s, int64_t ray_begin, int64_t n_rays,
                    int64_t img_offset);

// Device counters; 64-bit for atomicAdd.
struct DevStats {
    unsigned long long rays, acc, rej, fp64, slots, active;
    int32_t error_flag;
    int32_t pad;
};

// FP32 torus constants of one scene (the f_* fields of DevScene), carried in the kernel
// parameters when every ray of a launch shares one medium.
struct MedConst {
    float T_index, inv_T0, lr_pref, c2_pref, pref0;
    float nu[ODX_MAX_FREQ], inv_nu3[ODX_MAX_FREQ], rt_floor[ODX_MAX_FREQ];
    float inv_kc, ky, Atau, r_out;
    int32_t synch;
    int32_t spot;  // the launch's scenes are hot spots
};

struct TraceArgs {
    const DevScene *scenes;
    int32_t n_scenes;
    int32_t list_mode;     // 1: rays[n][4] = (alpha, beta, a, cos i) with scene 0 as prototype
    const double *rays;
    int64_t n_total;       // rays of the render (all scenes)
    int64_t id_begin, id_end;  // the global ray ids this launch traces; both 0: [0, n_total)
    odx_ray_record *records;
    double *image;         // may be null
    unsigned long long *queue;
    DevStats *stats;
    int32_t chunk;
    int32_t persistent;
    int32_t fp64_batch;
    int32_t single_medium;  // 1: every ray uses `med` (one scene, or list mode)
    MedConst med;
};

// The range of global ray ids a launch traces (id_begin = id_end = 0: every ray).
__host__ __device__ inline int64_t launch_first(const TraceArgs &a)
{
    return a.id_end > 0 ? a.id_begin : 0;
}
__host__ __device__ inline int64_t launch_count(const TraceArgs &a)
{
    return a.id_end > 0 ? a.id_end - a.id_begin : a.n_total;
}

// Fill a.single_medium and a.med from the host copy of scene 0.
void set_launch_medium(TraceArgs &a, const DevScene &scene0, bool single);
// True when every scene of the table folds to the same medium constants, bit for bit: the
// launch can then take the single-medium kernels (constants in the kernel parameters, the
// medium kind compiled in), which compute each ray as the per-lane-medium kernels do.
bool shared_medium(const DevScene *table, int32_t n_scenes);

// Launch the FP64 or mixed tracer (with its passes) on `stream`; when ev0/ev1 are given,
// they are recorded immediately before and after the tracing kernel itself.
cudaError_t launch_trace_fp64(const TraceArgs &args, int32_t nf_slots, const odx_launch &L,
                              int32_t num_sms, cudaStream_t st, cudaEvent_t ev0 = nullptr,
                              cudaEvent_t ev1 = nullptr);
cudaError_t launch_trace_mixed(const TraceArgs &args, int32_t nf_slots, const odx_launch &L,
                               int32_t num_sms, cudaStream_t st, cudaEvent_t ev0 = nullptr,
                               cudaEvent_t ev1 = nullptr);

// Image-integrated flux (spectra) and its frequency integral (light curves): spectra.cu.
cudaError_t launch_image_flux(const DevScene *scenes_dev, const void *planes_dev,
                              int32_t n_scenes, int32_t planes_per_scene, int64_t max_plane,
                              const double *image, double *partial, int32_t chunks,
                              double *flux, double *lum, cudaStream_t st);
size_t plane_ref_bytes();
void fill_plane_ref(void *dst, int64_t first, int64_t n, int32_t scene, int32_t j);

// Set the FP64 tracers' dynamic shared-memory limit on the current device (once per device,
// before any launch or stream capture).
cudaError_t prepare_fp64_kernels();

// FMA-chain peak microbenchmark: returns flop/s via *flops (synchronous).
cudaError_t run_fma_peak(int32_t precision, int32_t num_sms, double *flops);

}  // namespace odx
