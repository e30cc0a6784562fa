// Mixed-precision backward ray tracer for GB300 (sm_103a).
//
// GB300 executes FP32 at 63x the FP64 rate (78.5 vs 1.25 TFLOP/s measured), so the bulk
// of the Cash-Karp stages runs in FP32 with these FP64 / compensated parts:
//   - initial state and constants of motion (Section 2.2) in FP64;
//   - the state y and the transfer integrals tau, I kept as unevaluated float pairs
//     (hi + lo, ~48-bit) updated with error-free two-sums, so that the accumulation over
//     hundreds of steps does not add FP32 rounding (compensated sums);
//   - steps with r < r_switch (near the horizon and the photon orbits) in FP64 with the
//     FP64 tolerance rtol;
//   - the null-condition and Carter-constant checks and the disk redshift in FP64.
// Per-ray arithmetic depends only on the ray's own path (the FP32/FP64 choice is made per
// lane from its own radius), so results do not depend on the launch shape.
//
// An FP64 step costs a warp the same whether one lane or 32 take it, so lanes that need
// one wait until `fp64_batch` lanes of the warp need one (or no FP32 lane is left), and
// the warp then runs a single FP64 step for all of them.
#include <cuda_runtime.h>
#include <math.h>

#include "kerr_device.cuh"
#include "odx_internal.h"
#include "trace_common.cuh"
#include "trace_step.cuh"

namespace odx {

// (hi, lo) += d, error-free (Knuth two-sum, then renormalisation).
__device__ __forceinline__ void df_add(float &hi, float &lo, float d)
{
    const float s = hi + d;
    const float bp = s - hi;
    const float err = (hi - (s - bp)) + (d - bp);
    const float l = lo + err;
    const float t = s + l;
    lo = l - (t - s);
    hi = t;
}

__device__ __forceinline__ void df_set(float &hi, float &lo, double v)
{
    hi = (float)v;
    lo = (float)(v - (double)hi);
}

__device__ __forceinline__ double df_get(float hi, float lo) { return (double)hi + (double)lo; }

template <int NF>
struct RayM {
    float yh[6], yl[6];           // state as float pairs: r, theta, phi, t, p_r, p_theta
    float k1f[6];                 // FP32 first stage (valid when mode == 0)
    float th[NF + 1], tl[NF + 1]; // tau pairs
    float Ih[NF + 1], Il[NF + 1]; // invariant intensity pairs
    float kt1f[NF + 1], kI1f[NF + 1];
    float hf, hsf;                // FP32 step and error-scale step
    double hd, hsd;               // FP64 step and error-scale step
    int32_t mode;                 // 0: FP32 first stage and hf valid, 1: hd valid (FP64)
    float af, Lf, sgnf, r_switch, hmaxf, r_stopf, r_startf, rtolf;
    double a, L, Q0;
    double r_start, r_stop, r_in, r_out;
    double r_cross, phi_cross;
    int64_t id;
    int32_t scene, n_acc, n_rej, n_cross, n64;
};

template <int NF>
__device__ __forceinline__ void state_double(const RayM<NF> &R, double y[6], double *tau)
{
#pragma unroll
    for (int i = 0; i < 6; ++i) y[i] = df_get(R.yh[i], R.yl[i]);
#pragma unroll
    for (int k = 0; k < NF; ++k) tau[k] = df_get(R.th[k], R.tl[k]);
}

template <int NF>
__device__ __forceinline__ void write_result_m(const TraceArgs &A, const DevScene &S,
                                               const RayM<NF> &R, int32_t status,
                                               const double yend[6], double r_hit,
                                               double phi_hit, double g, double inten)
{
    RecordOut o;
    o.status = status;
    o.n_acc = R.n_acc;
    o.n_rej = R.n_rej;
    o.n_cross = R.n_cross;
    o.r_cross = R.r_cross;
    o.phi_cross = R.phi_cross;
    o.r_hit = r_hit;
    o.phi_hit = phi_hit;
    o.g = g;
    o.intensity = inten;
    o.H_end = null_violation(R.a, R.L, yend);
    o.Q_drift = (carter_q(R.a, R.L, yend) - R.Q0) / fmax(fabs(R.Q0), 1.0);
    store_record(A.records + R.id, o);
    if (A.image) {
        double *img = A.image + S.img_offset + (R.id - S.ray_begin);
        if constexpr (NF > 0) {
#pragma unroll
            for (int k = 0; k < NF; ++k) {
                if (k < S.s.n_freq) {
                    const double nu = S.s.freqs[k];
                    img[(int64_t)k * S.n_rays] = nu * nu * nu * df_get(R.Ih[k], R.Il[k]);
                }
            }
        } else {
            img[0] = inten;
        }
    }
}

// Equatorial crossing in FP32 (same method as the FP64 path, stopping at the FP32
// resolution of cos(theta)): returns the crossing state as doubles.
__device__ __noinline__ void locate_crossing32(const Geo<float> &g, const float yh[6],
                                               const float yl[6], const float k1[6], float h,
                                               double yc[6])
{
    float lo = 0.f, hi = h;
    float flo = cosf(yh[1]);
    float dy[6];
    ck_geo_increment<float>(g, yh, k1, h, dy);
    const float fhi = cosf(yh[1] + dy[1]);
    float sig = lo - flo * (hi - lo) / (fhi - flo);
    if (!(sig > lo && sig < hi)) sig = 0.5f * (lo + hi);
    for (int it = 0; it < 40; ++it) {
        ck_geo_increment<float>(g, yh, k1, sig, dy);
        float yt[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) yt[i] = yh[i] + dy[i];
        float sn, F;
        sincosf(yt[1], &sn, &F);
        if (fabsf(F) <= 3e-7f) break;
        if ((F > 0.f) == (flo > 0.f)) {
            lo = sig;
            flo = F;
        } else {
            hi = sig;
        }
        float f[6];
        geodesic_rhs<float>(g, yt[0], yt[1], yt[4], yt[5], f);
        const float dF = -sn * f[1];
        float nx = sig - F / dF;
        if (!(nx > lo && nx < hi)) nx = 0.5f * (lo + hi);
        if (hi - lo <= 1e-6f * h) break;
        sig = nx;
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) yc[i] = (double)yh[i] + ((double)yl[i] + (double)dy[i]);
}

__device__ __noinline__ void locate_crossing64m(const Geo<double> &g, const double y[6],
                                                const double k1[6], double h, double yc[6])
{
    double lo = 0.0, hi = h;
    double flo = cos(y[1]);
    double dy[6], y5[6];
    ck_geo_increment<double>(g, y, k1, h, dy);
    const double fhi = cos(y[1] + dy[1]);
    double sig = lo - flo * (hi - lo) / (fhi - flo);
    if (!(sig > lo && sig < hi)) sig = 0.5 * (lo + hi);
    for (int it = 0; it < 60; ++it) {
        ck_geo_increment<double>(g, y, k1, sig, dy);
#pragma unroll
        for (int i = 0; i < 6; ++i) y5[i] = y[i] + dy[i];
        double sn, F;
        sincos(y5[1], &sn, &F);
        if (fabs(F) <= 1e-14) break;
        if ((F > 0.0) == (flo > 0.0)) {
            lo = sig;
            flo = F;
        } else {
            hi = sig;
        }
        double f[6];
        geodesic_rhs<double>(g, y5[0], y5[1], y5[4], y5[5], f);
        const double dF = -sn * f[1];
        double nx = sig - F / dF;
        if (!(nx > lo && nx < hi)) nx = 0.5 * (lo + hi);
        if (hi - lo <= 1e-15 * h) break;
        sig = nx;
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) yc[i] = y[i] + dy[i];
}

// Disk hit with the crossing state yc (FP64): returns true when the ray stops on the disk.
template <int NF>
__device__ __forceinline__ bool disk_hit(const TraceArgs &A, const DevScene &S,
                                         const RayM<NF> &R, const double yc[6])
{
    if (S.s.emitter != ODX_EMIT_THIN_DISK || !(yc[0] >= R.r_in && yc[0] <= R.r_out)) return false;
    const double gz = disk_redshift(R.a, yc[0], R.L);
    const double g2 = gz * gz;
    const double inten = g2 * g2 * pow(yc[0], -S.s.q_emis);
    write_result_m<NF>(A, S, R, ODX_DISK_HIT, yc, yc[0], yc[2], gz, inten);
    return true;
}

// One FP32 Cash-Karp attempt.  Returns the new status.
template <int NF>
__device__ __forceinline__ int32_t step32(const TraceArgs &A, const DevScene &S, RayM<NF> &R,
                                          const MediumT<float> &mf)
{
    const Geo<float> g{R.af, R.Lf, R.sgnf};
    if (R.mode != 0) {  // (re)enter FP32: first stage in FP32
        derivs_stage<float, NF>(g, mf, R.yh, R.th, R.k1f, R.kt1f, R.kI1f);
        R.hf = (float)R.hd;
        R.hsf = R.hf;
        R.mode = 0;
    }
    const float h = R.hf;
    float dy[6], e[6], dtau[NF + 1], dI[NF + 1];
    ck_attempt<float, NF>(g, mf, R.yh, R.k1f, R.th, R.kt1f, R.kI1f, h, dy, e, dtau, dI);
    float errmax = 0.f;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const float sc = fabsf(R.yh[i]) + fabsf(R.hsf * R.k1f[i]) + 1e-30f;
        errmax = fmaxf(errmax, fabsf(e[i] / sc));
    }
    errmax /= R.rtolf;
    if (isnan(errmax)) errmax = INFINITY;
    if (!(errmax <= 1.f)) {
        ++R.n_rej;
        R.hf = fmaxf(0.9f * h * powf(errmax, -0.25f), 0.1f * h);
        return R.hf < 1e-12f ? ODX_NUMERR : ODX_RUNNING;
    }
    ++R.n_acc;
    const float h_next = (errmax > 1.89e-4f) ? 0.9f * h * powf(errmax, -0.2f) : 5.f * h;
    if ((cosf(R.yh[1]) > 0.f) != (cosf(R.yh[1] + dy[1]) > 0.f)) {
        double yc[6];
        locate_crossing32(g, R.yh, R.yl, R.k1f, h, yc);
        ++R.n_cross;
        if (R.n_cross == 1) {
            R.r_cross = yc[0];
            R.phi_cross = yc[2];
        }
        if (disk_hit<NF>(A, S, R, yc)) return ODX_DISK_HIT;
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) df_add(R.yh[i], R.yl[i], dy[i]);
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        df_add(R.th[k], R.tl[k], dtau[k]);
        df_add(R.Ih[k], R.Il[k], dI[k]);
    }
    if (R.yh[0] < R.r_stopf) return ODX_CAPTURED;
    derivs_stage<float, NF>(g, mf, R.yh, R.th, R.k1f, R.kt1f, R.kI1f);
    if (R.k1f[0] > 0.f && R.yh[0] > R.r_startf) return ODX_ESCAPED;
    R.hf = fminf(h_next, R.hmaxf * R.yh[0]);
    R.hsf = R.hf;
    return ODX_RUNNING;
}

// One FP64 Cash-Karp attempt on the pair state (FP64 tolerance rtol).  The first stage is
// evaluated afresh in FP64 (FP64 steps are rare and batched; keeping an FP64 first stage
// alive across the FP32 steps would cost 2 x (6 + 2 NF) registers on every step).
template <int NF>
__device__ __noinline__ int32_t step64(const TraceArgs &A, const DevScene &S, RayM<NF> &R)
{
    const Geo<double> g{R.a, R.L, (double)R.sgnf};
    MediumT<double> md{};
    if constexpr (NF > 0) load_medium_t<double>(S, R.a, md);
    double y[6], tau[NF + 1], k1[6], kt1[NF + 1], kI1[NF + 1];
    state_double<NF>(R, y, tau);
    derivs<double, NF>(g, md, y, tau, k1, kt1, kI1);
    if (R.mode != 1) {  // entering FP64
        R.hd = (double)R.hf;
        R.hsd = R.hd;
        R.mode = 1;
    }
    ++R.n64;
    const double h = R.hd;
    double dy[6], e[6], dtau[NF + 1], dI[NF + 1];
    ck_attempt<double, NF>(g, md, y, k1, tau, kt1, kI1, h, dy, e, dtau, dI);
    double errmax = 0.0;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const double sc = fabs(y[i]) + fabs(R.hsd * k1[i]) + 1e-30;
        errmax = fmax(errmax, fabs(e[i] / sc));
    }
    errmax /= S.s.rtol;
    if (isnan(errmax)) errmax = INFINITY;
    if (!(errmax <= 1.0)) {
        ++R.n_rej;
        R.hd = fmax(0.9 * h * pow(errmax, -0.25), 0.1 * h);
        return R.hd < 1e-12 ? ODX_NUMERR : ODX_RUNNING;
    }
    ++R.n_acc;
    const double h_next = (errmax > 1.89e-4) ? 0.9 * h * pow(errmax, -0.2) : 5.0 * h;
    if ((cos(y[1]) > 0.0) != (cos(y[1] + dy[1]) > 0.0)) {
        double yc[6];
        locate_crossing64m(g, y, k1, h, yc);
        ++R.n_cross;
        if (R.n_cross == 1) {
            R.r_cross = yc[0];
            R.phi_cross = yc[2];
        }
        if (disk_hit<NF>(A, S, R, yc)) return ODX_DISK_HIT;
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        y[i] += dy[i];
        df_set(R.yh[i], R.yl[i], y[i]);
    }
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        tau[k] += dtau[k];
        df_set(R.th[k], R.tl[k], tau[k]);
        df_set(R.Ih[k], R.Il[k], df_get(R.Ih[k], R.Il[k]) + dI[k]);
    }
    if (y[0] < R.r_stop) return ODX_CAPTURED;
    // escape test: dr/ds at the new point (sgn * Delta p_r / Sigma has the sign of sgn * p_r)
    if (R.sgnf * (float)y[4] > 0.f && y[0] > R.r_start) return ODX_ESCAPED;
    R.hd = fmin(h_next, S.s.hmax_frac * y[0]);
    R.hsd = R.hd;
    R.hf = (float)R.hd;
    return ODX_RUNNING;
}

// MINB: resident 128-thread blocks per SM the register allocation is capped for.
template <int NF, int MINB>
__global__ void __launch_bounds__(128, MINB) trace_mixed_kernel(TraceArgs A)
{
    const int lane = threadIdx.x & 31;
    RayM<NF> R;
    MediumT<float> mf{};
    bool live = false;
    WarpQueue q;
    q.init(A);
    unsigned long long my_slots = 0, my_active = 0, my_rays = 0, my_acc = 0, my_rej = 0,
                       my_64 = 0;

    for (;;) {
        int64_t id;
        q.refill(A, lane, live, id);
        if (id >= 0) {
            const int32_t sidx = find_scene(A, id);
            const DevScene &S = A.scenes[sidx];
            double alpha, beta, a, theta_obs;
            ray_inputs(A, S, id, alpha, beta, a, theta_obs);
            const double sgn = (S.s.convention == ODX_CONV_LITERAL) ? 1.0 : -1.0;
            const InitOut io = init_ray(a, S.s.r_obs, theta_obs, S.s.phi_obs, alpha, beta, sgn);
            R.id = id;
            R.scene = sidx;
            R.a = a;
            R.L = io.L;
            R.Q0 = io.Q;
            R.af = (float)a;
            R.Lf = (float)io.L;
            R.sgnf = (float)sgn;
#pragma unroll
            for (int i = 0; i < 6; ++i) df_set(R.yh[i], R.yl[i], io.y[i]);
#pragma unroll
            for (int k = 0; k < NF + 1; ++k) R.th[k] = R.tl[k] = R.Ih[k] = R.Il[k] = 0.f;
            R.r_start = io.y[0];
            R.r_stop = S.s.horizon_factor * horizon_radius(a);
            R.r_in = (S.s.r_in > 0.0) ? S.s.r_in : isco_radius(a);
            R.r_out = S.s.r_out;
            R.r_startf = (float)R.r_start;
            R.r_stopf = (float)R.r_stop;
            R.r_switch = (float)S.s.r_switch;
            R.hmaxf = (float)S.s.hmax_frac;
            R.rtolf = (float)S.s.rtol_fp32;
            R.r_cross = qnan();
            R.phi_cross = qnan();
            R.n_acc = R.n_rej = R.n_cross = R.n64 = 0;
            R.hd = fmin(S.s.h0, S.s.hmax_frac * io.y[0]);
            R.hsd = R.hd;
            R.hf = (float)R.hd;
            R.hsf = R.hf;
            R.mode = -1;
            if constexpr (NF > 0) load_medium_t<float>(S, a, mf);
            live = true;
        }
        const unsigned act = __ballot_sync(kFull, live);
        if (act == 0u) break;
        if (lane == 0) {
            my_slots += 32;
            my_active += __popc(act);
        }
        // per-lane precision of this step, from the lane's own radius
        const bool want64 = live && (R.yh[0] < R.r_switch);
        const unsigned b64 = __ballot_sync(kFull, want64);
        const unsigned b32 = act & ~b64;
        const bool run64 = b64 != 0u && (__popc(b64) >= A.fp64_batch || b32 == 0u);
        const bool mine = run64 ? want64 : (live && !want64);
        if (mine) {
            const DevScene &S = A.scenes[R.scene];
            int32_t status;
            if (run64) {
                // the FP64 step works on a copy: only this rare path pays for moving the ray
                // state through local memory, and the FP32 path keeps its registers
                RayM<NF> t = R;
                status = step64<NF>(A, S, t);
                R = t;
            } else {
                status = step32<NF>(A, S, R, mf);
            }
            if (status == ODX_RUNNING && R.n_acc + R.n_rej >= S.s.max_steps) status = ODX_MAXSTEPS;
            if (status != ODX_RUNNING) {
                if (status != ODX_DISK_HIT) {
                    double yend[6];
#pragma unroll
                    for (int i = 0; i < 6; ++i) yend[i] = df_get(R.yh[i], R.yl[i]);
                    write_result_m<NF>(A, S, R, status, yend, qnan(), qnan(), qnan(), 0.0);
                }
                my_rays += 1;
                my_acc += R.n_acc;
                my_rej += R.n_rej;
                my_64 += R.n64;
                live = false;
            }
        }
    }
    flush_stats(A, lane, my_rays, my_acc, my_rej, my_64, my_slots, my_active);
}

template <int NF>
cudaError_t launch_mixed_nf(const TraceArgs &args, const odx_launch &L, dim3 grid, cudaStream_t st)
{
    const dim3 block(L.block);
    switch (L.blocks_per_sm <= 2 ? 2 : (L.blocks_per_sm >= 4 ? 4 : 3)) {
    case 2: trace_mixed_kernel<NF, 2><<<grid, block, 0, st>>>(args); break;
    case 3: trace_mixed_kernel<NF, 3><<<grid, block, 0, st>>>(args); break;
    default: trace_mixed_kernel<NF, 4><<<grid, block, 0, st>>>(args); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_trace_mixed(const TraceArgs &args, int32_t nf_slots, const odx_launch &L,
                               int32_t num_sms, cudaStream_t st)
{
    if (L.block > 128) return cudaErrorInvalidValue;
    const dim3 grid = trace_grid(args, L, num_sms);
    switch (nf_slots) {
    case 0: return launch_mixed_nf<0>(args, L, grid, st);
    case 4: return launch_mixed_nf<4>(args, L, grid, st);
    case 8: return launch_mixed_nf<8>(args, L, grid, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace odx
