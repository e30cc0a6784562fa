// Pieces shared by the tracing kernels: the warp-level ray queue, scene lookup, ray inputs,
// vectorised record stores and statistics.
#pragma once

#include <cuda_runtime.h>

#include "kerr_device.cuh"
#include "odx_internal.h"

namespace odx {

__device__ __forceinline__ double qnan() { return __longlong_as_double(0x7ff8000000000000ULL); }

// Warp-uniform pool of ray indices [next, end) taken from the global queue.  In the
// non-persistent launch every thread owns the single ray with its global thread index.
struct WarpQueue {
    long long next, end;
    bool exhausted;

    __device__ __forceinline__ void init(const TraceArgs &)
    {
        next = end = 0;
        exhausted = false;
    }

    // Called by all 32 lanes together.  Lanes with live == false receive a ray index in id
    // (or keep -1 when the queue is drained).
    __device__ __forceinline__ void refill(const TraceArgs &A, int lane, bool live, int64_t &id)
    {
        id = -1;
        if (exhausted) return;
        // warp-coherent queue: a warp takes new rays only once all its lanes are done, so its
        // 32 lanes always trace neighbouring pixels that started together
        if (A.persistent == 3 && __ballot_sync(kFull, live) != 0u) return;
        // the launch traces global ids first .. first + count - 1; the queue counts from 0
        const long long first = launch_first(A), count = launch_count(A);
        if (!A.persistent) {
            const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
            if (!live && t < count) id = first + t;
            exhausted = true;
            return;
        }
        unsigned need = __ballot_sync(kFull, !live);
        // each pass either hands out rays or takes a new chunk; bounded by 32 lanes + 1
        for (int pass = 0; need != 0u && pass < 66; ++pass) {
            if (next >= end) {
                unsigned long long base = 0;
                if (lane == 0) base = atomicAdd(A.queue, (unsigned long long)A.chunk);
                base = __shfl_sync(kFull, base, 0);
                if ((long long)base >= count) {
                    exhausted = true;
                    break;
                }
                next = (long long)base;
                end = min((long long)base + A.chunk, count);
            }
            const int take = (int)min((long long)__popc(need), end - next);
            const unsigned below = (lane == 0) ? 0u : (0xffffffffu >> (32 - lane));
            const int rank = __popc(need & below);
            if (((need >> lane) & 1u) && rank < take) id = first + next + rank;
            next += take;
            need &= ~__ballot_sync(kFull, id >= 0);
        }
    }
};

__device__ __forceinline__ int32_t find_scene(const TraceArgs &A, int64_t id)
{
    if (A.list_mode || A.n_scenes == 1) return 0;
    int lo = 0, hi = A.n_scenes - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (A.scenes[mid].ray_begin <= id)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Observer and image-plane point of ray id.  Pixel centres:
// alpha_i = alpha_min + (i + 1/2)(alpha_max - alpha_min)/n_alpha.  Grid mode takes the
// scene's precomputed constants; list mode has its own (alpha, beta, a, cos i) per ray.
__device__ __forceinline__ ObsIn ray_observer(const TraceArgs &A, const DevScene &S, int64_t id)
{
    ObsIn o;
    o.r_obs = S.s.r_obs;
    o.spo = S.o_spo;
    o.cpo = S.o_cpo;
    if (A.list_mode) {
        const double *p = A.rays + 4 * id;
        o.alpha = p[0];
        o.beta = p[1];
        o.a = p[2];
        o.cto = p[3];
        o.sto = sqrt(fmax((1.0 - p[3]) * (1.0 + p[3]), 0.0));
        o.Ro = sqrt(o.r_obs * o.r_obs + o.a * o.a);
    } else {
        const int64_t local = id - S.ray_begin;
        const int64_t i = local % S.s.n_alpha, j = local / S.s.n_alpha;
        o.alpha = S.s.alpha_min + (((double)i + 0.5) * (S.s.alpha_max - S.s.alpha_min)) / S.s.n_alpha;
        o.beta = S.s.beta_min + (((double)j + 0.5) * (S.s.beta_max - S.s.beta_min)) / S.s.n_beta;
        o.a = S.s.a;
        o.sto = S.o_sto;
        o.cto = S.o_cto;
        o.Ro = S.o_Ro;
    }
    return o;
}

// Stop radius and ISCO of a ray's spin (the scene's precomputed values in grid mode).
__device__ __forceinline__ double ray_r_stop(const TraceArgs &A, const DevScene &S, double a)
{
    return A.list_mode ? S.s.horizon_factor * horizon_radius(a) : S.o_r_stop;
}
__device__ __forceinline__ double ray_r_isco(const TraceArgs &A, const DevScene &S, double a)
{
    return A.list_mode ? isco_radius(a) : S.o_r_isco;
}

// Image planes of a Novikov-Thorne disk hit at (r, g): B_nu(g T(r)) at each observed
// frequency (Liouville: I_nu / nu^3 invariant), zero for rays that miss the disk.  Returns
// the bolometric observed intensity g^4 (2 pi^4 / 15) T^4 for the record.
__device__ inline double nt_disk_planes(const DevScene &S, double *img, double a, double r_ms,
                                        double r, double g, bool hit)
{
    const double T = hit ? S.s.T0 * sqrt(sqrt(nt_flux_hat(a, r, r_ms))) : 0.0;
    if (img)
        for (int k = 0; k < S.s.n_freq; ++k) img[(int64_t)k * S.n_rays] = planck(S.s.freqs[k], g * T);
    const double gT = g * T;
    return hit ? 12.987878804533656 * gT * gT * gT * gT : 0.0;  // 2 pi^4 / 15
}

// ---- Keplerian hot spot (Section 4.4) -------------------------------------------------------
// max(d - 4 r_spot, -z) at state y (negative inside the spot) and d.  The photon at y reaches
// the image plane dt = sgn t later in coordinate time (t runs from 0 there with dt/ds =
// sgn dt/dlambda), so it left y at t_e = t_obs - sgn t, when the spot centre was at azimuth
// spot_phase + Omega t_e on the circle r = spot_r.  Distances in the pseudo-Cartesian
// coordinates x, y = sqrt(r^2 + a^2) (cos phi, sin phi), z = r cos theta.
__device__ inline double spot_region(const odx_scene &s, double sgn, const double y[6], double &d)
{
    const double rs = spot_orbit_radius(s);
    const double phs = s.spot_phase + spot_omega(s) * (s.t_obs - sgn * y[3]);
    const double Rs = sqrt(rs * rs + s.a * s.a), R = sqrt(y[0] * y[0] + s.a * s.a);
    double sp, cp, ss, cs, st, ct;
    sincos(y[2], &sp, &cp);
    sincos(phs, &ss, &cs);
    sincos(y[1], &st, &ct);
    const double dx = R * cp - Rs * cs, dy = R * sp - Rs * ss, z = y[0] * ct;
    d = sqrt(dx * dx + dy * dy + z * z);
    return fmax(d - 4.0 * s.spot_size, -z);
}

// Step cap near the spot: no step may carry a ray across it unseen, |h| <= (d - 4 r_spot) / 2,
// but not below r_spot / 4 (d from spot_region).
__device__ __forceinline__ double spot_cap(const odx_scene &s, double d)
{
    return fmax(0.5 * (d - 4.0 * s.spot_size), 0.25 * s.spot_size);
}
__device__ inline double spot_step_cap(const odx_scene &s, double sgn, const double y[6])
{
    double d;
    spot_region(s, sgn, y, d);
    return spot_cap(s, d);
}

// Redshift of gas co-rotating with the spot centre at Omega at (r, theta): g = 1 / (u^t
// (1 - Omega L)) (Eq. 2), u^t from u.u = -1; zero where that motion is not timelike.
__device__ inline double spot_redshift(const odx_scene &s, double r, double theta, double L)
{
    const double a = s.a;
    double st, ct;
    sincos(theta, &st, &ct);
    st = fmax(st, kSinFloor);
    const double Sig = r * r + a * a * ct * ct, Del = r * r - 2.0 * r + a * a;
    const double A = (r * r + a * a) * (r * r + a * a) - a * a * Del * st * st;
    const double Om = spot_omega(s);
    const double N = -(1.0 - 2.0 * r / Sig) - 2.0 * (2.0 * a * r * st * st / Sig) * Om +
                     A * st * st / Sig * Om * Om;
    return N < 0.0 ? sqrt(-N) / (1.0 - Om * L) : 0.0;
}

// Image planes of a spot hit: w B_nu(g T0) with w = C_norm exp(-d^2 / (2 r_spot^2)) at the
// entry point (I_nu / nu^3 invariant); zero for rays that miss.  Returns the bolometric
// intensity w (2 pi^4 / 15) (g T0)^4.
__device__ inline double spot_planes(const DevScene &S, double *img, double w, double g, bool hit)
{
    const double gT = hit ? g * S.s.T0 : 0.0;
    if (img)
        for (int k = 0; k < S.s.n_freq; ++k)
            img[(int64_t)k * S.n_rays] = hit ? w * planck(S.s.freqs[k], gT) : 0.0;
    return hit ? w * 12.987878804533656 * gT * gT * gT * gT : 0.0;  // 2 pi^4 / 15
}

struct RecordOut {
    int32_t status, n_acc, n_rej, n_cross;
    double r_cross, phi_cross, r_hit, phi_hit, g, intensity, H_end, Q_drift;
};

// One 80-byte record as five 16-byte stores (every sector written in full).
__device__ __forceinline__ void store_record(odx_ray_record *dst, const RecordOut &o)
{
    int4 *w = reinterpret_cast<int4 *>(dst);
    w[0] = make_int4(o.status, o.n_acc, o.n_rej, o.n_cross);
    double2 *d = reinterpret_cast<double2 *>(w + 1);
    d[0] = make_double2(o.r_cross, o.phi_cross);
    d[1] = make_double2(o.r_hit, o.phi_hit);
    d[2] = make_double2(o.g, o.intensity);
    d[3] = make_double2(o.H_end, o.Q_drift);
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ void flush_stats(const TraceArgs &A, int lane, unsigned long long rays,
                                            unsigned long long acc, unsigned long long rej,
                                            unsigned long long fp64, unsigned long long slots,
                                            unsigned long long active)
{
    rays = warp_sum(rays);
    acc = warp_sum(acc);
    rej = warp_sum(rej);
    fp64 = warp_sum(fp64);
    slots = warp_sum(slots);
    active = warp_sum(active);
    if (lane == 0) {
        atomicAdd(&A.stats->rays, rays);
        atomicAdd(&A.stats->acc, acc);
        atomicAdd(&A.stats->rej, rej);
        atomicAdd(&A.stats->fp64, fp64);
        atomicAdd(&A.stats->slots, slots);
        atomicAdd(&A.stats->active, active);
    }
}

inline dim3 trace_grid(const TraceArgs &A, const odx_launch &L, int32_t num_sms)
{
    if (L.persistent) return dim3((unsigned)(num_sms * L.blocks_per_sm));
    const long long nb = (launch_count(A) + L.block - 1) / L.block;
    return dim3((unsigned)(nb > 0 ? nb : 1));
}

}  // namespace odx
