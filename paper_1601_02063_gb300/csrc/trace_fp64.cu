// FP64 backward ray tracer for GB300 (sm_103a): persistent warps fed from a global ray queue
// (by default 32 consecutive rays once all lanes of the warp are done, so the warp's lanes
// trace neighbouring pixels together), one ray per lane, the Runge-Kutta state in registers.
//
// Per lane, one loop iteration is exactly one Cash-Karp attempt (Section 2.1: fifth-order
// Runge-Kutta with adaptive step size), so a rejected step costs its lane one iteration and
// never holds the other 31 lanes of the warp in a retry loop.  After an accepted step the
// lane runs the event checks (equatorial crossing, horizon, escape) and evaluates the
// right-hand side at the new point, which is both the escape test's dr/ds and the first
// stage of the next step.  Finished lanes are refilled between iterations: a ballot finds
// them, one lane takes `chunk` ray indices from the queue with a single atomicAdd, and the
// indices are handed out by rank within the ballot (with the warp-coherent queue only once
// the whole warp is done).
//
// Radiative transfer (Section 2.3, Eqs. 30-31) runs on the same stages as extra
// components: the optical depth tau_k needs its stage values (dI/ds depends on exp(-tau)),
// the invariant intensity only its weighted sums (the fifth-order increment and the error
// estimate), so only tau keeps per-stage slopes.  The intensities are under the step
// control (ODX_RT_CONTROLLED) and the medium ends at the stopping radius.
#include <cuda_runtime.h>
#include <math.h>

#include "kerr_device.cuh"
#include "odx_internal.h"
#include "trace_common.cuh"
#include "trace_step.cuh"

namespace odx {

template <int NF>
struct Ray64 {
    double y[6];      // r, theta, phi, t, p_r, p_theta
    double k1[6];     // dy/ds at y (first Cash-Karp stage)
    double tau[NF + 1];  // the intensities and the first stage's transfer slopes: shared memory
    double h, hs;     // next step; step used for the error scale of the current step
    double a, L, Q0, sgn;
    double r_start, r_stop, r_in, r_out;
    double r_cross, phi_cross;
    int64_t id;
    int32_t scene, n_acc, n_rej, n_cross;
};

// Equatorial crossing inside an accepted step: solve cos(theta(sigma)) = 0 for the
// fifth-order step of size sigma from the step start by Newton's method
// (d cos(theta)/ds = -sin(theta) dtheta/ds), kept in the sign bracket by bisection, to
// |cos(theta)| <= 1e-14 or 60 iterations.
__device__ __noinline__ void locate_crossing64(const Geo<double> &g, const double y[6],
                                               const double k1[6], double h, double yc[6])
{
    double lo = 0.0, hi = h;
    double flo = cos(y[1]);
    double y5[6], dy[6];
    ck_geo_increment<double>(g, y, k1, h, dy);
#pragma unroll
    for (int i = 0; i < 6; ++i) y5[i] = y[i] + dy[i];
    const double fhi = cos(y5[1]);
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
    for (int i = 0; i < 6; ++i) yc[i] = y5[i];
}

// For the hot spot, inten carries the Gaussian weight w of the entry point.
template <int NF>
__device__ __forceinline__ void write_result64(const TraceArgs &A, const DevScene &S,
                                               const Ray64<NF> &R, const double *I, int32_t status,
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
    const EndChecks ec = end_checks(R.a, R.L, yend);
    o.H_end = ec.H;
    o.Q_drift = (ec.Q - R.Q0) / fmax(fabs(R.Q0), 1.0);
    double *img = A.image ? A.image + S.img_offset + (R.id - S.ray_begin) : nullptr;
    if (S.s.emitter == ODX_EMIT_NT_DISK)
        o.intensity = nt_disk_planes(S, img, R.a, ray_r_isco(A, S, R.a), r_hit, g,
                                     status == ODX_DISK_HIT);
    if (S.s.emitter == ODX_EMIT_SPOT)
        o.intensity = spot_planes(S, img, inten, g, status == ODX_DISK_HIT);
    store_record(A.records + R.id, o);
    if (img && S.s.emitter != ODX_EMIT_NT_DISK && S.s.emitter != ODX_EMIT_SPOT) {
        if constexpr (NF > 0) {
            // synchrotron shell: the stages carry I_nu / (nu^3 Aj), nu in Hz
            const double Ij = S.s.emitter == ODX_EMIT_SYNCH ? synch_constants(S.s).Aj : 1.0;
#pragma unroll
            for (int k = 0; k < NF; ++k) {
                if (k < S.s.n_freq) {
                    const double nu = S.s.freqs[k];
                    img[(int64_t)k * S.n_rays] = nu * nu * nu * Ij * I[k * blockDim.x];
                }
            }
        } else {
            img[0] = inten;
        }
    }
}

// One Cash-Karp attempt as a loop over stages 2-6 around one inlined right-hand side (one
// copy of the FP64 stage code in the instruction cache).  Each stage's slopes are folded at
// once into the inputs of the later stages (acc[J]: stage J + 2, in shared memory, layout
// [J][component][thread], components r, theta, p_r, p_theta, tau_k: t and phi are read by no
// right-hand side), into the fifth-order sums and into the error estimates, so no stage
// slope is kept.  Same outputs as ck_attempt.
template <int NF>
__device__ __forceinline__ void ck_attempt_fold(const Geo<double> &g, const MediumT<double> &m,
                                                const double y[6], const double k1[6],
                                                const double *tau, const double *kt1,
                                                const double *kI1, int kstride, double h,
                                                double dy[6], double e[6], double *dtau,
                                                double *dI, double *eI, double *acc)
{
    constexpr int NG = 4 + NF;
    const int nt = blockDim.x, t = threadIdx.x;
    auto A_ = [&](int J, int c) -> double & { return acc[(J * NG + c) * nt + t]; };
    auto kc = [&](const double f[6], const double *ft, int c) {
        return c < 2 ? f[c] : (c < 4 ? f[c + 2] : ft[c - 4]);
    };
    // stage 1 (its transfer slopes kt1, kI1 with stride kstride)
#pragma unroll
    for (int c = 0; c < NG; ++c) {
        const double k = c < 4 ? kc(k1, nullptr, c) : kt1[(c - 4) * kstride];
        A_(0, c) = CK_A21 * k;
        A_(1, c) = CK_A31 * k;
        A_(2, c) = CK_A41 * k;
        A_(3, c) = CK_A51 * k;
        A_(4, c) = CK_A61 * k;
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        dy[i] = CK_B1 * k1[i];
        e[i] = CK_E1 * k1[i];
    }
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        dtau[k] = CK_B1 * kt1[k * kstride];
        dI[k] = CK_B1 * kI1[k * kstride];
        eI[k] = CK_E1 * kI1[k * kstride];
    }
#pragma unroll 1
    for (int st = 1; st < 6; ++st) {  // stages 2..6
        double yt[6], tt[NF + 1], f[6], ft[NF + 1], fI[NF + 1];
        yt[0] = y[0] + h * A_(st - 1, 0);
        yt[1] = y[1] + h * A_(st - 1, 1);
        yt[2] = y[2];
        yt[3] = y[3];
        yt[4] = y[4] + h * A_(st - 1, 2);
        yt[5] = y[5] + h * A_(st - 1, 3);
#pragma unroll
        for (int k = 0; k < NF; ++k) tt[k] = tau[k] + h * A_(st - 1, 4 + k);
        derivs<double, NF>(g, m, yt, tt, f, ft, fI);
        double b, ee;  // fifth-order weight and error weight of this stage
        switch (st) {
        case 1:  // b2 = e2 = 0
#pragma unroll
            for (int c = 0; c < NG; ++c) {
                const double k = kc(f, ft, c);
                A_(1, c) += CK_A32 * k;
                A_(2, c) += CK_A42 * k;
                A_(3, c) += CK_A52 * k;
                A_(4, c) += CK_A62 * k;
            }
            b = 0.0;
            ee = 0.0;
            break;
        case 2:
#pragma unroll
            for (int c = 0; c < NG; ++c) {
                const double k = kc(f, ft, c);
                A_(2, c) += CK_A43 * k;
                A_(3, c) += CK_A53 * k;
                A_(4, c) += CK_A63 * k;
            }
            b = CK_B3;
            ee = CK_E3;
            break;
        case 3:
#pragma unroll
            for (int c = 0; c < NG; ++c) {
                const double k = kc(f, ft, c);
                A_(3, c) += CK_A54 * k;
                A_(4, c) += CK_A64 * k;
            }
            b = CK_B4;
            ee = CK_E4;
            break;
        case 4:  // b5 = 0
#pragma unroll
            for (int c = 0; c < NG; ++c) A_(4, c) += CK_A65 * kc(f, ft, c);
            b = 0.0;
            ee = CK_E5;
            break;
        default:
            b = CK_B6;
            ee = CK_E6;
            break;
        }
        if (st != 1) {
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                dy[i] += b * f[i];
                e[i] += ee * f[i];
            }
#pragma unroll
            for (int k = 0; k < NF; ++k) {
                dtau[k] += b * ft[k];
                dI[k] += b * fI[k];
                eI[k] += ee * fI[k];
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        dy[i] *= h;
        e[i] *= h;
    }
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        dtau[k] *= h;
        dI[k] *= h;
        eI[k] *= h;
    }
}

// Shared memory of the FP64 tracer, per thread: the stage-input sums of ck_attempt_fold and
// the ray's medium constants (read by the right-hand side, kept out of the registers).
constexpr int kFp64MaxBlock = 256;  // the kernel's launch bound
inline size_t fp64_smem_bytes(int nf_slots, int block)
{
    // without transfer slots the medium is not read: the stage sums alone
    return ((size_t)(5 * (4 + nf_slots) + 3 * nf_slots) * sizeof(double) +
            (nf_slots > 0 ? sizeof(MediumT<double>) : 0)) * block;
}

template <int NF>
__global__ void __launch_bounds__(256) trace_fp64_kernel(TraceArgs A)
{
    extern __shared__ double acc_smem[];
    const int lane = threadIdx.x & 31;
    Ray64<NF> R;
    MediumT<double> *meds = reinterpret_cast<MediumT<double> *>(acc_smem + 5 * (4 + NF) * blockDim.x);
    MediumT<double> &m = meds[threadIdx.x];
    // per slot k: kt1 at [k], kI1 at [NF + k], the intensity I at [2 NF + k] (stride blockDim.x)
    double *const rt = reinterpret_cast<double *>(meds + blockDim.x) + threadIdx.x;
    double *const Kt = rt, *const KI = rt + NF * blockDim.x, *const Is = rt + 2 * NF * blockDim.x;
    const int ks = blockDim.x;
    bool live = false;
    WarpQueue q;
    q.init(A);

    unsigned long long my_slots = 0, my_active = 0;
    unsigned long long my_rays = 0, my_acc = 0, my_rej = 0;

    for (;;) {
        // ---- refill finished lanes from the queue (all 32 lanes together) ------------------
        int64_t id;
        q.refill(A, lane, live, id);
        if (id >= 0) {
            const int32_t sidx = find_scene(A, id);
            const DevScene &S = A.scenes[sidx];
            const ObsIn ob = ray_observer(A, S, id);
            const double a = ob.a;
            R.id = id;
            R.scene = sidx;
            R.a = a;
            R.sgn = (S.s.convention == ODX_CONV_LITERAL) ? 1.0 : -1.0;
            const InitOut io = init_ray(ob, R.sgn);
#pragma unroll
            for (int i = 0; i < 6; ++i) R.y[i] = io.y[i];
            R.L = io.L;
            R.Q0 = io.Q;
            R.r_start = io.y[0];
            const double r_isco = ray_r_isco(A, S, a);
            R.r_stop = ray_r_stop(A, S, a);
            R.r_in = (S.s.r_in > 0.0) ? S.s.r_in : r_isco;
            R.r_out = S.s.r_out;
            R.r_cross = qnan();
            R.phi_cross = qnan();
            R.n_acc = R.n_rej = R.n_cross = 0;
#pragma unroll
            for (int k = 0; k < NF + 1; ++k) R.tau[k] = 0.0;
#pragma unroll
            for (int k = 0; k < NF; ++k) Is[k * ks] = 0.0;
            if constexpr (NF > 0) load_medium_t<double>(S, r_isco, R.r_stop, m);
            const Geo<double> g{R.a, R.L, R.sgn};
            {
                double kt1[NF + 1], kI1[NF + 1];
                derivs<double, NF>(g, m, R.y, R.tau, R.k1, kt1, kI1);
#pragma unroll
                for (int k = 0; k < NF; ++k) {
                    Kt[k * ks] = kt1[k];
                    KI[k * ks] = kI1[k];
                }
            }
            R.h = fmin(S.s.h0, S.s.hmax_frac * R.y[0]);
            if (S.s.emitter == ODX_EMIT_SPOT) R.h = fmin(R.h, spot_step_cap(S.s, R.sgn, R.y));
            R.hs = R.h;
            live = true;
        }
        const unsigned act = __ballot_sync(kFull, live);
        if (act == 0u) break;
        if (lane == 0) {
            my_slots += 32;
            my_active += __popc(act);
        }

        if (live) {
            // ---- one Cash-Karp attempt ----------------------------------------------------------
            const DevScene &S = A.scenes[R.scene];
            const Geo<double> g{R.a, R.L, R.sgn};
            double y5[6], dy[6], e[6], dtau[NF + 1], dI[NF + 1], eI[NF + 1];
            const double h = R.h;
            ck_attempt_fold<NF>(g, m, R.y, R.k1, R.tau, Kt, KI, ks, h, dy, e, dtau, dI, eI,
                                acc_smem);
#pragma unroll
            for (int i = 0; i < 6; ++i) y5[i] = R.y[i] + dy[i];
            double errmax = 0.0;
            bool nan_err = false;  // fmax drops a NaN operand: track it, it rejects the step
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                const double sc = fabs(R.y[i]) + fabs(R.hs * R.k1[i]) + 1e-30;
                const double v = fabs(e[i] / sc);
                nan_err |= isnan(v);
                errmax = fmax(errmax, v);
            }
            // the intensities under the step control (ODX_RT_RIDE: infinite floors)
#pragma unroll
            for (int k = 0; k < NF; ++k) {
                const double sc = fabs(Is[k * ks]) + fabs(R.hs * KI[k * ks]) + m.I_floor[k];
                const double v = fabs(eI[k] / sc);
                nan_err |= isnan(v);
                errmax = fmax(errmax, v);
            }
            errmax /= S.s.rtol;
            if (nan_err || isnan(errmax)) errmax = INFINITY;

            int32_t status = ODX_RUNNING;
            if (errmax <= 1.0) {
                ++R.n_acc;
                const double h_next = (errmax > 1.89e-4) ? 0.9 * h * pow(errmax, -0.2) : 5.0 * h;
                if ((cos(R.y[1]) > 0.0) != (cos(y5[1]) > 0.0)) {  // equatorial crossing
                    double yc[6];
                    locate_crossing64(g, R.y, R.k1, h, yc);
                    ++R.n_cross;
                    if (R.n_cross == 1) {
                        R.r_cross = yc[0];
                        R.phi_cross = yc[2];
                    }
                    if (disk_emitter(S.s.emitter) && yc[0] >= R.r_in && yc[0] <= R.r_out) {
                        const double gz = disk_redshift(R.a, yc[0], R.L);
                        const double g2 = gz * gz;
                        const double inten = g2 * g2 * pow(yc[0], -S.s.q_emis);
                        write_result64<NF>(A, S, R, Is, ODX_DISK_HIT, yc, yc[0], yc[2], gz, inten);
                        status = ODX_DISK_HIT;
                    }
                }
                // hot spot: d_spot is the distance from the spot's centre at y5, the step's
                // end.  It stays infinite where the lower bound d >= |rho - R_s| keeps y5
                // outside the spot and the step cap from binding: there the exact distance
                // changes nothing and its three FP64 sincos are skipped.  In the spot's
                // pseudo-Cartesian coordinates x, y = sqrt(r^2 + a^2) (cos, sin) phi (no
                // sin theta), z = r cos theta, a point lies at rho = sqrt(r^2 + a^2) from the
                // z axis and the centre (z = 0) at R_s, so d^2 = (horizontal separation)^2
                // + z^2 >= (rho - R_s)^2 by the triangle inequality in the x-y plane.
                double d_spot = INFINITY;
                bool near_spot = false;
                if (status == ODX_RUNNING && S.s.emitter == ODX_EMIT_SPOT) {
                    const double Rs = (double)S.f_spot_Rs;  // FP32-rounded: 1e-6 margin
                    const double d_low =
                        fabs(sqrt(y5[0] * y5[0] + S.s.a * S.s.a) - Rs) - 1e-6 * Rs;
                    near_spot = 0.5 * (d_low - 4.0 * S.s.spot_size) <
                                fmin(h_next, S.s.hmax_frac * y5[0]);
                }
                if (near_spot && spot_region(S.s, R.sgn, y5, d_spot) < 0.0) {  // first entry
                    double yc[6];
                    locate_spot64(g, S.s, R.y, R.k1, h, yc, 60);
                    spot_region(S.s, R.sgn, yc, d_spot);
                    const double w = S.s.C_norm * exp(-d_spot * d_spot /
                                                      (2.0 * S.s.spot_size * S.s.spot_size));
                    write_result64<NF>(A, S, R, Is, ODX_DISK_HIT, yc, yc[0], yc[2],
                                       spot_redshift(S.s, yc[0], yc[1], R.L), w);
                    status = ODX_DISK_HIT;
                }
                if (status == ODX_RUNNING) {
#pragma unroll
                    for (int i = 0; i < 6; ++i) R.y[i] = y5[i];
#pragma unroll
                    for (int k = 0; k < NF; ++k) {
                        R.tau[k] += dtau[k];
                        Is[k * ks] += dI[k];
                    }
                    if (R.y[0] < R.r_stop) {
                        status = ODX_CAPTURED;
                    } else {
                        double kt1[NF + 1], kI1[NF + 1];
                        derivs<double, NF>(g, m, R.y, R.tau, R.k1, kt1, kI1);
#pragma unroll
                        for (int k = 0; k < NF; ++k) {
                            Kt[k * ks] = kt1[k];
                            KI[k * ks] = kI1[k];
                        }
                        if (R.k1[0] > 0.0 && R.y[0] > R.r_start) status = ODX_ESCAPED;
                    }
                    R.h = fmin(h_next, S.s.hmax_frac * R.y[0]);
                    if (S.s.emitter == ODX_EMIT_SPOT)
                        R.h = fmin(R.h, spot_cap(S.s, d_spot));  // R.y is y5
                    R.hs = R.h;
                }
            } else {
                ++R.n_rej;
                R.h = fmax(0.9 * h * pow(errmax, -0.25), 0.1 * h);
                if (R.h < 1e-12) status = ODX_NUMERR;
            }
            if (status == ODX_RUNNING && R.n_acc + R.n_rej >= S.s.max_steps)
                status = ODX_MAXSTEPS;
            if (status != ODX_RUNNING) {
                if (status != ODX_DISK_HIT)
                    write_result64<NF>(A, S, R, Is, status, R.y, qnan(), qnan(), qnan(), 0.0);
                my_rays += 1;
                my_acc += R.n_acc;
                my_rej += R.n_rej;
                live = false;
            }
        }
    }
    flush_stats(A, lane, my_rays, my_acc, my_rej, 0ull, my_slots, my_active);
}

cudaError_t launch_trace_fp64(const TraceArgs &args_in, int32_t nf_slots, const odx_launch &L_in,
                              int32_t num_sms, cudaStream_t st, cudaEvent_t ev0, cudaEvent_t ev1)
{
    TraceArgs args = args_in;
    if (args.chunk <= 0) args.chunk = 32;  // the FP64 tracer's default queue chunk
    // launch shape "auto": the warp-coherent queue (512^2 torus: 426 ms with lanes refilled
    // one by one, 348 ms one ray per thread, 306 ms coherent queue)
    odx_launch L = L_in;
    if (L.persistent == 2) L.persistent = 3;
    args.persistent = L.persistent;
    const dim3 block(L.block);
    const dim3 grid = trace_grid(args, L, num_sms);
    if (ev0) cudaEventRecord(ev0, st);
    if (L.block > kFp64MaxBlock) return cudaErrorInvalidValue;
    const size_t smem = fp64_smem_bytes(nf_slots, L.block);
    switch (nf_slots) {
    case 0: trace_fp64_kernel<0><<<grid, block, smem, st>>>(args); break;
    case 3: trace_fp64_kernel<3><<<grid, block, smem, st>>>(args); break;
    case 4: trace_fp64_kernel<4><<<grid, block, smem, st>>>(args); break;
    case 8: trace_fp64_kernel<8><<<grid, block, smem, st>>>(args); break;
    default: return cudaErrorInvalidValue;
    }
    if (ev1) cudaEventRecord(ev1, st);
    return cudaGetLastError();
}

// The FP64 tracers take up to 180 KB of dynamic shared memory (more than the default 48 KB)
// at the largest block: opt in once per device, before any launch or capture.
cudaError_t prepare_fp64_kernels()
{
    const void *fns[4] = {(const void *)trace_fp64_kernel<0>, (const void *)trace_fp64_kernel<3>,
                          (const void *)trace_fp64_kernel<4>, (const void *)trace_fp64_kernel<8>};
    const int nf[4] = {0, 3, 4, 8};
    for (int i = 0; i < 4; ++i) {
        const cudaError_t e = cudaFuncSetAttribute(fns[i], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)fp64_smem_bytes(nf[i], kFp64MaxBlock));
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace odx
