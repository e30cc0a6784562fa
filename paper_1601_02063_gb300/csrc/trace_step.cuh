// One Cash-Karp step of the geodesic plus radiative transfer, templated on the arithmetic
// type (double for the FP64 tracer and the FP64 region of the mixed tracer, float for the
// FP32 bulk of the mixed tracer).  Section 2.1 (Eqs. 4, 5, 9, 12, 14, 15 with the
// fifth-order adaptive Runge-Kutta scheme) and Section 2.3 (Eqs. 30-31).
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "kerr_device.cuh"
#include "trace_common.cuh"

namespace odx {

__device__ __forceinline__ float m_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double m_sqrt(double x) { return sqrt(x); }
// FP32 emissivity uses the hardware exponential and logarithm (relative error ~1e-6,
// far below the 1e-3 image tolerance of the reduced-precision path)
__device__ __forceinline__ float m_exp(float x) { return __expf(x); }
__device__ __forceinline__ double m_exp(double x) { return exp(x); }
__device__ __forceinline__ float m_log(float x) { return __logf(x); }
__device__ __forceinline__ double m_log(double x) { return log(x); }
__device__ __forceinline__ float m_expm1(float x) { return expm1f(x); }
__device__ __forceinline__ double m_expm1(double x) { return expm1(x); }
__device__ __forceinline__ float m_cos(float x) { return cosf(x); }
__device__ __forceinline__ double m_cos(double x) { return cos(x); }
__device__ __forceinline__ float m_pow(float x, float y) { return powf(x, y); }
__device__ __forceinline__ double m_pow(double x, double y) { return pow(x, y); }
// FP32 stages: the hardware sine/cosine (absolute error <= 2^-21.4 for |x| <= pi, theta stays
// in [0, pi] up to pole passages) is well inside the stages' 1e-6 tolerance; measured
// image error vs FP64 changes by 1 % of itself.  Crossing tests keep the accurate cosf.
__device__ __forceinline__ void m_sincos(float x, float *s, float *c) { __sincosf(x, s, c); }
__device__ __forceinline__ void m_sincos(double x, double *s, double *c) { sincos(x, s, c); }
// correctly rounded reciprocal (FP32: no division slow path) and reciprocal square root
__device__ __forceinline__ float m_rcp(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double m_rcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float m_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double m_rsqrt(double x) { return 1.0 / sqrt(x); }
// 1 - exp(-x) for x >= 0 given em = exp(-x): series below 1/32 (the FP32 cancellation
// there would cost up to 5 bits), expm1 in FP64
__device__ __forceinline__ float one_minus_exp(float x, float em)
{
    return x > 0.03125f ? 1.f - em : x * (1.f - x * (0.5f - x * (1.f / 6.f)));
}
__device__ __forceinline__ double one_minus_exp(double x, double em)
{
    return x > 0.5 ? 1.0 - em : -expm1(-x);
}

// Parameters of the emitting medium in the arithmetic type of the step: the analytic torus
// or the synchrotron shell (synch = 1: n_e / n_e0 and Theta_e take the torus's n_e and
// T_e forms; frequencies in GHz).
template <typename T>
struct MediumT {
    T ne_index, inv_2w2, T0, inv_T0, T_index, C_norm, r_isco;
    T freqs[ODX_MAX_FREQ];
    T I_floor[ODX_MAX_FREQ];  // error-scale floors of the intensities (rt_floor)
    T r_stop;                 // the medium ends inside the stopping radius
    int n_freq;
    int synch;
    T inv_kc, ky, Atau, r_out;
};

template <typename T>
__device__ __forceinline__ void load_medium_t(const DevScene &S, double r_isco, double r_stop,
                                              MediumT<T> &m)
{
    m.r_stop = (T)r_stop;
#pragma unroll
    for (int k = 0; k < ODX_MAX_FREQ; ++k) m.I_floor[k] = (T)S.rt_floor[k];
    m.ne_index = (T)S.s.ne_index;
    m.inv_2w2 = (T)(1.0 / (2.0 * S.s.theta_width * S.s.theta_width));
    m.T0 = (T)S.s.T0;
    m.inv_T0 = (T)(1.0 / S.s.T0);
    m.T_index = (T)S.s.T_index;
    m.C_norm = (T)S.s.C_norm;
    m.r_isco = (T)r_isco;
    m.n_freq = S.s.n_freq;
    m.synch = S.s.emitter == ODX_EMIT_SYNCH;
    const double nu_scale = m.synch ? 1.0 / kNuUnit : 1.0;
#pragma unroll
    for (int k = 0; k < ODX_MAX_FREQ; ++k) m.freqs[k] = (T)(S.s.freqs[k] * nu_scale);
    if (m.synch) {
        const SynchK q = synch_constants(S.s);
        m.inv_kc = (T)q.inv_kc;
        m.ky = (T)q.ky;
        m.Atau = (T)q.Atau;
        m.r_out = (T)S.s.r_out;
    } else {
        m.inv_kc = m.ky = m.Atau = m.r_out = T(0);
    }
}

// e^x K_2(x) = int_0^inf exp(-x (cosh t - 1)) cosh 2t dt (the integral representation of
// K_2, x > 0) by the trapezoidal rule with step hq on [0, inf).  The integrand is even and
// analytic in a strip about the real axis, so the error falls like exp(-2 pi d / hq), and
// for large x it is close to a Gaussian of width x^-1/2 whose trapezoid error is
// exp(-2 pi^2 / (x hq^2)): hq = min(1/4, x^-1/2 / 2) keeps the relative error below 3e-14
// in FP64 and hq = min(2/5, x^-1/2) below 3e-7 in FP32 for 1e-3 <= x <= 300 (checked
// against a library K_2).  The sum stops once x (cosh t - 1) - 2 t exceeds 40 (FP64) or
// 22 (FP32); the terms beyond fall faster than geometrically from below that size.
template <typename T>
__device__ __forceinline__ T k2_scaled(T x)
{
    constexpr bool f64 = sizeof(T) == 8;
    const T hq = fmin(f64 ? T(0.25) : T(0.4), (f64 ? T(0.5) : T(1)) * m_rsqrt(x));
    const T eh = m_exp(hq);
    const T cut = f64 ? T(40) : T(22);
    constexpr int kmax = f64 ? 64 : 40;
    T sum = T(0.5);  // t = 0 with the end weight 1/2
    T e = eh;        // exp(k hq)
    for (int k = 1; k < kmax; ++k) {
        const T ch = T(0.5) * (e + m_rcp(e));  // cosh(k hq)
        const T arg = x * (ch - T(1));
        if (arg - T(2) * hq * (T)k > cut) break;
        sum += m_exp(-arg) * (T(2) * ch * ch - T(1));  // cosh(2 k hq) = 2 cosh^2 - 1
        e *= eh;
    }
    return hq * sum;
}

// Transfer right-hand sides of the synchrotron shell at one stage (Eqs. 30-31 with Eqs.
// 37-39): nr = n_e / n_e0, iTh = 1 / Theta_e, ig = 1 / g, r <= r_out.  Per frequency, with
// x = nu0 / nu_c: M(x) = 4.0505 x^-1/6 (1 + 0.40 x^-1/4 + 0.5316 x^-1/2) exp(-1.8899 x^1/3),
// the exp(1 / Theta_e) of 1 / K_2 folded into the same exponential (no overflow for cold
// electrons); powers of x from w = x^-1/12.
template <typename T, int NF>
__device__ __forceinline__ void synch_rhs(const MediumT<T> &m, T r, T nr, T iTh, T ig,
                                          const T *tau, T *ftau, T *fI)
{
    const T P = nr * ig * m_rcp(k2_scaled<T>(iTh));
    const T inu_c = m.inv_kc * iTh * iTh * m_sqrt(r * m_rcp(nr));  // 1 / nu_c-hat
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        if (k < m.n_freq) {
            const T nu0 = m.freqs[k] * ig;
            const T x = nu0 * inu_c;
            const T w = m_exp(m_log(x) * T(-1.0 / 12.0));
            const T w2 = w * w, w3 = w2 * w, w6 = w3 * w3;
            const T Mp = T(4.0505) * w2 * (T(1) + T(0.40) * w3 + T(0.5316) * w6);
            const T jt = P * Mp * m_exp(iTh - T(1.8899) * m_rcp(w2 * w2)) * m_rcp(nu0 * nu0);
            ftau[k] = m.Atau * jt * m_expm1(m.ky * nu0 * iTh);  // Eq. 30, Kirchhoff
            fI[k] = jt * m_exp(-tau[k]);                        // Eq. 31
        } else {
            ftau[k] = T(0);
            fI[k] = T(0);
        }
    }
}

// Geodesic and transfer right-hand sides of one stage together, sharing sin(theta),
// cos(theta), Sigma, Delta and 1/Sigma between Eqs. 4-15 and the torus model (Eq. 2,
// Eqs. 30-31): the geodesic part is the same as geodesic_rhs.
template <typename T, int NF>
__device__ __forceinline__ void derivs(const Geo<T> &g, const MediumT<T> &m, const T y[6],
                                       const T *tau, T f[6], T *ftau, T *fI)
{
    if constexpr (NF == 0) {
        geodesic_rhs<T>(g, y[0], y[1], y[4], y[5], f);
    } else {
        const T r = y[0], pr = y[4], pth = y[5];
        T s, c;
        m_sincos(y[1], &s, &c);
        s = fmax(s, T(kSinFloor));
        const T a = g.a, L = g.L;
        const T r2 = r * r, a2 = a * a, s2 = s * s;
        const T Sig = r2 + a2 * c * c;
        const T Del = r2 - T(2) * r + a2;
        const T iSD = m_rcp(Sig * Del);
        const T iS = Del * iSD;
        const T iD = Sig * iSD;
        const T is = m_rcp(s);
        const T is2 = is * is;
        const T rr = r2 + a2;
        const T P = rr - a * L;
        const T q = L * is - a * s;
        const T pr2 = pr * pr, pth2 = pth * pth;
        const T F = Del * pr2 + pth2 + q * q - P * P * iD;
        const T kap = pth2 + L * L * is2 + a2 * s2;
        const T rm1 = r - T(1);
        const T twor = T(2) * r;
        f[0] = g.sgn * (Del * pr * iS);
        f[1] = g.sgn * (pth * iS);
        f[2] = g.sgn * ((twor * a + (Sig - twor) * L * is2) * iSD);
        f[3] = g.sgn * (T(1) + (twor * rr - twor * a * L) * iSD);
        f[4] = g.sgn * ((-kap * rm1 + twor * rr - T(2) * a * L) * iSD - T(2) * pr2 * rm1 * iS +
                        F * (rm1 * iSD + r * iS * iS));
        f[5] = g.sgn * (s * c * iS * (L * L * is2 * is2 - a2) - a2 * s * c * F * iS * iS);

        // the medium ends at the stopping radius (rays stop inside it)
        if (r < m.r_stop) {
#pragma unroll
            for (int k = 0; k < NF; ++k) ftau[k] = fI[k] = T(0);
            return;
        }
        // torus: Keplerian flow where r >= r_ISCO and timelike, else ZAMO; g from Eq. 2
        const T A = rr * rr - a2 * Del * s2;
        const T gtt = -(T(1) - twor * iS);
        const T gtp = -twor * a * s2 * iS;
        const T gpp = A * s2 * iS;
        T Om = m_rcp(r * m_sqrt(r) + a);
        T N = gtt + T(2) * gtp * Om + gpp * Om * Om;
        if (!(r >= m.r_isco && N < T(0))) {
            Om = twor * a * m_rcp(A);
            N = gtt + T(2) * gtp * Om + gpp * Om * Om;
        }
        const T ig = (T(1) - Om * L) * m_rsqrt(-N);  // 1/g = u^t (1 - Omega L)
        const T lr = m_log(r);
        const T ne = m_exp(-m.ne_index * lr - c * c * m.inv_2w2);
        const T iTe = m_exp(m.T_index * lr) * m.inv_T0;
        if (m.synch) {
            if (r <= m.r_out) {
                synch_rhs<T, NF>(m, r, ne, iTe, ig, tau, ftau, fI);
            } else {
#pragma unroll
                for (int k = 0; k < NF; ++k) ftau[k] = fI[k] = T(0);
            }
            return;
        }
        const T pref = m.C_norm * ne * ne * m_sqrt(iTe);  // C n_e^2 T^-1/2
#pragma unroll
        for (int k = 0; k < NF; ++k) {
            if (k < m.n_freq) {
                const T nu0 = m.freqs[k] * ig;
                const T x = nu0 * iTe;
                const T em = m_exp(-x);
                const T inu3 = m_rcp(nu0 * nu0 * nu0);
                ftau[k] = T(0.5) * pref * one_minus_exp(x, em) * inu3 * ig;  // Eq. 30
                fI[k] = pref * em * inu3 * ig * m_exp(-tau[k]);              // Eq. 31
            } else {
                ftau[k] = T(0);
                fI[k] = T(0);
            }
        }
    }
}

// Right-hand side evaluated out of line and returned by value: one copy of its code serves
// all six stages of a step, which keeps the FP32 stage loop inside the instruction cache.
template <typename T, int NF>
struct DerivOut {
    T f[6], ft[NF + 1], fI[NF + 1];
};
template <typename T, int NF>
struct TauIn {
    T t[NF + 1];
};

template <typename T, int NF>
__device__ __noinline__ DerivOut<T, NF> derivs_call(Geo<T> g, MediumT<T> m, T r, T th, T pr, T pth,
                                                    TauIn<T, NF> tau)
{
    DerivOut<T, NF> o;
    const T y[6] = {r, th, T(0), T(0), pr, pth};
    derivs<T, NF>(g, m, y, tau.t, o.f, o.ft, o.fI);
    return o;
}

// Stage evaluation: inline for FP64 (its pipe, not instruction fetch, bounds it), out of line
// for FP32.
template <typename T, int NF>
__device__ __forceinline__ void derivs_stage(const Geo<T> &g, const MediumT<T> &m, const T y[6],
                                             const T *tau, T f[6], T *ft, T *fI)
{
    if constexpr (sizeof(T) == 4) {
        TauIn<T, NF> ti;
#pragma unroll
        for (int k = 0; k < NF + 1; ++k) ti.t[k] = (k < NF) ? tau[k] : T(0);
        const DerivOut<T, NF> o = derivs_call<T, NF>(g, m, y[0], y[1], y[4], y[5], ti);
#pragma unroll
        for (int i = 0; i < 6; ++i) f[i] = o.f[i];
#pragma unroll
        for (int k = 0; k < NF; ++k) {
            ft[k] = o.ft[k];
            fI[k] = o.fI[k];
        }
    } else {
        derivs<T, NF>(g, m, y, tau, f, ft, fI);
    }
}

// One Cash-Karp attempt of size h from (y, tau) with first stage (k1, kt1, kI1).
// Returns the fifth-order increments dy (y5 = y + dy), the embedded error estimates e of the
// geodesic components and eI of the intensities, and the fifth-order increments dtau, dI of
// the transfer components.  tau needs its stage values (dI/ds depends on exp(-tau)); I only
// its weighted sums.
template <typename T, int NF>
__device__ __forceinline__ void ck_attempt(const Geo<T> &g, const MediumT<T> &m, const T y[6],
                                           const T k1[6], const T *tau, const T *kt1,
                                           const T *kI1, T h, T dy[6], T e[6], T *dtau, T *dI,
                                           T *eI)
{
    constexpr int N = NF + 1;
    T k2[6], k3[6], k4[6], k5[6], k6[6], yt[6];
    T t2[N], t3[N], t4[N], t5[N], t6[N], tt[N], fI[N], sI[N], sE[N];
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        sI[k] = T(CK_B1) * kI1[k];
        sE[k] = T(CK_E1) * kI1[k];
    }

#pragma unroll
    for (int i = 0; i < 6; ++i) yt[i] = y[i] + h * (T(CK_A21) * k1[i]);
#pragma unroll
    for (int k = 0; k < NF; ++k) tt[k] = tau[k] + h * (T(CK_A21) * kt1[k]);
    derivs_stage<T, NF>(g, m, yt, tt, k2, t2, fI);

#pragma unroll
    for (int i = 0; i < 6; ++i) yt[i] = y[i] + h * (T(CK_A31) * k1[i] + T(CK_A32) * k2[i]);
#pragma unroll
    for (int k = 0; k < NF; ++k) tt[k] = tau[k] + h * (T(CK_A31) * kt1[k] + T(CK_A32) * t2[k]);
    derivs_stage<T, NF>(g, m, yt, tt, k3, t3, fI);
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        sI[k] += T(CK_B3) * fI[k];
        sE[k] += T(CK_E3) * fI[k];
    }

#pragma unroll
    for (int i = 0; i < 6; ++i)
        yt[i] = y[i] + h * (T(CK_A41) * k1[i] + T(CK_A42) * k2[i] + T(CK_A43) * k3[i]);
#pragma unroll
    for (int k = 0; k < NF; ++k)
        tt[k] = tau[k] + h * (T(CK_A41) * kt1[k] + T(CK_A42) * t2[k] + T(CK_A43) * t3[k]);
    derivs_stage<T, NF>(g, m, yt, tt, k4, t4, fI);
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        sI[k] += T(CK_B4) * fI[k];
        sE[k] += T(CK_E4) * fI[k];
    }

#pragma unroll
    for (int i = 0; i < 6; ++i)
        yt[i] = y[i] + h * (T(CK_A51) * k1[i] + T(CK_A52) * k2[i] + T(CK_A53) * k3[i] +
                            T(CK_A54) * k4[i]);
#pragma unroll
    for (int k = 0; k < NF; ++k)
        tt[k] = tau[k] + h * (T(CK_A51) * kt1[k] + T(CK_A52) * t2[k] + T(CK_A53) * t3[k] +
                              T(CK_A54) * t4[k]);
    derivs_stage<T, NF>(g, m, yt, tt, k5, t5, fI);
#pragma unroll
    for (int k = 0; k < NF; ++k) sE[k] += T(CK_E5) * fI[k];  // b5 of stage 5 is 0

#pragma unroll
    for (int i = 0; i < 6; ++i)
        yt[i] = y[i] + h * (T(CK_A61) * k1[i] + T(CK_A62) * k2[i] + T(CK_A63) * k3[i] +
                            T(CK_A64) * k4[i] + T(CK_A65) * k5[i]);
#pragma unroll
    for (int k = 0; k < NF; ++k)
        tt[k] = tau[k] + h * (T(CK_A61) * kt1[k] + T(CK_A62) * t2[k] + T(CK_A63) * t3[k] +
                              T(CK_A64) * t4[k] + T(CK_A65) * t5[k]);
    derivs_stage<T, NF>(g, m, yt, tt, k6, t6, fI);
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        sI[k] += T(CK_B6) * fI[k];
        sE[k] += T(CK_E6) * fI[k];
    }

#pragma unroll
    for (int i = 0; i < 6; ++i) {
        dy[i] = h * (T(CK_B1) * k1[i] + T(CK_B3) * k3[i] + T(CK_B4) * k4[i] + T(CK_B6) * k6[i]);
        e[i] = h * (T(CK_E1) * k1[i] + T(CK_E3) * k3[i] + T(CK_E4) * k4[i] + T(CK_E5) * k5[i] +
                    T(CK_E6) * k6[i]);
    }
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        dtau[k] = h * (T(CK_B1) * kt1[k] + T(CK_B3) * t3[k] + T(CK_B4) * t4[k] + T(CK_B6) * t6[k]);
        dI[k] = h * sI[k];
        eI[k] = h * sE[k];
    }
}

// Geodesic-only fifth-order increment of a single Cash-Karp step of size h from y.
template <typename T>
__device__ __noinline__ void ck_geo_increment(const Geo<T> &g, const T y[6], const T k1[6], T h,
                                              T dy[6])
{
    const MediumT<T> m{};
    T e[6], z[1] = {T(0)}, d1[1], d2[1], d3[1];
    ck_attempt<T, 0>(g, m, y, k1, z, z, z, h, dy, e, d1, d2, d3);
}

// First entry into the hot spot inside an accepted step: bisection on the size of a single
// fifth-order step from the step start (the given number of halvings), ending inside;
// returns the state.
static __device__ __noinline__ void locate_spot64(const Geo<double> &g, const odx_scene &s,
                                           const double y[6], const double k1[6], double h,
                                           double yc[6], int halvings)
{
    double lo = 0.0, hi = h, dy[6], yt[6], d;
    for (int it = 0; it < halvings; ++it) {
        const double mid = 0.5 * (lo + hi);
        ck_geo_increment<double>(g, y, k1, mid, dy);
#pragma unroll
        for (int i = 0; i < 6; ++i) yt[i] = y[i] + dy[i];
        if (spot_region(s, g.sgn, yt, d) < 0.0)
            hi = mid;
        else
            lo = mid;
    }
    ck_geo_increment<double>(g, y, k1, hi, dy);
#pragma unroll
    for (int i = 0; i < 6; ++i) yc[i] = y[i] + dy[i];
}

// The same entry point by the Illinois variant of regula falsi on q(s), the spot region
// value (a distance in M) after a single fifth-order step of size s from the step start:
// q(0) > 0 outside, q(h) = q_end < 0 inside.  The bracket [lo, hi] always keeps hi inside;
// the search stops once q(hi) >= -tol (at most 40 evaluations) and returns the state at hi.
// The secant uses the Illinois weights (the value at an end kept twice in a row is halved);
// a secant point outside the open bracket falls back to the midpoint.
static __device__ __noinline__ void enter_spot64(const Geo<double> &g, const odx_scene &s,
                                          const double y[6], const double k1[6], double h,
                                          double q_end, double tol, double yc[6])
{
    double dy[6], yt[6], d;
    double lo = 0.0, hi = h;
    double flo = spot_region(s, g.sgn, y, d), fhi = q_end;  // secant weights
    double q_hi = q_end;                                   // q at hi itself
    int side = 0;
    for (int it = 0; it < 40 && q_hi < -tol; ++it) {
        double m = (lo * fhi - hi * flo) / (fhi - flo);
        if (!(m > lo && m < hi)) m = 0.5 * (lo + hi);
        ck_geo_increment<double>(g, y, k1, m, dy);
#pragma unroll
        for (int i = 0; i < 6; ++i) yt[i] = y[i] + dy[i];
        const double qm = spot_region(s, g.sgn, yt, d);
        if (qm < 0.0) {
            hi = m;
            fhi = q_hi = qm;
            if (side == -1) flo *= 0.5;
            side = -1;
        } else {
            lo = m;
            flo = qm;
            if (side == 1) fhi *= 0.5;
            side = 1;
        }
    }
    ck_geo_increment<double>(g, y, k1, hi, dy);
#pragma unroll
    for (int i = 0; i < 6; ++i) yc[i] = y[i] + dy[i];
}

}  // namespace odx
