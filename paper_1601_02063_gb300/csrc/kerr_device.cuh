// Device-side physics of the tracer: image-plane initial state, Kerr geodesic right-hand
// side, thin-disk redshift and analytic-torus transfer coefficients (Pu et al. 2016,
// Sections 2.1-2.3).  Written for the GB300 kernels; shares no code with the CPU oracle.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "odx_internal.h"

namespace odx {

constexpr double kSinFloor = 1e-8;  // Section 2.1: sin(theta) floored at 1e-8 near the poles
constexpr unsigned kFull = 0xffffffffu;

// Cash-Karp 4(5) tableau (Cash & Karp 1990), the adaptive fifth-order scheme of Section 2.1.
#define CK_A21 (1.0 / 5.0)
#define CK_A31 (3.0 / 40.0)
#define CK_A32 (9.0 / 40.0)
#define CK_A41 (3.0 / 10.0)
#define CK_A42 (-9.0 / 10.0)
#define CK_A43 (6.0 / 5.0)
#define CK_A51 (-11.0 / 54.0)
#define CK_A52 (5.0 / 2.0)
#define CK_A53 (-70.0 / 27.0)
#define CK_A54 (35.0 / 27.0)
#define CK_A61 (1631.0 / 55296.0)
#define CK_A62 (175.0 / 512.0)
#define CK_A63 (575.0 / 13824.0)
#define CK_A64 (44275.0 / 110592.0)
#define CK_A65 (253.0 / 4096.0)
#define CK_B1 (37.0 / 378.0)
#define CK_B3 (250.0 / 621.0)
#define CK_B4 (125.0 / 594.0)
#define CK_B6 (512.0 / 1771.0)
// fifth- minus fourth-order weights (the embedded error estimate)
#define CK_E1 (37.0 / 378.0 - 2825.0 / 27648.0)
#define CK_E3 (250.0 / 621.0 - 18575.0 / 48384.0)
#define CK_E4 (125.0 / 594.0 - 13525.0 / 55296.0)
#define CK_E5 (-277.0 / 14336.0)
#define CK_E6 (512.0 / 1771.0 - 1.0 / 4.0)

// Per-ray constants the right-hand side needs.
template <typename T>
struct Geo {
    T a, L, sgn;  // spin, angular momentum (E = 1), +1 literal / -1 physical direction
};

// Geodesic right-hand side ds-form: sgn * (r', theta', phi', t', p_r', p_theta') from
// Eqs. 4, 5, 12, 9, 14, 15 (E = 1, mu = 0).  The momentum equations carry the terms in
// F = 2 Sigma H that make them exactly Hamilton's equations off the null cone (they vanish
// on it); without them the constraint H = 0 is unstable on inward rays.
template <typename T>
__device__ __forceinline__ void geodesic_rhs(const Geo<T> &g, T r, T th, T pr, T pth, T f[6])
{
    T s, c;
    if constexpr (sizeof(T) == 8) {
        sincos(th, &s, &c);
    } else {
        __sincosf(th, &s, &c);  // see m_sincos in trace_step.cuh for the accuracy argument
    }
    s = fmax(s, T(kSinFloor));
    const T a = g.a, L = g.L;
    const T r2 = r * r, a2 = a * a;
    const T Sig = r2 + a2 * c * c;
    const T Del = r2 - T(2) * r + a2;
    T iSD, is;
    if constexpr (sizeof(T) == 8) {
        iSD = 1.0 / (Sig * Del);
        is = 1.0 / s;
    } else {  // correctly rounded reciprocals without the division slow path
        iSD = __frcp_rn(Sig * Del);
        is = __frcp_rn(s);
    }
    const T iS = Del * iSD;
    const T is2 = is * is;
    const T rr = r2 + a2;
    const T P = rr - a * L;
    const T q = L * is - a * s;
    const T pr2 = pr * pr, pth2 = pth * pth;
    const T F = Del * pr2 + pth2 + q * q - P * P * (Sig * iSD);
    const T kap = pth2 + L * L * is2 + a2 * s * s;
    const T rm1 = r - T(1);
    const T twor = T(2) * r;
    f[0] = g.sgn * (Del * pr * iS);
    f[1] = g.sgn * (pth * iS);
    f[2] = g.sgn * ((twor * a + (Sig - twor) * L * is2) * iSD);
    f[3] = g.sgn * (T(1) + (twor * rr - twor * a * L) * iSD);
    f[4] = g.sgn * ((-kap * rm1 + twor * rr - T(2) * a * L) * iSD - T(2) * pr2 * rm1 * iS +
                    F * (rm1 * iSD + r * iS * iS));
    f[5] = g.sgn * (s * c * iS * (L * L * is2 * is2 - a2) - a2 * s * c * F * iS * iS);
}

// Outer horizon and ISCO radius (prograde for a >= 0) of a disk rotating in +phi
// (Bardeen, Press & Teukolsky 1972, cited in Section 4.3).
__host__ __device__ __forceinline__ double horizon_radius(double a) { return 1.0 + sqrt(1.0 - a * a); }

__host__ __device__ __forceinline__ double isco_radius(double a)
{
    const double z1 = 1.0 + cbrt(1.0 - a * a) * (cbrt(1.0 + a) + cbrt(1.0 - a));
    const double z2 = sqrt(3.0 * a * a + z1 * z1);
    const double root = sqrt((3.0 - z1) * (3.0 + z1 + 2.0 * z2));
    return a >= 0.0 ? 3.0 + z2 - root : 3.0 + z2 + root;
}

// Eq. 2 for circular Keplerian orbits in the equatorial plane:
// g = 1 / (u^t (1 - Omega L)), Omega = 1/(r^1.5 + a).
__device__ __forceinline__ double disk_redshift(double a, double r, double L)
{
    const double rs = sqrt(r);
    const double r15 = r * rs;
    const double Om = 1.0 / (r15 + a);
    const double ut = (r15 + a) / (sqrt(rs * r) * sqrt(r15 - 3.0 * rs + 2.0 * a));
    return 1.0 / (ut * (1.0 - Om * L));
}

// Novikov-Thorne disk (Section 4.3): flux per unit proper area and time from one face of
// the disk at Boyer-Lindquist radius r, for unit accretion rate, in the closed form of
// Page & Thorne (1974) with x = sqrt(r), x0 = sqrt(r_ms) and the roots x1, x2, x3 of
// x^3 - 3x + 2a = 0; returned as 8 pi F / 3, which tends to r^-3 far out.  Zero inside r_ms.
__host__ __device__ inline double nt_flux_hat(double a, double r, double r_ms)
{
    if (!(r > r_ms)) return 0.0;
    const double x = sqrt(r), x0 = sqrt(r_ms);
    const double th = acos(a) / 3.0, third = 1.0471975511965976;  // pi / 3
    const double x1 = 2.0 * cos(th - third), x2 = 2.0 * cos(th + third), x3 = -2.0 * cos(th);
    double b = x - x0 - 1.5 * a * log(x / x0);
    b -= 3.0 * (x1 - a) * (x1 - a) / (x1 * (x1 - x2) * (x1 - x3)) * log((x - x1) / (x0 - x1));
    b -= 3.0 * (x2 - a) * (x2 - a) / (x2 * (x2 - x1) * (x2 - x3)) * log((x - x2) / (x0 - x2));
    b -= 3.0 * (x3 - a) * (x3 - a) / (x3 * (x3 - x1) * (x3 - x2)) * log((x - x3) / (x0 - x3));
    const double f = 1.5 * b / (x * x * (x * x * x - 3.0 * x + 2.0 * a));
    return (2.0 / 3.0) * f / r;  // 8 pi F / 3 with F = f / (4 pi r)
}

// Planck intensity B_nu(T) = 2 nu^3 / (exp(nu / T) - 1) (h = c = k = 1), 0 for T <= 0.
__host__ __device__ inline double planck(double nu, double T)
{
    return T > 0.0 ? 2.0 * nu * nu * nu / expm1(nu / T) : 0.0;
}

// Observer of one ray: spin, distance, sin and cos of theta_obs and phi_obs,
// Ro = sqrt(r_obs^2 + a^2), and the image-plane point (alpha, beta).
struct ObsIn {
    double a, r_obs, sto, cto, spo, cpo, Ro;
    double alpha, beta;
};

// Initial state of the ray through image-plane point (alpha, beta), Section 2.2:
// Eqs. 18-19 (observer grid -> Cartesian), 20-22 (-> Boyer-Lindquist), 24-26 (velocity of a
// ray perpendicular to the image plane), 7 (E, then scaled to 1), 8 (L), 4-5 (p_r, p_theta),
// 13 (Q).  In the physical convention the traced (real) photon moves opposite to Eqs. 24-26.
// cos(theta) = z'/r and the sine and cosine of phi - phi_obs come from the Cartesian point
// itself (the same values as the trigonometric functions of Eqs. 21-22, without them).
struct InitOut {
    double y[6];
    double L, Q;
};

__device__ __forceinline__ InitOut init_ray(const ObsIn &o, double sgn)
{
    const double a = o.a, sto = o.sto, cto = o.cto;
    const double D = o.Ro * sto - o.beta * cto;
    const double xp = D * o.cpo - o.alpha * o.spo;
    const double yp = D * o.spo + o.alpha * o.cpo;
    const double zp = o.r_obs * cto + o.beta * sto;
    const double w = xp * xp + yp * yp + zp * zp - a * a;
    const double r = sqrt(0.5 * (w + sqrt(w * w + 4.0 * a * a * zp * zp)));
    const double c = zp / r;
    const double th = acos(c);
    const double ph = atan2(yp, xp);
    const double s = fmax(sqrt(fmax((1.0 - c) * (1.0 + c), 0.0)), kSinFloor);
    const double rho2 = xp * xp + yp * yp;
    const double irho = rho2 > 0.0 ? rsqrt(rho2) : 0.0;
    const double cph = rho2 > 0.0 ? xp * irho : 1.0, sph = rho2 > 0.0 ? yp * irho : 0.0;
    const double cP = cph * o.cpo + sph * o.spo;  // cos(phi - phi_obs)
    const double sP = sph * o.cpo - cph * o.spo;  // sin(phi - phi_obs)
    const double R = sqrt(r * r + a * a);
    const double Sig = r * r + a * a * c * c;
    const double Del = r * r - 2.0 * r + a * a;
    // FP64 divisions are long sequences on this part: each reciprocal is taken once
    const double iSig = 1.0 / Sig, iDel = 1.0 / Del;
    double rd = sgn * (-(r * R * s * sto * cP + R * R * c * cto) * iSig);
    double td = sgn * ((r * s * cto - R * c * sto * cP) * iSig);
    double pd = sgn * (sto * sP / (R * s));
    const double E2 = ((Sig - 2.0 * r) * iSig * iDel) * (Sig * rd * rd + Sig * Del * td * td) +
                      Del * pd * pd * s * s;
    const double iE = rsqrt(E2);
    rd *= iE;
    td *= iE;
    pd *= iE;
    InitOut out;
    out.L = (Sig * Del * pd - 2.0 * a * r) * s * s / (Sig - 2.0 * r);
    out.y[0] = r;
    out.y[1] = th;
    out.y[2] = ph;
    out.y[3] = 0.0;
    out.y[4] = Sig * rd * iDel;
    out.y[5] = Sig * td;
    const double Ls = out.L / s;
    out.Q = out.y[5] * out.y[5] + (Ls * Ls - a * a) * c * c;
    return out;
}

// At the end of a ray (state y): the relative null violation H and the Carter constant Q,
// from one sincos of theta.
struct EndChecks {
    double H, Q;
};
__device__ __forceinline__ EndChecks end_checks(double a, double L, const double y[6])
{
    double s, c;
    sincos(y[1], &s, &c);
    s = fmax(s, kSinFloor);
    const double r = y[0];
    const double Del = r * r - 2.0 * r + a * a;
    const double t1 = Del * y[4] * y[4], t2 = y[5] * y[5];
    const double Ls = L / s;
    const double q = Ls - a * s;
    const double t3 = q * q;
    const double P = r * r + a * a - a * L;
    const double t4 = P * P / Del;
    EndChecks e;
    e.H = (t1 + t2 + t3 - t4) / (fabs(t1) + t2 + t3 + fabs(t4));
    e.Q = t2 + (Ls * Ls - a * a) * c * c;
    return e;
}

// ---- thermal synchrotron shell (Section 4.5) ---------------------------------------------
// CGS constants (CODATA 2018; G M_sun the IAU nominal value).
constexpr double kCgsC = 2.99792458e10, kCgsE = 4.803204712570263e-10, kCgsMe = 9.1093837015e-28,
                 kCgsMp = 1.67262192369e-24, kCgsH = 6.62607015e-27, kCgsGMsun = 1.3271244e26;
// The stages take frequencies in GHz and carry I-hat = (I_nu / nu^3) / Aj.
constexpr double kNuUnit = 1e9;

struct SynchK {
    double inv_kc;  // 1 / nu_c-hat at r = 1, n_e = n_e0, Theta_e = 1 (nu_c in GHz)
    double ky;      // h nu / k T_e = ky nu-hat / Theta_e
    double Atau;    // dtau/ds = Atau * (dI-hat/ds without exp(-tau)) * expm1(h nu0 / k T_e)
    double Aj;      // I_nu / nu^3 = Aj * I-hat (CGS, nu in Hz)
};

// With nr = n_e / n_e0, per unit path in r_g and nu0-hat the fluid-frame frequency in GHz:
//   j_nu / 4 pi = nu0 n_e e^2 / (sqrt(3) c K_2(1/Theta_e)) M(x_M)            (Eq. 37)
//   nu_c = 3 e B / (4 pi m_e c) Theta_e^2, B = B0 sqrt(nr / r)                (Eq. 39)
//   dI/ds = r_g j_nu / (4 pi g nu0^3) exp(-tau) = Aj nr M / (K_2 nu0-hat^2 g) exp(-tau)
//   dtau/ds = r_g alpha_nu / g = (c^2 / 2 h) expm1(h nu0 / k T_e) * (the same without exp)
// B0 = sqrt(8 pi n_e0 m_p c^2 / (6 beta_B)) from B^2 / 8 pi = n_e m_p c^2 / (6 beta_B r).
__host__ __device__ inline SynchK synch_constants(const odx_scene &s)
{
    const double pi = 3.14159265358979323846;
    const double rg = kCgsGMsun * s.mass / (kCgsC * kCgsC);
    const double B0 = sqrt(8.0 * pi * s.n_e0 * kCgsMp * kCgsC * kCgsC / (6.0 * s.beta_B));
    SynchK k;
    k.inv_kc = 4.0 * pi * kCgsMe * kCgsC * kNuUnit / (3.0 * kCgsE * B0);
    k.ky = kCgsH * kNuUnit / (kCgsMe * kCgsC * kCgsC);
    k.Aj = kCgsE * kCgsE * s.n_e0 * rg / (sqrt(3.0) * kCgsC * kNuUnit * kNuUnit);
    k.Atau = k.Aj * kCgsC * kCgsC / (2.0 * kCgsH);
    return k;
}

// ---- step control of the transfer equation (Section 2.3) ----------------------------------
// The invariant intensities I_k enter the Cash-Karp error norm with the scale
// |I_k| + |h dI_k/ds| + rt_floor(s, nu_k): the floor is kRtFloorFrac times the medium's
// source function at its temperature scale T0 seen at nu, B_nu(T0) / nu^3, in the units the
// stages carry (torus: 2 / (exp(nu / T0) - 1); synchrotron shell: the CGS value
// (2 h / c^2) / (exp(h nu / (T0 m_e c^2)) - 1) divided by Aj, nu in Hz), so that emission far
// below the medium's own intensity scale does not set the step.  ODX_RT_RIDE: infinite (the
// intensities stay out of the norm).
constexpr double kRtFloorFrac = 3e-5;
__host__ __device__ inline double rt_floor(const odx_scene &s, double nu)
{
    if (s.rt_control == ODX_RT_RIDE) return INFINITY;
    if (s.emitter == ODX_EMIT_SYNCH) {
        const double kT = s.T0 * kCgsMe * kCgsC * kCgsC;
        const double src = 2.0 * kCgsH / (kCgsC * kCgsC) / expm1(kCgsH * nu / kT);
        return kRtFloorFrac * src / synch_constants(s).Aj;
    }
    return kRtFloorFrac * 2.0 / expm1(nu / s.T0);
}

// ---- Keplerian hot spot (Section 4.4): the centre's circular equatorial orbit --------------
__host__ __device__ inline double spot_orbit_radius(const odx_scene &s)
{
    return s.spot_r > 0.0 ? s.spot_r : isco_radius(s.a);
}
__host__ __device__ inline double spot_omega(const odx_scene &s)
{
    const double rs = spot_orbit_radius(s);
    return 1.0 / (rs * sqrt(rs) + s.a);
}

}  // namespace odx
