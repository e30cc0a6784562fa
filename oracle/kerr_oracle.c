/*
 * kerr_oracle.c -- plain FP64 CPU oracle (test infrastructure only; see kerr_oracle.h).
 *
 * Every function follows a passage of Pu et al. 2016 ("Odyssey") in the paper's
 * order and notation, written for a reader to check by eye: no blocking, no fused
 * reformulation, no precomputed tables.  Readings of passages where the paper is
 * silent or ambiguous are marked "reading:" and listed in the design notes.
 *
 * State vector y = (r, theta, phi, t, p_r, p_theta), E = 1, mu = 0 (photons).
 * The traced parameter s grows from the observer toward the source.
 *   physical convention: the real photon moves outward with p_t = -1; it is traced
 *                        back in affine time, s = -lambda, dy/ds = -f(y).
 *   literal convention:  Eqs. 24-26 give the velocity of the traced photon itself,
 *                        s = lambda, dy/ds = +f(y).
 */
#include "kerr_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define N_GEO 6
#define N_MAX (N_GEO + 2 * ORC_MAX_FREQ)
#define SIN_FLOOR 1e-8 /* Section 2.1: sin(theta) is set to 1e-8 when it falls below 1e-8 */
#define M_PI_ORC 3.14159265358979323846

/* ------------------------------------------------------------------ */
/* Closed forms of the Kerr geometry                                  */
/* ------------------------------------------------------------------ */

/* Outer horizon r_+ = M + sqrt(M^2 - a^2), the larger root of Delta = 0 (Eq. 1). */
double orc_horizon(double a) { return 1.0 + sqrt(1.0 - a * a); }

/* Radius of the marginally stable (innermost stable) circular orbit for a disk that
 * rotates in +phi, from Bardeen, Press & Teukolsky 1972 (cited in Section 4.3). */
double orc_isco(double a)
{
    double z1 = 1.0 + cbrt(1.0 - a * a) * (cbrt(1.0 + a) + cbrt(1.0 - a));
    double z2 = sqrt(3.0 * a * a + z1 * z1);
    double root = sqrt((3.0 - z1) * (3.0 + z1 + 2.0 * z2));
    return (a >= 0.0) ? 3.0 + z2 - root : 3.0 + z2 + root;
}

/* ------------------------------------------------------------------ */
/* Cash-Karp embedded Runge-Kutta 4(5) tableau (Section 2.1 cites the  */
/* adaptive fifth-order scheme of Press et al. 1992; the coefficients   */
/* are those published by Cash & Karp 1990).                            */
/* ------------------------------------------------------------------ */
static const double CK_C[6] = {0.0, 1.0 / 5.0, 3.0 / 10.0, 3.0 / 5.0, 1.0, 7.0 / 8.0};
static const double CK_A[6][5] = {
    {0.0, 0.0, 0.0, 0.0, 0.0},
    {1.0 / 5.0, 0.0, 0.0, 0.0, 0.0},
    {3.0 / 40.0, 9.0 / 40.0, 0.0, 0.0, 0.0},
    {3.0 / 10.0, -9.0 / 10.0, 6.0 / 5.0, 0.0, 0.0},
    {-11.0 / 54.0, 5.0 / 2.0, -70.0 / 27.0, 35.0 / 27.0, 0.0},
    {1631.0 / 55296.0, 175.0 / 512.0, 575.0 / 13824.0, 44275.0 / 110592.0, 253.0 / 4096.0}};
static const double CK_B5[6] = {37.0 / 378.0, 0.0, 250.0 / 621.0, 125.0 / 594.0, 0.0,
                                512.0 / 1771.0};
static const double CK_B4[6] = {2825.0 / 27648.0, 0.0, 18575.0 / 48384.0, 13525.0 / 55296.0,
                                277.0 / 14336.0, 1.0 / 4.0};

void orc_ck_tableau(double c[6], double a[36], double b5[6], double b4[6])
{
    for (int i = 0; i < 6; ++i) {
        c[i] = CK_C[i];
        b5[i] = CK_B5[i];
        b4[i] = CK_B4[i];
        for (int j = 0; j < 6; ++j) a[6 * i + j] = (j < 5) ? CK_A[i][j] : 0.0;
    }
}

/* ------------------------------------------------------------------ */
/* Initial conditions, Section 2.2                                     */
/* ------------------------------------------------------------------ */

/* reading: pixel centres, alpha_i = alpha_min + (i + 1/2) (alpha_max - alpha_min) / N_alpha */
void orc_pixel_center(const orc_scene *sc, int32_t i, int32_t j, double *alpha, double *beta)
{
    *alpha = sc->alpha_min + (i + 0.5) * (sc->alpha_max - sc->alpha_min) / sc->n_alpha;
    *beta = sc->beta_min + (j + 0.5) * (sc->beta_max - sc->beta_min) / sc->n_beta;
}

/* Eqs. 18-19: image-plane point (x, y, z) = (alpha, beta, 0) -> black-hole Cartesian x'. */
void orc_observer_point(const orc_scene *sc, double alpha, double beta, double xyz[3])
{
    double x = alpha, y = beta, z = 0.0;
    double a = sc->a, ro = sc->r_obs, to = sc->theta_obs, po = sc->phi_obs;
    double D = (sqrt(ro * ro + a * a) - z) * sin(to) - y * cos(to); /* Eq. 19 */
    xyz[0] = D * cos(po) - x * sin(po);                             /* Eq. 18 */
    xyz[1] = D * sin(po) + x * cos(po);
    xyz[2] = (ro - z) * cos(to) + y * sin(to);
}

/*
 * Initial state of the ray through image-plane point (alpha, beta):
 * Eqs. 20-22 (Cartesian -> Boyer-Lindquist), Eqs. 24-26 (inward velocity),
 * Eq. 7 (E), Eq. 8 (L_z), Eqs. 4-5 (p_r, p_theta), Eq. 13 (Q).
 * reading: E is normalised to 1 by scaling the velocity (null rays are scale free).
 * reading: in the physical convention the real photon has velocity -v_in.
 */
void orc_init_ray(const orc_scene *sc, double alpha, double beta, double y0[6], double *L_out,
                  double *Q_out, double vin[3])
{
    double a = sc->a;
    double xp[3];
    orc_observer_point(sc, alpha, beta, xp);

    /* Eqs. 20-22 */
    double w = xp[0] * xp[0] + xp[1] * xp[1] + xp[2] * xp[2] - a * a;
    double r = sqrt((w + sqrt(w * w + 4.0 * a * a * xp[2] * xp[2])) / 2.0);
    double theta = acos(xp[2] / r);
    double phi = atan2(xp[1], xp[0]);

    /* Eqs. 24-26 with R = sqrt(r^2 + a^2), Phi = phi - phi_obs */
    double sint = fmax(sin(theta), SIN_FLOOR);
    double cost = cos(theta);
    double R = sqrt(r * r + a * a);
    double Phi = phi - sc->phi_obs;
    double Sigma = r * r + a * a * cost * cost;
    double Delta = r * r - 2.0 * r + a * a;
    double sto = sin(sc->theta_obs), cto = cos(sc->theta_obs);
    double rdot = -(r * R * sint * sto * cos(Phi) + R * R * cost * cto) / Sigma;
    double thdot = (r * sint * cto - R * cost * sto * cos(Phi)) / Sigma;
    double phdot = sto * sin(Phi) / (R * sint);
    if (vin) {
        vin[0] = rdot;
        vin[1] = thdot;
        vin[2] = phdot;
    }

    double sgn = (sc->convention == ORC_CONV_LITERAL) ? 1.0 : -1.0;
    rdot *= sgn;
    thdot *= sgn;
    phdot *= sgn;

    /* Eq. 7 with mu = 0, then scale so that E = 1 */
    double E2 = ((Sigma - 2.0 * r) / (Sigma * Delta)) * (Sigma * rdot * rdot +
                                                         Sigma * Delta * thdot * thdot) +
                Delta * phdot * phdot * sint * sint;
    double E = sqrt(E2);
    rdot /= E;
    thdot /= E;
    phdot /= E;

    /* Eq. 8 with E = 1 */
    double L = (Sigma * Delta * phdot - 2.0 * a * r) * sint * sint / (Sigma - 2.0 * r);

    y0[0] = r;
    y0[1] = theta;
    y0[2] = phi;
    y0[3] = 0.0;
    y0[4] = Sigma * rdot / Delta; /* Eq. 4 */
    y0[5] = Sigma * thdot;        /* Eq. 5 */
    *L_out = L;
    /* Eq. 13 with E = 1, mu = 0 */
    *Q_out = y0[5] * y0[5] + (L * L / (sint * sint) - a * a) * cost * cost;
}

/* ------------------------------------------------------------------ */
/* Geodesic right-hand side, Section 2.1                               */
/* ------------------------------------------------------------------ */

/*
 * f = d/dlambda (r, theta, phi, t, p_r, p_theta) from Eqs. 4, 5, 12, 9, 14, 15 with
 * E = 1, mu = 0 and the pole floor on sin(theta).
 *
 * reading: Eqs. 14-15 are Hamilton's equations for H = g^{mu nu} p_mu p_nu / 2 after the
 * null condition H = 0 was used to simplify them.  Off the null cone they differ from
 * -dH/dr and -dH/dtheta by terms proportional to
 *     F = 2 Sigma H = Delta p_r^2 + p_th^2 + (L csc - a sin)^2 - ((r^2 + a^2) - a L)^2 / Delta,
 * and with those terms H Sigma Delta is conserved, so a truncation error made at radius r1
 * grows like (r1 / r2)^4 by radius r2 on an inward ray (a ray aimed at the hole from
 * r = 1000 escapes at rtol 1e-8).  The terms in F below restore Hamilton's equations
 * exactly; they vanish on the null cone, so the geodesics are those of Eqs. 14-15.
 */
void orc_geodesic_rhs(double a, double L, const double y[6], double f[6])
{
    double r = y[0], theta = y[1], pr = y[4], pth = y[5];
    double sint = fmax(sin(theta), SIN_FLOOR);
    double cost = cos(theta);
    double Sigma = r * r + a * a * cost * cost;
    double Delta = r * r - 2.0 * r + a * a;
    double kappa = pth * pth + L * L / (sint * sint) + a * a * sint * sint; /* below Eq. 15 */
    double P = (r * r + a * a) - a * L;
    double F = Delta * pr * pr + pth * pth + (L / sint - a * sint) * (L / sint - a * sint) -
               P * P / Delta;

    f[0] = Delta * pr / Sigma;                                                  /* Eq. 4 */
    f[1] = pth / Sigma;                                                         /* Eq. 5 */
    f[2] = (2.0 * a * r + (Sigma - 2.0 * r) * L / (sint * sint)) / (Sigma * Delta); /* Eq. 12 */
    f[3] = 1.0 + (2.0 * r * (r * r + a * a) - 2.0 * a * r * L) / (Sigma * Delta);  /* Eq. 9 */
    f[4] = (-kappa * (r - 1.0) + 2.0 * r * (r * r + a * a) - 2.0 * a * L) / (Sigma * Delta) -
           2.0 * pr * pr * (r - 1.0) / Sigma                                     /* Eq. 14 */
           + F * ((r - 1.0) / (Sigma * Delta) + r / (Sigma * Sigma));
    f[5] = (sint * cost / Sigma) * (L * L / (sint * sint * sint * sint) - a * a) /* Eq. 15 */
           - a * a * sint * cost * F / (Sigma * Sigma);
}

/* ------------------------------------------------------------------ */
/* Emitters                                                            */
/* ------------------------------------------------------------------ */

/* Eq. 2 for an equatorial Keplerian disk (Section 4.3, circular orbits of Cunningham
 * 1975 / Bardeen et al. 1972): u = u^t (1, 0, 0, Omega), Omega = 1/(r^1.5 + a);
 * with p_t = -1, p_phi = L:  g = (p.u)|inf / (p.u)|em = 1 / (u^t (1 - Omega L)). */
double orc_disk_redshift(double a, double r, double L)
{
    double r15 = pow(r, 1.5);
    double Omega = 1.0 / (r15 + a);
    double ut = (r15 + a) / (pow(r, 0.75) * sqrt(r15 - 3.0 * sqrt(r) + 2.0 * a));
    return 1.0 / (ut * (1.0 - Omega * L));
}

/* ---- Novikov-Thorne disk (Section 4.3) ---------------------------------------------------
 * Circular prograde equatorial orbits (Bardeen, Press & Teukolsky 1972): specific energy E,
 * angular momentum L and angular velocity Omega.  Page & Thorne (1974): the flux from one
 * face for accretion rate Mdot is F = Mdot f / (4 pi r) with
 *   f(r) = -dOmega/dr (E - Omega L)^-2  int_{r_ms}^{r} (E - Omega L) dL/dr' dr'.
 * Here: derivatives by five-point central differences in long double, the integral by
 * adaptive Simpson quadrature (tolerance 1e-12 of the integral); returned as
 * 8 pi F / 3 for Mdot = 1. */
double orc_circ_E(double a, double r)
{
    double rs = sqrt(r);
    return (r * rs - 2.0 * rs + a) / (pow(r, 0.75) * sqrt(r * rs - 3.0 * rs + 2.0 * a));
}

double orc_circ_L(double a, double r)
{
    double rs = sqrt(r);
    return (r * r - 2.0 * a * rs + a * a) / (pow(r, 0.75) * sqrt(r * rs - 3.0 * rs + 2.0 * a));
}

static long double circ_Omega(double a, long double r) { return 1.0L / (powl(r, 1.5L) + a); }

static long double circ_Ll(double a, long double r)
{
    long double rs = sqrtl(r);
    return (r * r - 2.0L * a * rs + (long double)a * a) /
           (powl(r, 0.75L) * sqrtl(r * rs - 3.0L * rs + 2.0L * a));
}

static long double circ_El(double a, long double r)
{
    long double rs = sqrtl(r);
    return (r * rs - 2.0L * rs + a) / (powl(r, 0.75L) * sqrtl(r * rs - 3.0L * rs + 2.0L * a));
}

/* five-point central difference with step 1e-4 r */
static long double ddr(long double (*fn)(double, long double), double a, long double r)
{
    long double h = 1e-4L * r;
    return (-fn(a, r + 2 * h) + 8 * fn(a, r + h) - 8 * fn(a, r - h) + fn(a, r - 2 * h)) /
           (12 * h);
}

static long double pt_integrand(double a, long double r)
{
    return (circ_El(a, r) - circ_Omega(a, r) * circ_Ll(a, r)) * ddr(circ_Ll, a, r);
}

static long double simpson_rec(double a, long double lo, long double hi, long double flo,
                               long double fmid, long double fhi, long double whole,
                               long double tol, int depth)
{ /* tol: absolute, halved per level (1e-12 of the whole integral at the top) */
    long double mid = 0.5L * (lo + hi), lm = 0.5L * (lo + mid), rm = 0.5L * (mid + hi);
    long double flm = pt_integrand(a, lm), frm = pt_integrand(a, rm);
    long double left = (mid - lo) / 6.0L * (flo + 4.0L * flm + fmid);
    long double right = (hi - mid) / 6.0L * (fmid + 4.0L * frm + fhi);
    if (depth <= 0 || fabsl(left + right - whole) <= 15.0L * tol)
        return left + right + (left + right - whole) / 15.0L;
    return simpson_rec(a, lo, mid, flo, flm, fmid, left, 0.5L * tol, depth - 1) +
           simpson_rec(a, mid, hi, fmid, frm, fhi, right, 0.5L * tol, depth - 1);
}

double orc_nt_flux(double a, double r)
{
    double rms = orc_isco(a);
    if (!(r > rms)) return 0.0;
    long double lo = rms, hi = r, mid = 0.5L * (lo + hi);
    long double flo = pt_integrand(a, lo), fmid = pt_integrand(a, mid), fhi = pt_integrand(a, hi);
    long double whole = (hi - lo) / 6.0L * (flo + 4.0L * fmid + fhi);
    long double tol = 1e-12L * fabsl(whole) + 1e-30L;
    long double integral = simpson_rec(a, lo, hi, flo, fmid, fhi, whole, tol, 24);
    long double eol = circ_El(a, r) - circ_Omega(a, r) * circ_Ll(a, r);
    long double f = -ddr(circ_Omega, a, r) / (eol * eol) * integral;
    return (double)(2.0L * f / (3.0L * r)); /* 8 pi F / 3 with F = f / (4 pi r) */
}

/* ------------------------------------------------------------------ */
/* Thermal synchrotron shell (Section 4.5), CGS units                  */
/* ------------------------------------------------------------------ */
#define CGS_C 2.99792458e10        /* speed of light, cm s^-1 (exact)          */
#define CGS_E 4.803204712570263e-10 /* elementary charge, esu                   */
#define CGS_ME 9.1093837015e-28     /* electron mass, g                         */
#define CGS_MP 1.67262192369e-24    /* proton mass, g                           */
#define CGS_H 6.62607015e-27        /* Planck constant, erg s (exact)           */
#define CGS_GMSUN 1.3271244e26      /* G M_sun, cm^3 s^-2 (IAU nominal)          */

static long double k2_integrand(long double x, long double t)
{ /* exp(-x (cosh t - 1)) cosh 2t: the integrand of K_2 without its factor exp(-x) */
    return expl(-x * (coshl(t) - 1.0L)) * coshl(2.0L * t);
}

/* Nodes and weights of the 16-point Gauss-Legendre rule on [-1, 1]: the roots of P_16 by
 * Newton's method from the usual cosine guesses, w = 2 / ((1 - x^2) P_16'(x)^2). */
static void gauss_legendre16(long double x[16], long double w[16])
{
    const int n = 16;
    for (int i = 0; i < n / 2; ++i) {
        long double z = cosl(3.14159265358979323846264338327950288L * (i + 0.75L) / (n + 0.5L));
        long double dp = 1.0L;
        for (int it = 0; it < 100; ++it) {
            long double p0 = 1.0L, p1 = z; /* P_0, P_1 -> P_n by the three-term recurrence */
            for (int k = 2; k <= n; ++k) {
                long double p2 = ((2.0L * k - 1.0L) * z * p1 - (k - 1.0L) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0L);
            long double dz = p1 / dp;
            z -= dz;
            if (fabsl(dz) < 1e-19L) break;
        }
        x[i] = -z;
        x[n - 1 - i] = z;
        w[i] = w[n - 1 - i] = 2.0L / ((1.0L - z * z) * dp * dp);
    }
}

/* Modified Bessel function of the second kind of order 2, from its integral representation
 * K_n(x) = int_0^inf exp(-x cosh t) cosh(n t) dt (x > 0): 16-point Gauss-Legendre on eight
 * equal panels of [0, t_max], t_max where the integrand has fallen below e^-45 of its value
 * at 0 (relative error ~1e-15 against a library K_2 for 1e-3 <= x <= 100). */
double orc_bessel_k2(double x)
{
    if (!(x > 0.0)) return NAN;
    long double xl = x, hi = 1.0L;
    while (xl * (coshl(hi) - 1.0L) - 2.0L * hi < 45.0L) hi += 0.25L;
    long double gx[16], gw[16];
    gauss_legendre16(gx, gw);
    long double integral = 0.0L, width = hi / 8.0L;
    for (int p = 0; p < 8; ++p) {
        long double mid = (p + 0.5L) * width;
        for (int i = 0; i < 16; ++i)
            integral += 0.5L * width * gw[i] * k2_integrand(xl, mid + 0.5L * width * gx[i]);
    }
    return (double)(expl(-xl) * integral);
}

/* Gravitational radius G M / c^2 in cm for a mass in solar masses. */
double orc_r_g(double mass) { return CGS_GMSUN * mass / (CGS_C * CGS_C); }

/* Section 4.5: thermal synchrotron emissivity of a relativistic Maxwellian (the angle-
 * averaged fit of Mahadevan et al. 1996 that the paper prints),
 *   j_nu = nu 4 pi n e^2 / (sqrt(3) c K_2(1/Theta_e)) M(x_M),  x_M = nu / nu_c,
 *   M(x) = 4.0505 x^-1/6 (1 + 0.40 x^-1/4 + 0.5316 x^-1/2) exp(-1.8899 x^1/3),
 *   nu_c = 3 e B / (4 pi m_e c) Theta_e^2,
 * and the absorption coefficient from Kirchhoff's law, alpha_nu = j_nu / B_nu(T_e).
 * reading: the printed j_nu is the emissivity integrated over all directions (its integral
 * over nu is the synchrotron power of a Maxwell-Juttner electron, (4/3) sigma_T c U_B
 * <gamma^2 beta^2>); the transfer equation and Kirchhoff's law take the emissivity per
 * steradian, j_nu / 4 pi, which is what this function returns.
 * reading: the density and temperature follow power laws in r with the torus's polar
 * profile, and B from equipartition with a fraction of the ions' virial energy,
 * B^2 / 8 pi = n_e m_p c^2 / (6 beta_B r) (the profiles of the cited shell model are not
 * printed); no emission beyond r_out. */
typedef struct {
    double n, Theta, nu_c, K2; /* n_e [cm^-3], Theta_e, nu_c [Hz], K_2(1 / Theta_e) */
} synch_local;

static synch_local synch_at(const orc_scene *sc, double r, double cost)
{
    synch_local q;
    double w = sc->theta_width;
    q.n = sc->n_e0 * pow(r, -sc->ne_index) * exp(-cost * cost / (2.0 * w * w));
    q.Theta = sc->T0 * pow(r, -sc->T_index);
    double B = sqrt(8.0 * M_PI_ORC * q.n * CGS_MP * CGS_C * CGS_C / (6.0 * sc->beta_B * r));
    q.nu_c = 3.0 * CGS_E * B / (4.0 * M_PI_ORC * CGS_ME * CGS_C) * q.Theta * q.Theta;
    q.K2 = orc_bessel_k2(1.0 / q.Theta);
    return q;
}

static void synch_coeffs_at(const synch_local *q, double nu0, double *j, double *alpha)
{
    double x = nu0 / q->nu_c;
    double M = 4.0505 / pow(x, 1.0 / 6.0) * (1.0 + 0.40 / pow(x, 0.25) + 0.5316 / sqrt(x)) *
               exp(-1.8899 * cbrt(x));
    double jnu = nu0 * 4.0 * M_PI_ORC * q->n * CGS_E * CGS_E / (sqrt(3.0) * CGS_C * q->K2) * M;
    /* B_nu(T) = (2 h nu^3 / c^2) / (exp(h nu / k T) - 1), k T = Theta m_e c^2 */
    double Bnu = 2.0 * CGS_H * nu0 * nu0 * nu0 / (CGS_C * CGS_C) /
                 expm1(CGS_H * nu0 / (q->Theta * CGS_ME * CGS_C * CGS_C));
    *j = jnu / (4.0 * M_PI_ORC);
    *alpha = *j / Bnu;
}

void orc_synch_coeffs(const orc_scene *sc, double r, double cost, double nu0, double *j,
                      double *alpha)
{
    synch_local q = synch_at(sc, r, cost);
    synch_coeffs_at(&q, nu0, j, alpha);
}

/* ------------------------------------------------------------------ */
/* Keplerian hot spot (Section 4.4)                                    */
/* ------------------------------------------------------------------ */
static double spot_radius(const orc_scene *sc)
{
    return (sc->spot_r > 0.0) ? sc->spot_r : orc_isco(sc->a);
}

/* Keplerian angular velocity of the spot centre's circular equatorial orbit (prograde). */
double orc_spot_omega(const orc_scene *sc) { return 1.0 / (pow(spot_radius(sc), 1.5) + sc->a); }

/* A photon that reaches the observer at t_obs left the point y at coordinate time
 * t_e = t_obs - dt, dt the coordinate time it spends between y and the image plane: the
 * traced t runs from 0 at the image plane with dt/ds = sgn dt/dlambda, so dt = sgn t.
 * The spot centre at t_e sits at azimuth spot_phase + Omega t_e on the circle r = spot_r,
 * theta = pi/2.  Distances in the pseudo-Cartesian coordinates the paper prints:
 * x = sqrt(r^2 + a^2) cos phi, y = sqrt(r^2 + a^2) sin phi, z = r cos theta.
 * reading: the spot is the region d < 4 r_spot, z > 0 where the paper defines its
 * emission; it is optically thick, so a ray ends where it first enters that region.
 * Returns max(d - 4 r_spot, -z): negative inside. */
double orc_spot_region(const orc_scene *sc, double sgn, const double y[6], double *d_out)
{
    double a = sc->a, rs = spot_radius(sc);
    double t_e = sc->t_obs - sgn * y[3];
    double phs = sc->spot_phase + orc_spot_omega(sc) * t_e;
    double Rs = sqrt(rs * rs + a * a), R = sqrt(y[0] * y[0] + a * a);
    double dx = R * cos(y[2]) - Rs * cos(phs);
    double dy = R * sin(y[2]) - Rs * sin(phs);
    double z = y[0] * cos(y[1]);
    double d = sqrt(dx * dx + dy * dy + z * z);
    if (d_out) *d_out = d;
    return fmax(d - 4.0 * sc->spot_size, -z);
}

/* Redshift of the spot's gas, g = 1 / (u^t (1 - Omega L)) (Eq. 2) for gas co-rotating with
 * the centre at Omega at the point (r, theta); 0 where that motion is not timelike. */
static double spot_redshift(const orc_scene *sc, double r, double theta, double L)
{
    double a = sc->a, sint = fmax(sin(theta), SIN_FLOOR), cost = cos(theta);
    double Sigma = r * r + a * a * cost * cost;
    double Delta = r * r - 2.0 * r + a * a;
    double A = (r * r + a * a) * (r * r + a * a) - a * a * Delta * sint * sint;
    double Om = orc_spot_omega(sc);
    double N = -(1.0 - 2.0 * r / Sigma) - 2.0 * (2.0 * a * r * sint * sint / Sigma) * Om +
               A * sint * sint / Sigma * Om * Om;
    if (!(N < 0.0)) return 0.0;
    return sqrt(-N) / (1.0 - Om * L);
}

/* reading: torus velocity field.  Keplerian Omega(r) at BL radius r where r >= r_ISCO
 * and the orbit is timelike at (r, theta); the zero-angular-momentum observer
 * Omega = 2 a r / A elsewhere.  u^t from u.u = -1 with the metric of Eq. 1. */
static void torus_flow(double a, double r_isco, double r, double sint, double cost, double *ut,
                       double *Omega)
{
    double Sigma = r * r + a * a * cost * cost;
    double Delta = r * r - 2.0 * r + a * a;
    double A = (r * r + a * a) * (r * r + a * a) - a * a * Delta * sint * sint;
    double gtt = -(1.0 - 2.0 * r / Sigma);
    double gtp = -2.0 * a * r * sint * sint / Sigma;
    double gpp = A * sint * sint / Sigma;
    double Om = 1.0 / (pow(r, 1.5) + a);
    double N = gtt + 2.0 * gtp * Om + gpp * Om * Om;
    if (!(r >= r_isco && N < 0.0)) {
        Om = 2.0 * a * r / A;
        N = gtt + 2.0 * gtp * Om + gpp * Om * Om;
    }
    *Omega = Om;
    *ut = 1.0 / sqrt(-N);
}

/* ------------------------------------------------------------------ */
/* One ray                                                             */
/* ------------------------------------------------------------------ */
typedef struct {
    const orc_scene *sc;
    double a, L, sgn, r_isco, r_horizon;
    double r_stop; /* the ray stops inside this radius; the medium ends there too */
    int n; /* number of integrated components: 6 geodesic + 2 per frequency (RT) */
    int n_rt;
    double I_floor[ORC_MAX_FREQ]; /* error-scale floor of each invariant intensity */
} ray_ctx;

/* reading: the invariant intensities of the transfer equation are under the step control
 * (the paper integrates Eqs. 30-31 along with the geodesic and names no error norm for
 * them).  Each I_k enters the error norm with the scale |I_k| + |h dI_k/ds| + I_floor_k,
 * I_floor_k = RT_FLOOR_FRAC times the source function of the medium at its temperature
 * scale T0 seen at nu_k, B_nu(T0) / nu^3 (the test medium: its source function eps /
 * kappa), so that emission far below the medium's own intensity scale does not set the
 * step.  tau_k stays out of the norm: its error reaches I_k only through exp(-tau_k), which
 * the estimate of I_k already carries.  With the transfer components outside the norm
 * (ORC_RT_RIDE, the earlier reading) the steps follow the geodesic alone and the
 * intensities of rays through steep emission (the shadow's edge of the torus, the inner
 * synchrotron shell) are good to 1e-3 - 1e-2 only, even at rtol 1e-8. */
#define RT_FLOOR_FRAC 3e-5

static double source_scale(const orc_scene *sc, double nu)
{
    if (sc->emitter == ORC_EMIT_CONST) return sc->T0 / sc->C_norm;
    if (sc->emitter == ORC_EMIT_SYNCH)
        return 2.0 * CGS_H / (CGS_C * CGS_C) / expm1(CGS_H * nu / (sc->T0 * CGS_ME * CGS_C * CGS_C));
    return 2.0 / expm1(nu / sc->T0); /* torus: B_nu(T) = 2 nu^3 / (exp(nu / T) - 1) */
}

/* dy/ds for the geodesic and, for RT emitters, Eqs. 30-31 per frequency:
 *   dtau/ds = alpha_0(nu_0) / g,   dI/ds = j_0(nu_0) / (g nu_0^3) exp(-tau),
 * with nu_0 = nu_obs / g the frequency in the fluid frame.
 * reading: the nu in Eq. 31 is the local frequency nu_0 (both in j and in nu^3). */
static void derivs(const ray_ctx *rc, int n, const double *y, double *dy)
{
    double f[6];
    orc_geodesic_rhs(rc->a, rc->L, y, f);
    for (int i = 0; i < N_GEO; ++i) dy[i] = rc->sgn * f[i];
    if (rc->n_rt == 0 || n == N_GEO) return;
    /* reading: rays stop at r < horizon_factor r_+, and the medium ends there: no emission
     * or absorption inside that radius.  The last step of a captured ray ends somewhere
     * inside it, at a radius that depends on the step sequence; without this the intensity
     * of such rays would depend on that step. */
    if (y[0] < rc->r_stop) {
        for (int k = 0; k < rc->n_rt; ++k) dy[N_GEO + 2 * k] = dy[N_GEO + 2 * k + 1] = 0.0;
        return;
    }

    const orc_scene *sc = rc->sc;
    if (sc->emitter == ORC_EMIT_CONST) {
        for (int k = 0; k < rc->n_rt; ++k) {
            dy[N_GEO + 2 * k] = sc->C_norm;
            dy[N_GEO + 2 * k + 1] = sc->T0 * exp(-y[N_GEO + 2 * k]);
        }
        return;
    }

    /* analytic thermal torus: n_e, T_e, thermal j_nu, Kirchhoff alpha_nu = j_nu / B_nu */
    double r = y[0];
    double sint = fmax(sin(y[1]), SIN_FLOOR);
    double cost = cos(y[1]);
    double ut, Omega;
    torus_flow(rc->a, rc->r_isco, r, sint, cost, &ut, &Omega);
    double g = 1.0 / (ut * (1.0 - Omega * rc->L)); /* Eq. 2 */
    if (sc->emitter == ORC_EMIT_SYNCH) {
        /* lengths in r_g: d/ds per r_g of path = (per cm) * r_g */
        double rg = orc_r_g(sc->mass);
        synch_local q;
        if (r <= sc->r_out) q = synch_at(sc, r, cost);
        for (int k = 0; k < rc->n_rt; ++k) {
            double nu0 = sc->freqs[k] / g, jnu = 0.0, anu = 0.0;
            if (r <= sc->r_out) synch_coeffs_at(&q, nu0, &jnu, &anu);
            double tau = y[N_GEO + 2 * k];
            dy[N_GEO + 2 * k] = anu * rg / g;                                    /* Eq. 30 */
            dy[N_GEO + 2 * k + 1] = jnu / (nu0 * nu0 * nu0) * rg / g * exp(-tau); /* Eq. 31 */
        }
        return;
    }
    double w = sc->theta_width;
    double ne = pow(r, -sc->ne_index) * exp(-cost * cost / (2.0 * w * w));
    double Te = sc->T0 * pow(r, -sc->T_index);
    for (int k = 0; k < rc->n_rt; ++k) {
        double nu0 = sc->freqs[k] / g;
        double jnu = sc->C_norm * ne * ne / sqrt(Te) * exp(-nu0 / Te);
        /* B_nu = 2 nu^3 / (exp(nu/T) - 1); j/B written with expm1 so that it stays
         * finite where exp(nu/T) overflows near the horizon */
        double anu = sc->C_norm * ne * ne / sqrt(Te) * (-expm1(-nu0 / Te)) /
                     (2.0 * nu0 * nu0 * nu0);
        double tau = y[N_GEO + 2 * k];
        dy[N_GEO + 2 * k] = anu / g;                                         /* Eq. 30 */
        dy[N_GEO + 2 * k + 1] = jnu / (nu0 * nu0 * nu0) / g * exp(-tau);     /* Eq. 31 */
    }
}

/* One Cash-Karp step of size h from y (derivative k1 = dy/ds at y): fifth-order
 * solution y5 and embedded error estimate yerr = y5 - y4. */
static void ck_step(const ray_ctx *rc, int n, const double *y, const double *k1, double h,
                    double *y5, double *yerr)
{
    double k[6][N_MAX], ytmp[N_MAX];
    memcpy(k[0], k1, sizeof(double) * n);
    for (int st = 1; st < 6; ++st) {
        for (int i = 0; i < n; ++i) {
            double acc = 0.0;
            for (int j = 0; j < st; ++j) acc += CK_A[st][j] * k[j][i];
            ytmp[i] = y[i] + h * acc;
        }
        derivs(rc, n, ytmp, k[st]);
    }
    for (int i = 0; i < n; ++i) {
        double s5 = 0.0, s4 = 0.0;
        for (int j = 0; j < 6; ++j) {
            s5 += CK_B5[j] * k[j][i];
            s4 += CK_B4[j] * k[j][i];
        }
        y5[i] = y[i] + h * s5;
        yerr[i] = h * (s5 - s4);
    }
}

/* reading: localise the equatorial crossing inside an accepted step by re-taking single
 * Cash-Karp steps of size sigma from the step start and solving cos(theta(sigma)) = 0
 * with Newton's method (d cos(theta)/ds = -sin(theta) dtheta/ds), kept inside the sign
 * bracket by bisection, to |cos(theta)| <= 1e-14 or 60 iterations. */
static void locate_crossing(const ray_ctx *rc, const double *y, const double *k1, double h,
                            double *ycross, double *sigma_out)
{
    double lo = 0.0, hi = h;
    double flo = cos(y[1]);
    double y5[N_MAX], yerr[N_MAX], dy[N_MAX];
    ck_step(rc, N_GEO, y, k1, h, y5, yerr);
    double fhi = cos(y5[1]);
    double sigma = lo - flo * (hi - lo) / (fhi - flo);
    if (!(sigma > lo && sigma < hi)) sigma = 0.5 * (lo + hi);
    for (int it = 0; it < 60; ++it) {
        ck_step(rc, N_GEO, y, k1, sigma, y5, yerr);
        double F = cos(y5[1]);
        if (fabs(F) <= 1e-14) break;
        if ((F > 0.0) == (flo > 0.0)) {
            lo = sigma;
            flo = F;
        } else {
            hi = sigma;
            fhi = F;
        }
        derivs(rc, N_GEO, y5, dy);
        double dF = -sin(y5[1]) * dy[1];
        double next = sigma - F / dF;
        if (!(next > lo && next < hi)) next = 0.5 * (lo + hi);
        if (hi - lo <= 1e-15 * h) break;
        sigma = next;
    }
    memcpy(ycross, y5, sizeof(double) * N_GEO);
    *sigma_out = sigma;
}

/* relative violation of the null condition H = 0, using the separated form
 * 2 Sigma H = Delta p_r^2 + p_th^2 + (L csc - a sin)^2 - ((r^2 + a^2) - a L)^2 / Delta,
 * divided by the sum of the magnitudes of its terms */
static double null_violation(double a, double L, const double *y)
{
    double r = y[0], pr = y[4], pth = y[5];
    double sint = fmax(sin(y[1]), SIN_FLOOR);
    double Delta = r * r - 2.0 * r + a * a;
    double t1 = Delta * pr * pr, t2 = pth * pth;
    double t3 = (L / sint - a * sint) * (L / sint - a * sint);
    double t4 = ((r * r + a * a) - a * L) * ((r * r + a * a) - a * L) / Delta;
    return (t1 + t2 + t3 - t4) / (fabs(t1) + t2 + t3 + fabs(t4));
}

static double carter_q(double a, double L, const double *y)
{
    double sint = fmax(sin(y[1]), SIN_FLOOR);
    double cost = cos(y[1]);
    return y[5] * y[5] + (L * L / (sint * sint) - a * a) * cost * cost; /* Eq. 13 */
}

/*
 * Trace one ray with adaptive Cash-Karp steps and Numerical-Recipes style step control:
 *   yscal_i = |y_i| + |h dy_i/ds| + 1e-30 over the six geodesic components,
 *   errmax = max_i |yerr_i / yscal_i| / rtol,
 *   reject if errmax > 1: h <- max(0.9 h errmax^-1/4, 0.1 h),
 *   accept: h_next = 0.9 h errmax^-1/5 if errmax > 1.89e-4 else 5 h,
 *   and before every step |h| <= hmax_frac * r.
 * Events after every accepted step, in this order: equatorial crossing (thin disk hit
 * stops the ray), horizon r < horizon_factor * r_+, escape (dr/ds > 0 and r > r_start).
 * If path arrays are given, every accepted state is recorded.
 */
static int trace_core(const orc_scene *sc, double alpha, double beta, orc_result *out,
                      int32_t max_pts, double *s_pts, double *y_pts, int32_t *n_pts)
{
    ray_ctx rc;
    rc.sc = sc;
    rc.a = sc->a;
    rc.sgn = (sc->convention == ORC_CONV_LITERAL) ? 1.0 : -1.0;
    rc.r_isco = orc_isco(sc->a);
    rc.r_horizon = orc_horizon(sc->a);
    rc.n_rt = (sc->emitter == ORC_EMIT_TORUS || sc->emitter == ORC_EMIT_CONST ||
               sc->emitter == ORC_EMIT_SYNCH)
                  ? sc->n_freq
                  : 0;
    rc.n = N_GEO + 2 * rc.n_rt;
    rc.r_stop = sc->horizon_factor * rc.r_horizon;
    for (int k = 0; k < rc.n_rt; ++k)
        rc.I_floor[k] = RT_FLOOR_FRAC * source_scale(sc, sc->freqs[k]);

    double y[N_MAX], Q0, L;
    memset(y, 0, sizeof(y));
    orc_init_ray(sc, alpha, beta, y, &L, &Q0, NULL);
    rc.L = L;

    double r_in = (sc->r_in > 0.0) ? sc->r_in : rc.r_isco;
    double r_start = y[0];
    double r_stop = rc.r_stop;

    memset(out, 0, sizeof(*out));
    out->r_cross = out->phi_cross = NAN;
    out->r_hit = out->phi_hit = out->g = NAN;
    out->intensity = 0.0;
    out->L = L;
    out->Q0 = Q0;

    int status = ORC_RUNNING;
    int n_acc = 0, n_rej = 0, n_cross = 0;
    double h = sc->h0, s = 0.0;
    double k1[N_MAX], y5[N_MAX], yerr[N_MAX], yscal[N_GEO + ORC_MAX_FREQ], dy[N_MAX];
    int np = 0;
    if (s_pts && np < max_pts) {
        s_pts[np] = s;
        memcpy(y_pts + (size_t)np * rc.n, y, sizeof(double) * rc.n);
        ++np;
    }

    while (status == ORC_RUNNING) {
        if (n_acc + n_rej >= sc->max_steps) {
            status = ORC_MAXSTEPS;
            break;
        }
        if (h > sc->hmax_frac * y[0]) h = sc->hmax_frac * y[0];
        if (sc->emitter == ORC_EMIT_SPOT) {
            /* reading: no step may carry a ray across the spot unseen, |h| <= (d - 4 r_spot)
             * / 2 (a photon moves at most ~1 in these coordinates per unit affine parameter
             * away from the hole), but not below r_spot / 4 */
            double d;
            orc_spot_region(sc, rc.sgn, y, &d);
            double cap = fmax(0.5 * (d - 4.0 * sc->spot_size), 0.25 * sc->spot_size);
            if (h > cap) h = cap;
        }
        derivs(&rc, rc.n, y, k1);
        for (int i = 0; i < N_GEO; ++i) yscal[i] = fabs(y[i]) + fabs(h * k1[i]) + 1e-30;
        for (int k = 0; k < rc.n_rt; ++k) {
            int iI = N_GEO + 2 * k + 1;
            yscal[N_GEO + k] = fabs(y[iI]) + fabs(h * k1[iI]) + rc.I_floor[k];
        }

        double errmax;
        for (;;) {
            ck_step(&rc, rc.n, y, k1, h, y5, yerr);
            errmax = 0.0;
            int nan_err = 0; /* fmax drops a NaN operand: a NaN component rejects the step */
            for (int i = 0; i < N_GEO; ++i) {
                double v = fabs(yerr[i] / yscal[i]);
                if (isnan(v)) nan_err = 1;
                errmax = fmax(errmax, v);
            }
            if (sc->rt_control == ORC_RT_CONTROLLED) {
                for (int k = 0; k < rc.n_rt; ++k) {
                    int iI = N_GEO + 2 * k + 1;
                    double v = fabs(yerr[iI] / yscal[N_GEO + k]);
                    if (isnan(v)) nan_err = 1;
                    errmax = fmax(errmax, v);
                }
            }
            errmax /= sc->rtol;
            if (nan_err || isnan(errmax)) errmax = INFINITY;
            if (errmax <= 1.0) break;
            ++n_rej;
            h = fmax(0.9 * h * pow(errmax, -0.25), 0.1 * h);
            if (h < 1e-12) {
                status = ORC_NUMERR;
                break;
            }
            if (n_acc + n_rej >= sc->max_steps) {
                status = ORC_MAXSTEPS;
                break;
            }
        }
        if (status != ORC_RUNNING) break;
        ++n_acc;
        double h_next = (errmax > 1.89e-4) ? 0.9 * h * pow(errmax, -0.2) : 5.0 * h;

        /* equatorial crossing */
        if ((cos(y[1]) > 0.0) != (cos(y5[1]) > 0.0)) {
            double yc[N_MAX], sig;
            locate_crossing(&rc, y, k1, h, yc, &sig);
            ++n_cross;
            if (n_cross == 1) {
                out->r_cross = yc[0];
                out->phi_cross = yc[2];
            }
            if ((sc->emitter == ORC_EMIT_THIN_DISK || sc->emitter == ORC_EMIT_NT_DISK) &&
                yc[0] >= r_in && yc[0] <= sc->r_out) {
                status = ORC_DISK_HIT;
                out->r_hit = yc[0];
                out->phi_hit = yc[2];
                out->g = orc_disk_redshift(sc->a, yc[0], L);
                out->intensity = pow(out->g, 4.0) * pow(yc[0], -sc->q_emis);
                if (sc->emitter == ORC_EMIT_NT_DISK) {
                    /* blackbody at T(r) seen at g T (I_nu / nu^3 invariant along the ray) */
                    double T = sc->T0 * pow(orc_nt_flux(sc->a, yc[0]), 0.25);
                    double gT = out->g * T;
                    for (int k = 0; k < sc->n_freq; ++k) {
                        double nu = sc->freqs[k];
                        out->I_nu[k] = 2.0 * nu * nu * nu / expm1(nu / gT);
                    }
                    out->intensity = 2.0 * pow(3.14159265358979323846, 4.0) / 15.0 * pow(gT, 4.0);
                }
                memcpy(y, yc, sizeof(double) * N_GEO);
                s += sig;
                break;
            }
        }

        /* hot spot: first entry into the opaque spot, located by bisection on the size of a
         * single Cash-Karp step from the step start (60 halvings) */
        if (sc->emitter == ORC_EMIT_SPOT && orc_spot_region(sc, rc.sgn, y5, NULL) < 0.0) {
            double lo = 0.0, hi = h, yt[N_MAX], yerr_t[N_MAX];
            for (int it = 0; it < 60; ++it) {
                double mid = 0.5 * (lo + hi);
                ck_step(&rc, N_GEO, y, k1, mid, yt, yerr_t);
                if (orc_spot_region(sc, rc.sgn, yt, NULL) < 0.0)
                    hi = mid;
                else
                    lo = mid;
            }
            ck_step(&rc, N_GEO, y, k1, hi, yt, yerr_t);
            double d;
            orc_spot_region(sc, rc.sgn, yt, &d);
            status = ORC_DISK_HIT;
            out->r_hit = yt[0];
            out->phi_hit = yt[2];
            out->g = spot_redshift(sc, yt[0], yt[1], L);
            /* reading: the spot emits the printed Gaussian profile times a blackbody at T0,
             * seen as I_nu = g^3 I_em(nu / g) = w B_nu(g T0) */
            double w = sc->C_norm * exp(-d * d / (2.0 * sc->spot_size * sc->spot_size));
            double gT = out->g * sc->T0;
            for (int k = 0; k < sc->n_freq; ++k) {
                double nu = sc->freqs[k];
                out->I_nu[k] = (gT > 0.0) ? w * 2.0 * nu * nu * nu / expm1(nu / gT) : 0.0;
            }
            out->intensity = w * 2.0 * pow(3.14159265358979323846, 4.0) / 15.0 * pow(gT, 4.0);
            memcpy(y, yt, sizeof(double) * N_GEO);
            s += hi;
            break;
        }

        memcpy(y, y5, sizeof(double) * rc.n);
        s += h;
        h = h_next;
        if (s_pts && np < max_pts) {
            s_pts[np] = s;
            memcpy(y_pts + (size_t)np * rc.n, y, sizeof(double) * rc.n);
            ++np;
        }

        if (y[0] < r_stop) {
            status = ORC_CAPTURED;
            break;
        }
        derivs(&rc, N_GEO, y, dy);
        if (dy[0] > 0.0 && y[0] > r_start) {
            status = ORC_ESCAPED;
            break;
        }
    }

    out->status = status;
    out->n_acc = n_acc;
    out->n_rej = n_rej;
    out->n_cross = n_cross;
    out->s_end = s;
    memcpy(out->y_end, y, sizeof(double) * N_GEO);
    out->H_end = null_violation(sc->a, L, y);
    out->Q_drift = (carter_q(sc->a, L, y) - Q0) / fmax(fabs(Q0), 1.0);
    for (int k = 0; k < rc.n_rt; ++k) {
        double nu = sc->freqs[k];
        out->tau_nu[k] = y[N_GEO + 2 * k];
        out->I_nu[k] = (sc->emitter == ORC_EMIT_CONST) ? y[N_GEO + 2 * k + 1]
                                                       : nu * nu * nu * y[N_GEO + 2 * k + 1];
    }
    if (n_pts) *n_pts = np;
    return 0;
}

int orc_trace_ray(const orc_scene *sc, double alpha, double beta, orc_result *out)
{
    return trace_core(sc, alpha, beta, out, 0, NULL, NULL, NULL);
}

int orc_trace_path(const orc_scene *sc, double alpha, double beta, int32_t max_pts,
                   double *s_pts, double *y_pts, int32_t *n_pts, orc_result *out)
{
    return trace_core(sc, alpha, beta, out, max_pts, s_pts, y_pts, n_pts);
}

/* Whole image (or the listed pixel indices p = j * n_alpha + i), one ray per pixel. */
int orc_render(const orc_scene *sc, const int64_t *pixels, int64_t n, orc_result *out,
               int32_t n_threads)
{
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 8)
#endif
    for (int64_t q = 0; q < n; ++q) {
        int64_t p = pixels ? pixels[q] : q;
        int32_t i = (int32_t)(p % sc->n_alpha), j = (int32_t)(p / sc->n_alpha);
        double alpha, beta;
        orc_pixel_center(sc, i, j, &alpha, &beta);
        orc_trace_ray(sc, alpha, beta, &out[q]);
    }
    return 0;
}

/* Explicit ray list rays[n][4] = (alpha, beta, a, cos i); the other scene fields from proto. */
int orc_trace_list(const orc_scene *proto, const double *rays, int64_t n, orc_result *out,
                   int32_t n_threads)
{
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 8)
#endif
    for (int64_t q = 0; q < n; ++q) {
        orc_scene sc = *proto;
        sc.a = rays[4 * q + 2];
        sc.theta_obs = acos(rays[4 * q + 3]);
        orc_trace_ray(&sc, rays[4 * q], rays[4 * q + 1], &out[q]);
    }
    return 0;
}

/* reading of "tau about 1 at the middle frequency": choose the emissivity normalisation C
 * so that a static, flat-space path along the equator from r_+ to r_outer has optical
 * depth 1 at frequency nu:  C = 1 / int alpha_nu(r, pi/2)|_{C=1} dr.
 * Composite Simpson rule in u = ln r with 200000 intervals. */
double orc_torus_norm(double a, double nu, double ne_index, double T0, double T_index,
                      double r_outer)
{
    const int n = 200000;
    double u0 = log(orc_horizon(a)), u1 = log(r_outer);
    double du = (u1 - u0) / n, sum = 0.0;
    for (int i = 0; i <= n; ++i) {
        double r = exp(u0 + i * du);
        double ne = pow(r, -ne_index);
        double Te = T0 * pow(r, -T_index);
        double anu = ne * ne / sqrt(Te) * (-expm1(-nu / Te)) / (2.0 * nu * nu * nu);
        double wgt = (i == 0 || i == n) ? 1.0 : ((i % 2) ? 4.0 : 2.0);
        sum += wgt * anu * r; /* dr = r du */
    }
    return 1.0 / (sum * du / 3.0);
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
