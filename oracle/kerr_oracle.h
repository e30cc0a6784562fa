/*
 * kerr_oracle.h -- plain, slow FP64 CPU oracle for backward ray tracing and
 * radiative transfer in Kerr spacetime (Pu, Yun, Younsi & Yoon 2016, "Odyssey").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may include, link or
 * call this code: only the test suite, the smoke check and the CPU-baseline leg
 * of the benchmark use it.  It shares no source, header, table or helper with
 * the CUDA library; the two sides meet only through the scene numbers a caller
 * passes to each.
 *
 * Units: G = c = M = 1 (Section 2).  The traced photon has E = 1.  The synchrotron shell
 * (Section 4.5) evaluates its coefficients in CGS and scales path lengths by r_g.
 *
 * Pins of the synchrotron shell (tests/test_oracle_synch.py): K_2 against a library Bessel
 * routine; the emissivity's frequency integral against the synchrotron power of a
 * Maxwell-Juttner gas (Thomson cross-section, to the fit's few per cent); Kirchhoff's law;
 * the optically thick limit of an isothermal shell (Rayleigh-Jeans intensity, redshifted).
 */
#ifndef KERR_ORACLE_H
#define KERR_ORACLE_H

#include <stdint.h>

#define ORC_MAX_FREQ 8

/* ray status after tracing */
#define ORC_RUNNING 0
#define ORC_ESCAPED 1
#define ORC_CAPTURED 2
#define ORC_DISK_HIT 3
#define ORC_MAXSTEPS 4
#define ORC_NUMERR 5

/* emission models */
#define ORC_EMIT_NONE 0      /* grid projection / shadow: geodesics only        */
#define ORC_EMIT_THIN_DISK 1 /* opaque Keplerian equatorial disk, I = g^4 r^-q  */
#define ORC_EMIT_TORUS 2     /* analytic thermal torus, RT Eqs. 30-31           */
#define ORC_EMIT_CONST 3     /* test medium: dtau/ds = kappa, dI/ds = eps e^-tau */
#define ORC_EMIT_NT_DISK 4   /* Novikov-Thorne disk: blackbody at T0 (8 pi F / 3)^1/4 */
#define ORC_EMIT_SYNCH 5     /* Keplerian shell, thermal synchrotron (Section 4.5, CGS) */
#define ORC_EMIT_SPOT 6      /* optically thick Keplerian hot spot (Section 4.4)       */

/* step control of the transfer components */
#define ORC_RT_CONTROLLED 0 /* invariant intensities in the error norm (default)        */
#define ORC_RT_RIDE 1       /* geodesic components only; tau and I ride on its steps   */

/* sign conventions for the traced photon (see the direction reading in the design notes) */
#define ORC_CONV_PHYSICAL 0 /* real outgoing photon, traced back in affine time */
#define ORC_CONV_LITERAL 1  /* future-directed inward photon, Eqs. 24-26 as printed */

typedef struct {
    double a, r_obs, theta_obs, phi_obs;
    double alpha_min, alpha_max, beta_min, beta_max;
    int32_t n_alpha, n_beta;
    int32_t emitter;
    int32_t n_freq;
    double freqs[ORC_MAX_FREQ];
    double r_in, r_out, q_emis;        /* thin disk; r_in <= 0 means r_ISCO(a) */
    double ne_index, theta_width;      /* torus: n_e = r^-ne_index exp(-cos^2/(2 w^2)) */
    double T0, T_index;                /* torus: T_e = T0 r^-T_index */
    double C_norm;                     /* torus emissivity normalisation;
                                          const medium: kappa = C_norm, eps = T0 */
    double rtol, h0, hmax_frac, horizon_factor;
    int32_t max_steps;
    int32_t convention;
    /* synchrotron shell: n_e = n_e0 r^-ne_index exp(-cos^2/(2 w^2)) [cm^-3],
     * Theta_e = T0 r^-T_index, B^2 / 8 pi = n_e m_p c^2 / (6 beta_B r) [G], black-hole mass
     * [solar masses] (lengths in r_g = G M / c^2), freqs in Hz, emission for r <= r_out */
    double n_e0, beta_B, mass;
    /* hot spot: centre on the equatorial circular orbit of radius spot_r (<= 0: r_ISCO),
     * azimuth spot_phase + Omega t; Gaussian width spot_size (r_spot); the image is the one
     * seen at observer time t_obs; emitted I_nu = C_norm exp(-d^2 / (2 r_spot^2)) B_nu(T0) */
    double spot_r, spot_size, spot_phase, t_obs;
    /* step control of the transfer equation (torus, shell, test medium): ORC_RT_CONTROLLED
     * puts the invariant intensities into the error norm; ORC_RT_RIDE leaves them out (they
     * ride on the geodesic's steps) */
    int32_t rt_control;
    int32_t pad_;
} orc_scene;

typedef struct {
    int32_t status, n_acc, n_rej, n_cross;
    double r_cross, phi_cross;         /* first equatorial crossing (NaN if none) */
    double r_hit, phi_hit, g, intensity; /* thin-disk hit (NaN / 0 otherwise)      */
    double H_end, Q_drift;             /* relative null violation, relative Q drift */
    double s_end;                      /* affine length traced                     */
    double L, Q0;                      /* constants of motion of the ray (E = 1)   */
    double y_end[6];                   /* r, theta, phi, t, p_r, p_theta at the end */
    double I_nu[ORC_MAX_FREQ];         /* observed I_nu = nu^3 * invariant I      */
    double tau_nu[ORC_MAX_FREQ];
} orc_result;

double orc_horizon(double a);
double orc_isco(double a);
void orc_ck_tableau(double c[6], double a[36], double b5[6], double b4[6]);
void orc_pixel_center(const orc_scene *sc, int32_t i, int32_t j, double *alpha, double *beta);
void orc_observer_point(const orc_scene *sc, double alpha, double beta, double xyz[3]);
void orc_init_ray(const orc_scene *sc, double alpha, double beta, double y0[6], double *L,
                  double *Q, double vin[3]);
void orc_geodesic_rhs(double a, double L, const double y[6], double f[6]);
double orc_disk_redshift(double a, double r, double L);
/* Page-Thorne flux of one face of the Novikov-Thorne disk for unit accretion rate, as
 * 8 pi F(r) / 3, by quadrature of the Page & Thorne (1974) integral; 0 inside r_ISCO. */
double orc_nt_flux(double a, double r);
/* Specific energy and angular momentum of prograde circular equatorial orbits (E = 1
 * normalisation of the photon does not enter; Bardeen, Press & Teukolsky 1972). */
double orc_circ_E(double a, double r);
double orc_circ_L(double a, double r);
/* Thermal synchrotron (Section 4.5): K_2 by quadrature of its integral definition, the
 * gravitational radius in cm, and the emission / absorption coefficients in the fluid frame
 * (CGS; j per steradian) at BL position (r, cos theta) and local frequency nu0 [Hz]. */
double orc_bessel_k2(double x);
double orc_r_g(double mass);
void orc_synch_coeffs(const orc_scene *sc, double r, double cost, double nu0, double *j,
                      double *alpha);
/* Hot spot (Section 4.4): the region function max(d - 4 r_spot, -z) at state y (t = y[3])
 * for the traced direction sign sgn, and the spot centre's orbital angular velocity. */
double orc_spot_region(const orc_scene *sc, double sgn, const double y[6], double *d);
double orc_spot_omega(const orc_scene *sc);
double orc_torus_norm(double a, double nu, double ne_index, double T0, double T_index,
                      double r_outer);
int orc_trace_ray(const orc_scene *sc, double alpha, double beta, orc_result *out);
int orc_trace_path(const orc_scene *sc, double alpha, double beta, int32_t max_pts,
                   double *s_pts, double *y_pts, int32_t *n_pts, orc_result *out);
int orc_render(const orc_scene *sc, const int64_t *pixels, int64_t n, orc_result *out,
               int32_t n_threads);
int orc_trace_list(const orc_scene *proto, const double *rays, int64_t n, orc_result *out,
                   int32_t n_threads);
int orc_max_threads(void);

#endif
