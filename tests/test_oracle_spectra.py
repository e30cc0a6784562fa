"""Pins of the spectra / light-curve oracle (oracle/spectra.py, Section 4.4): the image
integral of a constant image, of the Schwarzschild shadow (solid angle 27 pi / r_obs^2 of
the capture region, Section 4.2), and the trapezoid rule over frequency on closed forms."""
import math

import numpy as np

from oracle import spectra as S
from paper_1601_02063_gb300 import workloads as W


def test_constant_image_flux_is_window_solid_angle():
    sc = W.scene(n_alpha=37, n_beta=23, alpha_min=-7.0, alpha_max=11.0, beta_min=-3.0,
                 beta_max=5.0, r_obs=500.0)
    img = np.full((1, 37 * 23), 2.5)
    F = S.image_flux(sc, img)
    assert math.isclose(F[0], 2.5 * 18.0 * 8.0 / 500.0 ** 2, rel_tol=1e-14)


def test_schwarzschild_shadow_solid_angle(orc):
    """Capture mask integrated over the image = solid angle of the shadow, a disk of radius
    3 sqrt(3) M on the image plane at large r_obs (pixelisation error ~ perimeter x pixel)."""
    n = 160
    sc = W.scene(a=0.0, theta_obs=math.radians(60), n_alpha=n, n_beta=n, alpha_min=-7.0,
                 alpha_max=7.0, beta_min=-7.0, beta_max=7.0, emitter="none", r_obs=1000.0)
    res = orc.render(sc)
    mask = (res["status"] == 2).astype(np.float64)[None, :]
    F = S.image_flux(sc, mask)[0]
    exact = 27.0 * math.pi / sc["r_obs"] ** 2
    pix = 14.0 / n
    assert abs(F - exact) < 2.0 * math.pi * math.sqrt(27.0) * pix / sc["r_obs"] ** 2, (F, exact)


def test_light_curve_trapezoid_closed_forms():
    sc = W.torus_512()
    nu = np.asarray(sc["freqs"])
    # linear F(nu): the trapezoid rule is exact
    F = 3.0 + 2.0 * nu
    exact = 3.0 * (nu[-1] - nu[0]) + (nu[-1] ** 2 - nu[0] ** 2)
    assert math.isclose(S.light_curve_point(sc, F), exact, rel_tol=1e-14)
    # F = nu^2 on a fine grid: error of the composite rule is sum h^3 / 6
    sc2 = dict(sc, freqs=list(np.linspace(0.5, 2.0, 8)))
    nu2 = np.asarray(sc2["freqs"])
    h = np.diff(nu2)
    got = S.light_curve_point(sc2, nu2 ** 2)
    exact2 = (nu2[-1] ** 3 - nu2[0] ** 3) / 3.0
    assert math.isclose(got - exact2, float(np.sum(h ** 3)) / 6.0, rel_tol=1e-9)
    # one plane: F itself
    assert S.light_curve_point(W.scene(), np.array([4.25])) == 4.25


# ---- Novikov-Thorne disk (Section 4.3): the oracle's Page-Thorne flux ------------------------

def test_page_thorne_radiative_efficiency(orc):
    """Energy radiated to infinity by both faces, int 4 pi r F E dr = Mdot (1 - E_ms): the
    binding energy of the innermost stable orbit (Page & Thorne 1974), with f = 1.5 r Fhat."""
    from scipy.integrate import quad
    for a in (0.0, 0.5, 0.9, 0.998):
        rms = orc.isco(a)
        g = lambda r: 1.5 * r * orc.nt_flux(a, r) * orc.circ_E(a, r)
        tot = quad(g, rms, 50.0, limit=200, epsrel=1e-10)[0]
        tot += quad(lambda u: g(math.exp(u)) * math.exp(u), math.log(50.0), math.log(1e7),
                    limit=200, epsrel=1e-10)[0]
        tot += 1.5e-7  # tail beyond 1e7: f -> 1.5 / r^2
        assert abs(tot - (1.0 - orc.circ_E(a, rms))) < 2e-7, (a, tot, 1.0 - orc.circ_E(a, rms))


def test_page_thorne_boundary_and_newtonian_limit(orc):
    for a in (0.0, 0.9):
        rms = orc.isco(a)
        assert orc.nt_flux(a, rms) == 0.0 and orc.nt_flux(a, 0.9 * rms) == 0.0
        # zero torque at r_ms: F grows like (r - r_ms)^2
        e = 1e-3
        ratio = orc.nt_flux(a, rms * (1 + e)) / orc.nt_flux(a, rms * (1 + e / 2))
        assert abs(ratio - 4.0) < 0.02, ratio
    # far out the Newtonian disk: 8 pi F / 3 = r^-3 (1 - C / sqrt(r) + D / r + ...), the
    # inner boundary entering through the constants: c(r) = (1 - F r^3) sqrt(r) = C - D /
    # sqrt(r) converges, its steps shrinking by sqrt(10) per decade of r
    for a in (0.0, 0.9):
        c = [(1.0 - orc.nt_flux(a, r) * r ** 3) * math.sqrt(r) for r in (1e5, 1e6, 1e7)]
        assert 0.0 < c[2] < 10.0
        assert abs((c[0] - c[1]) / (c[1] - c[2]) - math.sqrt(10.0)) < 0.1, c


def test_nt_disk_pixel_is_planck_at_gT(orc):
    """A ray hitting the Novikov-Thorne disk carries B_nu(g T(r)) at every frequency."""
    sc = W.scene(emitter="nt_disk", freqs=[0.1, 0.3, 1.0, 3.0], T0=1.0, r_out=30.0)
    r = orc.trace_ray(sc, 6.0, 2.0)
    assert r.status == 3
    T = sc["T0"] * orc.nt_flux(sc["a"], r.r_hit) ** 0.25
    for k, nu in enumerate(sc["freqs"]):
        planck = 2.0 * nu ** 3 / math.expm1(nu / (r.g * T))
        assert math.isclose(r.I_nu[k], planck, rel_tol=1e-14)
    assert math.isclose(r.intensity, 2 * math.pi ** 4 / 15 * (r.g * T) ** 4, rel_tol=1e-14)
