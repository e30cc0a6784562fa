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
