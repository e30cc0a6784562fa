"""Pins of the oracle's whole integrator against results fixed by general relativity and
the paper: capture boundaries (Section 4.2), weak-field deflection, the first
equatorial crossing from Carter's separated equations, redshift of the thin disk
(Section 4.3, Figure 5), conservation of H and Q (Section 2.1) and the radiative
transfer solution (Section 2.3)."""
import json
import math
import os

import numpy as np
import pytest
from scipy.integrate import quad
from scipy.optimize import brentq

from paper_1601_02063_gb300 import workloads as W

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
ESCAPED, CAPTURED, DISK_HIT = 1, 2, 3


def _boundary_rho(orc, scene, psis, lo=0.5, hi=12.0, iters=44):
    """Bisect, along image-plane directions psi, the radius rho where rays switch from
    captured (inside) to escaped (outside).  Returns rho per psi."""
    psis = np.asarray(psis, dtype=float)
    lo = np.full(len(psis), lo)
    hi = np.full(len(psis), hi)
    cosi = math.cos(scene["theta_obs"])
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        rays = np.stack([mid * np.cos(psis), mid * np.sin(psis), np.full_like(mid, scene["a"]),
                         np.full_like(mid, cosi)], axis=1)
        st = orc.trace_list(scene, rays)["status"]
        assert np.all((st == CAPTURED) | (st == ESCAPED)), st
        inside = st == CAPTURED
        lo = np.where(inside, mid, lo)
        hi = np.where(inside, hi, mid)
    return 0.5 * (lo + hi)


def _constants(orc, scene, alpha, beta):
    _, L, Q, _ = orc.init_ray(scene, alpha, beta)
    return L, Q


def test_schwarzschild_capture_radius(orc):
    """a = 0: rays are captured iff b = sqrt(lambda^2 + eta) < 3 sqrt(3) M, i.e. the shadow
    is alpha^2 + beta^2 = 27 for a distant observer (Section 4.2)."""
    b2 = GOLDEN["schwarzschild_shadow_alpha2_plus_beta2"]["value"]
    sc = W.scene(a=0.0, theta_obs=math.radians(60.0), emitter="none", rtol=1e-10)
    psis = np.linspace(0.1, 2 * math.pi, 7, endpoint=False)
    rho = _boundary_rho(orc, sc, psis)
    for p, r in zip(psis, rho):
        L, Q = _constants(orc, sc, r * math.cos(p), r * math.sin(p))
        assert abs(math.sqrt(L * L + Q) - math.sqrt(b2)) < 1e-6


def _bardeen_curve(a):
    """Spherical photon orbits of Kerr (Bardeen 1973): constants (xi, eta) of the orbit at
    radius r, for r between the prograde and retrograde equatorial photon orbits."""
    xi = lambda r: (r * r * (3 - r) - a * a * (r + 1)) / (a * (r - 1))
    eta = lambda r: r ** 3 * (4 * a * a - r * (r - 3) ** 2) / (a * a * (r - 1) ** 2)
    r_pro = 2 * (1 + math.cos(2.0 / 3.0 * math.acos(-a)))
    r_ret = 2 * (1 + math.cos(2.0 / 3.0 * math.acos(a)))
    return xi, eta, r_pro, r_ret


@pytest.mark.parametrize("a", [0.5, 0.9, 0.998])
@pytest.mark.parametrize("inc", [30.0, 60.0, 90.0])
def test_kerr_shadow_boundary_is_bardeen_curve(orc, a, inc):
    """The capture boundary consists of rays whose constants (lambda, eta) = (L, Q) are those
    of a spherical photon orbit; the shadow is displaced toward +alpha (prograde photons,
    L > 0, arrive on the alpha < 0 side and skim closer)."""
    sc = W.scene(a=a, theta_obs=math.radians(inc), emitter="none", rtol=1e-10,
                 horizon_factor=1.0005)
    xi, eta, r_pro, r_ret = _bardeen_curve(a)
    psis = np.array([0.05, 0.8, 1.7, 2.6, math.pi - 0.05, 4.0, 5.0])
    rho = _boundary_rho(orc, sc, psis, lo=0.3, hi=10.0)
    for p, r in zip(psis, rho):
        L, Q = _constants(orc, sc, r * math.cos(p), r * math.sin(p))
        rc = brentq(lambda x: xi(x) - L, r_pro * (1 + 1e-12), r_ret * (1 - 1e-12))
        assert abs(eta(rc) - Q) < 2e-5 * max(1.0, abs(Q)), (p, L, Q, eta(rc))
    assert rho[0] > rho[4]


def test_kerr_shadow_equatorial_endpoints(orc):
    """Edge-on (i = 90 deg) the boundary on the beta = 0 line is the pair of equatorial
    circular photon orbits: lambda = xi(r_pro) on the alpha < 0 side and xi(r_ret) on the
    alpha > 0 side."""
    a = 0.9
    sc = W.scene(a=a, theta_obs=math.radians(90.0), emitter="none", rtol=1e-10)
    xi, _, r_pro, r_ret = _bardeen_curve(a)
    assert abs(r_pro - 1.5578546) < 1e-6 and abs(r_ret - 3.9102679) < 1e-6
    rho = _boundary_rho(orc, sc, [math.pi, 0.0], lo=0.3, hi=10.0, iters=46)
    L_left, _ = _constants(orc, sc, -rho[0], 0.0)
    L_right, _ = _constants(orc, sc, rho[1], 0.0)
    assert abs(L_left - xi(r_pro)) < 1e-5 and abs(xi(r_pro) - 2.8444) < 1e-4
    assert abs(L_right - xi(r_ret)) < 1e-5 and abs(xi(r_ret) + 6.8323) < 1e-4


def test_literal_convention_mirrors_the_shadow(orc):
    """Read literally (inward velocity, p_t = -E), the traced photon is the mirror image
    of the physical one: the shadow is displaced toward -alpha instead of +alpha."""
    kw = dict(a=0.9, theta_obs=math.radians(90.0), emitter="none", rtol=1e-9)
    rho_p = _boundary_rho(orc, W.scene(**kw), [0.0, math.pi], lo=0.3, hi=10.0, iters=30)
    rho_l = _boundary_rho(orc, W.scene(convention="literal", **kw), [0.0, math.pi],
                          lo=0.3, hi=10.0, iters=30)
    assert rho_p[0] > rho_p[1] and rho_l[0] < rho_l[1]
    assert abs(rho_p[0] - rho_l[1]) < 1e-6 and abs(rho_p[1] - rho_l[0]) < 1e-6


@pytest.mark.parametrize("b", [1.0e2, 1.0e3, 1.0e4])
def test_weak_field_deflection(orc, b):
    """a = 0, equatorial ray from r_obs = 1e6: the total change in phi equals the orbit
    integral  int du / sqrt(b^-2 - u^2 (1 - 2u))  (u = 1/r) between the actual end radii and
    the turning point, and approaches pi + 4/b + (15 pi/4)/b^2 + (128/3)/b^3 from r = infinity."""
    sc = W.scene(a=0.0, r_obs=1.0e6, theta_obs=math.pi / 2, emitter="none", rtol=1e-11)
    res = orc.trace_ray(sc, b, 0.0)
    assert res.status == ESCAPED
    y0, L, _, _ = orc.init_ray(sc, b, 0.0)
    bb = abs(L)
    umax = brentq(lambda u: bb ** -2 - u * u * (1 - 2 * u), 0.0, 2.0 / bb, xtol=1e-16)

    def leg(u0):
        # substitution u = umax (1 - t^2) removes the inverse square root at the turning point
        f = lambda t: 2 * umax * t / math.sqrt(bb ** -2 - (umax * (1 - t * t)) ** 2
                                               * (1 - 2 * umax * (1 - t * t)))
        return quad(f, 0.0, math.sqrt(1 - u0 / umax), epsabs=0, epsrel=1e-13, limit=200)[0]

    dphi = leg(1.0 / y0[0]) + leg(1.0 / res.y_end[0])
    assert abs(abs(res.y_end[2] - y0[2]) - dphi) < 1e-9
    # asymptotic series check (finite observer distance changes it by O(b / r_obs))
    series = math.pi + 4 / bb + 15 * math.pi / 4 / bb ** 2 + 128 / 3 / bb ** 3
    full = 2 * leg(0.0)
    assert abs(full - series) < 200 / bb ** 4 + 1e-12


def test_direct_crossing_radius_from_carter_separation(orc):
    """For rays that reach the equator before any radial or polar turning point, Mino-time
    separation gives  int_{r_c}^{r_0} dr / sqrt(R(r)) = int_{theta_0}^{pi/2} dtheta / sqrt(Theta)
    with R = ((r^2 + a^2) - a L)^2 - Delta (Q + (L - a)^2), Theta = Q + a^2 cos^2 - L^2 cot^2.
    The crossing radius solved from it matches the integrator's first crossing."""
    a = 0.9
    sc = W.scene(a=a, theta_obs=math.radians(60.0), emitter="none", rtol=1e-11)
    checked = 0
    for alpha, beta in [(2.0, -6.0), (-5.0, -8.0), (8.0, -3.0), (-9.0, -12.0), (0.7, -4.5),
                        (12.0, -14.0)]:
        y0, L, Q, _ = orc.init_ray(sc, alpha, beta)
        res = orc.trace_ray(sc, alpha, beta)
        r0, th0 = y0[0], y0[1]
        R = lambda r: ((r * r + a * a) - a * L) ** 2 - (r * r - 2 * r + a * a) * (Q + (L - a) ** 2)
        Th = lambda t: Q + a * a * math.cos(t) ** 2 - L * L / math.tan(t) ** 2
        ths = np.linspace(th0, math.pi / 2, 400)
        if not all(Th(t) > 0 for t in ths):
            continue
        G = quad(lambda t: 1 / math.sqrt(Th(t)), th0, math.pi / 2, epsabs=0, epsrel=1e-13,
                 limit=200)[0]
        I = lambda rc: quad(lambda r: 1 / math.sqrt(R(r)), rc, r0, epsabs=0, epsrel=1e-13,
                            limit=400, points=[min(r0, 50.0)])[0]
        # lowest radius reachable without a radial turning point
        rs = np.geomspace(r0, 1.0 + math.sqrt(1 - a * a), 20000)
        bad = np.nonzero([R(r) <= 0 for r in rs])[0]
        r_lo = (rs[bad[0] - 1] if len(bad) else rs[-1]) * (1 + 1e-9)
        if I(r_lo) < G:
            continue  # the ray turns in r before it reaches the equator
        rc = brentq(lambda x: I(x) - G, r_lo, r0 - 1, xtol=1e-14)
        assert abs(res.r_cross - rc) < 1e-9 * rc, (alpha, beta, res.r_cross, rc)
        checked += 1
    assert checked >= 4


def test_face_on_schwarzschild_disk_redshift(orc):
    """Face-on (i = 0) around a = 0 every ray has L = 0, so g = 1/u^t = sqrt(1 - 3M/r) at the
    disk radius where it lands."""
    sc = W.scene(a=0.0, theta_obs=0.0, n_alpha=24, n_beta=24, r_in=6.0, r_out=50.0,
                 alpha_min=-40, alpha_max=40, beta_min=-40, beta_max=40)
    res = orc.render(sc)
    hit = res["status"] == DISK_HIT
    assert hit.sum() > 200
    g_exact = np.sqrt(1 - 3 / res["r_hit"][hit])
    assert np.max(np.abs(res["g"][hit] - g_exact)) < 1e-12


def test_thin_disk_redshift_figure(orc):
    """Section 4.3, Figure 5: a = 0, cos(i) = 0.25, disk r_ISCO..50 M: the approaching
    (alpha < 0) side is blueshifted, the receding side redshifted; the directly seen disk
    spans the figure's contour range of g and of radius."""
    fig = GOLDEN["thin_disk_redshift_figure"]
    sc = W.scene(a=fig["a"], theta_obs=math.acos(fig["cos_theta_obs"]), r_out=fig["r_out"],
                 n_alpha=64, n_beta=32, alpha_min=-55, alpha_max=55, beta_min=-30, beta_max=30)
    res = orc.render(sc)
    hit = res["status"] == DISK_HIT
    g = res["g"].reshape(32, 64)
    alpha = np.linspace(-55, 55, 64, endpoint=False) + 110 / 128
    left = hit.reshape(32, 64) & (alpha < -8)[None, :]
    right = hit.reshape(32, 64) & (alpha > 8)[None, :]
    assert np.median(g[left]) > 1.0 > np.median(g[right])
    lo, hi = fig["gamma_contours"]
    assert res["g"][hit].min() < lo + 0.05 and res["g"][hit].max() > hi - 0.05
    assert res["r_hit"][hit].min() >= orc.isco(0.0) - 1e-12
    assert res["r_hit"][hit].max() <= fig["r_out"]


def test_conservation_on_thin_disk_image(orc):
    """E and L are exact constants in this formulation; H = 0 and Carter's Q must be kept by
    the integrator: relative violations <= 1e-6 on every ray at rtol 1e-8."""
    res = orc.render(W.thin_disk_64())
    assert np.max(np.abs(res["H_end"])) < 1e-6
    assert np.max(np.abs(res["Q_drift"])) < 1e-6
    st = np.bincount(res["status"], minlength=6)
    assert st[ESCAPED] > 0 and st[CAPTURED] > 0 and st[DISK_HIT] > 0
    assert st[4] == 0 and st[5] == 0


def test_isco_bounds_disk_hits(orc):
    res = orc.render(W.thin_disk_64())
    hit = res["status"] == DISK_HIT
    assert res["r_hit"][hit].min() >= orc.isco(0.9) and res["r_hit"][hit].max() <= 20.0


def test_constant_medium_closed_form(orc):
    """Eqs. 30-31 with constant coefficients dtau/ds = kappa, dI/ds = eps exp(-tau) integrate to
    tau = kappa s, I = (eps / kappa)(1 - exp(-kappa s)) over the traced affine length s
    (escaping rays: the medium fills the whole path).  Riding on the geodesic's steps
    (outside the error norm) the intensity's error is the fifth-order truncation in kappa h:
    doubling kappa multiplies it by about 2^5.  Under the step control it stays below the
    tolerance at both opacities (here the geodesic's own steps are short enough)."""
    eps = 0.7
    rays = [(-14.0, 9.0), (10.0, 3.0), (12.0, -8.0)]
    for mode in ("ride", "controlled"):
        errs = {}
        for kappa in (1e-3, 2e-3):
            sc = W.scene(emitter="const", freqs=[1.0, 2.0], C_norm=kappa, T0=eps,
                         rt_control=mode)
            errs[kappa] = []
            for alpha, beta in rays:
                res = orc.trace_ray(sc, alpha, beta)
                assert res.status == 1  # escaped
                s = res.s_end
                assert abs(res.tau_nu[0] - kappa * s) < 1e-13 * kappa * s
                expect = eps / kappa * (-math.expm1(-kappa * s))
                errs[kappa].append(abs(res.I_nu[1] - expect) / expect)
        if mode == "ride":
            assert max(errs[1e-3]) < 1e-10
            ratio = np.array(errs[2e-3]) / np.array(errs[1e-3])
            assert np.all((ratio > 16) & (ratio < 128)), ratio
            ride = errs
        else:
            assert max(errs[1e-3] + errs[2e-3]) < 1e-9, errs
            assert max(errs[2e-3]) <= max(ride[2e-3]), (errs, ride)


def test_medium_ends_at_the_stopping_radius(orc):
    """A captured ray stops at the end of the first step inside r_stop = 1.01 r_+, at a radius
    that depends on the step sequence; the medium ends at r_stop, so the optical depth of a
    constant medium is kappa times the affine length to r_stop alone, whatever the
    tolerance.  That length comes from a separate trace of the geodesic alone (no medium) at
    rtol 1e-12: its recorded points, linear in r across the last (1e-4 long) step.  The step
    that crosses r_stop carries a kink of the integrand, resolved by the intensity's step
    control to the tolerance's level."""
    kappa, eps = 1e-3, 0.7
    sc = W.scene(emitter="const", freqs=[1.0], C_norm=kappa, T0=eps)
    r_stop = 1.01 * orc.horizon(0.9)
    s_pts, y_pts, _ = orc.trace_path(dict(sc, emitter="none", freqs=[], rtol=1e-12), 1.0, 1.0)
    inside = np.nonzero(y_pts[:, 0] < r_stop)[0][0]
    s0, s1 = s_pts[inside - 1], s_pts[inside]
    r0, r1 = y_pts[inside - 1, 0], y_pts[inside, 0]
    assert s1 - s0 < 1e-3
    s_stop = s0 + (r0 - r_stop) / (r0 - r1) * (s1 - s0)
    tau_stop = kappa * s_stop
    I_stop = eps / kappa * (-math.expm1(-tau_stop))
    for rtol in (1e-8, 1e-10):
        res = orc.trace_ray(dict(sc, rtol=rtol), 1.0, 1.0)
        assert res.status == 2  # captured
        assert res.s_end > s_stop  # the last step ends inside r_stop ...
        assert abs(res.tau_nu[0] - tau_stop) < 1e-8 * tau_stop  # ... the medium does not
        assert abs(res.I_nu[0] - I_stop) < 1e-8 * I_stop


def _torus_sources(a, L, r, th, nu, C):
    """Emission and absorption of the analytic torus at (r, theta), computed from the
    configuration's definitions with the fluid four-velocity normalised numerically."""
    s, c = max(math.sin(th), 1e-8), math.cos(th)
    Sig, Del = r * r + a * a * c * c, r * r - 2 * r + a * a
    gtt = -(1 - 2 * r / Sig)
    gtp = -2 * a * r * s * s / Sig
    gpp = ((r * r + a * a) ** 2 - a * a * Del * s * s) * s * s / Sig
    r_isco = 3 + math.sqrt(3 * a * a + (1 + (1 - a * a) ** (1 / 3) * ((1 + a) ** (1 / 3)
                                                                        + (1 - a) ** (1 / 3))) ** 2)
    z1 = 1 + (1 - a * a) ** (1 / 3) * ((1 + a) ** (1 / 3) + (1 - a) ** (1 / 3))
    r_isco -= math.sqrt((3 - z1) * (3 + z1 + 2 * math.sqrt(3 * a * a + z1 * z1)))
    Om = 1 / (r ** 1.5 + a)
    N = gtt + 2 * gtp * Om + gpp * Om * Om
    if not (r >= r_isco and N < 0):
        Om = -gtp / gpp
        N = gtt + 2 * gtp * Om + gpp * Om * Om
    ut = 1 / math.sqrt(-N)
    g = 1 / (ut * (1 - Om * L))
    ne = r ** -1.5 * math.exp(-c * c / (2 * 0.3 ** 2))
    T = 10 * r ** -0.84
    nu0 = nu / g
    j = C * ne * ne / math.sqrt(T) * math.exp(-nu0 / T)
    alpha_abs = j * math.expm1(nu0 / T) / (2 * nu0 ** 3) if nu0 / T < 700 else 0.0
    return g, j, alpha_abs, nu0


def test_torus_radiative_transfer_formal_solution(orc):
    """Section 2.3: along the recorded path, tau(s) = int alpha_0 / g ds (Eq. 29 with
    -k.u = 1/g) and the formal solution (Eq. 28, no background) I = int S e^-tau dtau must
    equal what the integrator carried as extra components (Eqs. 30-31)."""
    a = 0.94
    C = orc.torus_norm(a)
    sc = W.scene(a=a, theta_obs=math.radians(30.0), emitter="torus", freqs=[0.5, 1.0, 2.0],
                 C_norm=C, hmax_frac=0.004, rtol=1e-10)
    for alpha, beta in [(6.0, 2.0), (-3.0, -9.0)]:
        s, y, res = orc.trace_path(sc, alpha, beta)
        L = res.L
        for k, nu in enumerate([0.5, 1.0, 2.0]):
            vals = np.array([_torus_sources(a, L, yy[0], yy[1], nu, C) for yy in y])
            g, j, al, nu0 = vals.T
            dtau = al / g
            tau = np.concatenate([[0.0], np.cumsum(0.5 * (dtau[1:] + dtau[:-1]) * np.diff(s))])
            # the integrator's own tau along the path agrees with the quadrature
            assert abs(tau[-1] - res.tau_nu[k]) < 2e-4 * max(res.tau_nu[k], 1e-3)
            assert np.max(np.abs(tau - y[:, 6 + 2 * k])) < 2e-4 * max(res.tau_nu[k], 1e-3)
            # Eq. 28 integrated in tau with the source function S = eta / chi, expressed
            # back along s: dI = (j / nu0^3) / g e^-tau ds
            integrand = j / nu0 ** 3 / g * np.exp(-tau)
            I_inv = np.sum(0.5 * (integrand[1:] + integrand[:-1]) * np.diff(s))
            assert abs(nu ** 3 * I_inv - res.I_nu[k]) < 2e-4 * res.I_nu[k]


@pytest.mark.parametrize("emitter", ["torus", "synch"])
def test_intensities_converge_under_the_step_control(orc, emitter):
    """The transfer equation's intensities are part of the error norm: the image then
    converges with the tolerance pixel by pixel (rtol 1e-8 against 1e-10 within 2e-6 of
    each pixel, or of 1e-3 of the image's brightest pixel for dark ones).  Riding on the
    geodesic's steps instead, the same two tolerances differ by up to ~1e-2 on the torus's
    shadow and the inner shell, where the emission varies faster than the geodesic."""
    if emitter == "torus":
        sc = dict(W.torus_512("fp64"), n_alpha=24, n_beta=24, alpha_min=-8.0, alpha_max=8.0,
                  beta_min=-8.0, beta_max=8.0)
    else:
        sc = W.synch_shell(a=0.0, n=16, precision="fp64")
    nf = len(sc["freqs"])
    worst = {}
    for mode in ("ride", "controlled"):
        lo = orc.render(dict(sc, rtol=1e-8, rt_control=mode))
        hi = orc.render(dict(sc, rtol=1e-10, rt_control=mode))
        assert np.array_equal(lo["status"], hi["status"])
        Il, Ih = lo["I_nu"][:, :nf], hi["I_nu"][:, :nf]
        rel = np.abs(Il - Ih) / np.maximum(np.abs(Ih), 1e-3 * np.abs(Ih).max(axis=0))
        worst[mode] = rel.max()
    assert worst["controlled"] < 2e-6, worst
    assert worst["ride"] > 1e-4, worst
