"""Pins of the oracle's building blocks against what mathematics and the paper fix.

Each check is computed here from first principles (a different route from the oracle's
code), so that a dropped term, a wrong sign or a swapped index in the oracle fails it.
"""
import math
from fractions import Fraction

import numpy as np
import pytest
from scipy.optimize import brentq

from paper_1601_02063_gb300 import workloads as W


def _frac(x):
    return Fraction(x).limit_denominator(200000)


def test_cash_karp_tableau_order_conditions(orc):
    """Cash & Karp 1990: row sums equal c; the fifth-order weights satisfy the quadrature
    conditions sum b c^k = 1/(k+1) for k <= 4 and the fourth-order ones for k <= 3, plus the
    tree conditions of order <= 4 (exact rational arithmetic)."""
    c, A, b5, b4 = orc.ck_tableau()
    c = [_frac(v) for v in c]
    A = [[_frac(v) for v in row] for row in A]
    b5 = [_frac(v) for v in b5]
    b4 = [_frac(v) for v in b4]
    for i in range(6):
        assert sum(A[i][:i]) == c[i]
    for b, order in ((b5, 5), (b4, 4)):
        for k in range(order):
            assert sum(bi * ci ** k for bi, ci in zip(b, c)) == Fraction(1, k + 1)
        # order-3 tree: sum b_i a_ij c_j = 1/6
        s3 = sum(b[i] * A[i][j] * c[j] for i in range(6) for j in range(i))
        assert s3 == Fraction(1, 6)
        # order-4 trees
        assert sum(b[i] * c[i] * A[i][j] * c[j] for i in range(6) for j in range(i)) == \
            Fraction(1, 8)
        assert sum(b[i] * A[i][j] * c[j] ** 2 for i in range(6) for j in range(i)) == \
            Fraction(1, 12)
        assert sum(b[i] * A[i][j] * A[j][k] * c[k] for i in range(6) for j in range(i)
                   for k in range(j)) == Fraction(1, 24)
    assert b5 != b4


def _hamiltonian(a, y, L, E=1.0):
    """H = g^{mu nu} p_mu p_nu / 2 for Kerr in Boyer-Lindquist coordinates, written from
    the inverse metric components (not from the separated form the oracle uses)."""
    r, th, _, _, pr, pth = y
    s, c = math.sin(th), math.cos(th)
    Sig = r * r + a * a * c * c
    Del = r * r - 2 * r + a * a
    A = (r * r + a * a) ** 2 - a * a * Del * s * s
    gtt = -A / (Sig * Del)
    gtp = -2 * a * r / (Sig * Del)
    gpp = (Del - a * a * s * s) / (Sig * Del * s * s)
    pt, pp = -E, L
    return 0.5 * (Del / Sig * pr * pr + pth * pth / Sig + gtt * pt * pt + 2 * gtp * pt * pp
                  + gpp * pp * pp)


def _fd(fun, x, h):
    return (fun(x + h) - fun(x - h)) / (2 * h)


@pytest.mark.parametrize("on_shell", [True, False])
def test_rhs_is_hamiltons_equations(orc, on_shell):
    """The six ODEs of Section 2.1 are Hamilton's equations: dx/dlambda = dH/dp,
    dp/dlambda = -dH/dx (phi-dot = dH/dL, t-dot = -dH/dE), checked by central
    differences of H.  Off the null cone too (see the reading of Eqs. 14-15)."""
    rng = np.random.default_rng(7)
    for _ in range(40):
        a = rng.uniform(-0.99, 0.99)
        r = rng.uniform(2.5, 60.0)
        th = rng.uniform(0.2, math.pi - 0.2)
        L = rng.uniform(-8, 8)
        pth = rng.uniform(-6, 6)
        Del = r * r - 2 * r + a * a
        s = math.sin(th)
        rest = pth ** 2 + (L / s - a * s) ** 2 - ((r * r + a * a) - a * L) ** 2 / Del
        if on_shell:
            if rest > 0:
                continue
            pr = math.sqrt(-rest / Del) * rng.choice([-1, 1])
        else:
            pr = rng.uniform(-3, 3)
        y = np.array([r, th, 0.3, 5.0, pr, pth])
        f = orc.geodesic_rhs(a, L, y)
        H = lambda yy, LL=L, E=1.0: _hamiltonian(a, yy, LL, E)

        def along(k, h):
            e = np.zeros(6)
            e[k] = 1.0
            return _fd(lambda t: H(y + t * e), 0.0, h)

        num = np.array([
            along(4, 1e-5),                                  # r-dot = dH/dp_r
            along(5, 1e-5),                                  # theta-dot = dH/dp_theta
            _fd(lambda l: H(y, l), L, 1e-5),                 # phi-dot = dH/dL
            -_fd(lambda e: H(y, L, e), 1.0, 1e-5),           # t-dot = dH/dp_t = -dH/dE
            -along(0, 1e-5 * r),                             # p_r-dot = -dH/dr
            -along(1, 1e-5),                                 # p_theta-dot = -dH/dtheta
        ])
        scale = np.abs(num) + 1e-3 * np.max(np.abs(num))
        assert np.all(np.abs(f - num) <= 2e-7 * scale), (f, num)


def _eq14_eq15_as_printed(a, y, L):
    """Eqs. 14-15 exactly as printed (E = 1, mu = 0, kappa from the state)."""
    r, th, _, _, pr, pth = y
    s, c = math.sin(th), math.cos(th)
    Sig = r * r + a * a * c * c
    Del = r * r - 2 * r + a * a
    kap = pth ** 2 + L * L / s ** 2 + a * a * s * s
    prdot = (-kap * (r - 1) + 2 * r * (r * r + a * a) - 2 * a * L) / (Sig * Del) \
        - 2 * pr * pr * (r - 1) / Sig
    pthdot = s * c / Sig * (L * L / s ** 4 - a * a)
    return prdot, pthdot


def test_rhs_equals_printed_eq14_on_null_cone(orc):
    """On the null cone the oracle's momentum equations equal Eqs. 14-15 as printed;
    off it they differ (by the terms in F that keep the flow Hamiltonian)."""
    rng = np.random.default_rng(11)
    n_on = 0
    for _ in range(60):
        a = rng.uniform(-0.99, 0.99)
        r, th = rng.uniform(2.5, 40), rng.uniform(0.3, 2.8)
        L, pth = rng.uniform(-6, 6), rng.uniform(-5, 5)
        Del, s = r * r - 2 * r + a * a, math.sin(th)
        rest = pth ** 2 + (L / s - a * s) ** 2 - ((r * r + a * a) - a * L) ** 2 / Del
        if rest > 0:
            continue
        pr = math.sqrt(-rest / Del)
        y = np.array([r, th, 0.0, 0.0, pr, pth])
        f = orc.geodesic_rhs(a, L, y)
        p1, p2 = _eq14_eq15_as_printed(a, y, L)
        assert abs(f[4] - p1) <= 1e-10 * (abs(p1) + 1)
        assert abs(f[5] - p2) <= 1e-10 * (abs(p2) + 1)
        y_off = y.copy()
        y_off[4] *= 1.01
        f_off = orc.geodesic_rhs(a, L, y_off)
        p1_off, _ = _eq14_eq15_as_printed(a, y_off, L)
        assert abs(f_off[4] - p1_off) > 1e-8 * (abs(p1_off) + 1)
        n_on += 1
    assert n_on > 20


def _bl_from_cartesian(a, x, y, z):
    """Eqs. 20-22 restated: oblate-spheroidal (Boyer-Lindquist) r, theta, phi."""
    w = x * x + y * y + z * z - a * a
    r = math.sqrt((w + math.sqrt(w * w + 4 * a * a * z * z)) / 2)
    return r, math.acos(z / r), math.atan2(y, x)


@pytest.mark.parametrize("a,inc,phio", [(0.9, 60.0, 0.0), (0.5, 17.0, 1.1), (0.0, 85.0, -2.0)])
def test_initial_velocity_is_derivative_of_straight_line(orc, a, inc, phio):
    """Eqs. 24-26 are the BL velocities of a point moving with unit speed along the line
    of sight toward the hole: the image-plane z axis mapped by Eq. 18.  The test builds
    that direction from the rotation angles of the text, maps points along the line with
    Eqs. 20-22 and differentiates numerically."""
    sc = W.scene(a=a, theta_obs=math.radians(inc), phi_obs=phio, r_obs=1000.0)
    to = math.radians(inc)
    # unit vector from the observer toward the origin: -(observer direction)
    d = -np.array([math.sin(to) * math.cos(phio), math.sin(to) * math.sin(phio), math.cos(to)])
    for alpha, beta in [(3.0, 2.0), (-7.5, 4.2), (12.0, -9.0)]:
        x0 = orc.observer_point(sc, alpha, beta)
        y0, L, Q, vin = orc.init_ray(sc, alpha, beta)
        h = 1e-3
        p = _bl_from_cartesian(a, *(x0 + h * d))
        m = _bl_from_cartesian(a, *(x0 - h * d))
        num = np.array([(p[i] - m[i]) / (2 * h) for i in range(3)])
        assert np.allclose(vin, num, rtol=1e-7, atol=1e-12), (vin, num)
        # the mapped start point itself (Eqs. 20-22)
        r0, th0, ph0 = _bl_from_cartesian(a, *x0)
        assert abs(y0[0] - r0) < 1e-9 and abs(y0[1] - th0) < 1e-12
        assert abs(y0[2] - ph0) < 1e-12


def test_observer_point_is_a_rigid_motion(orc):
    """Eq. 18 is a reflection and two rotations plus a translation: distances between
    image-plane points are preserved, and the image centre lies at distance
    sqrt(r_obs^2 + a^2 sin^2 theta_obs) from the origin along the observer direction."""
    sc = W.scene(a=0.7, theta_obs=math.radians(40.0), phi_obs=0.4)
    pts = [(0.0, 0.0), (5.0, 0.0), (0.0, 5.0), (3.0, -4.0)]
    X = [orc.observer_point(sc, *p) for p in pts]
    for i in range(4):
        for j in range(4):
            d_img = math.dist(pts[i], pts[j])
            assert abs(np.linalg.norm(X[i] - X[j]) - d_img) < 1e-9
    to, ro = math.radians(40.0), 1000.0
    expect = math.sqrt((ro ** 2 + 0.49) * math.sin(to) ** 2 + ro ** 2 * math.cos(to) ** 2)
    assert abs(np.linalg.norm(X[0]) - expect) < 1e-9


def test_initial_state_is_null_and_matches_flat_space_limit(orc):
    """H(y0) = 0; at a large observer distance the constants of motion approach the
    flat-space impact parameters: L = -alpha sin(i), p_theta = beta,
    Q = beta^2 + (alpha^2 - a^2) cos^2 i (Bardeen's celestial coordinates with
    alpha = -lambda csc i for the physically traced photon)."""
    for a, inc in [(0.9, 60.0), (0.3, 25.0), (0.998, 80.0)]:
        sc = W.scene(a=a, theta_obs=math.radians(inc), r_obs=1.0e6)
        to = math.radians(inc)
        for alpha, beta in [(4.0, 3.0), (-6.0, 1.5), (0.5, -8.0)]:
            y0, L, Q, _ = orc.init_ray(sc, alpha, beta)
            H = _hamiltonian(a, y0, L)
            scale = 0.5 * (y0[0] ** 2) / (y0[0] ** 2)  # |g^tt E^2| / 2 ~ 1/2 far away
            assert abs(H) < 1e-13 * scale * 10
            assert abs(L - (-alpha * math.sin(to))) < 1e-4
            assert abs(y0[5] - beta) < 1e-4
            assert abs(Q - (beta ** 2 + (alpha ** 2 - a * a) * math.cos(to) ** 2)) < 1e-3


def test_face_on_schwarzschild_has_zero_angular_momentum(orc):
    sc = W.scene(a=0.0, theta_obs=0.0)
    for alpha, beta in [(3.0, 4.0), (-1.0, 0.25), (10.0, -10.0)]:
        _, L, _, _ = orc.init_ray(sc, alpha, beta)
        assert L == 0.0


def test_literal_convention_flips_angular_momentum(orc):
    """The two readings of the traced direction differ only in the sign of the velocity:
    at a = 0 the literal reading's L is exactly minus the physical one."""
    for alpha, beta in [(3.0, 4.0), (-6.0, 2.0)]:
        _, Lp, Qp, _ = orc.init_ray(W.scene(a=0.0), alpha, beta)
        _, Ll, Ql, _ = orc.init_ray(W.scene(a=0.0, convention="literal"), alpha, beta)
        assert Ll == -Lp and abs(Ql - Qp) < 1e-12


@pytest.mark.parametrize("a,expect", [(0.0, 6.0), (0.9, 2.320883), (0.94, 2.023593),
                                      (0.998, 1.236971), (0.7, 3.393128)])
def test_isco_is_root_of_marginal_stability_polynomial(orc, a, expect):
    """r_ISCO solves r^2 - 6 M r + 8 a sqrt(M r) - 3 a^2 = 0 (Bardeen, Press & Teukolsky
    1972), root above the photon orbit; the oracle uses the closed form."""
    poly = lambda r: r * r - 6 * r + 8 * a * math.sqrt(r) - 3 * a * a
    root = brentq(poly, 1.0 + 1e-9 if a > 0.99 else 1.5, 9.0) if a > 0 else 6.0
    if a > 0.9:
        # the polynomial has a second, spurious root below the prograde photon orbit
        root = brentq(poly, 1.1, 9.0)
    assert abs(orc.isco(a) - root) < 1e-12 * root
    assert abs(orc.isco(a) - expect) < 1e-6


def test_horizon(orc):
    for a in (0.0, 0.5, 0.94, 0.998):
        rp = orc.horizon(a)
        assert abs(rp * rp - 2 * rp + a * a) < 1e-14 and rp >= 1.0


def test_disk_redshift_from_metric(orc):
    """g = 1/(u^t (1 - Omega L)) for a circular equatorial orbit with Omega = 1/(r^1.5 + a):
    here u^t comes from the normalisation u.u = -1 with the metric components of Eq. 1,
    not from the closed form used by the oracle."""
    for a in (0.0, 0.5, 0.9, -0.5):
        for r in (orc.isco(a) + 0.01, 7.0, 19.0):
            for L in (-4.0, 0.0, 3.0):
                Sig, Del = r * r, r * r - 2 * r + a * a
                gtt = -(1 - 2 * r / Sig)
                gtp = -2 * a * r / Sig
                gpp = (r * r + a * a + 2 * a * a * r / Sig)
                Om = 1.0 / (r ** 1.5 + a)
                ut = 1.0 / math.sqrt(-(gtt + 2 * gtp * Om + gpp * Om * Om))
                g = 1.0 / (ut * (1 - Om * L))
                assert abs(orc.disk_redshift(a, r, L) - g) < 1e-12 * g


def test_torus_normalisation_by_independent_quadrature(orc):
    """The emissivity normalisation (optical depth 1 along the static equatorial path from
    r_+ to 1000 M at nu = 1) against scipy's adaptive quadrature of the same integral."""
    from scipy.integrate import quad
    for a in (0.94, 0.998):
        rp = orc.horizon(a)

        def alpha_nu(r, nu=1.0):
            ne = r ** -1.5
            T = 10.0 * r ** -0.84
            j = ne * ne / math.sqrt(T) * math.exp(-nu / T)
            B = 2 * nu ** 3 / math.expm1(nu / T)
            return j / B

        val = sum(quad(alpha_nu, lo, hi, limit=200, epsabs=0, epsrel=1e-12)[0]
                  for lo, hi in [(rp, 10), (10, 100), (100, 1000)])
        assert abs(orc.torus_norm(a) - 1.0 / val) < 1e-9 / val
