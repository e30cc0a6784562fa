"""Pins of the thermal-synchrotron shell in the oracle (Section 4.5): K_2 against SciPy's
Bessel routine; the emissivity fit's frequency integral against the synchrotron power of a
Maxwell-Juttner electron gas (Larmor power with the Thomson cross-section); Kirchhoff's law;
and the optically thick limit of a ray, the Rayleigh-Jeans intensity 2 nu^2 k T g / c^2 of
an isothermal shell surface."""
import math

import numpy as np
import pytest
from scipy import integrate, special

from paper_1601_02063_gb300 import workloads as W

# CGS constants typed here from CODATA 2018 (independent of the oracle's copies)
C = 2.99792458e10
ME = 9.1093837015e-28
MP = 1.67262192369e-24
H = 6.62607015e-27
SIGMA_T = 6.6524587321e-25


@pytest.mark.parametrize("x", [1e-3, 0.01, 0.1, 0.5, 1.0, 2.0, 5.0, 10.0, 30.0, 80.0])
def test_bessel_k2_matches_scipy(orc, x):
    assert math.isclose(orc.bessel_k2(x), special.kn(2, x), rel_tol=1e-13)


def _mj_gamma2beta2(theta):
    """<gamma^2 beta^2> over the Maxwell-Juttner distribution gamma^2 beta exp(-gamma/theta)."""
    w = lambda g: g * g * math.sqrt(1.0 - 1.0 / (g * g)) * math.exp(-(g - 1.0) / theta)
    lo, hi = 1.0, 1.0 + 200.0 * theta
    num = integrate.quad(lambda g: (g * g - 1.0) * w(g), lo, hi, limit=400)[0]
    den = integrate.quad(w, lo, hi, limit=400)[0]
    return num / den


def test_emissivity_integrates_to_synchrotron_power(orc):
    """4 pi int j_nu dnu = n (4/3) sigma_T c (B^2 / 8 pi) <gamma^2 beta^2> for relativistic
    electrons (Theta_e = 100, where the fit's universal form applies); the fit is good to a
    few per cent, a dropped term, a wrong power of x or a lost 4 pi is not."""
    sc = W.synch_shell()
    sc.update(T0=100.0, T_index=0.0, ne_index=0.0, n_e0=1e6, theta_width=1e3)
    r = 50.0
    n = sc["n_e0"]
    B2 = 8.0 * math.pi * n * MP * C * C / (6.0 * sc["beta_B"] * r)
    nu_c = 3.0 * 4.803204712570263e-10 * math.sqrt(B2) / (4.0 * math.pi * ME * C) * 100.0 ** 2
    f = lambda lx: orc.synch_coeffs(sc, r, 0.0, nu_c * math.exp(lx))[0] * nu_c * math.exp(lx)
    P_nu = 4.0 * math.pi * integrate.quad(f, math.log(1e-6), math.log(1e5), limit=400)[0]
    P = n * 4.0 / 3.0 * SIGMA_T * C * B2 / (8.0 * math.pi) * _mj_gamma2beta2(100.0)
    assert abs(P_nu / P - 1.0) < 0.03, P_nu / P


@pytest.mark.parametrize("r,nu", [(2.0, 150e9), (20.0, 340e9), (300.0, 1e12), (5.0, 1e15)])
def test_kirchhoff_source_function_is_planck(orc, r, nu):
    sc = W.synch_shell()
    j, al = orc.synch_coeffs(sc, r, 0.3, nu)
    kT = sc["T0"] * r ** -sc["T_index"] * ME * C * C
    B_nu = 2.0 * H * nu ** 3 / C ** 2 / math.expm1(H * nu / kT)
    assert j > 0 and al > 0
    assert math.isclose(j / al, B_nu, rel_tol=1e-12)


def test_no_emission_beyond_shell(orc):
    """A ray that never enters r <= r_out gathers nothing."""
    sc = W.synch_shell()
    sc.update(r_out=5.0, alpha_min=40.0, alpha_max=41.0, beta_min=40.0, beta_max=41.0,
              n_alpha=1, n_beta=1)
    res = orc.render(sc)
    assert res["status"][0] == 1
    assert np.all(res["I_nu"][0, :3] == 0.0) and np.all(res["tau_nu"][0, :3] == 0.0)


def test_optically_thick_isothermal_shell_is_rayleigh_jeans(orc):
    """Nearly face-on view of a uniform, isothermal, very opaque shell of radius 500 M around a
    Schwarzschild hole: the ray stops seeing anything within a few M of entering, where the
    flow is at rest to 1e-5 (near the pole), so I_nu = nu^3 B_nu0(T) / nu0^3 with
    nu0 = nu / g, g = sqrt(1 - 2 / 500): the Rayleigh-Jeans value 2 nu^2 k T g / c^2 to
    h nu / k T ~ 1e-9.  Small steps keep the optical depth per step below ~0.7 (Eqs. 30-31
    integrated as Runge-Kutta components are accurate only while it stays small).  At
    340 GHz the tau = 1 layer is ~5 M deep; at 150 GHz it is 0.3 M deep, thinner than the
    step that straddles the shell's sharp edge, which limits that frequency to ~3e-3."""
    sc = W.synch_shell(a=0.0)
    sc.update(theta_obs=0.01, r_obs=2000.0, alpha_min=0.4, alpha_max=0.6, beta_min=0.4,
              beta_max=0.6, n_alpha=1, n_beta=1, ne_index=0.0, T_index=0.0, T0=10.0,
              n_e0=1e8, theta_width=1e3, hmax_frac=2e-4, max_steps=400000,
              freqs=[150e9, 340e9])
    res = orc.render(sc)
    g = math.sqrt(1.0 - 2.0 / 500.0)
    kT = 10.0 * ME * C * C
    for k, nu in enumerate(sc["freqs"]):
        assert res["tau_nu"][0, k] > 30.0
        rj = 2.0 * nu * nu * kT * g / C ** 2
        tol = 1e-4 if nu > 200e9 else 5e-3
        assert abs(res["I_nu"][0, k] / rj - 1.0) < tol, (nu, res["I_nu"][0, k] / rj)


def test_shell_intensities_resolve_jumps_to_the_tolerance(orc):
    """The sensitivity the FP64 parity bar of the shell allows for: the oracle at rtol 1e-8
    and at 1e-8 (1 + 1e-14) agrees within 1e-8 on at least 99 % of a 40 x 36 shell image
    and within 1e-6 on every pixel (the rejection cascades at the flow's and the shell's
    jumps end at slightly different points)."""
    sc = dict(W.synch_shell(a=0.0, precision="fp64"), n_alpha=40, n_beta=36)
    a = orc.render(sc)
    b = orc.render(dict(sc, rtol=1e-8 * (1.0 + 1e-14)))
    for k in range(3):
        rel = np.abs(a["I_nu"][:, k] - b["I_nu"][:, k]) / np.abs(a["I_nu"][:, k])
        assert np.mean(rel <= 1e-8) >= 0.99 and rel.max() <= 1e-6, (k, rel.max())
