"""Seeded synthetic workloads shared by the CUDA path and the oracle.

This module holds only scene parameters and seeded random draws: none of the
method's arithmetic.  Quantities that the method derives (r_ISCO for a disk with
``r_in = 0``, the torus emissivity normalisation when ``C_norm`` is None) are left
for each side to compute with its own code.

The scenes follow the workloads of Pu et al. 2016: thin Keplerian disk around a Kerr
hole seen from r = 1000 M (Sections 4.1-4.3, Table 1's grid-projection workload),
analytic thermal flow for the radiative transfer of Section 2.3, a many-scene
parameter sweep, and a 4096^2 near-edge-on case.  All randomness draws from numpy's
PCG64 with an explicit seed.
"""
from __future__ import annotations

import math

import numpy as np

SEED = 20160109

_DEFAULTS = dict(
    a=0.9, r_obs=1000.0, theta_obs=math.radians(60.0), phi_obs=0.0,
    alpha_min=-15.0, alpha_max=15.0, beta_min=-15.0, beta_max=15.0,
    n_alpha=64, n_beta=64, emitter="thin_disk", freqs=[],
    r_in=0.0, r_out=20.0, q_emis=3.0,
    ne_index=1.5, theta_width=0.3, T0=10.0, T_index=0.84, C_norm=None, nu_norm=1.0,
    rtol=1e-8, h0=1.0, hmax_frac=0.1, horizon_factor=1.01, max_steps=100000,
    convention="physical", precision="fp64",
    # transfer components under the step control ("controlled") or riding on the geodesic's
    # steps ("ride")
    rt_control="controlled",
    # reduced-precision controls (ignored by the FP64 path)
    rtol_fp32=1e-6, r_switch=0.0,
    # synchrotron shell: n_e at r = 1 [cm^-3], field parameter beta_B, mass [M_sun]
    n_e0=3e7, beta_B=10.0, mass=4e6,
    # hot spot: orbit radius (<= 0: r_ISCO), Gaussian width r_spot, phase at t = 0, the
    # observer time of the image
    spot_r=0.0, spot_size=0.5, spot_phase=0.0, t_obs=0.0,
)


def scene(**kw) -> dict:
    """A scene dict with the defaults above overridden by ``kw``."""
    unknown = set(kw) - set(_DEFAULTS)
    if unknown:
        raise KeyError(f"unknown scene keys: {sorted(unknown)}")
    d = dict(_DEFAULTS)
    d.update(kw)
    d["freqs"] = list(d["freqs"])
    return d


def thin_disk_64() -> dict:
    """Kerr a=0.9, r_obs=1000, i=60 deg, 64x64 over [-15,15]^2, thin Keplerian disk from
    r_ISCO to 20 M with emissivity r^-3, Cash-Karp rtol 1e-8."""
    return scene()


def torus_512(precision: str = "fp64") -> dict:
    """a=0.94, i=30 deg, r_obs=1000, 512x512 over [-20,20]^2; analytic Keplerian torus
    n_e = r^-1.5 exp(-cos^2 / (2 0.3^2)), T_e = 10 r^-0.84, thermal emission with Kirchhoff
    absorption at nu in {0.5, 1, 2}; stop at 1.01 r_+ or on escape."""
    return scene(a=0.94, theta_obs=math.radians(30.0), alpha_min=-20.0, alpha_max=20.0,
                 beta_min=-20.0, beta_max=20.0, n_alpha=512, n_beta=512, emitter="torus",
                 freqs=[0.5, 1.0, 2.0], precision=precision)


def torus_hard_4096(precision: str = "mixed") -> dict:
    """a=0.998, i=85 deg, 4096x4096 over [-20,20]^2, torus as above at 8 log-spaced
    frequencies in [0.25, 4]."""
    freqs = [float(v) for v in np.geomspace(0.25, 4.0, 8)]
    return scene(a=0.998, theta_obs=math.radians(85.0), alpha_min=-20.0, alpha_max=20.0,
                 beta_min=-20.0, beta_max=20.0, n_alpha=4096, n_beta=4096, emitter="torus",
                 freqs=freqs, precision=precision)


def projection_1024(precision: str = "fp64") -> dict:
    """The paper's timing workload (Section 5, Table 1): grid projection (geodesics only, the
    first equatorial crossing recorded) at a = 0.95, i = 60 deg, r_obs = 1000, 1024x1024.
    The paper states neither the field of view nor the tolerance; here [-15, 15]^2 and
    rtol 1e-8 as in the other scenes."""
    return scene(a=0.95, theta_obs=math.radians(60.0), n_alpha=1024, n_beta=1024,
                 emitter="none", precision=precision)


def nt_disk(r_out: float = 20.0, n: int = 512, precision: str = "mixed") -> dict:
    """Novikov-Thorne disk spectrum (Section 4.3, the spectra figure): a = 0.999, i = 85 deg,
    r_obs = 1000, disk r_ISCO .. r_out, temperature scale T0 = 1, 8 log-spaced frequencies in
    [0.02, 3]; window [-(r_out + 2), r_out + 2]^2 at n x n."""
    w = r_out + 2.0
    freqs = [float(v) for v in np.geomspace(0.02, 3.0, 8)]
    return scene(a=0.999, theta_obs=math.radians(85.0), alpha_min=-w, alpha_max=w, beta_min=-w,
                 beta_max=w, n_alpha=n, n_beta=n, emitter="nt_disk", r_out=r_out, T0=1.0,
                 freqs=freqs, precision=precision)


def synch_shell(a: float = 0.0, n: int = 256, precision: str = "mixed",
                freqs=(150e9, 340e9, 1000e9)) -> dict:
    """Keplerian shell with thermal synchrotron emission (Section 4.5) around a 4e6 M_sun
    black hole seen at i = 60 deg: n_e = 3e7 r^-1.1 cm^-3, Theta_e = 100 r^-0.84, field from
    B^2 / 8 pi = n_e m_p c^2 / (6 beta_B r) with beta_B = 10, shell out to 500 M, images
    at 150, 340 and 1000 GHz over +-15 M (optical depth through the shell about 6, 1 and
    0.1).  The 1000 GHz emissivity, exp(-1.8899 x^1/3) with x ~ r^2.7, changes by a factor
    ~2 per 0.1 r step near the hole; the intensities' step control resolves it."""
    return scene(a=a, theta_obs=math.radians(60.0), alpha_min=-15.0, alpha_max=15.0,
                 beta_min=-15.0, beta_max=15.0, n_alpha=n, n_beta=n, emitter="synch",
                 freqs=list(freqs), r_out=500.0, ne_index=1.1, theta_width=10.0, T0=100.0,
                 T_index=0.84, n_e0=3e7, beta_B=10.0, mass=4e6, precision=precision)


def hot_spot(t_obs: float = 0.0, a: float = 0.0, n: int = 128, precision: str = "fp64") -> dict:
    """Optically thick Keplerian hot spot (Section 4.4): centre on the circular equatorial
    orbit at r_ISCO, r_spot = 0.5 M (the spot is the region d < 4 r_spot, z > 0), seen at
    i = 60 deg over [-10, 10]^2 M at observer time t_obs; blackbody at T0 = 1 times the
    Gaussian profile, 8 frequencies log-spaced in [0.1, 10]."""
    freqs = [float(v) for v in np.geomspace(0.1, 10.0, 8)]
    return scene(a=a, theta_obs=math.radians(60.0), alpha_min=-10.0, alpha_max=10.0,
                 beta_min=-10.0, beta_max=10.0, n_alpha=n, n_beta=n, emitter="spot",
                 freqs=freqs, T0=1.0, C_norm=1.0, spot_r=0.0, spot_size=0.5,
                 spot_phase=0.0, t_obs=t_obs, precision=precision)


def sweep_64(seed: int = SEED, precision: str = "mixed") -> list[dict]:
    """64 thin-disk scenes: resolution from {128,256,512,1024}^2, a ~ U[0, 0.998],
    i ~ U[5, 85] deg, disk and window as in the 64x64 thin-disk scene."""
    rng = np.random.Generator(np.random.PCG64(seed))
    res = rng.choice([128, 256, 512, 1024], size=64)
    spins = rng.uniform(0.0, 0.998, size=64)
    incl = rng.uniform(5.0, 85.0, size=64)
    return [scene(a=float(a), theta_obs=math.radians(float(i)), n_alpha=int(n), n_beta=int(n),
                  precision=precision)
            for n, a, i in zip(res, spins, incl)]


def training_rays(n: int, seed: int = SEED + 1) -> np.ndarray:
    """n rays (alpha, beta, a, cos i): alpha, beta ~ U[-20, 20], a ~ U[0, 0.998],
    i ~ U[1, 89] deg.  Returns float64 [n, 4]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = np.empty((n, 4), dtype=np.float64)
    out[:, 0] = rng.uniform(-20.0, 20.0, n)
    out[:, 1] = rng.uniform(-20.0, 20.0, n)
    out[:, 2] = rng.uniform(0.0, 0.998, n)
    out[:, 3] = np.cos(np.radians(rng.uniform(1.0, 89.0, n)))
    return out


def surrogate_scene_2048() -> dict:
    """Inference image for the learned transfer function: 2048^2 thin disk, a=0.7,
    i=45 deg, window [-20,20]^2."""
    return scene(a=0.7, theta_obs=math.radians(45.0), alpha_min=-20.0, alpha_max=20.0,
                 beta_min=-20.0, beta_max=20.0, n_alpha=2048, n_beta=2048, precision="mixed")


def sample_pixels(n_pix: int, k: int, seed: int = SEED + 2) -> np.ndarray:
    """k distinct flat pixel indices out of n_pix, sorted."""
    rng = np.random.Generator(np.random.PCG64(seed))
    k = min(k, n_pix)
    return np.sort(rng.choice(n_pix, size=k, replace=False)).astype(np.int64)
