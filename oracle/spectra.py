"""Spectra and light curves from rendered images, written out from their definitions
(Section 4.4: a light curve integrates the intensity over the frequency bins of each image;
a spectrum is the image-integrated intensity per frequency).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The flux density of one image plane at the observer is the intensity summed over the image
times the solid angle of a pixel, dOmega = dalpha dbeta / r_obs^2 (alpha, beta in units of M
on the image plane at distance r_obs):

    F_j = dalpha dbeta / r_obs^2 * sum_pixels I_j(pixel)

and a light-curve point is F integrated over the image's frequencies (trapezoid rule over
nu; with one plane, F itself).  Sums are exactly rounded (math.fsum).
"""
from __future__ import annotations

import math

import numpy as np


def pixel_solid_angle(scene: dict) -> float:
    da = (scene["alpha_max"] - scene["alpha_min"]) / scene["n_alpha"]
    db = (scene["beta_max"] - scene["beta_min"]) / scene["n_beta"]
    return da * db / (scene["r_obs"] * scene["r_obs"])


def planes_of(scene: dict) -> int:
    return len(scene["freqs"]) if scene["emitter"] in ("torus", "nt_disk", "synch", "spot") else 1


def image_planes(scene: dict, results: np.ndarray) -> np.ndarray:
    """[planes][n_beta * n_alpha] image from oracle results in pixel order: I_nu per
    frequency for the torus, the Novikov-Thorne disk and the synchrotron shell, the thin-disk
    intensity otherwise."""
    if scene["emitter"] in ("torus", "nt_disk", "synch", "spot"):
        return np.ascontiguousarray(results["I_nu"][:, :planes_of(scene)].T)
    return np.ascontiguousarray(results["intensity"][None, :])


def image_flux(scene: dict, planes: np.ndarray) -> np.ndarray:
    """F_j for every plane j of one scene's image ([planes][pixels])."""
    w = pixel_solid_angle(scene)
    return np.array([math.fsum(np.asarray(p, dtype=np.float64).ravel()) * w for p in planes])


def light_curve_point(scene: dict, flux: np.ndarray) -> float:
    """Trapezoid rule of F over the scene's frequencies; one plane: F itself."""
    if len(flux) < 2:
        return float(flux[0])
    nu = np.asarray(scene["freqs"], dtype=np.float64)
    return math.fsum(0.5 * (flux[j] + flux[j + 1]) * (nu[j + 1] - nu[j])
                     for j in range(len(flux) - 1))
