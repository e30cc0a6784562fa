"""Per-pixel parity of reduced-precision images against the FP64 oracle.

Bar (the benchmark spec, reading C17): 1e-4 relative per pixel away from the critical curve.  A
pixel is *stable* when the oracle gives the same ray status at its four corners.  The
relative error of an intensity is |I - I_ref| / max(|I_ref|, 1e-3 I_max), I_max the brightest
reference pixel of that frequency plane: pixels darker than 1e-3 of the brightest are held
to an absolute 1e-7 of it instead of a relative bar on a vanishing value.
"""
from __future__ import annotations

import math

import numpy as np

REL_PIXEL = 1e-4
DARK = 1e-3


def corner_status(orc, sc: dict, pixels=None) -> np.ndarray:
    """Oracle status of the four corners of the given flat pixels (all if None): [4, n]."""
    na, nb = sc["n_alpha"], sc["n_beta"]
    if pixels is None:
        pixels = np.arange(na * nb)
    j, i = np.divmod(np.asarray(pixels), na)
    da = (sc["alpha_max"] - sc["alpha_min"]) / na
    db = (sc["beta_max"] - sc["beta_min"]) / nb
    a0 = sc["alpha_min"] + (i + 0.5) * da
    b0 = sc["beta_min"] + (j + 0.5) * db
    out = []
    for sa, sb in ((-0.5, -0.5), (0.5, -0.5), (-0.5, 0.5), (0.5, 0.5)):
        rays = np.stack([a0 + sa * da, b0 + sb * db, np.full(a0.size, sc["a"]),
                         np.full(a0.size, math.cos(sc["theta_obs"]))], axis=1)
        out.append(orc.trace_list(dict(sc, precision="fp64"), rays)["status"])
    return np.array(out)


def stable(orc, sc: dict, pixels=None) -> np.ndarray:
    st = corner_status(orc, sc, pixels)
    return np.all(st == st[0], axis=0)


def pixel_rel(I: np.ndarray, I_ref: np.ndarray, I_max: float) -> np.ndarray:
    return np.abs(I - I_ref) / np.maximum(np.abs(I_ref), DARK * I_max)


def check_planes(img_planes, ref_planes, mask, label, frac_ok=0.999, worst=1e-3):
    """img_planes, ref_planes: [planes, n]; mask: pixels held to the bar.  Asserts that at
    least frac_ok of them are within REL_PIXEL and all within `worst`; returns the fraction
    above REL_PIXEL per plane (printed)."""
    fracs = []
    for k, (I, R) in enumerate(zip(img_planes, ref_planes)):
        rel = pixel_rel(I, R, np.abs(R).max())[mask]
        above = float(np.mean(rel > REL_PIXEL))
        fracs.append(above)
        print(f"{label} plane {k}: {mask.sum()} stable pixels, {above:.4%} above {REL_PIXEL:g}, "
              f"max {rel.max():.2e}")
        assert 1.0 - above >= frac_ok and rel.max() <= worst, (label, k, above, rel.max())
    return fracs
