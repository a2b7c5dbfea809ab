"""Observables of the time-averaged jet (Sec. 3, "Self-similarity in
multicomponent turbulent jets").

These act on the time-averaged fields <phi> and <u_z> that the step kernel
accumulates (option ``average``): the centre-line profiles, whose inverse
grows linearly downstream of the potential core (the paper fits slopes of
about 1/(6.5 D)), and the radial profiles at a given distance from the
nozzle, which the paper fits with Gaussians exp(-k (r / (z - z0))^2)
(k = 75 for the velocity at 12 D; k = 80 / 200 for the phase field).

Post-processing on the host (numpy), outside the time-stepping path.  Fields
are arrays shaped (nz, ny, nx), z the jet axis.
"""
from __future__ import annotations

import numpy as np


def centerline(field: np.ndarray, cx: float, cy: float) -> np.ndarray:
    """Values along the jet axis x = cx, y = cy (bilinear in x, y), one per z plane."""
    nz, ny, nx = field.shape
    x0, y0 = int(np.floor(cx)), int(np.floor(cy))
    fx, fy = cx - x0, cy - y0
    x1, y1 = min(x0 + 1, nx - 1), min(y0 + 1, ny - 1)
    return ((1 - fx) * (1 - fy) * field[:, y0, x0] + fx * (1 - fy) * field[:, y0, x1] +
            (1 - fx) * fy * field[:, y1, x0] + fx * fy * field[:, y1, x1])


def radial_profile(field: np.ndarray, z: int, cx: float, cy: float, dr: float = 1.0,
                   r_max: float | None = None):
    """Azimuthal average of the plane z in rings of width dr around (cx, cy).
    Returns (ring centres r, mean values)."""
    plane = field[z]
    ny, nx = plane.shape
    Y, X = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    r = np.sqrt((X - cx) ** 2 + (Y - cy) ** 2)
    if r_max is None:
        r_max = min(cx, cy, nx - 1 - cx, ny - 1 - cy)
    edges = np.arange(0.0, r_max + dr, dr)
    k = np.digitize(r.ravel(), edges) - 1
    ok = (k >= 0) & (k < len(edges) - 1)
    sums = np.bincount(k[ok], weights=plane.ravel()[ok], minlength=len(edges) - 1)
    counts = np.bincount(k[ok], minlength=len(edges) - 1)
    keep = counts > 0
    centres = 0.5 * (edges[:-1] + edges[1:])
    return centres[keep], sums[keep] / counts[keep]


def gaussian_exponent(r: np.ndarray, profile: np.ndarray, z: float, z0: float = 0.0) -> float:
    """Least-squares k of profile / profile(0) = exp(-k (r / (z - z0))^2), fitted on
    log(profile / peak) over the points where the profile exceeds 5 % of its peak."""
    peak = profile[0]
    eta2 = (r / (z - z0)) ** 2
    sel = profile > 0.05 * peak
    y = np.log(profile[sel] / peak)
    x = eta2[sel]
    return float(-np.sum(x * y) / np.sum(x * x))


def inverse_slope(z: np.ndarray, values: np.ndarray, z_min: float, z_max: float) -> float:
    """Slope of the straight-line fit of 1 / values over z_min <= z <= z_max."""
    sel = (z >= z_min) & (z <= z_max)
    return float(np.polyfit(z[sel], 1.0 / values[sel], 1)[0])
