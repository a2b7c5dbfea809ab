"""Seeded synthetic workloads: initial fields and run parameters.

This module holds no arithmetic of the lattice Boltzmann step.  It builds the
initial macroscopic fields (density, velocity, phase field) and the parameter
sets of the workloads the paper simulates (Sec. 3, Table 1), so that the
CUDA library, its tests and the benchmark all start from the same inputs.

Conventions: fields are numpy float64 arrays shaped (nz, ny, nx) (x fastest in
memory), vectors (3, nz, ny, nx); phi in [-1, 1], +1 = component A.
Boundary faces are named by strings in the order (-x, +x, -y, +y, -z, +z):
"periodic", "inlet" (only -z), "outflow", "free_slip".
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence, Tuple

import numpy as np

FACE_NAMES = ("periodic", "inlet", "outflow", "free_slip")
U_CHAR = 0.05  # characteristic jet speed of the paper's runs (Table 1, rows 4-5)


def viscosity_from_reynolds(u: float, d: float, re: float) -> float:
    """Kinematic viscosity of a jet of speed u and diameter d at Reynolds number re (Re = u d / nu)."""
    return u * d / re


def omega_from_viscosity(nu: float) -> float:
    """BGK frequency for viscosity nu in lattice units, nu = (1/3)(1/omega - 1/2) (Sec. 2)."""
    return 1.0 / (3.0 * nu + 0.5)


def sigma_from_weber(u: float, d: float, we: float, rho: float = 1.0) -> float:
    """Surface tension for Weber number we = rho u^2 d / sigma."""
    return rho * u * u * d / we


@dataclasses.dataclass
class Workload:
    """One simulation case: grid, physics parameters, boundaries and length."""

    name: str
    nx: int
    ny: int
    nz: int
    omega: float
    sigma: float
    width: float = 3.0                      # interface width W (Gamma = 1/W)
    normal_eps: float = 1e-2                # regularisation of the interface normal
    faces: Tuple[str, ...] = ("periodic",) * 6
    inlet_u: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    inlet_diameter: float = 0.0
    inlet_cx: float = 0.0
    inlet_cy: float = 0.0
    noise_amp: float = 0.0
    seed: int = 0
    steps: int = 100
    kind: str = "droplet"                   # "droplet" | "jet"
    radius: float = 0.0                     # droplet radius (droplet kind)

    @property
    def nodes(self) -> int:
        return self.nx * self.ny * self.nz

    def fields(self):
        """Initial (rho, u, phi) of this workload."""
        if self.kind == "jet":
            return jet_fields(self.nx, self.ny, self.nz)
        return droplet_fields(self.nx, self.ny, self.nz, self.radius, self.width)


def droplet_fields(nx: int, ny: int, nz: int, radius: float, width: float = 3.0,
                   center: Sequence[float] | None = None):
    """A droplet of component A at rest: phi = -tanh(2 (r - R) / W) with r the
    distance of each node from the centre (default: box centre nx/2, ny/2, nz/2)."""
    if center is None:
        center = (nx / 2.0, ny / 2.0, nz / 2.0)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    r = np.sqrt((x - center[0]) ** 2 + (y - center[1]) ** 2 + (z - center[2]) ** 2)
    phi = -np.tanh(2.0 * (r - radius) / width)
    rho = np.ones((nz, ny, nx))
    u = np.zeros((3, nz, ny, nx))
    return rho, u, phi


def cylinder_fields(nx: int, ny: int, nz: int, radius: float, width: float = 3.0):
    """A cylinder of component A along z (quasi-2D Laplace case), at rest."""
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    r = np.sqrt((x - nx / 2.0) ** 2 + (y - ny / 2.0) ** 2)
    phi = -np.tanh(2.0 * (r - radius) / width)
    return np.ones((nz, ny, nx)), np.zeros((3, nz, ny, nx)), phi


def jet_fields(nx: int, ny: int, nz: int):
    """Quiescent component B filling the box (the jet enters through the inlet)."""
    return np.ones((nz, ny, nx)), np.zeros((3, nz, ny, nx)), -np.ones((nz, ny, nx))


def random_smooth_fields(nx: int, ny: int, nz: int, seed: int, amp_rho: float = 1e-3,
                         amp_u: float = 1e-2, amp_pi: float = 0.0, modes: int = 3,
                         phi_mode: str = "smooth"):
    """Seeded smooth periodic perturbations (a few low Fourier modes per field).
    Returns (rho, u, pi, phi); pi is zero unless amp_pi > 0."""
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")

    def field():
        out = np.zeros((nz, ny, nx))
        for _ in range(modes):
            kx, ky, kz = (rng.integers(0, 3) for _ in range(3))
            ph = rng.uniform(0, 2 * math.pi)
            a = rng.uniform(-1, 1)
            out += a * np.cos(2 * math.pi * (kx * x / nx + ky * y / ny + kz * z / nz) + ph)
        return out / modes

    rho = 1.0 + amp_rho * field()
    u = np.stack([amp_u * field() for _ in range(3)])
    pi = np.stack([amp_pi * field() for _ in range(6)])
    if phi_mode == "smooth":
        phi = np.tanh(2.0 * field())
    else:
        phi = -np.ones((nz, ny, nx))
    return rho, u, pi, phi


def droplet_workload(n: int = 32, radius: float = 8.0, omega: float = 1.6, sigma: float = 0.01,
                     width: float = 3.0, steps: int = 100) -> Workload:
    """Static droplet in a periodic box (radius 8, W = 3, omega 1.6, sigma 0.01 at n = 32)."""
    return Workload(name=f"droplet{n}", nx=n, ny=n, nz=n, omega=omega, sigma=sigma, width=width,
                    faces=("periodic",) * 6, steps=steps, kind="droplet", radius=radius)


def jet_workload(nx: int = 192, ny: int = 192, nz: int = 384, diameter: float = 16.0,
                 u: float = U_CHAR, re: float = 5000.0, we: float = 100.0, noise: float = 0.01,
                 seed: int = 1, width: float = 3.0, steps: int = 2000,
                 side: str = "free_slip") -> Workload:
    """Axisymmetric jet: nozzle of diameter D centred on the z = 0 face, inflow u
    along +z with uniform random velocity noise, outflow at the top, side walls."""
    nu = viscosity_from_reynolds(u, diameter, re)
    return Workload(name=f"jet{nx}x{ny}x{nz}", nx=nx, ny=ny, nz=nz,
                    omega=omega_from_viscosity(nu), sigma=sigma_from_weber(u, diameter, we),
                    width=width, faces=(side, side, side, side, "inlet", "outflow"),
                    inlet_u=(0.0, 0.0, u), inlet_diameter=diameter, inlet_cx=nx / 2.0,
                    inlet_cy=ny / 2.0, noise_amp=noise, seed=seed, steps=steps, kind="jet")


def weber_sweep(nx: int = 512, ny: int = 512, nz: int = 1024, diameter: float = 40.0,
                webers: Sequence[float] = (10.0, 100.0, 500.0, 2000.0), seed: int = 2,
                steps: int = 500) -> List[Workload]:
    """The large jet at Re = 5000 for several Weber numbers (set through sigma)."""
    return [jet_workload(nx, ny, nz, diameter=diameter, we=we, seed=seed, steps=steps)
            for we in webers]


def batched_ensemble(count: int = 64, seed: int = 4, edges: Sequence[int] = (48, 64, 96, 128),
                     steps: int = 200) -> List[Workload]:
    """Independent periodic droplets and jets of uneven cubic sizes: edge uniform
    in `edges`, droplet or jet with equal odds, We log-uniform in [10, 2000]."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        e = int(rng.choice(edges))
        we = float(math.exp(rng.uniform(math.log(10.0), math.log(2000.0))))
        if rng.random() < 0.5:
            r = 0.25 * e
            w = droplet_workload(e, radius=r, omega=1.6, sigma=sigma_from_weber(U_CHAR, 2 * r, we),
                                 steps=steps)
            w.name = f"droplet{e}_{k}"
        else:
            d = float(round(0.15 * e))
            w = jet_workload(e, e, e, diameter=d, we=we, seed=seed * 1000 + k, steps=steps,
                             side="periodic")
            w.name = f"jet{e}_{k}"
        out.append(w)
    return out


def crop_jet(w: Workload, nx: int, ny: int, nz: int, diameter: float | None = None) -> Workload:
    """The same jet on a smaller box with the nozzle kept centred."""
    d = w.inlet_diameter if diameter is None else diameter
    return dataclasses.replace(w, name=f"jet{nx}x{ny}x{nz}", nx=nx, ny=ny, nz=nz,
                               inlet_diameter=d, inlet_cx=nx / 2.0, inlet_cy=ny / 2.0)
