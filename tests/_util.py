"""Shared helpers of the tests: workload -> oracle parameters, error norms."""
from __future__ import annotations

import numpy as np

import oracle
from paper_2403_15773_gb300 import inputs

_FACE = {"periodic": oracle.PERIODIC, "inlet": oracle.INLET, "outflow": oracle.OUTFLOW,
         "free_slip": oracle.FREE_SLIP}


def oracle_params(w: inputs.Workload, **over) -> oracle.Params:
    kw = dict(nx=w.nx, ny=w.ny, nz=w.nz, omega=w.omega, sigma=w.sigma,
              gamma=(1.0 / w.width) if w.width > 0 else 0.0,
              faces=[_FACE[f] for f in w.faces], inlet_u=w.inlet_u,
              inlet_diameter=w.inlet_diameter, inlet_cx=w.inlet_cx, inlet_cy=w.inlet_cy,
              inlet_width=w.width if w.width > 0 else 3.0, noise_amp=w.noise_amp, seed=w.seed,
              normal_eps=w.normal_eps)
    kw.update(over)
    return oracle.make_params(**kw)


def oracle_sim(w: inputs.Workload, fields=None, **over) -> oracle.OracleSim:
    s = oracle.OracleSim(oracle_params(w, **over))
    rho, u, phi = w.fields() if fields is None else fields
    s.set_state(rho, u, phi)
    return s


def scaled_max_error(x, ref, scale) -> float:
    """max |x - ref| / scale."""
    return float(np.max(np.abs(np.asarray(x, dtype=np.float64) - ref)) / scale)
