"""Workload recipes: the jet parameters reproduce the consistent rows of the
paper's Table 1 (Sec. 3), and the synthetic ensembles are seeded."""
import os

import numpy as np

from paper_2403_15773_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_table1_rows_reproduced():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "table1_parameters.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 2
    for sim, U, sigma, nu, D, Re, We in rows:
        w = inputs.jet_workload(400, 400, 800, diameter=float(D), u=float(U), re=float(Re),
                                we=float(We))
        nu_w = (1.0 / 3.0) * (1.0 / w.omega - 0.5)
        assert abs(nu_w - float(nu)) < 1e-12
        assert abs(w.sigma - float(sigma)) < 1e-15


def test_jet_config_parameters():
    w = inputs.jet_workload()
    assert (w.nx, w.ny, w.nz) == (192, 192, 384)
    assert abs((1.0 / 3.0) * (1.0 / w.omega - 0.5) - 1.6e-4) < 1e-15
    assert abs(w.omega - 1.998082) < 1e-6
    assert abs(w.sigma - 4e-4) < 1e-15
    assert w.faces == ("free_slip",) * 4 + ("inlet", "outflow")
    assert w.inlet_cx == 96 and w.inlet_cy == 96 and w.inlet_diameter == 16
    # Mach number of the jet stays far below the 0.6 threshold of Sec. 3
    assert w.inlet_u[2] / (1.0 / 3.0) ** 0.5 < 0.1


def test_weber_sweep_sigmas():
    ws = inputs.weber_sweep()
    assert [round(w.sigma, 12) for w in ws] == [1e-2, 1e-3, 2e-4, 5e-5]
    assert all(abs(w.omega - 1.995211) < 1e-6 for w in ws)


def test_batched_ensemble_seeded():
    a = inputs.batched_ensemble()
    b = inputs.batched_ensemble()
    assert len(a) == 64
    assert [(w.name, w.nx, w.sigma) for w in a] == [(w.name, w.nx, w.sigma) for w in b]
    assert {w.nx for w in a} <= {48, 64, 96, 128}
    assert all(w.nx == w.ny == w.nz for w in a)
    kinds = {w.kind for w in a}
    assert kinds == {"droplet", "jet"}


def test_droplet_fields_shape_and_profile():
    rho, u, phi = inputs.droplet_fields(32, 32, 32, 8.0, 3.0)
    assert rho.shape == (32, 32, 32) and u.shape == (3, 32, 32, 32)
    assert phi[16, 16, 16] > 0.9999 and phi[0, 0, 0] < -0.9999
    assert np.all(np.abs(phi) <= 1.0)
