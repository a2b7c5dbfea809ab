"""Batched ensembles and the tile autotuner.

Every node's arithmetic is the same in whatever tile (and launch) it is
computed, so each grid of a batch must be bitwise equal to the same grid run
alone, and autotuning (which only recomputes the current step into the spare
buffer) must leave the trajectory unchanged."""
import numpy as np
import pytest
import torch

import paper_2403_15773_gb300 as tslb
from paper_2403_15773_gb300 import inputs
from _util import oracle_sim

pytestmark = pytest.mark.gpu


def small_ensemble():
    ws = [
        inputs.droplet_workload(24, radius=6.0, sigma=0.02),
        inputs.jet_workload(32, 32, 32, diameter=6, we=300, seed=11, side="periodic"),
        inputs.droplet_workload(40, radius=10.0, omega=1.9, sigma=0.005),
        inputs.jet_workload(48, 36, 40, diameter=8, we=50, seed=12),
        inputs.droplet_workload(16, radius=4.0, omega=1.2),
        inputs.jet_workload(30, 44, 20, diameter=6, we=1000, seed=13),
    ]
    return ws


def single_run(w, steps, **kw):
    s = tslb.Simulation(w, **kw)
    rho, u, phi = w.fields()
    s.set_state(torch.from_numpy(rho), torch.from_numpy(u), torch.from_numpy(phi))
    s.step(steps)
    out = s.fields_numpy()
    sums = s.sums()
    s.close()
    return out, sums


@pytest.mark.parametrize("block_warps,tile_z,plain", [(8, 16, False), (12, 32, False), (8, 0, False),
                                                     (12, 24, True), (8, 40, True)])
def test_batch_equals_each_grid_alone(block_warps, tile_z, plain):
    ws = small_ensemble()
    b = tslb.BatchSimulation(ws, block_warps=block_warps, tile_z=tile_z, plain_stores=plain)
    for i, w in enumerate(ws):
        rho, u, phi = w.fields()
        b.set_state(i, rho, u, phi)
    b.step(30)
    assert b.kernel_launches == 30
    for i, w in enumerate(ws):
        got = b.fields_numpy(i)
        ref, ref_sums = single_run(w, 30)
        for k in range(4):
            assert np.array_equal(got[k], ref[k]), (i, k)
        # totals: each thread sums at most 64 planes in FP32 before the FP64
        # reduction, and that grouping follows the tile shape
        m, p = b.sums(i)
        eps32 = 2.0 ** -24
        assert abs(m - ref_sums[0]) <= 64 * eps32 * float(np.sum(np.abs(ref[0] - 1.0))) + 1e-9
        assert abs(p - ref_sums[1]) <= 64 * eps32 * float(np.sum(np.abs(ref[3]))) + 1e-9
    b.close()


def test_batch_grid_matches_oracle():
    ws = small_ensemble()
    b = tslb.BatchSimulation(ws)
    for i, w in enumerate(ws):
        b.set_state(i, *w.fields())
    b.step(60)
    for i in (1, 3):
        g = b.fields_numpy(i)
        s = oracle_sim(ws[i])
        s.step(60)
        r = s.moments()
        e_rho = np.max(np.abs(g[0] - r[0])) / np.max(np.abs(r[0]))
        e_u = np.max(np.abs(g[1] - r[1])) / max(np.max(np.abs(r[1])), 0.05)
        e_phi = np.max(np.abs(g[3] - r[3]))
        assert max(e_rho, e_u, e_phi) < 1e-5, (i, e_rho, e_u, e_phi)
    b.close()


def test_autotune_does_not_change_the_trajectory():
    w = inputs.jet_workload(64, 48, 80, diameter=10, seed=21)
    ref, _ = single_run(w, 25)
    s = tslb.Simulation(w)
    rho, u, phi = w.fields()
    s.set_state(torch.from_numpy(rho), torch.from_numpy(u), torch.from_numpy(phi))
    s.step(5)
    nw, tz, plain = s.autotune(4)
    assert nw in (8, 12, 16) and 8 <= tz <= 128 and plain in (0, 1)
    assert s.t == 5
    s.step(20)
    got = s.fields_numpy()
    s.close()
    for k in range(4):
        assert np.array_equal(got[k], ref[k])


def test_batch_autotune_keeps_state():
    ws = small_ensemble()[:3]
    a = tslb.BatchSimulation(ws)
    b = tslb.BatchSimulation(ws)
    for sim in (a, b):
        for i, w in enumerate(ws):
            sim.set_state(i, *w.fields())
        sim.step(4)
    a.autotune(2)
    a.step(10)
    b.step(10)
    for i in range(len(ws)):
        ga, gb = a.fields_numpy(i), b.fields_numpy(i)
        for k in range(4):
            assert np.array_equal(ga[k], gb[k])
    a.close()
    b.close()


def test_batch_step_after_autotune_runs_every_tile():
    """The autotuner re-runs the same step many times; afterwards the next
    step must again take every tile (its tile counter rearmed): a new state
    set after tuning is stepped, not left at the trials' result."""
    ws = small_ensemble()[:3]
    new = [inputs.random_smooth_fields(w.nx, w.ny, w.nz, seed=40 + i, amp_rho=1e-3, amp_u=1e-2)
           for i, w in enumerate(ws)]
    a = tslb.BatchSimulation(ws)
    for i, w in enumerate(ws):
        a.set_state(i, *w.fields())
    a.autotune(2)
    b = tslb.BatchSimulation(ws)
    for sim in (a, b):
        for i, (rho, u, _, _) in enumerate(new):
            sim.set_state(i, rho, u, ws[i].fields()[2])
        sim.step(1)
    for i in range(len(ws)):
        ga, gb = a.fields_numpy(i), b.fields_numpy(i)
        for k in range(4):
            assert np.array_equal(ga[k], gb[k]), (i, k)
    a.close()
    b.close()


def test_full_ensemble_in_the_benchmark_configuration():
    """The 64-grid ensemble of the benchmark, autotuned as bench.py does: after
    three steps its smallest grid, a jet and its largest grid equal the same
    grids run alone, bit for bit."""
    ws = inputs.batched_ensemble()
    b = tslb.BatchSimulation(ws)
    for i, w in enumerate(ws):
        b.set_state(i, *w.fields())
    nw, tz, plain = b.autotune(3)
    assert nw in (8, 12) and plain in (0, 1)
    b.step(3)
    sizes = [w.nodes for w in ws]
    jets = [i for i, w in enumerate(ws) if w.kind == "jet"]
    picks = {int(np.argmin(sizes)), int(np.argmax(sizes)), jets[0]}
    for i in sorted(picks):
        got = b.fields_numpy(i)
        ref, _ = single_run(ws[i], 3)
        for k in range(4):
            assert np.array_equal(got[k], ref[k]), (i, k)
    b.close()


def test_batch_one_load_path_form_equals_per_tile_form():
    """A batch whose grids all load every tile by TMA (16-byte rows; periodic
    grids wider than a tile, through the side boxes) runs 12-warp
    staged-store steps in the kernel compiled for TMA loads alone: the same
    bits and sums as the per-tile kernel (option per_tile_loads); one narrow
    periodic grid in the batch (its only tile wraps both ways) keeps the
    per-tile kernel for the whole batch."""
    ws = [inputs.droplet_workload(48, radius=11.0),
          inputs.jet_workload(56, 48, 40, diameter=8, we=300, seed=11, side="periodic"),
          inputs.jet_workload(72, 50, 30, diameter=10, we=50, seed=12)]
    runs = []
    for per_tile in (False, True):
        b = tslb.BatchSimulation(ws, block_warps=12, tile_z=24, per_tile_loads=per_tile)
        for i, w in enumerate(ws):
            b.set_state(i, *w.fields())
        form = b.step_form()
        b.step(20)
        runs.append((form, [b.fields_numpy(i) for i in range(len(ws))], [b.sums(i) for i in range(len(ws))]))
        b.close()
    assert runs[0][0] == (12, 24, 0, 1), runs[0][0]
    assert runs[1][0][3] == 0, runs[1][0]
    for i in range(len(ws)):
        for k in range(4):
            assert np.array_equal(runs[0][1][i][k], runs[1][1][i][k]), (i, k)
        assert runs[0][2][i] == runs[1][2][i]
    b = tslb.BatchSimulation(ws + [inputs.droplet_workload(24, radius=6.0)], block_warps=12)
    assert b.step_form()[3] == 0
    b.close()
