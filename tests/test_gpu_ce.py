"""Parity of the Chapman-Enskog closure (Sec. 2.1: a2_neq from the strain rate
of j, 5 stored fields) on the GPU with the FP64 oracle run with the same
closure.  Same error norms and bar as the projection closure: rho relative to
max|rho|, u relative to max(max|u|, 0.05), phi absolute, 1e-5 after 100
steps; and on their own scales u relative to max|u_ref| (where that exceeds
1e-4) and the stored rho - 1 relative to max|rho_ref - 1|."""
import numpy as np
import pytest
import torch

import oracle
import paper_2403_15773_gb300 as tslb
from paper_2403_15773_gb300 import inputs
from _util import oracle_params, oracle_sim

pytestmark = pytest.mark.gpu
TOL = 1e-5
CE = "chapman_enskog"


def gpu_run(w, steps, fields=None, **kw):
    rho, u, phi = w.fields() if fields is None else fields
    sim = tslb.Simulation(w, closure=CE, **kw)
    sim.set_state(torch.from_numpy(np.asarray(rho)), torch.from_numpy(np.asarray(u)),
                  torch.from_numpy(np.asarray(phi)))
    sim.step(steps)
    out = sim.fields_numpy()
    if kw.get("storage", "fp32") == "fp32":  # the stored rho - 1 (raw state, field 0)
        raw = sim.get_state()[:4 * w.nodes].view(torch.float32)
        out = out + (raw.double().cpu().numpy().reshape(out[0].shape),)
    sums = sim.sums()
    launches = sim.kernel_launches
    sim.close()
    return out, sums, launches


def errors(g, r):
    e_rho = np.max(np.abs(g[0] - r[0])) / np.max(np.abs(r[0]))
    e_u = np.max(np.abs(g[1] - r[1])) / max(np.max(np.abs(r[1])), 0.05)
    e_phi = np.max(np.abs(g[3] - r[3]))
    return e_rho, e_u, e_phi


def check_parity(w, steps, fields=None, **kw):
    g, sums, launches = gpu_run(w, steps, fields, **kw)
    assert g[2] is None
    s = oracle_sim(w, fields=fields, ce_neq=True)
    s.step(steps)
    r = s.moments()
    e = errors(g, r)
    umax = np.max(np.abs(r[1]))
    eu = np.max(np.abs(g[1] - r[1])) / umax if umax > 1e-4 else None
    d_gpu = g[4] if len(g) > 4 else g[0] - 1.0
    ed = np.max(np.abs(d_gpu - (r[0] - 1.0))) / np.max(np.abs(r[0] - 1.0))
    print(f"CE parity {w.name} {w.nx}x{w.ny}x{w.nz} {steps} steps: err rho {e[0]:.2e} u {e[1]:.2e} "
          f"phi {e[2]:.2e} | own scale: u {'-' if eu is None else f'{eu:.2e}'}, rho-1 {ed:.2e}")
    assert launches == steps
    assert max(e) < TOL, f"{w.name}: err rho {e[0]:.2e} u {e[1]:.2e} phi {e[2]:.2e}"
    assert eu is None or eu < TOL, f"{w.name}: err u on max|u_ref| {eu:.2e}"
    assert ed < TOL, f"{w.name}: err rho - 1 on max|rho_ref - 1| {ed:.2e}"
    m_ref, p_ref, _ = s.sums()
    assert abs(sums[0] - m_ref) / m_ref < 1e-6
    assert abs(sums[1] - p_ref) / np.sum(np.abs(r[3])) < 1e-6
    return e


def test_droplet_32_periodic_100_steps():
    check_parity(inputs.droplet_workload(), 100)


def test_jet_all_boundaries_100_steps():
    """Free-slip sides, inlet with 1 % noise, outflow: every ghost rule."""
    w = inputs.jet_workload(48, 40, 44, diameter=12, we=100, noise=0.01, seed=3)
    check_parity(w, 100)


def test_jet_crop_of_the_192x192x384_geometry():
    w = inputs.crop_jet(inputs.jet_workload(), 64, 64, 64)
    check_parity(w, 100)


def test_ragged_tiles_mixed_faces():
    """33 x 17 x 29: partial tiles in every direction, periodic x, free-slip y,
    outflow z, an off-centre droplet in a random smooth flow."""
    w = inputs.droplet_workload(8, radius=6.0)
    w.nx, w.ny, w.nz = 33, 17, 29
    w.faces = ("periodic", "periodic", "free_slip", "free_slip", "outflow", "outflow")
    w.name = "ragged"
    rho0, u0, _, _ = inputs.random_smooth_fields(33, 17, 29, seed=8, amp_rho=2e-3, amp_u=2e-2)
    _, _, phi = inputs.droplet_fields(33, 17, 29, 6.0, 3.0, center=(13.0, 8.0, 15.0))
    check_parity(w, 100, fields=(rho0, u0, phi))


@pytest.mark.parametrize("dims,faces", [
    ((48, 40, 1), ("periodic",) * 6),
    ((2, 30, 20), ("free_slip", "free_slip", "periodic", "periodic", "outflow", "outflow")),
    ((70, 3, 5), ("periodic", "periodic", "free_slip", "free_slip", "periodic", "periodic")),
])
def test_thin_and_small_grids(dims, faces):
    nx, ny, nz = dims
    w = inputs.droplet_workload(8, radius=5.0)
    w.nx, w.ny, w.nz, w.faces, w.name = nx, ny, nz, faces, f"small{nx}x{ny}x{nz}"
    rho0, u0, _, phi = inputs.random_smooth_fields(nx, ny, nz, seed=21, amp_rho=2e-3, amp_u=2e-2)
    check_parity(w, 50, fields=(rho0, u0, phi))


def test_rest_state_is_bitwise_fixed():
    w = inputs.droplet_workload(24)
    for phi0 in (1.0, -1.0):
        g, _, _ = gpu_run(w, 40, fields=(np.ones((24, 24, 24)), np.zeros((3, 24, 24, 24)),
                                         np.full((24, 24, 24), phi0)))
        assert np.all(g[0] == 1.0) and np.all(g[1] == 0.0) and np.all(g[3] == phi0)


@pytest.mark.parametrize("tile_z,block_warps", [(1, 8), (7, 8), (0, 12), (13, 12)])
def test_fields_independent_of_tiling(tile_z, block_warps):
    """Every node's arithmetic is the same in whatever tile it lands."""
    w = inputs.jet_workload(64, 50, 40, diameter=10, noise=0.01, seed=5)
    ref, _, _ = gpu_run(w, 30)
    got, _, _ = gpu_run(w, 30, tile_z=tile_z, block_warps=block_warps)
    for k in (0, 1, 3):
        assert np.array_equal(got[k], ref[k]), k


def test_checkpoint_is_five_fields_and_resumes_bitwise():
    w = inputs.jet_workload(40, 36, 30, diameter=10, noise=0.01, seed=4)
    rho, u, phi = w.fields()
    a = tslb.Simulation(w, closure=CE)
    a.set_state(torch.from_numpy(rho), torch.from_numpy(u), torch.from_numpy(phi))
    assert a.state_bytes() == 5 * w.nodes * 4 + 8
    a.step(7)
    buf = a.get_state()
    a.step(9)
    ref = a.fields_numpy()
    b = tslb.Simulation(w, closure=CE)
    b.put_state(buf)
    assert b.t == 7
    b.step(9)
    got = b.fields_numpy()
    for k in (0, 1, 3):
        assert np.array_equal(got[k], ref[k])
    with pytest.raises(tslb.TslbError):
        tslb.tslb_get_moments(a.ctx, 0, 0, torch.empty(6 * w.nodes, device="cuda").data_ptr(), 1)
    a.close()
    b.close()


@pytest.mark.parametrize("storage", ["fp16", "bf16"])
def test_16bit_storage_against_fp32(storage):
    """5 stored fields in 16 bits: rms error on the parity scales within 16
    unit roundoffs of the storage format after 300 steps of a droplet."""
    eps = {"fp16": 2.0 ** -11, "bf16": 2.0 ** -8}[storage]
    w = inputs.droplet_workload(48, radius=12.0)
    f32, _, _ = gpu_run(w, 300)
    g, _, _ = gpu_run(w, 300, storage=storage)
    scales = [1.0, max(np.abs(f32[1]).max(), 0.05), None, 1.0]
    for k in (0, 1, 3):
        d = np.abs(g[k] - f32[k]) / scales[k]
        rms = float(np.sqrt(np.mean(d * d)))
        print(f"CE {storage} field {k}: max {d.max():.2e} rms {rms:.2e}")
        assert rms < 16 * eps, (storage, k, rms)


def test_time_averages_match_oracle():
    w = inputs.jet_workload(40, 36, 30, diameter=10, noise=0.01, seed=6)
    rho, u, phi = w.fields()
    sim = tslb.Simulation(w, closure=CE, average=True)
    sim.set_state(torch.from_numpy(rho), torch.from_numpy(u), torch.from_numpy(phi))
    s = oracle_sim(w, ce_neq=True)
    acc_phi = np.zeros_like(phi)
    acc_uz = np.zeros_like(phi)
    for _ in range(20):
        sim.step(1)
        s.step(1)
        r = s.moments()
        acc_phi += r[3]
        acc_uz += r[1][2]
    aphi, auz, n = sim.averages()
    sim.close()
    assert n == 20
    assert np.max(np.abs(aphi - acc_phi / 20)) < TOL
    assert np.max(np.abs(auz - acc_uz / 20)) / 0.05 < TOL


def test_full_size_jet_sampled_step():
    """The 192 x 192 x 384 jet in the benchmark's launch configuration (the
    tile shape its autotuner picks): after 60 steps, one more step checked
    node by node at 3000 sampled nodes (faces, nozzle, interior) against the
    oracle's single-step evaluation from the same stored state."""
    w = inputs.jet_workload()
    rho, u, phi = w.fields()
    sim = tslb.Simulation(w, closure=CE)
    sim.set_state(torch.from_numpy(rho), torch.from_numpy(u), torch.from_numpy(phi))
    shape = sim.autotune(6)
    sim.step(60)
    before = sim.fields_numpy()
    t = sim.t
    sim.step(1)
    after = sim.fields_numpy()
    sim.close()
    nx, ny, nz = w.nx, w.ny, w.nz
    rng = np.random.default_rng(1)
    pts = [rng.integers(0, [nx, ny, nz], size=(1500, 3))]
    for axis, val in ((0, 0), (0, nx - 1), (1, 0), (1, ny - 1), (2, 0), (2, 1), (2, nz - 1)):
        p = rng.integers(0, [nx, ny, nz], size=(150, 3))
        p[:, axis] = val
        pts.append(p)
    pts.append(np.stack([rng.integers(88, 104, 200), rng.integers(88, 104, 200), rng.integers(0, 6, 200)], 1))
    P = np.concatenate(pts)
    idx = P[:, 0] + nx * (P[:, 1] + ny * P[:, 2])
    flat = lambda a: a.reshape(a.shape[0], -1) if a.ndim == 4 else a.reshape(-1)
    N = w.nodes
    out = oracle.step_sample(oracle_params(w, ce_neq=True), t, flat(before[0]), flat(before[1]),
                             np.zeros(6 * N), flat(before[3]), idx)
    e_rho = np.max(np.abs(flat(after[0])[idx] - out[:, 0])) / np.max(np.abs(out[:, 0]))
    e_u = np.max(np.abs(flat(after[1])[:, idx].T - out[:, 1:4])) / max(np.max(np.abs(out[:, 1:4])), 0.05)
    e_phi = np.max(np.abs(flat(after[3])[idx] - out[:, 10]))
    print(f"CE parity full-size sampled step, tile {shape}: err rho {e_rho:.2e} u {e_u:.2e} phi {e_phi:.2e}")
    assert max(e_rho, e_u, e_phi) < TOL, (e_rho, e_u, e_phi)


def test_departs_from_projection_closure_as_the_oracle_does():
    """The GPU's difference between the two closures is the oracle's."""
    w = inputs.droplet_workload(24, radius=7.0, sigma=0.01)
    g_ce, _, _ = gpu_run(w, 60)
    sim = tslb.Simulation(w)
    rho, u, phi = w.fields()
    sim.set_state(torch.from_numpy(rho), torch.from_numpy(u), torch.from_numpy(phi))
    sim.step(60)
    g_pr = sim.fields_numpy()
    sim.close()
    r_ce = oracle_sim(w, ce_neq=True)
    r_ce.step(60)
    r_pr = oracle_sim(w)
    r_pr.step(60)
    d_gpu = g_ce[1] - g_pr[1]
    d_orc = r_ce.moments()[1] - r_pr.moments()[1]
    assert np.max(np.abs(d_gpu - d_orc)) < 1e-3 * np.max(np.abs(d_orc)) + 1e-7


@pytest.mark.parametrize("block_warps", [8, 12])
def test_plain_store_form_parity(block_warps):
    """The plain-store form (the one the autotuner picks for this closure on
    FP32 grids): parity with the oracle on every ghost rule of the jet, and on
    ragged tiles with mirror faces."""
    w = inputs.jet_workload(48, 40, 44, diameter=12, we=100, noise=0.01, seed=3)
    check_parity(w, 100, plain_stores=True, block_warps=block_warps)
    w = inputs.droplet_workload(8, radius=6.0)
    w.nx, w.ny, w.nz = 36, 17, 29
    w.faces = ("free_slip", "free_slip", "free_slip", "free_slip", "outflow", "outflow")
    w.name = "ragged_mirror"
    rho0, u0, _, _ = inputs.random_smooth_fields(36, 17, 29, seed=8, amp_rho=2e-3, amp_u=2e-2)
    _, _, phi = inputs.droplet_fields(36, 17, 29, 6.0, 3.0, center=(13.0, 8.0, 15.0))
    check_parity(w, 60, fields=(rho0, u0, phi), plain_stores=True, block_warps=block_warps)


@pytest.mark.parametrize("block_warps", [8, 12])
def test_staged_stores_equal_plain_stores(block_warps):
    """FP32 grids with 16-byte rows write finished planes through a staging box
    and one TMA store per plane; the plain-store form writes the same bits."""
    for w in (inputs.jet_workload(64, 50, 40, diameter=10, noise=0.01, seed=5),
              inputs.droplet_workload(48, radius=12.0)):
        a, sa, _ = gpu_run(w, 12, block_warps=block_warps)
        b, sb, _ = gpu_run(w, 12, block_warps=block_warps, plain_stores=True)
        for k in (0, 1, 3):
            assert np.array_equal(a[k], b[k])
        assert sa == sb
