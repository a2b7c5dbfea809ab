"""The z-slab decomposition on the GPU: a domain split into slab contexts
(halo faces toward their neighbours, ghost planes written by
tslb_halo_unpack from the neighbours' tslb_halo_pack messages before every
step) advances exactly like one context holding the whole domain.  The slabs
are contexts of one process on one GPU exchanging through device copies
(slabs.exchange_in_process): no kernel waits for another, the exchange is
ordered by the host between steps.  Every node's arithmetic is the same, so
the fields are bitwise equal; the summed totals agree to the rounding of the
kernel's per-thread partial sums."""
import numpy as np
import pytest
import torch

import paper_2403_15773_gb300 as tslb
from paper_2403_15773_gb300 import inputs, slabs

pytestmark = pytest.mark.gpu


def _case(name):
    if name.startswith("jet"):
        nx, ny, nz = (48, 40, 44) if name == "jet" else (33, 20, 24)
        w = inputs.jet_workload(nx, ny, nz, diameter=10, we=100, noise=0.01, seed=9)
        rho, u, pi, _ = inputs.random_smooth_fields(nx, ny, nz, seed=3, amp_rho=1e-2, amp_u=1e-2, amp_pi=5e-4)
        _, _, phi = inputs.droplet_fields(nx, ny, nz, 6.0, 3.0, center=(nx / 2.0, ny / 2.0, 0.6 * nz))
        return w, (rho, u, pi, phi), False
    w = inputs.droplet_workload(48, radius=10.0)
    w.ny, w.nz = 44, 40
    rho, u, pi, _ = inputs.random_smooth_fields(48, 44, 40, seed=4, amp_rho=1e-2, amp_u=1e-2, amp_pi=5e-4)
    _, _, phi = inputs.droplet_fields(48, 44, 40, 10.0, 3.0, center=(20.0, 22.0, 38.0))  # across the z wrap
    return w, (rho, u, pi, phi), True


@pytest.mark.parametrize("name,parts", [("jet", 2), ("jet", 3), ("jet_ragged", 2), ("droplet", 2)])
def test_slab_contexts_equal_one_context(name, parts):
    w, (rho, u, pi, phi), periodic = _case(name)
    steps = 30
    whole = tslb.Simulation(w, graph_steps=1)
    whole.set_state(rho, u, phi, pi)
    whole.step(steps)
    ref = whole.fields_numpy()
    ref_sums = whole.sums()
    whole.close()

    sims, parts_ = [], [slabs.partition(w.nz, parts, r, periodic_z=periodic) for r in range(parts)]
    for sl in parts_:
        s = tslb.Simulation(slabs.slab_workload(w, sl), graph_steps=1)
        z = slice(sl.z0, sl.z1)
        s.set_state(rho[z], u[:, z], phi[z], pi[:, z])
        sims.append(s)
    for _ in range(steps):
        slabs.exchange_in_process(sims)
        for s in sims:
            s.step(1)
    got = [s.fields_numpy() for s in sims]
    sums = [s.sums() for s in sims]
    for s in sims:
        s.close()
    for k in range(4):
        axis = 0 if k in (0, 3) else 1
        cat = np.concatenate([g[k] for g in got], axis=axis)
        assert np.array_equal(cat, ref[k]), (name, parts, k)
    # the step kernel sums each thread's nodes along its z march in FP32 before
    # the FP64 block and grid sums, so other slab boundaries round differently
    # (~1e-9 relative): the parity tests' tolerance of the totals
    m = sum(x[0] for x in sums)
    p = sum(x[1] for x in sums)
    assert abs(m - ref_sums[0]) / ref_sums[0] < 1e-6
    assert abs(p - ref_sums[1]) / float(np.sum(np.abs(ref[3]))) < 1e-6


def test_halo_calls_are_checked():
    w = inputs.jet_workload(32, 24, 16, diameter=8)
    s = tslb.Simulation(w)
    buf = torch.empty(tslb.tslb_halo_values(s.ctx), dtype=torch.float32, device="cuda")
    assert buf.numel() == 12 * 32 * 24
    with pytest.raises(tslb.TslbError) as ei:  # before any state
        tslb.tslb_halo_pack(s.ctx, 0, buf.data_ptr(), 1)
    assert ei.value.status == tslb.TSLB_ERR_STATE
    s.set_state(*w.fields())
    tslb.tslb_halo_pack(s.ctx, 1, buf.data_ptr(), 1)
    with pytest.raises(tslb.TslbError) as ei:  # the inlet face has no ghost planes to fill
        tslb.tslb_halo_unpack(s.ctx, 0, buf.data_ptr(), 1)
    assert ei.value.status == tslb.TSLB_ERR_INVALID_ARG
    s.close()
