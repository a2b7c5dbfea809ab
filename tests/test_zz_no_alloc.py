"""tslb_field_sums_noalloc: FP64 totals of caller-owned fields without any
device allocation.

It exists for callers that must not allocate device memory when they ask for
the totals: cudaMalloc / cudaFree synchronise the whole device (an
asynchronous solver loop cannot afford that), and a process whose device
memory sits in another allocator's pool may have nothing left to allocate.
The check: its result equals the context's tslb_sums on the same state, on
two calls in a row (the second after more steps, so the shared scratch holds
the first call's partials when it starts).
"""
import numpy as np
import pytest
import torch

import paper_2403_15773_gb300 as tslb
from paper_2403_15773_gb300 import inputs

REL_TOL = 1e-6  # the tolerance of the FP64 sums in the parity tests


@pytest.mark.gpu
def test_noalloc_sums_match_context_sums_on_two_calls():
    w = inputs.jet_workload(48, 40, 44, diameter=12, we=100, noise=0.01, seed=3)
    rho0, u0, phi0 = w.fields()
    sim = tslb.Simulation(w)
    sim.set_state(torch.from_numpy(rho0), torch.from_numpy(u0), torch.from_numpy(phi0))
    out = torch.zeros(2, dtype=torch.float64, device="cuda")  # the caller's output buffer
    for call in range(2):
        sim.step(25)
        rho, _, _ = sim.moments()
        phi = sim.phi()
        mass, phi_total = sim.sums()  # existing entry point (context workspace)
        tslb.tslb_field_sums_noalloc(rho.data_ptr(), phi.data_ptr(), w.nodes, out.data_ptr(), 0)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert abs(got[0] - mass) / mass < REL_TOL, (call, got[0], mass)
        assert abs(got[1] - phi_total) / float(torch.sum(torch.abs(phi.double()))) < REL_TOL, \
            (call, got[1], phi_total)
    sim.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    """n above 16384 x 16384 values is refused before any GPU work."""
    with pytest.raises(tslb.TslbError) as ei:
        tslb.tslb_field_sums_noalloc(1, 1, 16384 * 16384 + 1, 1, 0)
    assert ei.value.status == tslb.TSLB_ERR_INVALID_ARG
    assert "268435456" in tslb.tslb_last_error(None)
    with pytest.raises(tslb.TslbError):
        tslb.tslb_field_sums_noalloc(1, 1, 0, 1, 0)
