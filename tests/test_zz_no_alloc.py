"""tslb_field_sums_noalloc: FP64 totals of caller-owned fields without any
device allocation.

It exists for callers that must not allocate device memory when they ask for
the totals: cudaMalloc / cudaFree synchronise the whole device (an
asynchronous solver loop cannot afford that), and a process whose device
memory sits in another allocator's pool may have nothing left to allocate.
The checks:
  - its result equals the context's tslb_sums on the same state and an FP64
    host sum of the same fields, on two calls in a row (the second after more
    steps, so the shared scratch holds the first call's partials when it
    starts), and the device's free memory is the same before and after the
    second call;
  - on fields whose totals are exact in FP64 whatever the summation order
    (multiples of 2^-10), it returns those totals exactly, with the last block
    of 16384 values partly filled, exactly filled, and with the scratch full
    (n = 16384 x 16384).
"""
import numpy as np
import pytest
import torch

import paper_2403_15773_gb300 as tslb
from paper_2403_15773_gb300 import inputs

REL_TOL = 1e-6   # the tolerance of the FP64 sums against the context sums in the parity tests
HOST_TOL = 1e-12  # FP64 against FP64: only the summation order differs
CHUNK = 16384     # values per block partial of the entry point's scratch
MAX_N = CHUNK * CHUNK


@pytest.mark.gpu
def test_noalloc_sums_match_context_and_host_sums_on_two_calls():
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
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        tslb.tslb_field_sums_noalloc(rho.data_ptr(), phi.data_ptr(), w.nodes, out.data_ptr(), 0)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        if call == 1:  # (the first call may load the library's kernels onto the device)
            assert free1 == free0, (free0, free1)
        got = out.cpu().numpy()
        h_rho = rho.double().cpu().numpy()
        h_phi = phi.double().cpu().numpy()
        scale_phi = float(np.sum(np.abs(h_phi)))
        assert abs(got[0] - mass) / mass < REL_TOL, (call, got[0], mass)
        assert abs(got[1] - phi_total) / scale_phi < REL_TOL, (call, got[1], phi_total)
        assert abs(got[0] - np.sum(h_rho)) / np.sum(h_rho) < HOST_TOL, (call, got[0], np.sum(h_rho))
        assert abs(got[1] - np.sum(h_phi)) / scale_phi < HOST_TOL, (call, got[1], np.sum(h_phi))
    sim.close()


def _exact_fields(n):
    """a[i] = ((37 i) mod 1000) / 1024 and b[i] = -((13 i) mod 999) / 1024 on
    the device (FP32, exact), and their totals from the periods of the two
    sequences in integer arithmetic.  Every partial sum of these values is a
    multiple of 2^-10 below 2^43, so any FP64 summation order is exact."""
    i = torch.arange(n, dtype=torch.int64, device="cuda")
    a = ((i * 37) % 1000).to(torch.float32) / 1024.0
    b = -((i * 13) % 999).to(torch.float32) / 1024.0
    del i

    def total(mult, period):
        full, rest = divmod(n, period)
        per = sum((mult * k) % period for k in range(period))
        return full * per + sum((mult * k) % period for k in range(rest))

    return a, b, total(37, 1000) / 1024.0, -total(13, 999) / 1024.0


@pytest.mark.gpu
@pytest.mark.parametrize("n", [CHUNK * 5 + 77, CHUNK * 64, MAX_N])
def test_noalloc_sums_exact_on_full_and_partial_blocks(n):
    a, b, ta, tb = _exact_fields(n)
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    for _ in range(2):
        torch.cuda.synchronize()
        tslb.tslb_field_sums_noalloc(a.data_ptr(), b.data_ptr(), n, out.data_ptr(), 0)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert got[0] == ta and got[1] == tb, (n, got, ta, tb)
    del a, b
    torch.cuda.empty_cache()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    """n above 16384 x 16384 values is refused before any GPU work."""
    with pytest.raises(tslb.TslbError) as ei:
        tslb.tslb_field_sums_noalloc(1, 1, MAX_N + 1, 1, 0)
    assert ei.value.status == tslb.TSLB_ERR_INVALID_ARG
    assert "268435456" in tslb.tslb_last_error(None)
    with pytest.raises(tslb.TslbError):
        tslb.tslb_field_sums_noalloc(1, 1, 0, 1, 0)
