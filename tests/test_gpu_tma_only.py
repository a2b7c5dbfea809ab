"""The step kernel compiled for TMA tile loads alone against the kernel that
chooses its load path tile by tile.

By default (option per_tile_loads = 0) a single grid whose tiles all load by
TMA in the 12-warp form -- the kernel's own tile set-up, run once per tile at
tslb_init, decides -- runs 12-warp staged-store steps in a kernel with no
element-wise load path.  The checks: that form is the one tslb_step_form
reports where it applies (FP32 with mirror and copy faces, FP32 across
periodic faces through the side boxes, 16-bit storage) and is not where a
tile must load element by element (a periodic grid narrower than one tile;
16-bit storage across periodic faces, which has no side boxes; rows that are
not a multiple of 16 bytes; 8-warp blocks; plain stores); and after 12 steps
its stored state and FP64 sums equal, bit for bit, those of the per-tile
kernel (per_tile_loads = 1), also for slab depths that leave every
remainder of the march unrolled by four.  The oracle parity of the form comes from the
12-warp parity tests, which run it wherever it applies."""
import pytest
import torch

import paper_2403_15773_gb300 as tslb
from paper_2403_15773_gb300 import inputs

pytestmark = pytest.mark.gpu
STEPS = 12


def run(w, storage="fp32", **kw):
    sim = tslb.Simulation(w, storage=storage, **kw)
    rho, u, phi = w.fields()
    sim.set_state(torch.from_numpy(rho), torch.from_numpy(u), torch.from_numpy(phi))
    form = sim.step_form()
    sim.step(STEPS)
    state = sim.get_state().cpu().clone()
    sums = sim.sums()
    sim.close()
    return form, state, sums


def close_totals(got, ref):
    """FP64 totals of the same state summed over other tiles: each thread adds
    at most 64 planes in FP32 before the FP64 reduction, and that grouping
    follows the tile shape."""
    for x, y in zip(got, ref):
        assert abs(x - y) <= 64 * 2.0 ** -24 * abs(y), (got, ref)


def jet72(side="free_slip"):  # 72 columns: 16-byte rows in FP32 and 16 bits; ragged x and y tiles
    return inputs.jet_workload(72, 50, 30, diameter=10, noise=0.01, seed=4, side=side)


# (storage, workload, whether the TMA-only form applies)
CASES = [
    ("fp32", jet72, True),
    ("fp32", lambda: inputs.jet_workload(56, 48, 40, diameter=10, noise=0.01, seed=5, side="periodic"), True),
    ("fp32", lambda: inputs.droplet_workload(48, radius=11.0), True),
    ("fp16", jet72, True),
    ("bf16", jet72, True),
    ("fp32", lambda: inputs.droplet_workload(24, radius=6.0), False),   # x0 = 0 and x0 + 31 >= nx: both wraps
    ("fp16", lambda: inputs.droplet_workload(48, radius=11.0), False),  # 16-bit: no side boxes
    ("fp32", lambda: inputs.jet_workload(70, 50, 30, diameter=10, noise=0.01, seed=4), False),  # 280-byte rows
]


@pytest.mark.parametrize("storage,make,applies", CASES)
def test_tma_only_form_equals_per_tile_form(storage, make, applies):
    w = make()
    fa, a, sa = run(w, storage)
    fb, b, sb = run(w, storage, per_tile_loads=True)
    assert fa[0] == 12 and fa[2] == 0, fa
    assert fa[3] == (1 if applies else 0), (w.nx, w.ny, w.nz, storage, fa)
    assert fb[3] == 0, fb
    assert torch.equal(a, b)
    assert sa == sb


@pytest.mark.parametrize("kw", [dict(block_warps=8), dict(plain_stores=True)])
def test_other_forms_choose_per_tile(kw):
    w = jet72()
    fa, a, sa = run(w, **kw)
    assert fa[3] == 0, fa
    fb, b, sb = run(w)
    assert fb[3] == 1, fb
    assert torch.equal(a, b)
    close_totals(sa, sb)


def test_autotuned_12_warp_form_reports_tma_only():
    w = jet72()
    sim = tslb.Simulation(w)
    rho, u, phi = w.fields()
    sim.set_state(torch.from_numpy(rho), torch.from_numpy(u), torch.from_numpy(phi))
    nw, tz, pl = sim.autotune(2)
    form = sim.step_form()
    assert form[:3] == (nw, tz, pl)
    assert form[3] == (1 if (nw, pl) == (12, 0) else 0), form
    sim.close()


@pytest.mark.parametrize("tile_z", [1, 2, 3, 4, 5, 6, 7, 9, 30])
def test_tma_only_form_independent_of_slab_depth(tile_z):
    """The TMA-only form unrolls its plane march by four: slab depths whose
    march (tile_z + 3 planes) leaves every remainder mod 4, and the single
    slab of the whole grid, give the same bits as the per-tile form in its
    default slabs."""
    w = jet72()
    fa, a, sa = run(w, tile_z=tile_z)
    assert fa[3] == 1 and fa[1] == tile_z, fa
    fb, b, sb = run(w, per_tile_loads=True)
    assert fb[3] == 0, fb
    assert torch.equal(a, b)
    close_totals(sa, sb)


def test_time_sums_keep_the_per_tile_form():
    """The TMA-only form keeps no time sums of phi and u_z: with the option
    average on, the same grid runs the per-tile form (whose averages the
    parity tests check against the oracle)."""
    w = jet72()
    fa, a, sa = run(w, average=True)
    assert fa[0] == 12 and fa[3] == 0, fa
    fb, b, sb = run(w)
    assert fb[3] == 1, fb
    assert torch.equal(a, b)
    assert sa == sb
