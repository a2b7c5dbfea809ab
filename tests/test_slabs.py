"""The z-slab decomposition (the multi-GPU runs the paper names as future
work, Sec. 4 and 5) on CPU ranks: gloo ranks each advance an FP64 oracle slab
with ghost planes, exchange the ghost planes of every step through
``slabs.exchange`` (the messages ``slabs.send_planes`` / ``ghost_planes``
describe: one plane of the ten moment fields, two planes of phi), and must
match the oracle run on the whole domain.  The moments of the second ghost
plane are never exchanged, so the match also pins the halo depths."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2403_15773_gb300 import inputs, slabs
from _util import oracle_params

P, IN, OUT = oracle.PERIODIC, oracle.INLET, oracle.OUTFLOW
_FACE = {"periodic": P, "inlet": IN, "outflow": OUT, "free_slip": oracle.FREE_SLIP}


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case(name):
    if name == "jet":
        w = inputs.jet_workload(16, 14, 20, diameter=6, we=100, noise=0.01, seed=7)
        rho, u, pi, _ = inputs.random_smooth_fields(16, 14, 20, seed=5, amp_rho=1e-2, amp_u=1e-2, amp_pi=5e-4)
        _, _, phi = inputs.droplet_fields(16, 14, 20, 4.0, 3.0, center=(8.0, 7.0, 11.0))
        return w, (rho, u, pi, phi), False
    w = inputs.droplet_workload(12, radius=4.0)
    w.nz = 16
    rho, u, pi, _ = inputs.random_smooth_fields(12, 12, 16, seed=6, amp_rho=1e-2, amp_u=1e-2, amp_pi=5e-4)
    _, _, phi = inputs.droplet_fields(12, 12, 16, 4.0, 3.0, center=(6.0, 6.0, 15.0))  # across the z wrap
    return w, (rho, u, pi, phi), True


def _whole_domain(w, fields, steps):
    rho, u, pi, phi = fields
    s = oracle.OracleSim(oracle_params(w))
    s.set_state(rho, u, phi, pi=pi)
    s.step(steps)
    return s.moments()


def _worker(rank, world, port, name, steps, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, fields, periodic = _case(name)
        slab = slabs.partition(w.nz, world, rank, periodic_z=periodic)
        lo = 2 if slab.lower is not None else 0
        hi = 2 if slab.upper is not None else 0
        n = slab.planes
        # the slab plus its ghost planes, one oracle box; a face toward a
        # neighbour gets any rule (its ghost planes are rewritten every step)
        faces = [_FACE[f] for f in w.faces]
        if periodic:
            faces[4] = faces[5] = OUT
        if lo:
            faces[4] = OUT
        if hi:
            faces[5] = OUT
        prm = oracle_params(w, nz=n + lo + hi, faces=faces)
        zs = np.arange(slab.z0 - lo, slab.z1 + hi) % w.nz
        rho, u, pi, phi = fields
        sim = oracle.OracleSim(prm)
        sim.set_state(rho[zs], u[:, zs], phi[zs], pi=pi[:, zs])
        nxy = w.nx * w.ny

        for t in range(steps):
            r, uu, pp, ph = (a.copy() for a in sim.moments())

            def pack(side):
                m, (a, b) = slabs.send_planes(n, side)
                mom = np.concatenate([r[None, lo + m], uu[:, lo + m], pp[:, lo + m]]).reshape(-1)
                return torch.from_numpy(np.concatenate([mom, ph[lo + a].reshape(-1), ph[lo + b].reshape(-1)]))

            def unpack(side, msg):
                m, (a, b) = slabs.ghost_planes(n, side)
                v = msg.numpy()
                mom = v[:slabs.MOMENT_FIELDS * nxy].reshape(slabs.MOMENT_FIELDS, w.ny, w.nx)
                r[lo + m], uu[:, lo + m], pp[:, lo + m] = mom[0], mom[1:4], mom[4:10]
                ph[lo + a] = v[slabs.MOMENT_FIELDS * nxy:(slabs.MOMENT_FIELDS + 1) * nxy].reshape(w.ny, w.nx)
                ph[lo + b] = v[(slabs.MOMENT_FIELDS + 1) * nxy:].reshape(w.ny, w.nx)

            vals = (slabs.MOMENT_FIELDS + slabs.PHI_PLANES) * nxy
            slabs.exchange(slab, pack, unpack, lambda: torch.empty(vals, dtype=torch.float64), dist)
            sim.set_state(r, uu, ph, pi=pp, t0=t)
            sim.step(1)
        got = sim.moments()
        ref = _whole_domain(w, fields, steps)
        sl = slice(lo, lo + n)
        err = max(float(np.max(np.abs(got[0][sl] - ref[0][slab.z0:slab.z1]))),
                  float(np.max(np.abs(got[1][:, sl] - ref[1][:, slab.z0:slab.z1]))),
                  float(np.max(np.abs(got[2][:, sl] - ref[2][:, slab.z0:slab.z1]))),
                  float(np.max(np.abs(got[3][sl] - ref[3][slab.z0:slab.z1]))))
        out[rank] = err
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("name,world", [("jet", 2), ("jet", 3), ("droplet", 2)])
def test_oracle_slabs_match_the_whole_domain(name, world):
    """jet: inlet on the first slab, outflow on the last, a middle slab with
    two halo faces at world 3; droplet: a periodic z axis split in two, both
    cuts between the same two ranks, a droplet across the wrap."""
    oracle.build()
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, name, 12, out), nprocs=world, join=True)
        errs = dict(out)
    assert sorted(errs) == list(range(world))
    assert max(errs.values()) < 1e-13, errs


def test_partition_covers_the_domain_once():
    for nz, world in ((20, 2), (21, 4), (384, 8), (9, 4)):
        parts = [slabs.partition(nz, world, r) for r in range(world)]
        assert parts[0].z0 == 0 and parts[-1].z1 == nz
        assert all(a.z1 == b.z0 for a, b in zip(parts, parts[1:]))
        assert all(p.planes >= 2 for p in parts) and max(p.planes for p in parts) - min(p.planes for p in parts) <= 1
        assert parts[0].lower is None and parts[-1].upper is None
    ring = [slabs.partition(12, 3, r, periodic_z=True) for r in range(3)]
    assert [(p.lower, p.upper) for p in ring] == [(2, 1), (0, 2), (1, 0)]
    with pytest.raises(ValueError):
        slabs.partition(5, 3, 0)


def test_slab_workload_faces():
    w = inputs.jet_workload(32, 32, 40)
    first, mid, last = (slabs.slab_workload(w, slabs.partition(40, 3, r)) for r in range(3))
    assert first.faces[4:] == ("inlet", "halo") and mid.faces[4:] == ("halo", "halo")
    assert last.faces[4:] == ("halo", "outflow") and first.faces[:4] == w.faces[:4]
    assert first.nz + mid.nz + last.nz == 40
