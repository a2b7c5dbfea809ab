"""Throughput benchmark of the fused multicomponent TSLB step on GB300.

Default workload: the large-jet Weber sweep, four jets on a 512 x 512 x 1024
grid (268 M nodes each; nozzle D = 40 on the z = 0 face, u = 0.05, Re = 5000,
We = 10, 100, 500 and 2000 through sigma, 1 % inlet noise, free-slip sides,
outflow), FP32 storage, all four resident in HBM (94 GB of state).  One
benchmark step is one lattice Boltzmann time step of each of the four jets
(four fused kernel launches, 1.07 G lattice updates).  The forms measured
beside it (16-bit storage, the Chapman-Enskog closure, the paper's two-sweep
design, the batched ensemble) run on the 192 x 192 x 384 jet.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl tslb|reference]

Prints one JSON line (rank 0).  Under torchrun each rank advances its own
replica of the workload on its own GPU (the method needs no exchange between
independent jets); the value is the total lattice updates of all ranks over
the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GLUPS and % of HBM roofline on 1 GB300, FP32 vs FP16-storage vs batched"
UNIT = "GLUPS"
FIELDS = 11  # stored values per node: rho - 1, u (3), P (6), phi
# committed ncu summaries of the step kernel per storage type (DRAM bytes per node)
PROFILE_SUMMARIES = {"fp32": os.path.join(ROOT, "profiles", "step_kernel_fp32.txt"),
                     "fp16": os.path.join(ROOT, "profiles", "step_kernel_fp16.txt")}
TX = 28  # interior columns of a step-kernel tile
KERNEL_SOURCES = [os.path.join(ROOT, "paper_2403_15773_gb300", "csrc", f)
                  for f in ("tslb_step.cu", "tslb_device.cuh", "tslb_internal.h")]


def kernel_source_sha() -> str:
    """Hash of the step kernel's code (comments and whitespace removed, so that
    a comment edit does not orphan the ncu summary taken on the same code)."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(f, encoding="utf-8") as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def profiled_traffic(nodes: int, storage: str = "fp32"):
    """DRAM bytes per launch of the step kernel of `storage` from its committed
    ncu summary, scaled to `nodes`, if it was taken on the current kernel
    source (None for a storage type without one)."""
    path = PROFILE_SUMMARIES.get(storage)
    try:
        txt = open(path).read() if path else None
    except OSError:
        return None
    if txt is None:
        return None
    sha = re.search(r"kernel_source_sha:\s*(\w+)", txt)
    bpn = re.search(r"dram_bytes_per_node:\s*([0-9.eE+-]+)", txt)
    if not sha or not bpn or sha.group(1) != kernel_source_sha():
        return None
    return float(bpn.group(1)) * nodes


def profiled_fp32_ops(storage: str = "fp32"):
    """FP32 lane operations per staged node of the step kernel of `storage`
    from its committed ncu summary (instruction counts), if it was taken on the
    current kernel source."""
    path = PROFILE_SUMMARIES.get(storage)
    try:
        txt = open(path).read() if path else ""
    except OSError:
        return None
    sha = re.search(r"kernel_source_sha:\s*(\w+)", txt)
    ops = re.search(r"fp32_lane_ops_per_staged_node:\s*([0-9.eE+-]+)", txt)
    if not sha or not ops or sha.group(1) != kernel_source_sha():
        return None
    return float(ops.group(1))


def staged_per_node(nx: int, ny: int, nz: int, block_warps: int, tile_z: int) -> float:
    """Nodes the step kernel's tiles stage (32 columns x 2 block_warps rows x
    (slab + 2) planes each) per interior node of the grid."""
    ty = 2 * block_warps - 2
    tz = min(tile_z, nz) if tile_z > 0 else nz
    bx, by = -(-nx // TX), -(-ny // ty)
    planes = sum(min(tz, nz - k * tz) + 2 for k in range(-(-nz // tz)))
    return bx * 32 * by * 2 * block_warps * planes / (nx * ny * nz)


class ClockSampler:
    """nvidia-smi clock / throttle samples of one GPU during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.samples = []
        if self.proc is None:
            return False
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.samples.append(parts)
        return False

    def summary(self):
        if not getattr(self, "samples", None):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4) if s[5 + k].lower() == "active"})
        pw = [float(s[3]) for s in self.samples if re.match(r"^[0-9.]+$", s[3])]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples),
                "power_w_max": max(pw) if pw else None}


# ----------------------------------------------------------------- workloads

def workloads_by_name(name: str):
    """The grids one benchmark step advances (the Weber sweep: four)."""
    from paper_2403_15773_gb300 import inputs
    if name == "weber512":
        return inputs.weber_sweep()
    return [workload_by_name(name)]


def workload_by_name(name: str):
    from paper_2403_15773_gb300 import inputs
    if name == "jet192":
        return inputs.jet_workload()
    if name == "jet128":
        return inputs.jet_workload(128, 128, 256)
    if name == "jet512":
        return inputs.weber_sweep()[1]
    if name == "droplet32":
        return inputs.droplet_workload()
    raise SystemExit(f"unknown workload {name}")


def describe_all(ws) -> str:
    if len(ws) == 1:
        return describe(ws[0])
    w = ws[0]
    wes = "/".join(f"{w.inlet_u[2] ** 2 * w.inlet_diameter / x.sigma:g}" for x in ws)
    return (f"Weber sweep: {len(ws)} jets {w.nx}x{w.ny}x{w.nz}, We {wes} (sigma "
            f"{'/'.join(f'{x.sigma:.3g}' for x in ws)}), faces {'/'.join(w.faces)}, omega {w.omega:.6f}, "
            f"W {w.width:g}, nozzle D {w.inlet_diameter:g}, u {w.inlet_u[2]:g}, noise {w.noise_amp:g}; "
            f"all resident, one step = one time step of each jet")


def describe(w) -> str:
    return (f"{w.kind} {w.nx}x{w.ny}x{w.nz}, faces {'/'.join(w.faces)}, omega {w.omega:.6f}, "
            f"sigma {w.sigma:.3g}, W {w.width:g}" +
            (f", nozzle D {w.inlet_diameter:g}, u {w.inlet_u[2]:g}, noise {w.noise_amp:g}"
             if w.kind == "jet" else f", R {w.radius:g}"))


# ------------------------------------------------------------- CPU oracle leg

def oracle_params_of(w, ce_neq=False):
    import oracle
    faces = {"periodic": oracle.PERIODIC, "inlet": oracle.INLET, "outflow": oracle.OUTFLOW,
             "free_slip": oracle.FREE_SLIP}
    return oracle.make_params(w.nx, w.ny, w.nz, w.omega, w.sigma, 1.0 / w.width,
                              [faces[f] for f in w.faces], w.inlet_u, w.inlet_diameter, w.inlet_cx,
                              w.inlet_cy, w.width, w.noise_amp, w.seed, normal_eps=w.normal_eps,
                              ce_neq=ce_neq)


def oracle_sample_workload(w, dims=(64, 64, 32)):
    """A bounded sample of the workload for the CPU oracle: the lower part of
    the domain around the nozzle (same physics, fewer nodes)."""
    from paper_2403_15773_gb300 import inputs
    if w.kind == "jet":
        return inputs.crop_jet(w, *dims)
    return w


def _oracle_rate(s_w, budget_s: float):
    """GLUPS of the FP64 oracle on workload s_w (steps fitted to about budget_s), steps, seconds."""
    import oracle
    sim = oracle.OracleSim(oracle_params_of(s_w))
    rho, u, phi = s_w.fields()
    sim.set_state(rho, u, phi)
    sim.step(1)                     # the first step also starts the thread pool
    t0 = time.perf_counter()
    sim.step(2)
    one = (time.perf_counter() - t0) / 2
    n = max(1, min(1000, int(budget_s / max(one, 1e-6))))
    t0 = time.perf_counter()
    sim.step(n)
    dt = time.perf_counter() - t0
    return s_w.nodes * n / dt / 1e9, n, dt


def cpu_baseline(w, budget_s: float = 12.0):
    """The oracle on the host cores: the headline figure on a crop of the
    workload around the nozzle with every core, and beside it the same crop on
    one thread and the 32^3 static droplet in full (every core)."""
    import oracle
    from paper_2403_15773_gb300 import inputs
    s_w = oracle_sample_workload(w)
    glups, n, dt = _oracle_rate(s_w, budget_s)
    crop = f"{s_w.nx}x{s_w.ny}x{s_w.nz} crop of the workload around the nozzle"
    cores = oracle.threads()
    out = {"value": glups, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"FP64 oracle (paper-literal 27+7 population push), {n} steps of a {crop}, {dt:.1f} s"}
    try:
        oracle.set_threads(1)
        g1, n1, dt1 = _oracle_rate(s_w, budget_s / 4)
    finally:
        oracle.set_threads(cores)
    out["single_thread"] = {"value": g1, "unit": UNIT, "cores": 1, "sample": f"{n1} steps of the {crop}, {dt1:.1f} s"}
    d = inputs.droplet_workload()
    gd, nd, dtd = _oracle_rate(d, budget_s / 4)
    out["droplet32"] = {"value": gd, "unit": UNIT, "cores": cores,
                        "sample": f"{nd} steps of the periodic {d.nx}^3 static droplet in full, {dtd:.1f} s"}
    return out


# ------------------------------------------------------------- multi-rank

def max_over_ranks(value: float, dist, device) -> float:
    """The largest `value` over all ranks (every rank gets it)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(nodes_per_rank: int, world: int, steps: int, ms_max: float) -> float:
    """Lattice updates of all ranks over the slowest rank's time, in GLUPS."""
    return nodes_per_rank * world * steps / (ms_max * 1e-3) / 1e9


# ------------------------------------------------------------------ GPU leg

def variant_form(name: str):
    """(storage, scheme, closure) of a measured form: fp32 / fp16 / bf16
    storage, two_sweep (the paper's population design), ce[_fp16|_bf16] (the
    Chapman-Enskog closure, 5 stored fields)."""
    if name == "two_sweep":
        return "fp32", "two_sweep", "projection"
    if name.startswith("ce"):
        return (name[3:] or "fp32"), "fused", "chapman_enskog"
    return name, "fused", "projection"


def stored_bytes_per_node(name: str) -> int:
    """Algorithmic HBM bytes per node and step of a form: every stored value
    read once and written once (two_sweep: 11 moments + 34 populations)."""
    st, scheme, closure = variant_form(name)
    if scheme == "two_sweep":
        return (11 + 34) * 2 * 4
    return (5 if closure == "chapman_enskog" else FIELDS) * 2 * (4 if st == "fp32" else 2)


def run_gpu(args, ws, storage: str, world: int, dist, tile=None, steps=None):
    """Times `steps` benchmark steps of the grids `ws`, all resident at once:
    each benchmark step advances every grid by one time step (one fused
    launch per grid, the grids in turn on one stream).  The tile shape is
    autotuned on the first grid (unless given) and used for all of them."""
    import torch
    import paper_2403_15773_gb300 as tslb
    steps = args.steps if steps is None else steps
    stream = torch.cuda.Stream()
    st, scheme, closure = variant_form(storage)
    two = scheme == "two_sweep"
    tile = dict(tile or {})
    if not tile and not two and (args.block_warps or args.tile_z):
        tile = {"block_warps": args.block_warps, "tile_z": args.tile_z, "plain_stores": int(args.plain_stores)}
    cache = {}

    def start_fields(w):  # grids of one jet geometry share their initial fields
        key = (w.kind, w.nx, w.ny, w.nz, w.radius, w.width)
        if key not in cache:
            cache.clear()
            cache[key] = tuple(torch.from_numpy(a.astype(np.float32)) for a in w.fields())
        return cache[key]

    def make(w):
        sim = tslb.Simulation(w, storage=st, stream=stream,
                              block_warps=0 if two else tile.get("block_warps", 0),
                              tile_z=0 if two else tile.get("tile_z", 0), scheme=scheme, closure=closure,
                              plain_stores=bool(tile.get("plain_stores", 0)) and not two)
        sim.set_state(*start_fields(w))
        return sim

    sims = [make(ws[0])]
    tuned = False
    if not two and not tile:
        nw, tz, pl = sims[0].autotune(6)  # tile shape chosen by timing; the state does not change
        tile = {"block_warps": nw, "tile_z": tz, "plain_stores": pl}
        tuned = True
    sims += [make(w) for w in ws[1:]]
    if not two:  # 1: the step kernel compiled for TMA tile loads alone runs
        tile["tma_only"] = sims[0].step_form()[3]
    cache.clear()
    for sim in sims:
        sim.step(args.warmup)
        sim.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    launches0 = sum(sim.kernel_launches for sim in sims)
    start = torch.cuda.Event(enable_timing=True)
    marks = [torch.cuda.Event(enable_timing=True) for _ in sims]
    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")) if world > 1 else torch.cuda.current_device())
    with sampler:
        barrier()
        start.record(stream)
        for sim, mark in zip(sims, marks):
            sim.step(steps)
            mark.record(stream)
        marks[-1].synchronize()
        barrier()
    ms = start.elapsed_time(marks[-1])
    per = [start.elapsed_time(marks[0])] + [marks[k - 1].elapsed_time(marks[k]) for k in range(1, len(marks))]
    launches = sum(sim.kernel_launches for sim in sims) - launches0
    ok = True
    for sim in sims:
        m, p = sim.sums()
        ok = ok and math.isfinite(m) and math.isfinite(p)
        sim.close()
    del sims
    torch.cuda.empty_cache()
    ms = max_over_ranks(ms, dist, torch.device("cuda", torch.cuda.current_device()))
    if two:
        tile = {"block_warps": 8, "tile_z": 0, "plain_stores": 0}
    return {"ms": ms, "per_grid_ms": per, "launches": launches, "clocks": sampler.summary(), "finite": ok,
            "shape": tile, "autotuned": tuned, "steps": steps}


def run_batched(args):
    """The ensemble of independent uneven grids advanced together (one
    persistent launch per step, graph-replayed, autotuned tiles), against the
    same grids advanced one after another with the plain FP32 path, each in
    the tile shape the autotuner picks for its kind of grid (edge and faces)."""
    import torch
    import paper_2403_15773_gb300 as tslb
    from paper_2403_15773_gb300 import inputs
    ws = inputs.batched_ensemble()
    steps = args.batch_steps
    stream = torch.cuda.Stream()
    b = tslb.BatchSimulation(ws, stream=stream)
    for i, w in enumerate(ws):
        b.set_state(i, *w.fields())
    shape = b.autotune(3)
    batch_form = b.step_form()
    b.step(args.warmup)
    b.synchronize()
    st, sp = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = b.kernel_launches
    st.record(stream)
    b.step(steps)
    sp.record(stream)
    sp.synchronize()
    ms_batch = st.elapsed_time(sp)
    launches = b.kernel_launches - l0
    b.close()
    nodes = sum(w.nodes for w in ws)
    tuned = {}  # (edge, faces) -> tile shape of the single-grid path
    ms_seq = 0.0
    for w in ws:
        key = (w.nx, w.ny, w.nz, tuple(w.faces))
        rho, u, phi = w.fields()
        if key not in tuned:
            s = tslb.Simulation(w, stream=stream)
            s.set_state(torch.from_numpy(rho), torch.from_numpy(u), torch.from_numpy(phi))
            tuned[key] = s.autotune(3)
            s.close()
        nw, tz, pl = tuned[key]
        s = tslb.Simulation(w, stream=stream, block_warps=nw, tile_z=tz, plain_stores=bool(pl))
        s.set_state(torch.from_numpy(rho), torch.from_numpy(u), torch.from_numpy(phi))
        s.step(args.warmup)
        s.synchronize()
        st.record(stream)
        s.step(steps)
        sp.record(stream)
        sp.synchronize()
        ms_seq += st.elapsed_time(sp)
        s.close()
    torch.cuda.empty_cache()
    g_batch = nodes * steps / (ms_batch * 1e-3) / 1e9
    g_seq = nodes * steps / (ms_seq * 1e-3) / 1e9
    peak, _ = measured_peaks()
    return {"storage": "fp32", "instances": len(ws), "nodes": nodes, "steps": steps, "value": g_batch,
            "unit": UNIT, "ms_per_step": ms_batch / steps,
            "hbm_frac": FIELDS * 8 * nodes / (ms_batch * 1e-3 / steps) / 1e9 / peak,
            "sequential_fp32_value": g_seq, "speedup_vs_sequential_fp32": g_batch / g_seq,
            "sequential_tiles": "each grid in the tile shape the autotuner picks for its edge and faces "
                                f"({len(tuned)} kinds), one grid after another on one stream",
            "gpu_launches": launches,
            "autotuned": {"block_warps": shape[0], "tile_z": shape[1], "plain_stores": shape[2],
                          "tma_only": batch_form[3]},
            "workload": "64 cubic grids, edges uniform in {48, 64, 96, 128}, periodic droplets (R = edge/4) "
                        "and jets (D = 0.15 edge, periodic sides), We log-uniform in [10, 2000], seed 4"}


def run_e2e(args, ws, storage: str, world: int = 1, dist=None, shape=None):
    """Same metric through the public C ABI with host buffers: per grid, upload
    the initial fields from pinned memory, run the steps, read rho, u and phi
    back into pinned memory and take the FP64 sums.  `shape` is the tile shape
    of the device-timed run (so both time the same kernel)."""
    import torch
    import paper_2403_15773_gb300 as tslb
    stream = torch.cuda.Stream()
    shape = shape or {}
    sims = [tslb.Simulation(w, storage=storage, stream=stream, block_warps=shape.get("block_warps", 0),
                            tile_z=shape.get("tile_z", 0), plain_stores=bool(shape.get("plain_stores", 0)))
            for w in ws]
    inputs_of = {}
    for w in ws:
        key = (w.kind, w.nx, w.ny, w.nz, w.radius, w.width)
        if key not in inputs_of:
            inputs_of[key] = tuple(torch.from_numpy(a.astype(np.float32).reshape(-1)).pin_memory()
                                   for a in w.fields())
    nmax = max(w.nodes for w in ws)
    out_rho = torch.empty(nmax, dtype=torch.float32).pin_memory()
    out_u = torch.empty(3 * nmax, dtype=torch.float32).pin_memory()
    out_phi = torch.empty(nmax, dtype=torch.float32).pin_memory()

    def job(steps):
        for w, sim in zip(ws, sims):
            rho, u, phi = inputs_of[(w.kind, w.nx, w.ny, w.nz, w.radius, w.width)]
            sim.set_state_host(rho, u, phi)
            sim.step(steps)
            sim.moments_host(out_rho, out_u, None)
            sim.phi_host(out_phi)
            sim.sums()

    job(min(args.warmup, 16))  # warm-up of the whole path (graph capture, first touch of pinned pages)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    job(args.steps)
    dt = time.perf_counter() - t0
    for sim in sims:
        sim.close()
    del sims
    torch.cuda.empty_cache()
    dt = max_over_ranks(dt * 1e3, dist, torch.device("cuda", torch.cuda.current_device())) * 1e-3
    nodes = sum(w.nodes for w in ws)
    h2d = 5 * nodes * 4
    d2h = 5 * nodes * 4 + 16 * len(ws)
    return {"value": whole_job_rate(nodes, world, args.steps, dt * 1e3), "unit": UNIT,
            "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
            "note": "one job per timed region: per grid, set_state from pinned host buffers, the steps, "
                    "get_moments (rho, u) + get_phi into pinned host buffers, FP64 sums; bytes per step "
                    "are the job's copies divided by the steps"}


def variant_line(w, storage, res, base_glups):
    steps = res["steps"]
    glups = w.nodes * steps / (res["ms"] * 1e-3) / 1e9
    bpn = stored_bytes_per_node(storage)
    st, scheme, closure = variant_form(storage)
    peak, _ = measured_peaks()
    ach = bpn * w.nodes / (res["ms"] * 1e-3 / steps) / 1e9
    return {"storage": st, "scheme": scheme, "closure": closure, "value": glups, "unit": UNIT,
            "speedup_vs_fp32": glups / base_glups, "ms_per_step": res["ms"] / steps, "steps": steps,
            "bytes_per_node": bpn, "hbm_frac": ach / peak, "gpu_launches": res["launches"],
            "tile": res["shape"], "state_gb": (45 * 4 if scheme == "two_sweep" else bpn) * w.nodes / 1e9}


def oracle_errors(w, storages, steps=200):
    """Max errors against the FP64 oracle of each storage form on a small crop
    of the workload (48^3 around the nozzle, D 8), same physics."""
    import torch
    import oracle
    import paper_2403_15773_gb300 as tslb
    from paper_2403_15773_gb300 import inputs
    c = inputs.crop_jet(w, 48, 48, 48, diameter=8) if w.kind == "jet" else w
    rho, u, phi = c.fields()
    refs = {}
    out = {}
    for name in storages:
        st, scheme, closure = variant_form(name)
        ce = closure == "chapman_enskog"
        if ce not in refs:  # each closure against the oracle run with it
            ref = oracle.OracleSim(oracle_params_of(c, ce_neq=ce))
            ref.set_state(rho, u, phi)
            ref.step(steps)
            refs[ce] = ref.moments()
        r = refs[ce]
        sim = tslb.Simulation(c, storage=st, scheme=scheme, closure=closure)
        sim.set_state(torch.from_numpy(rho), torch.from_numpy(u), torch.from_numpy(phi))
        sim.step(steps)
        g = sim.fields_numpy()
        sim.close()
        out[name] = {"rho": float(np.max(np.abs(g[0] - r[0])) / np.max(np.abs(r[0]))),
                     "u": float(np.max(np.abs(g[1] - r[1])) / max(np.max(np.abs(r[1])), 0.05)),
                     "phi": float(np.max(np.abs(g[3] - r[3]))),
                     "rho_rms": float(np.sqrt(np.mean((g[0] - r[0]) ** 2)) / np.max(np.abs(r[0]))),
                     "u_rms": float(np.sqrt(np.mean((g[1] - r[1]) ** 2)) / max(np.max(np.abs(r[1])), 0.05)),
                     "phi_rms": float(np.sqrt(np.mean((g[3] - r[3]) ** 2)))}
    case = (f"{c.nx}x{c.ny}x{c.nz} crop of the workload (nozzle D {c.inlet_diameter:g}), {steps} steps; max "
            f"and rms error (rho / max rho, u / max(max u, 0.05), phi)")
    return out, case


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500,
                    help="timed benchmark steps (Weber sweep: one time step of each of the four jets)")
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="tslb", choices=["tslb", "reference"])
    ap.add_argument("--workload", default="weber512",
                    help="weber512 (the four 512x512x1024 jets), jet512 (one of them, We 100), jet192, "
                         "jet128, droplet32")
    ap.add_argument("--storage", default="fp32", choices=["fp32", "fp16", "bf16"])
    ap.add_argument("--variants", default="fp32,fp16,bf16,two_sweep,ce,ce_fp16",
                    help="forms measured on the variant workload: fp32, fp16, bf16 storage, "
                         "two_sweep (the paper's population design), ce, ce_fp16, ce_bf16 (the "
                         "Chapman-Enskog closure, 5 stored fields) ('' for none)")
    ap.add_argument("--variant-workload", default="jet192")
    ap.add_argument("--variant-steps", type=int, default=500)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-oracle-error", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-fma-peak", action="store_true")
    ap.add_argument("--batch-steps", type=int, default=200)
    ap.add_argument("--block-warps", type=int, default=0)
    ap.add_argument("--tile-z", type=int, default=0)
    ap.add_argument("--plain-stores", action="store_true",
                    help="with --block-warps / --tile-z: the FP32 step kernel form without the store staging box")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    ws = workloads_by_name(args.workload)

    if args.impl == "reference":
        # the reference arm is the FP64 CPU oracle; under torchrun only rank 0 runs it
        if rank != 0:
            return
        return reference_arm(args, ws)

    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    import paper_2403_15773_gb300 as tslb
    tslb.lib()  # build / load the CUDA library before timing

    res = run_gpu(args, ws, args.storage, world, dist)
    nodes = sum(w.nodes for w in ws)
    e2e = None if args.no_e2e else run_e2e(args, ws, args.storage, world, dist, res["shape"])

    variants = {}
    vlist = [s for s in args.variants.split(",") if s]
    wv = workload_by_name(args.variant_workload)
    base_v = None
    if vlist and world == 1:
        base = run_gpu(args, [wv], "fp32", world, dist, steps=args.variant_steps)
        base_v = wv.nodes * base["steps"] / (base["ms"] * 1e-3) / 1e9
        for v in vlist:
            r = base if v == "fp32" else run_gpu(args, [wv], v, world, dist, steps=args.variant_steps)
            variants[v] = variant_line(wv, v, r, base_v)
            variants[v]["workload"] = describe(wv)
    if not args.no_batched and world == 1:
        variants["batched"] = run_batched(args)
        if base_v:
            variants["batched"]["speedup_vs_fp32"] = variants["batched"]["value"] / base_v
    errs = None
    if rank == 0 and not args.no_oracle_error:
        err_ws = ws[1] if len(ws) > 1 else ws[0]
        errs, err_case = oracle_errors(err_ws, [args.storage])
        if vlist:
            verrs, vcase = oracle_errors(wv, [v for v in vlist])
            for v in vlist:
                variants[v]["oracle_err"] = verrs[v]
                variants[v]["oracle_err_case"] = vcase
    for v in variants:
        if v.startswith("ce"):
            variants[v]["note"] = ("Chapman-Enskog closure of a2_neq (Sec. 2.1): 5 stored fields, P "
                                   "neither stored nor read; a different closure, so oracle_err is "
                                   "against the oracle run with the same closure")
    if "two_sweep" in variants and base_v:
        variants["two_sweep"]["note"] = ("the paper's design on this GPU: collide+push into 34 population "
                                         "arrays, then their moments; fused speedup over it = "
                                         f"{base_v / variants['two_sweep']['value']:.2f}x")
    fma = None
    if not args.no_fma_peak and rank == 0:
        fma = {"packed": tslb.tslb_fp32_lane_rate(1), "scalar": tslb.tslb_fp32_lane_rate(0)}
    if dist is not None:
        dist.barrier()
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    K = res["steps"]
    sec = res["ms"] * 1e-3
    glups = whole_job_rate(nodes, world, K, res["ms"])
    bpn = FIELDS * 2 * (4 if args.storage == "fp32" else 2)
    per_launch = sec / max(res["launches"], 1) if res["launches"] else sec / (K * len(ws))
    n_grid = ws[0].nodes
    peak, peak_kind = measured_peaks()
    achieved = bpn * n_grid / per_launch / 1e9
    traffic = profiled_traffic(n_grid, args.storage)
    line = {
        "metric": METRIC, "value": glups, "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": res["ms"] / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.storage == "fp32" else "f32 (" + args.storage + " storage)",
        "data": "synthetic",
        "config": {"workload": describe_all(ws), "grids": len(ws), "nodes_per_grid": n_grid,
                   "updates_per_step": nodes, "storage": args.storage, "tile": res["shape"],
                   "tile_autotuned": res["autotuned"],
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "l2": f"state {bpn * n_grid / 1e9:.2f} GB per grid (two buffers) > 126 MB L2: "
                         "inputs larger than L2, no flush"},
        "per_grid": [{"sigma": w.sigma, "value": w.nodes * K / (ms * 1e-3) / 1e9, "ms_per_step": ms / K}
                     for w, ms in zip(ws, res["per_grid_ms"])],
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "note": f"{bpn} algorithmic bytes per node ({FIELDS} stored values read and "
                             f"written) x {n_grid} nodes per launch / mean launch time over the timed "
                             f"region ({res['launches']} launches); peak {peak_kind} (MEASURED_PEAKS.json "
                             f"hbm_gbs); traffic: ncu DRAM bytes per node of the same kernel scaled to the "
                             f"grid (null when the kernel changed since the capture)"},
        "oracle_err": None if errs is None else {"case": err_case, args.storage: errs[args.storage]},
        "gpu_launches": res["launches"],
        "clocks": res["clocks"],
        "variants": variants,
    }
    if fma is not None:
        ops_staged = profiled_fp32_ops(args.storage)
        sh = res["shape"]
        ratio = staged_per_node(ws[0].nx, ws[0].ny, ws[0].nz, sh["block_warps"], sh["tile_z"])
        ops = None if ops_staged is None else ops_staged * ratio
        line["fp32_roofline"] = {
            "bound": "alu", "unit": "FP32 lane-FMA/s", "peak": fma["packed"], "peak_scalar": fma["scalar"],
            "ops_per_update": ops, "staged_per_node": ratio,
            "achieved": None if ops is None else ops * n_grid / per_launch,
            "frac": None if ops is None else ops * n_grid / per_launch / fma["packed"],
            "note": "peak: this run's tslb_fp32_lane_rate (independent FMA chains; packed f32x2 and "
                    "scalar); ops_per_update: FP32 lane operations (packed x 2) per staged node "
                    "counted by ncu on the same kernel source (null when it changed since) x the "
                    "nodes the timed tile shape stages per interior node"}
    if e2e is not None:
        line["e2e"] = e2e
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(ws[1] if len(ws) > 1 else ws[0])
    if not res["finite"]:
        line["error"] = "non-finite sums"
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def reference_arm(args, ws):
    """The FP64 CPU oracle timed as it stands on the host cores: each benchmark
    step is one oracle time step of a bounded sample of each grid of the
    workload (a 32^3 crop around the nozzle)."""
    import oracle
    sims = []
    for w in ws:
        s_w = oracle_sample_workload(w, (32, 32, 32))
        sim = oracle.OracleSim(oracle_params_of(s_w))
        rho, u, phi = s_w.fields()
        sim.set_state(rho, u, phi)
        sims.append((s_w, sim))
    for _, sim in sims:
        sim.step(args.warmup)
    t0 = time.perf_counter()
    for _, sim in sims:
        sim.step(args.steps)
    dt = time.perf_counter() - t0
    nodes = sum(s_w.nodes for s_w, _ in sims)
    v = nodes * args.steps / dt / 1e9
    s0 = sims[0][0]
    sample = (f"{s0.nx}x{s0.ny}x{s0.nz} crop around the nozzle of each of the {len(ws)} grid(s) of the "
              f"workload per step")
    cb = {"value": v, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle", "sample": sample}
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference", "config": {"workload": describe_all(ws), "sample": sample},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
