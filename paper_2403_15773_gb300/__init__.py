"""Python binding of the GB300 multicomponent thread-safe lattice Boltzmann
library (arXiv 2403.15773).

The binding only marshals arguments: every step of the method runs in the
CUDA kernels of ``_build/libtslb.so`` behind the C ABI of ``include/tslb.h``.
The functions ``tslb_*`` below carry the names of the C entry points;
:class:`Simulation` is a convenience wrapper that keeps the device workspace
in a PyTorch tensor and issues work on a PyTorch stream.

There is no CPU fallback: if the CUDA library cannot be built or loaded, the
functions raise.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

import numpy as np

from . import build as _build

__all__ = [
    "TSLB_OK", "TslbError", "Grid", "Boundary", "Options", "lib", "library_path",
    "tslb_default_options", "tslb_workspace_bytes", "tslb_init", "tslb_set_state", "tslb_step",
    "tslb_get_moments", "tslb_get_phi", "tslb_sums", "tslb_get_time", "tslb_state_bytes",
    "tslb_get_state", "tslb_put_state", "tslb_synchronize", "tslb_destroy", "tslb_last_error",
    "tslb_status_string", "tslb_kernel_launches", "tslb_field_sums_noalloc",
    "tslb_batch_workspace_bytes", "tslb_init_batch", "tslb_batch_set_state", "tslb_batch_get_moments",
    "tslb_batch_get_phi", "tslb_batch_sums", "tslb_batch_count", "tslb_autotune",
    "tslb_step_form", "tslb_get_averages", "tslb_reset_averages", "tslb_fp32_lane_rate", "tslb_halo_values", "tslb_halo_pack",
    "tslb_halo_unpack", "Simulation", "BatchSimulation", "SYMBOLS",
]

TSLB_OK, TSLB_ERR_INVALID_ARG, TSLB_ERR_OOM, TSLB_ERR_CUDA, TSLB_ERR_UNSTABLE, TSLB_ERR_TIMEOUT, \
    TSLB_ERR_STATE = range(7)
TSLB_LATTICE_D3Q27_D3Q7 = 0
STORAGE = {"fp32": 0, "fp16": 1, "bf16": 2}
CLOSURES = {"projection": 0, "chapman_enskog": 1}
FACES = {"periodic": 0, "inlet": 1, "outflow": 2, "free_slip": 3, "halo": 4}

SYMBOLS = ("tslb_default_options", "tslb_workspace_bytes", "tslb_init", "tslb_set_state", "tslb_step",
           "tslb_get_moments", "tslb_get_phi", "tslb_sums", "tslb_get_time", "tslb_state_bytes",
           "tslb_get_state", "tslb_put_state", "tslb_synchronize", "tslb_destroy", "tslb_last_error",
           "tslb_status_string", "tslb_kernel_launches", "tslb_field_sums_noalloc",
           "tslb_batch_workspace_bytes", "tslb_init_batch", "tslb_batch_set_state", "tslb_batch_get_moments",
           "tslb_batch_get_phi", "tslb_batch_sums", "tslb_batch_count", "tslb_autotune",
           "tslb_step_form", "tslb_get_averages", "tslb_reset_averages", "tslb_fp32_lane_rate", "tslb_halo_values",
           "tslb_halo_pack", "tslb_halo_unpack")


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32)]


class Boundary(ctypes.Structure):
    _fields_ = [("face", ctypes.c_int32 * 6), ("inlet_u", ctypes.c_float * 3),
                ("inlet_diameter", ctypes.c_float), ("inlet_cx", ctypes.c_float),
                ("inlet_cy", ctypes.c_float), ("noise_amp", ctypes.c_float), ("seed", ctypes.c_uint64)]


class Options(ctypes.Structure):
    _fields_ = [("storage", ctypes.c_int32), ("interface_width", ctypes.c_float),
                ("normal_eps", ctypes.c_float), ("field_scale", ctypes.c_float * 4),
                ("check_every", ctypes.c_int32), ("tile_z", ctypes.c_int32),
                ("graph_steps", ctypes.c_int32), ("block_warps", ctypes.c_int32),
                ("scheme", ctypes.c_int32), ("average", ctypes.c_int32), ("closure", ctypes.c_int32),
                ("test_tma_stall", ctypes.c_int32), ("plain_stores", ctypes.c_int32),
                ("per_tile_loads", ctypes.c_int32), ("cuda_stream", ctypes.c_void_p)]


class TslbError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"tslb status {status}: {msg}")
        self.status = status


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB_PATH


def lib() -> ctypes.CDLL:
    """Load (building first if needed) the CUDA library."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = ctypes.CDLL(path)
            P, VP = ctypes.POINTER, ctypes.c_void_p
            L.tslb_default_options.argtypes = [P(Options)]
            L.tslb_default_options.restype = None
            L.tslb_workspace_bytes.argtypes = [P(Grid), P(Options)]
            L.tslb_workspace_bytes.restype = ctypes.c_size_t
            L.tslb_init.argtypes = [P(VP), P(Grid), ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                    P(Boundary), P(Options), VP, ctypes.c_size_t]
            L.tslb_set_state.argtypes = [VP, VP, VP, VP, VP, ctypes.c_int]
            L.tslb_step.argtypes = [VP, ctypes.c_int64]
            L.tslb_get_moments.argtypes = [VP, VP, VP, VP, ctypes.c_int]
            L.tslb_get_phi.argtypes = [VP, VP, ctypes.c_int]
            L.tslb_sums.argtypes = [VP, P(ctypes.c_double), P(ctypes.c_double)]
            L.tslb_get_time.argtypes = [VP, P(ctypes.c_int64)]
            L.tslb_state_bytes.argtypes = [VP]
            L.tslb_state_bytes.restype = ctypes.c_size_t
            L.tslb_get_state.argtypes = [VP, VP, ctypes.c_int]
            L.tslb_put_state.argtypes = [VP, VP, ctypes.c_int]
            L.tslb_synchronize.argtypes = [VP]
            L.tslb_destroy.argtypes = [VP]
            L.tslb_last_error.argtypes = [VP]
            L.tslb_last_error.restype = ctypes.c_char_p
            L.tslb_status_string.argtypes = [ctypes.c_int]
            L.tslb_status_string.restype = ctypes.c_char_p
            L.tslb_kernel_launches.argtypes = [VP]
            L.tslb_kernel_launches.restype = ctypes.c_int64
            L.tslb_field_sums_noalloc.argtypes = [VP, VP, ctypes.c_int64, VP, VP]
            L.tslb_field_sums_noalloc.restype = ctypes.c_int
            L.tslb_batch_workspace_bytes.argtypes = [ctypes.c_int32, P(Grid), P(Options)]
            L.tslb_batch_workspace_bytes.restype = ctypes.c_size_t
            L.tslb_init_batch.argtypes = [P(VP), ctypes.c_int32, P(Grid), ctypes.c_int, P(ctypes.c_double),
                                          P(ctypes.c_double), P(Boundary), P(Options), VP, ctypes.c_size_t]
            L.tslb_batch_set_state.argtypes = [VP, ctypes.c_int32, VP, VP, VP, VP, ctypes.c_int]
            L.tslb_batch_get_moments.argtypes = [VP, ctypes.c_int32, VP, VP, VP, ctypes.c_int]
            L.tslb_batch_get_phi.argtypes = [VP, ctypes.c_int32, VP, ctypes.c_int]
            L.tslb_batch_sums.argtypes = [VP, ctypes.c_int32, P(ctypes.c_double), P(ctypes.c_double)]
            L.tslb_batch_count.argtypes = [VP]
            L.tslb_batch_count.restype = ctypes.c_int32
            L.tslb_autotune.argtypes = [VP, ctypes.c_int32, P(ctypes.c_int32), P(ctypes.c_int32), P(ctypes.c_int32)]
            L.tslb_step_form.argtypes = [VP, P(ctypes.c_int32), P(ctypes.c_int32), P(ctypes.c_int32),
                                         P(ctypes.c_int32)]
            L.tslb_get_averages.argtypes = [VP, ctypes.c_int32, VP, VP, P(ctypes.c_int64), ctypes.c_int]
            L.tslb_get_averages.restype = ctypes.c_int
            L.tslb_reset_averages.argtypes = [VP]
            L.tslb_reset_averages.restype = ctypes.c_int
            L.tslb_fp32_lane_rate.argtypes = [ctypes.c_int32, VP, P(ctypes.c_double)]
            L.tslb_fp32_lane_rate.restype = ctypes.c_int
            L.tslb_halo_values.argtypes = [VP]
            L.tslb_halo_values.restype = ctypes.c_size_t
            L.tslb_halo_pack.argtypes = [VP, ctypes.c_int32, VP, ctypes.c_int]
            L.tslb_halo_pack.restype = ctypes.c_int
            L.tslb_halo_unpack.argtypes = [VP, ctypes.c_int32, VP, ctypes.c_int]
            L.tslb_halo_unpack.restype = ctypes.c_int
            for name in ("tslb_init_batch", "tslb_batch_set_state", "tslb_batch_get_moments", "tslb_batch_get_phi",
                         "tslb_batch_sums", "tslb_autotune", "tslb_step_form"):
                getattr(L, name).restype = ctypes.c_int
            for name in ("tslb_init", "tslb_set_state", "tslb_step", "tslb_get_moments", "tslb_get_phi",
                         "tslb_sums", "tslb_get_time", "tslb_get_state", "tslb_put_state",
                         "tslb_synchronize", "tslb_destroy"):
                getattr(L, name).restype = ctypes.c_int
            _lib = L
    return _lib


def _check(status: int, ctx=None):
    if status != TSLB_OK:
        msg = lib().tslb_last_error(ctx)
        raise TslbError(status, msg.decode() if msg else "")


# ---------------------------------------------------------------- C names

def tslb_default_options() -> Options:
    o = Options()
    lib().tslb_default_options(ctypes.byref(o))
    return o


def tslb_workspace_bytes(grid: Grid, opt: Optional[Options] = None) -> int:
    return int(lib().tslb_workspace_bytes(ctypes.byref(grid), ctypes.byref(opt) if opt else None))


def tslb_init(grid: Grid, omega: float, sigma: float, bc: Optional[Boundary] = None,
              opt: Optional[Options] = None, workspace: int = 0, workspace_bytes: int = 0) -> int:
    ctx = ctypes.c_void_p()
    st = lib().tslb_init(ctypes.byref(ctx), ctypes.byref(grid), TSLB_LATTICE_D3Q27_D3Q7, float(omega),
                         float(sigma), ctypes.byref(bc) if bc else None, ctypes.byref(opt) if opt else None,
                         ctypes.c_void_p(workspace or None), ctypes.c_size_t(workspace_bytes))
    _check(st, None)
    return ctx.value


def tslb_set_state(ctx: int, rho: int, u: int, pi: int, phi: int, on_device: int):
    _check(lib().tslb_set_state(ctx, rho, u, pi or None, phi, int(on_device)), ctx)


def tslb_step(ctx: int, n: int):
    _check(lib().tslb_step(ctx, int(n)), ctx)


def tslb_get_moments(ctx: int, rho: int, u: int, pi: int, on_device: int):
    _check(lib().tslb_get_moments(ctx, rho or None, u or None, pi or None, int(on_device)), ctx)


def tslb_get_phi(ctx: int, phi: int, on_device: int):
    _check(lib().tslb_get_phi(ctx, phi, int(on_device)), ctx)


def tslb_sums(ctx: int):
    m, p = ctypes.c_double(), ctypes.c_double()
    _check(lib().tslb_sums(ctx, ctypes.byref(m), ctypes.byref(p)), ctx)
    return m.value, p.value


def tslb_get_time(ctx: int) -> int:
    t = ctypes.c_int64()
    _check(lib().tslb_get_time(ctx, ctypes.byref(t)), ctx)
    return t.value


def tslb_state_bytes(ctx: int) -> int:
    return int(lib().tslb_state_bytes(ctx))


def tslb_get_state(ctx: int, dst: int, on_device: int):
    _check(lib().tslb_get_state(ctx, dst, int(on_device)), ctx)


def tslb_put_state(ctx: int, src: int, on_device: int):
    _check(lib().tslb_put_state(ctx, src, int(on_device)), ctx)


def tslb_synchronize(ctx: int):
    _check(lib().tslb_synchronize(ctx), ctx)


def tslb_destroy(ctx: int):
    _check(lib().tslb_destroy(ctx), None)


def tslb_last_error(ctx: Optional[int]) -> str:
    m = lib().tslb_last_error(ctx)
    return m.decode() if m else ""


def tslb_status_string(status: int) -> str:
    return lib().tslb_status_string(int(status)).decode()


def tslb_kernel_launches(ctx: int) -> int:
    return int(lib().tslb_kernel_launches(ctx))


def tslb_field_sums_noalloc(rho: int, phi: int, n: int, out: int, stream: int = 0):
    """FP64 totals of caller-owned FP32 device fields into out[0..1] (device),
    without any device allocation: for callers that cannot allocate at that
    point (see include/tslb.h).  Asynchronous on `stream`."""
    _check(lib().tslb_field_sums_noalloc(rho, phi, int(n), out, stream or None), None)


def tslb_batch_workspace_bytes(grids, opt: Optional[Options] = None) -> int:
    arr = (Grid * len(grids))(*grids)
    return int(lib().tslb_batch_workspace_bytes(len(grids), arr, ctypes.byref(opt) if opt else None))


def tslb_init_batch(grids, omegas, sigmas, bcs=None, opt: Optional[Options] = None, workspace: int = 0,
                    workspace_bytes: int = 0) -> int:
    n = len(grids)
    ctx = ctypes.c_void_p()
    g = (Grid * n)(*grids)
    om = (ctypes.c_double * n)(*[float(x) for x in omegas])
    sg = (ctypes.c_double * n)(*[float(x) for x in sigmas])
    b = (Boundary * n)(*bcs) if bcs is not None else None
    st = lib().tslb_init_batch(ctypes.byref(ctx), n, g, TSLB_LATTICE_D3Q27_D3Q7, om, sg, b,
                               ctypes.byref(opt) if opt else None, ctypes.c_void_p(workspace or None),
                               ctypes.c_size_t(workspace_bytes))
    _check(st, None)
    return ctx.value


def tslb_batch_set_state(ctx: int, i: int, rho: int, u: int, pi: int, phi: int, on_device: int):
    _check(lib().tslb_batch_set_state(ctx, int(i), rho, u, pi or None, phi, int(on_device)), ctx)


def tslb_batch_get_moments(ctx: int, i: int, rho: int, u: int, pi: int, on_device: int):
    _check(lib().tslb_batch_get_moments(ctx, int(i), rho or None, u or None, pi or None, int(on_device)), ctx)


def tslb_batch_get_phi(ctx: int, i: int, phi: int, on_device: int):
    _check(lib().tslb_batch_get_phi(ctx, int(i), phi, int(on_device)), ctx)


def tslb_batch_sums(ctx: int, i: int):
    m, p = ctypes.c_double(), ctypes.c_double()
    _check(lib().tslb_batch_sums(ctx, int(i), ctypes.byref(m), ctypes.byref(p)), ctx)
    return m.value, p.value


def tslb_batch_count(ctx: int) -> int:
    return int(lib().tslb_batch_count(ctx))


def tslb_step_form(ctx: int):
    """The step kernel form of the next step: (block_warps, tile_z,
    plain_stores, tma_only)."""
    v = [ctypes.c_int32() for _ in range(4)]
    _check(lib().tslb_step_form(ctx, *(ctypes.byref(x) for x in v)), ctx)
    return tuple(x.value for x in v)


def tslb_autotune(ctx: int, steps_per_trial: int = 8):
    """Returns the chosen (block_warps, tile_z, plain_stores)."""
    nw, tz, pl = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(lib().tslb_autotune(ctx, int(steps_per_trial), ctypes.byref(nw), ctypes.byref(tz), ctypes.byref(pl)),
           ctx)
    return nw.value, tz.value, pl.value


def tslb_get_averages(ctx: int, i: int, phi_sum: int, uz_sum: int, on_device: int) -> int:
    n = ctypes.c_int64()
    _check(lib().tslb_get_averages(ctx, int(i), phi_sum or None, uz_sum or None, ctypes.byref(n), int(on_device)),
           ctx)
    return n.value


def tslb_reset_averages(ctx: int):
    _check(lib().tslb_reset_averages(ctx), ctx)


def tslb_halo_values(ctx: int) -> int:
    return int(lib().tslb_halo_values(ctx))


def tslb_halo_pack(ctx: int, side: int, dst: int, on_device: int):
    _check(lib().tslb_halo_pack(ctx, int(side), dst, int(on_device)), ctx)


def tslb_halo_unpack(ctx: int, side: int, src: int, on_device: int):
    _check(lib().tslb_halo_unpack(ctx, int(side), src, int(on_device)), ctx)


def tslb_fp32_lane_rate(packed: int, stream: int = 0) -> float:
    """FP32 fused multiply-adds per second of the current device over all
    lanes (packed = 1: the packed f32x2 form); synchronises."""
    r = ctypes.c_double()
    _check(lib().tslb_fp32_lane_rate(int(packed), stream or None, ctypes.byref(r)), None)
    return r.value


# ------------------------------------------------------------ convenience

def _boundary_from(workload) -> Boundary:
    b = Boundary()
    for k, f in enumerate(workload.faces):
        b.face[k] = FACES[f]
    for a in range(3):
        b.inlet_u[a] = float(workload.inlet_u[a])
    b.inlet_diameter = float(workload.inlet_diameter)
    b.inlet_cx = float(workload.inlet_cx)
    b.inlet_cy = float(workload.inlet_cy)
    b.noise_amp = float(workload.noise_amp)
    b.seed = int(workload.seed)
    return b


class Simulation:
    """One simulation context on the current CUDA device.

    ``workload`` is an :class:`inputs.Workload` (grid, omega, sigma, faces,
    inlet).  The workspace is a torch uint8 tensor owned by this object; work
    is issued on ``stream`` (a ``torch.cuda.Stream``; default: a new one).
    """

    def __init__(self, workload, storage: str = "fp32", stream=None, tile_z: int = 0,
                 graph_steps: int = 0, check_every: int = 0, field_scale=None, block_warps: int = 0,
                 average: bool = False, scheme: str = "fused", closure: str = "projection",
                 test_tma_stall: int = 0, plain_stores: bool = False, per_tile_loads: bool = False):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("Simulation needs a CUDA device")
        self.workload = workload
        self.grid = Grid(workload.nx, workload.ny, workload.nz)
        self.N = workload.nx * workload.ny * workload.nz
        self.stream = stream if stream is not None else torch.cuda.Stream()
        o = tslb_default_options()
        o.storage = STORAGE[storage]
        o.interface_width = float(workload.width)
        o.normal_eps = float(getattr(workload, "normal_eps", 1e-2))
        o.tile_z = int(tile_z)
        o.graph_steps = int(graph_steps)
        o.check_every = int(check_every)
        o.block_warps = int(block_warps)
        o.average = 1 if average else 0
        o.scheme = {"fused": 0, "two_sweep": 1}[scheme]
        o.closure = CLOSURES[closure]
        o.test_tma_stall = int(test_tma_stall)
        o.plain_stores = 1 if plain_stores else 0
        o.per_tile_loads = 1 if per_tile_loads else 0
        self.closure = closure
        if field_scale is not None:
            for g in range(4):
                o.field_scale[g] = float(field_scale[g])
        o.cuda_stream = ctypes.c_void_p(self.stream.cuda_stream)
        self.options = o
        nbytes = tslb_workspace_bytes(self.grid, o)
        if nbytes == 0:
            raise TslbError(TSLB_ERR_INVALID_ARG, "invalid grid or options")
        self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        base = self._ws.data_ptr()
        off = (-base) % 256
        self.ctx = tslb_init(self.grid, workload.omega, workload.sigma, _boundary_from(workload), o,
                             base + off, nbytes)

    # -- state
    def set_state(self, rho, u, phi, pi=None):
        """rho[N], u[3, N], phi[N] (torch tensors on any device, or numpy)."""
        import torch
        dev = torch.device("cuda")

        def prep(a, n):
            if a is None:
                return None
            t = torch.as_tensor(a)
            t = t.to(device=dev, dtype=torch.float32).contiguous().reshape(-1)
            if t.numel() != n:
                raise ValueError(f"expected {n} values, got {t.numel()}")
            return t

        N = self.N
        r, uu, ph, pp = prep(rho, N), prep(u, 3 * N), prep(phi, N), prep(pi, 6 * N)
        torch.cuda.current_stream().synchronize()  # inputs written on the current stream
        tslb_set_state(self.ctx, r.data_ptr(), uu.data_ptr(), pp.data_ptr() if pp is not None else 0,
                       ph.data_ptr(), 1)
        self.stream.synchronize()  # the temporaries above may be freed after this

    def set_state_host(self, rho, u, phi, pi=None):
        """Host (numpy / CPU tensor, pinned or pageable) inputs through the C ABI."""
        ptr = lambda a: a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data
        tslb_set_state(self.ctx, ptr(rho), ptr(u), ptr(pi) if pi is not None else 0, ptr(phi), 0)

    def step(self, n: int = 1):
        tslb_step(self.ctx, n)

    def moments(self):
        """(rho[N], u[3, N], pi[6, N]) as float32 CUDA tensors; pi is None
        under the Chapman-Enskog closure (P is not part of its state)."""
        import torch
        N = self.N
        rho = torch.empty(N, dtype=torch.float32, device="cuda")
        u = torch.empty(3 * N, dtype=torch.float32, device="cuda")
        if self.closure == "chapman_enskog":
            tslb_get_moments(self.ctx, rho.data_ptr(), u.data_ptr(), 0, 1)
            return rho, u.view(3, N), None
        pi = torch.empty(6 * N, dtype=torch.float32, device="cuda")
        tslb_get_moments(self.ctx, rho.data_ptr(), u.data_ptr(), pi.data_ptr(), 1)
        return rho, u.view(3, N), pi.view(6, N)

    def moments_host(self, rho, u, pi):
        ptr = lambda a: (a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data) if a is not None else 0
        tslb_get_moments(self.ctx, ptr(rho), ptr(u), ptr(pi), 0)

    def phi(self):
        import torch
        out = torch.empty(self.N, dtype=torch.float32, device="cuda")
        tslb_get_phi(self.ctx, out.data_ptr(), 1)
        return out

    def phi_host(self, phi):
        tslb_get_phi(self.ctx, phi.data_ptr() if hasattr(phi, "data_ptr") else phi.ctypes.data, 0)

    def fields_numpy(self):
        """(rho, u, pi, phi) as float64 numpy arrays shaped like the grid."""
        rho, u, pi = self.moments()
        ph = self.phi()
        s = (self.workload.nz, self.workload.ny, self.workload.nx)
        f = lambda t, lead: None if t is None else t.double().cpu().numpy().reshape(lead + s)
        return f(rho, ()), f(u, (3,)), f(pi, (6,)), f(ph, ())

    def sums(self):
        return tslb_sums(self.ctx)

    @property
    def t(self) -> int:
        return tslb_get_time(self.ctx)

    @property
    def kernel_launches(self) -> int:
        return tslb_kernel_launches(self.ctx)

    def state_bytes(self) -> int:
        return tslb_state_bytes(self.ctx)

    def get_state(self):
        import torch
        buf = torch.empty(self.state_bytes(), dtype=torch.uint8, device="cuda")
        tslb_get_state(self.ctx, buf.data_ptr(), 1)
        return buf

    def put_state(self, buf):
        tslb_put_state(self.ctx, buf.data_ptr(), 1 if buf.is_cuda else 0)

    def synchronize(self):
        tslb_synchronize(self.ctx)

    def autotune(self, steps_per_trial: int = 8):
        """Pick the fastest kernel form (block size, store path) and slab depth;
        the state is unchanged.  Returns (block_warps, tile_z, plain_stores)."""
        return tslb_autotune(self.ctx, steps_per_trial)

    def step_form(self):
        """(block_warps, tile_z, plain_stores, tma_only) of the next step's
        kernel; tma_only: the kernel compiled for TMA tile loads alone."""
        return tslb_step_form(self.ctx)

    def averages(self):
        """Time averages (<phi>, <u_z>) as float64 numpy arrays shaped like the
        grid, and the number of steps they cover (needs average=True)."""
        import torch
        w = self.workload
        a = torch.empty(2 * self.N, dtype=torch.float64, device="cuda")
        n = tslb_get_averages(self.ctx, 0, a.data_ptr(), a.data_ptr() + 8 * self.N, 1)
        s = (w.nz, w.ny, w.nx)
        a = a.cpu().numpy()
        k = max(n, 1)
        return a[:self.N].reshape(s) / k, a[self.N:].reshape(s) / k, n

    def reset_averages(self):
        tslb_reset_averages(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            tslb_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchSimulation:
    """Many independent grids (a list of :class:`inputs.Workload`) advanced
    together: one persistent launch per time step, graph-replayed."""

    def __init__(self, workloads, stream=None, tile_z: int = 0, block_warps: int = 0, graph_steps: int = 0,
                 plain_stores: bool = False, per_tile_loads: bool = False):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("BatchSimulation needs a CUDA device")
        self.workloads = list(workloads)
        widths = {float(w.width) for w in self.workloads}
        eps = {float(getattr(w, "normal_eps", 1e-2)) for w in self.workloads}
        if len(widths) != 1 or len(eps) != 1:
            raise ValueError("a batch shares the interface width and the normal regularisation")
        self.grids = [Grid(w.nx, w.ny, w.nz) for w in self.workloads]
        self.stream = stream if stream is not None else torch.cuda.Stream()
        o = tslb_default_options()
        o.interface_width = widths.pop()
        o.normal_eps = eps.pop()
        o.tile_z = int(tile_z)
        o.block_warps = int(block_warps)
        o.graph_steps = int(graph_steps)
        o.plain_stores = 1 if plain_stores else 0
        o.per_tile_loads = 1 if per_tile_loads else 0
        o.cuda_stream = ctypes.c_void_p(self.stream.cuda_stream)
        self.options = o
        nbytes = tslb_batch_workspace_bytes(self.grids, o)
        if nbytes == 0:
            raise TslbError(TSLB_ERR_INVALID_ARG, "invalid grids or options")
        self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        base = self._ws.data_ptr()
        off = (-base) % 256
        self.ctx = tslb_init_batch(self.grids, [w.omega for w in self.workloads], [w.sigma for w in self.workloads],
                                   [_boundary_from(w) for w in self.workloads], o, base + off, nbytes)

    @property
    def nodes(self) -> int:
        return sum(w.nodes for w in self.workloads)

    def set_state(self, i: int, rho, u, phi, pi=None):
        import torch
        n = self.workloads[i].nodes
        prep = lambda a, k: None if a is None else torch.as_tensor(a).to("cuda", torch.float32).contiguous().reshape(-1)
        r, uu, ph, pp = prep(rho, n), prep(u, 3 * n), prep(phi, n), prep(pi, 6 * n)
        torch.cuda.current_stream().synchronize()
        tslb_batch_set_state(self.ctx, i, r.data_ptr(), uu.data_ptr(), pp.data_ptr() if pp is not None else 0,
                             ph.data_ptr(), 1)
        self.stream.synchronize()

    def step(self, n: int = 1):
        tslb_step(self.ctx, n)

    def autotune(self, steps_per_trial: int = 4):
        return tslb_autotune(self.ctx, steps_per_trial)

    def step_form(self):
        """(block_warps, tile_z of the first grid, plain_stores, tma_only) of
        the next step's kernel."""
        return tslb_step_form(self.ctx)

    def fields_numpy(self, i: int):
        import torch
        w = self.workloads[i]
        n = w.nodes
        rho = torch.empty(n, dtype=torch.float32, device="cuda")
        u = torch.empty(3 * n, dtype=torch.float32, device="cuda")
        pi = torch.empty(6 * n, dtype=torch.float32, device="cuda")
        phi = torch.empty(n, dtype=torch.float32, device="cuda")
        tslb_batch_get_moments(self.ctx, i, rho.data_ptr(), u.data_ptr(), pi.data_ptr(), 1)
        tslb_batch_get_phi(self.ctx, i, phi.data_ptr(), 1)
        s = (w.nz, w.ny, w.nx)
        f = lambda t, lead: t.double().cpu().numpy().reshape(lead + s)
        return f(rho, ()), f(u, (3,)), f(pi, (6,)), f(phi, ())

    def sums(self, i: int):
        return tslb_batch_sums(self.ctx, i)

    @property
    def t(self) -> int:
        return tslb_get_time(self.ctx)

    @property
    def kernel_launches(self) -> int:
        return tslb_kernel_launches(self.ctx)

    def synchronize(self):
        tslb_synchronize(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            tslb_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
