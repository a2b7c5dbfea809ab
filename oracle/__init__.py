"""FP64 CPU oracle of the multicomponent thread-safe LB step (arXiv 2403.15773).

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only code allowed to import this module.
The product library never imports it and shares no code with it: the oracle
is plain C (``tslb_oracle.c``) in FP64 that keeps the paper's 27 + 7
population arrays and advances them with the literal push of Sec. 2 (Eq.
pushLB, eqts, noneqts, neq_final; Sec. 2.2 Eq. intcapturing, antidiff).

Every function of the C file is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_*.py`` against closed forms, invariants and printed values.
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tslb_oracle.c")
_HDR = os.path.join(_HERE, "tslb_oracle.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

PERIODIC, INLET, OUTFLOW, FREE_SLIP = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile ``tslb_oracle.c`` with gcc (OpenMP when available)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))):
        return _LIB_PATH
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        raise RuntimeError("oracle build: no C compiler found")
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = [cc, "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("omega", ctypes.c_double), ("sigma", ctypes.c_double), ("gamma", ctypes.c_double),
        ("face", ctypes.c_int * 6),
        ("inlet_u", ctypes.c_double * 3),
        ("inlet_diameter", ctypes.c_double),
        ("inlet_cx", ctypes.c_double), ("inlet_cy", ctypes.c_double),
        ("inlet_width", ctypes.c_double),
        ("noise_amp", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("ext_force", ctypes.c_double * 3),
        ("normal_eps", ctypes.c_double),
        ("ce_neq", ctypes.c_int),
    ]


_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.POINTER(ctypes.c_int64)
_U32 = ctypes.POINTER(ctypes.c_uint32)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            l = ctypes.CDLL(build())
            l.orc_create.restype = ctypes.c_void_p
            l.orc_create.argtypes = [ctypes.POINTER(Params)]
            l.orc_destroy.argtypes = [ctypes.c_void_p]
            l.orc_set_state.argtypes = [ctypes.c_void_p, _D, _D, _D, _D, ctypes.c_int64]
            l.orc_set_state.restype = ctypes.c_int
            l.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_int]
            l.orc_get_moments.argtypes = [ctypes.c_void_p, _D, _D, _D, _D]
            l.orc_sums.argtypes = [ctypes.c_void_p, _D, _D, _D]
            l.orc_time.argtypes = [ctypes.c_void_p]
            l.orc_time.restype = ctypes.c_int64
            l.orc_threads.restype = ctypes.c_int
            l.orc_set_threads.argtypes = [ctypes.c_int]
            l.orc_set_threads.restype = None
            l.orc_step_sample.argtypes = [ctypes.POINTER(Params), ctypes.c_int64, _D, _D, _D, _D,
                                          ctypes.c_int64, _I64, _D]
            l.orc_step_sample.restype = ctypes.c_int
            l.orc_lattice.argtypes = [_D, _D, _D, _D]
            l.orc_post_populations.argtypes = [ctypes.c_double, _D, _D, _D, ctypes.c_double, _D]
            l.orc_feq3.argtypes = [ctypes.c_double, _D, _D]
            l.orc_interface.argtypes = [_D, ctypes.c_double, ctypes.c_double, _D, _D, _D, _D, _D]
            l.orc_philox4x32_10.argtypes = [_U32, _U32, _U32]
            l.orc_ce_neq.argtypes = [_D, ctypes.c_double, _D]
            l.orc_inlet_state.argtypes = [ctypes.POINTER(Params), ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int64, _D, _D]
            _lib = l
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _f64(a, n=None) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def make_params(nx, ny, nz, omega, sigma=0.0, gamma=0.0, faces=(0, 0, 0, 0, 0, 0),
                inlet_u=(0.0, 0.0, 0.0), inlet_diameter=0.0, inlet_cx=0.0, inlet_cy=0.0,
                inlet_width=3.0, noise_amp=0.0, seed=0, ext_force=(0.0, 0.0, 0.0),
                normal_eps=1e-2, ce_neq=False) -> Params:
    p = Params()
    p.nx, p.ny, p.nz = int(nx), int(ny), int(nz)
    p.omega, p.sigma, p.gamma = float(omega), float(sigma), float(gamma)
    for k in range(6):
        p.face[k] = int(faces[k])
    for a in range(3):
        p.inlet_u[a] = float(inlet_u[a])
        p.ext_force[a] = float(ext_force[a])
    p.inlet_diameter = float(inlet_diameter)
    p.inlet_cx, p.inlet_cy = float(inlet_cx), float(inlet_cy)
    p.inlet_width = float(inlet_width)
    p.noise_amp = float(noise_amp)
    p.seed = int(seed)
    p.normal_eps = float(normal_eps)
    p.ce_neq = 1 if ce_neq else 0
    return p


class OracleSim:
    """A running oracle simulation on an (nx, ny, nz) grid (x fastest)."""

    def __init__(self, params: Params):
        self.params = params
        self.shape = (params.nz, params.ny, params.nx)
        self.N = params.nx * params.ny * params.nz
        self._h = lib().orc_create(ctypes.byref(params))
        if not self._h:
            raise ValueError("oracle rejected the parameters")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    def set_state(self, rho, u, phi, pi=None, t0: int = 0):
        N = self.N
        r, uu, ph = _f64(rho, N), _f64(u, 3 * N), _f64(phi, N)
        pp = _f64(pi, 6 * N) if pi is not None else None
        lib().orc_set_state(self._h, _dp(r), _dp(uu), _dp(pp) if pp is not None else None, _dp(ph), int(t0))

    def step(self, n: int = 1):
        lib().orc_step(self._h, int(n))

    @property
    def t(self) -> int:
        return int(lib().orc_time(self._h))

    def moments(self):
        """(rho[N], u[3,N], pi[6,N], phi[N]) as grid-shaped arrays (…, nz, ny, nx)."""
        N = self.N
        rho, u, pi, phi = (np.empty(N), np.empty(3 * N), np.empty(6 * N), np.empty(N))
        lib().orc_get_moments(self._h, _dp(rho), _dp(u), _dp(pi), _dp(phi))
        s = self.shape
        return rho.reshape(s), u.reshape((3,) + s), pi.reshape((6,) + s), phi.reshape(s)

    def sums(self):
        m, ph, j = ctypes.c_double(), ctypes.c_double(), np.empty(3)
        lib().orc_sums(self._h, ctypes.byref(m), ctypes.byref(ph), _dp(j))
        return m.value, ph.value, j


def step_sample(params: Params, t: int, rho, u, pi, phi, idx) -> np.ndarray:
    """New (rho, u, P, phi) at the flat node indices ``idx`` after one step from
    the given full stored state at step ``t``; shape (len(idx), 11)."""
    N = params.nx * params.ny * params.nz
    r, uu, pp, ph = _f64(rho, N), _f64(u, 3 * N), _f64(pi, 6 * N), _f64(phi, N)
    ix = np.ascontiguousarray(np.asarray(idx, dtype=np.int64))
    out = np.empty((ix.size, 11))
    rc = lib().orc_step_sample(ctypes.byref(params), int(t), _dp(r), _dp(uu), _dp(pp), _dp(ph),
                               ix.size, ix.ctypes.data_as(_I64), _dp(out))
    if rc != 0:
        raise ValueError("oracle step_sample rejected its input")
    return out


def lattice():
    c27, w27, c7, w7 = np.empty(81), np.empty(27), np.empty(21), np.empty(7)
    lib().orc_lattice(_dp(c27), _dp(w27), _dp(c7), _dp(w7))
    return c27.reshape(27, 3), w27, c7.reshape(7, 3), w7


def post_populations(rho, u_raw, pi6, force, omega) -> np.ndarray:
    f = np.empty(27)
    lib().orc_post_populations(float(rho), _dp(_f64(u_raw, 3)), _dp(_f64(pi6, 6)),
                               _dp(_f64(force, 3)), float(omega), _dp(f))
    return f


def feq3(rho, u) -> np.ndarray:
    f = np.empty(27)
    lib().orc_feq3(float(rho), _dp(_f64(u, 3)), _dp(f))
    return f


def interface(phi27, sigma, eps=1e-2):
    g, h, n, k, F = np.empty(3), np.empty(6), np.empty(3), ctypes.c_double(), np.empty(3)
    lib().orc_interface(_dp(_f64(phi27, 27)), float(sigma), float(eps), _dp(g), _dp(h), _dp(n),
                        ctypes.byref(k), _dp(F))
    return g, h, n, k.value, F


def ce_neq(j27, omega) -> np.ndarray:
    """Chapman-Enskog a2_neq (xx, yy, zz, xy, xz, yz) from the momentum j of the
    27 neighbours (27 x 3, oracle direction order)."""
    out = np.empty(6)
    lib().orc_ce_neq(_dp(_f64(j27, 81)), float(omega), _dp(out))
    return out


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    o = np.empty(4, dtype=np.uint32)
    lib().orc_philox4x32_10(c.ctypes.data_as(_U32), k.ctypes.data_as(_U32), o.ctypes.data_as(_U32))
    return o


def inlet_state(params: Params, x: int, y: int, t: int):
    u = np.empty(3)
    ph = ctypes.c_double()
    lib().orc_inlet_state(ctypes.byref(params), int(x), int(y), int(t), _dp(u), ctypes.byref(ph))
    return u, ph.value


def threads() -> int:
    return int(lib().orc_threads())


def set_threads(n: int) -> None:
    """Threads of the later steps (timing only: the results do not depend on it)."""
    lib().orc_set_threads(int(n))
