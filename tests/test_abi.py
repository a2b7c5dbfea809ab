"""The C ABI library builds for sm_103a, loads, and exports every entry point
declared in include/tslb.h; host-side argument checking works without a GPU."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2403_15773_gb300 as tslb
from paper_2403_15773_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"TSLB_API\s+[\w\s\*]*?\b(tslb_\w+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_the_abi():
    names = declared_symbols()
    for n in ("tslb_init", "tslb_step", "tslb_get_moments", "tslb_get_phi", "tslb_sums", "tslb_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol():
    path = build.build()
    L = ctypes.CDLL(path)
    for n in declared_symbols():
        assert hasattr(L, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (tslb_\w+)", out))
    assert set(declared_symbols()) <= exported


def test_binding_names_match_header():
    assert sorted(tslb.SYMBOLS) == declared_symbols()
    for n in declared_symbols():
        assert callable(getattr(tslb, n))


def test_default_options():
    o = tslb.tslb_default_options()
    assert o.storage == 0 and abs(o.interface_width - 3.0) < 1e-7 and abs(o.normal_eps - 1e-2) < 1e-9
    assert o.check_every == 0 and o.tile_z == 0 and o.graph_steps == 0 and o.block_warps == 0


def test_workspace_bytes():
    g = tslb.Grid(32, 32, 32)
    b = tslb.tslb_workspace_bytes(g)
    N = 32 ** 3
    assert b >= 2 * 11 * N * 4 + N * 4
    o = tslb.tslb_default_options()
    o.storage = tslb.STORAGE["fp16"]
    b16 = tslb.tslb_workspace_bytes(g, o)
    assert 2 * 11 * N * 2 <= b16 < b
    assert tslb.tslb_workspace_bytes(tslb.Grid(0, 4, 4)) == 0


def _bc(faces):
    b = tslb.Boundary()
    for k, f in enumerate(faces):
        b.face[k] = tslb.FACES[f]
    return b


@pytest.mark.parametrize("case", [
    dict(omega=2.5),
    dict(omega=0.0),
    dict(sigma=-1.0),
    dict(faces=("inlet", "outflow", "periodic", "periodic", "periodic", "periodic")),
    dict(faces=("periodic", "outflow", "periodic", "periodic", "periodic", "periodic")),
    dict(grid=(1, 8, 8), faces=("free_slip", "free_slip", "periodic", "periodic", "periodic", "periodic")),
    dict(grid=(8, 8, 0)),
    dict(faces=("halo", "halo", "periodic", "periodic", "periodic", "periodic")),
    dict(faces=("periodic", "periodic", "periodic", "periodic", "halo", "periodic")),
])
def test_init_rejects_invalid_arguments_before_touching_the_gpu(case):
    g = tslb.Grid(*case.get("grid", (8, 8, 8)))
    bc = _bc(case.get("faces", ("periodic",) * 6))
    with pytest.raises(tslb.TslbError) as ei:
        tslb.tslb_init(g, case.get("omega", 1.5), case.get("sigma", 0.0), bc)
    assert ei.value.status == tslb.TSLB_ERR_INVALID_ARG
    assert tslb.tslb_last_error(None)


def test_status_strings():
    assert tslb.tslb_status_string(0) == "ok"
    assert "invalid" in tslb.tslb_status_string(1)


def test_product_code_does_not_use_the_oracle():
    pkg = os.path.join(ROOT, "paper_2403_15773_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".h", ".cuh", ".cpp")):
                src = open(os.path.join(dirpath, fn)).read()
                assert "import oracle" not in src and "tslb_oracle" not in src, fn


def test_kernel_options_are_checked_before_touching_the_gpu():
    g = tslb.Grid(8, 8, 8)
    for kw in (dict(closure=2), dict(closure=1, block_warps=16), dict(closure=1, scheme=1), dict(plain_stores=2),
               dict(plain_stores=-1), dict(per_tile_loads=2), dict(per_tile_loads=-1)):
        o = tslb.tslb_default_options()
        for k, v in kw.items():
            setattr(o, k, v)
        with pytest.raises(tslb.TslbError) as ei:
            tslb.tslb_init(g, 1.5, 0.0, None, o)
        assert ei.value.status == tslb.TSLB_ERR_INVALID_ARG


def test_halo_faces_need_the_fused_projection_step():
    g = tslb.Grid(8, 8, 8)
    bc = _bc(("periodic",) * 4 + ("halo", "outflow"))
    for kw in (dict(closure=1), dict(scheme=1)):
        o = tslb.tslb_default_options()
        for k, v in kw.items():
            setattr(o, k, v)
        with pytest.raises(tslb.TslbError) as ei:
            tslb.tslb_init(g, 1.5, 0.0, bc, o)
        assert ei.value.status == tslb.TSLB_ERR_INVALID_ARG
    with pytest.raises(tslb.TslbError):
        tslb.tslb_init_batch([g], [1.5], [0.0], [bc])


def test_workspace_holds_the_ghost_planes_of_halo_faces():
    """A single grid's workspace is sized for halo z faces (four ghost planes
    after each field of both state buffers), whatever faces it gets."""
    g = tslb.Grid(16, 12, 10)
    N, nxy = 16 * 12 * 10, 16 * 12
    assert tslb.tslb_workspace_bytes(g) >= 2 * 11 * (N + 4 * nxy) * 4
    o = tslb.tslb_default_options()
    o.storage = tslb.STORAGE["fp16"]
    assert tslb.tslb_workspace_bytes(g, o) >= 2 * 11 * (N + 4 * nxy) * 2


def test_chapman_enskog_state_is_five_fields():
    g = tslb.Grid(32, 32, 32)
    N = 32 ** 3
    o = tslb.tslb_default_options()
    full = tslb.tslb_workspace_bytes(g, o)
    o.closure = tslb.CLOSURES["chapman_enskog"]
    ce = tslb.tslb_workspace_bytes(g, o)
    assert 2 * 5 * N * 4 <= ce and full - ce >= 2 * 6 * N * 4


def test_ctypes_structs_match_the_c_layout(tmp_path):
    """Offsets and sizes of the option, boundary and grid structs as gcc lays
    them out from the header, against the binding's ctypes structures."""
    structs = {"tslb_options": tslb.Options, "tslb_boundary": tslb.Boundary, "tslb_grid": tslb.Grid}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "tslb.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("  return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l}
    for cname, cls in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)
