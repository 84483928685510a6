"""Host-side checks of the C ABI (CPU only, no GPU calls).

The library must build for sm_103a, load, and export every function that
include/vans.h declares.  The parameter validation and the size queries run on
the host and are checked here too, as is the independence of oracle and
CUDA path (no shared sources, no imports either way)."""
import ctypes
import os
import re

import pytest

from paper_1406_6438_gb300 import build as B
from paper_1406_6438_gb300._binding import Params, load_library

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "vans.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(vans_[a-z_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return load_library()


def test_library_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 30
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings_and_version(lib):
    assert lib.vans_version().decode().startswith("vans-gb300")
    for code in (0, -1, -2, -3, -4, -5, -6):
        assert lib.vans_status_string(code)
    assert lib.vans_status_string(-99) == b"unknown status"


def _sizes(lib, **kw):
    p = Params(**kw).c()
    return lib.vans_state_floats(ctypes.byref(p)), lib.vans_workspace_bytes(ctypes.byref(p))


def test_size_queries(lib):
    sf, wb = _sizes(lib, q=9, nx=4096, ny=4096, tau=0.6)
    pitch = 4128                       # 8 + round_up(4096, 128) + 1, rounded up to 32
    assert sf == 9 * 4096 * pitch
    assert wb == (2 * sf + 4096 * pitch + 64 + 3 * 256) * 4   # states, eps, status, monitor partials
    sf3, _ = _sizes(lib, q=19, nx=256, ny=256, nz=256, tau=0.6, wall_mask=6)
    assert sf3 == 19 * 256 * 256 * 320  # D3Q19: column 0 on a 128-byte line, 32 + 256 + 1 -> 320
    # ragged nx: rows still start on 128-byte boundaries
    sfr, _ = _sizes(lib, q=9, nx=37, ny=5, tau=0.7)
    assert sfr % 64 == 0 and sfr >= 9 * 5 * (4 + 37 + 2)


@pytest.mark.parametrize("bad", [
    dict(q=7, nx=4, ny=4), dict(q=9, nx=0, ny=4), dict(q=9, nx=4, ny=4, nz=2),
    dict(q=9, nx=4, ny=4, tau=0.5), dict(q=9, nx=4, ny=4, tau=float("nan")),
    dict(q=9, nx=4, ny=4, drag_mode=3), dict(q=9, nx=4, ny=4, drag_mode=1, k_mode=0, d_p=0.0),
    dict(q=9, nx=4, ny=4, drag_mode=1, k_mode=1, K=-1.0), dict(q=9, nx=4, ny=4, wall_mask=4),
    dict(q=19, nx=4, ny=4, nz=4, wall_mask=9),
])
def test_invalid_parameters_rejected_on_host(lib, bad):
    kw = dict(tau=0.8)
    kw.update(bad)
    p = Params(**kw).c()
    assert lib.vans_state_floats(ctypes.byref(p)) == -1
    assert lib.vans_workspace_bytes(ctypes.byref(p)) == 0
    h = ctypes.c_void_p()
    rc = lib.vans_create(ctypes.byref(p), ctypes.c_void_p(256), 1 << 30, None, ctypes.byref(h))
    assert rc == -1 and not h.value


def test_x_walls_unsupported(lib):
    p = Params(q=9, nx=8, ny=8, wall_mask=1).c()
    h = ctypes.c_void_p()
    assert lib.vans_create(ctypes.byref(p), ctypes.c_void_p(256), 1 << 30, None,
                           ctypes.byref(h)) == -5


def test_workspace_checks(lib):
    p = Params(q=9, nx=8, ny=8).c()
    need = lib.vans_workspace_bytes(ctypes.byref(p))
    h = ctypes.c_void_p()
    # misaligned or too small workspace: rejected before any CUDA call
    assert lib.vans_create(ctypes.byref(p), ctypes.c_void_p(256 + 4), need, None, ctypes.byref(h)) == -1
    assert lib.vans_create(ctypes.byref(p), ctypes.c_void_p(256), need - 4, None, ctypes.byref(h)) == -1
    assert lib.vans_create(ctypes.byref(p), None, need, None, ctypes.byref(h)) == -1
    assert lib.vans_create(ctypes.byref(p), ctypes.c_void_p(256), need, None, None) == -1
    # null handles
    assert lib.vans_step(None, 1) == -1
    assert lib.vans_set_eps(None, None) == -1
    assert lib.vans_cells(None) == -1


def test_batch_sizes(lib):
    ps = [Params(q=9, nx=64 + 7 * k, ny=32 + 3 * k, wall_mask=2, tau=0.7).c() for k in range(5)]
    arr = (type(ps[0]) * 5)(*ps)
    assert lib.vans_batch_workspace_bytes(arr, 5) > 0
    assert lib.vans_batch_workspace_bytes(arr, 0) == 0
    bad = (type(ps[0]) * 1)(Params(q=19, nx=8, ny=8, nz=8).c())
    assert lib.vans_batch_workspace_bytes(bad, 1) == 0


def test_oracle_and_cuda_path_share_nothing():
    """The oracle is independent of the CUDA path: no includes, imports or
    sources in common."""
    csrc = os.path.join(ROOT, "paper_1406_6438_gb300", "csrc")
    for f in os.listdir(csrc):
        text = open(os.path.join(csrc, f)).read()
        assert "oracle" not in text.lower(), f
    pkg = os.path.join(ROOT, "paper_1406_6438_gb300")
    for f in os.listdir(pkg):
        if f.endswith(".py"):
            text = open(os.path.join(pkg, f)).read()
            assert not re.search(r"^\s*(import|from)\s+oracle", text, re.M), f
    ora = open(os.path.join(ROOT, "oracle", "vans_oracle.c")).read()
    assert "vans.h" not in ora and "csrc" not in ora
    ora_py = open(os.path.join(ROOT, "oracle", "__init__.py")).read()
    assert "paper_1406_6438_gb300" not in ora_py


def test_plates_on_nodes_parameters(lib):
    """wall_kind 1 (plates on nodes): y walls only, ny >= 3, single domain."""
    assert lib.vans_state_floats(ctypes.byref(Params(q=9, nx=8, ny=5, wall_mask=2,
                                                     wall_kind=1).c())) > 0
    for bad in (dict(wall_mask=0), dict(ny=2), dict(wall_kind=2)):
        kw = dict(q=9, nx=8, ny=5, wall_mask=2, wall_kind=1)
        kw.update(bad)
        assert lib.vans_state_floats(ctypes.byref(Params(**kw).c())) == -1
    # z walls with plates on nodes, and batches, are refused
    assert lib.vans_state_floats(ctypes.byref(Params(q=19, nx=8, ny=5, nz=4, wall_mask=6,
                                                     wall_kind=1).c())) == -1
    one = (type(Params().c()) * 1)(Params(q=9, nx=8, ny=5, wall_mask=2, wall_kind=1).c())
    assert lib.vans_batch_workspace_bytes(one, 1) == 0


def _header_struct_fields(name):
    """Field names of `typedef struct { ... } name;` in include/vans.h, in order."""
    import re
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    m = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + r"\s*;", src)
    assert m, name
    fields = []
    for decl in m.group(1).split(";"):
        decl = " ".join(decl.split())
        if not decl:
            continue
        names = decl.split(" ", 1)[1]            # drop the type; "nx, ny, nz" or "g[3]"
        for n in names.split(","):
            fields.append(re.sub(r"\[.*\]", "", n).strip().lstrip("*"))
    return fields


def test_binding_structs_mirror_the_header():
    """The ctypes mirrors of vans_params and vans_launch list the header's
    fields in the header's order (a field added on one side only would shift
    every later one)."""
    from paper_1406_6438_gb300 import _binding as B
    assert [f for f, _ in B._CLaunch._fields_] == _header_struct_fields("vans_launch")
    assert [f for f, _ in B._CParams._fields_] == _header_struct_fields("vans_params")


@pytest.mark.parametrize("lang,std", [("c", "-std=c99"), ("c++", "-std=c++17")])
def test_header_compiles_as_plain_c_and_cpp(tmp_path, lang, std):
    """include/vans.h is a plain C header (C99 types only) usable from C++
    too: a translation unit that declares every struct compiles warning-free."""
    import shutil
    import subprocess
    cc = "gcc" if lang == "c" else "g++"
    if shutil.which(cc) is None:
        pytest.skip(cc + " not found")
    src = tmp_path / "use_vans.c"
    src.write_text('#include "vans.h"\n'
                   "int main(void) { vans_params p; vans_launch l; (void)p; (void)l;\n"
                   "  return (int)sizeof(vans_launch); }\n")
    r = subprocess.run([cc, std, "-Wall", "-Wextra", "-pedantic", "-Werror", "-x", lang,
                        "-I", os.path.join(ROOT, "include"), "-c", str(src), "-o",
                        str(tmp_path / "use_vans.o")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
