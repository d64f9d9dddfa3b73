"""CPU checks of the C-ABI library: it builds, loads without a GPU, exports
every symbol that include/fdtd.h declares, and validates arguments on the
host (no compute calls)."""
import ctypes
import os
import re

import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def fd():
    import __graft_entry__

    __graft_entry__._lib_builder().build()
    import paper_0904_0939_gb300 as fd

    return fd


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "fdtd.h")).read()
    return sorted(set(re.findall(r"FDTD_API\s+[\w\s\*]*?\b(fdtd_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ["fdtd_create", "fdtd_set_potential", "fdtd_init_symmetric", "fdtd_evolve",
                     "fdtd_observables", "fdtd_upsample", "fdtd_backward"]:
        assert required in names


def test_library_exports_every_declared_symbol(fd):
    lib = ctypes.CDLL(fd.LIB_PATH)
    for name in declared_symbols():
        assert hasattr(lib, name), name
    assert set(fd.EXPORTED) | {"fdtd_last_error"} >= set(declared_symbols())


def test_last_error_copies_into_the_callers_buffer(fd):
    """fdtd_last_error(h, buf, n): full length returned, the copy truncated
    and NUL-terminated (checked after a failed create, no GPU needed)."""
    o = fd.default_options(check_every=0)
    h = ctypes.c_void_p()
    desc = fd.Lattice(8, 4.0, fd.F32).desc()
    rc = fd.lib.fdtd_create(ctypes.byref(desc), 1, ctypes.byref(o), None, 0, None, ctypes.byref(h))
    assert rc < 0
    full = fd.lib.fdtd_last_error(None, None, 0)
    assert full > 0
    msg = fd.last_error(None)
    assert len(msg) == full
    small = ctypes.create_string_buffer(8)
    assert fd.lib.fdtd_last_error(None, small, 8) == full
    assert small.value == msg.encode()[:7]


def test_default_options(fd):
    o = fd.default_options()
    assert o.check_every == 100 and o.tol == pytest.approx(1e-6) and o.tol_relative == 1
    assert o.reimpose_parity == 1 and o.batched == 0


def _size(fd, lats, **kw):
    arr = (fd.LatticeDesc * len(lats))(*[l.desc() for l in lats])
    size = ctypes.c_size_t()
    o = fd.default_options(**kw)
    rc = fd.lib.fdtd_workspace_size(arr, len(lats), ctypes.byref(o), ctypes.byref(size))
    return rc, size.value


def test_workspace_size_grows_with_lattice(fd):
    rc1, s1 = _size(fd, [fd.Lattice(32, 10.0, fd.F32)])
    rc2, s2 = _size(fd, [fd.Lattice(64, 10.0, fd.F32)])
    rc3, s3 = _size(fd, [fd.Lattice(64, 10.0, fd.F64)])
    assert rc1 == rc2 == rc3 == 0
    assert s2 - s1 >= 3 * (64**3 - 32**3) * 4 and s3 - s2 >= 5 * 64**3 * 4
    rc4, s4 = _size(fd, [fd.Lattice(32, 10.0, fd.F32)], backward_steps=400)
    assert rc4 == 0 and s4 > s1 + 20 * 32**3 * 4  # sqrt(T) checkpoints + segment


def test_host_side_validation(fd):
    # von Neumann bound dtau < m a^2 / 3 (Sec. III)
    a = 10.0 / 32
    rc, _ = _size(fd, [fd.Lattice(32, 10.0, fd.F32, dtau=a * a / 3 * 1.0001)])
    assert rc == fd.ERR_UNSTABLE_DT
    rc, _ = _size(fd, [fd.Lattice(32, 10.0, fd.F32, dtau=a * a / 3 * 0.99)])
    assert rc == fd.OK
    rc, _ = _size(fd, [fd.Lattice(0, 10.0, fd.F32)])
    assert rc == fd.ERR_INVALID_ARG
    rc, _ = _size(fd, [fd.Lattice(8, -1.0, fd.F32)])
    assert rc == fd.ERR_INVALID_ARG
    rc, _ = _size(fd, [fd.Lattice(8, 1.0, 7)])
    assert rc == fd.ERR_INVALID_ARG
    rc, _ = _size(fd, [fd.Lattice(8, 1.0, fd.F32)], check_every=0)
    assert rc == fd.ERR_INVALID_ARG
    assert "check_every" in fd.last_error(None)
    rc, _ = _size(fd, [fd.Lattice(32, 10.0, fd.F32, dtau=a * a / 3 * 1.0001)])
    assert "von Neumann" in fd.last_error(None)
    # tile shapes: 64 or 128 wide, 16 or 32 high, 32 only with 64-wide tiles
    for kw, ok in ((dict(tile_x=64, tile_y=32), True), (dict(tile_x=128), True), (dict(tile_y=16), True),
                   (dict(tile_x=96), False), (dict(tile_y=8), False), (dict(tile_x=128, tile_y=32), False)):
        rc, _ = _size(fd, [fd.Lattice(32, 10.0, fd.F32)], **kw)
        assert (rc == fd.OK) == ok, kw
        if not ok:
            assert rc == fd.ERR_INVALID_ARG and "tile" in fd.last_error(None)


def test_create_rejects_bad_workspace(fd):
    arr = (fd.LatticeDesc * 1)(fd.Lattice(8, 4.0, fd.F32).desc())
    o = fd.default_options()
    h = ctypes.c_void_p()
    rc = fd.lib.fdtd_create(arr, 1, ctypes.byref(o), None, 0, None, ctypes.byref(h))
    assert rc == fd.ERR_WORKSPACE and not h.value
    rc = fd.lib.fdtd_create(arr, 1, ctypes.byref(o), ctypes.c_void_p(0x1001), 1 << 30, None, ctypes.byref(h))
    assert rc == fd.ERR_WORKSPACE


def test_null_handle_calls_fail_cleanly(fd):
    assert fd.lib.fdtd_evolve(None, 10, None) == fd.ERR_INVALID_ARG
    assert fd.lib.fdtd_destroy(None) == fd.ERR_INVALID_ARG
    assert fd.lib.fdtd_set_potential(None, 0, None, 0, 0) == fd.ERR_INVALID_ARG


def _struct_fields(text, name):
    body = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + r";", text).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    return re.findall(r"\b(\w+)(?:\s*\[\s*\d+\s*\])?\s*;", body)


def test_struct_layouts_match_the_header(fd, tmp_path):
    """Size and every field offset of the public structs, as gcc lays them
    out from include/fdtd.h, equal the ctypes definitions of the binding."""
    import shutil
    import subprocess

    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    text = open(os.path.join(ROOT, "include", "fdtd.h")).read()
    pairs = {"fdtd_lattice_desc": fd.LatticeDesc, "fdtd_options": fd.Options, "fdtd_obs": fd.Obs,
             "fdtd_stats": fd.Stats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "fdtd.h"', "int main(void) {"]
    for cname in pairs:
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f in _struct_fields(text, cname):
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for row in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        cname, field, value = row.split()
        got[(cname, field)] = int(value)
    for cname, cls in pairs.items():
        assert got[(cname, "sizeof")] == ctypes.sizeof(cls), cname
        names = _struct_fields(text, cname)
        assert names == [f for f, _ in cls._fields_], cname
        for f in names:
            assert got[(cname, f)] == getattr(cls, f).offset, (cname, f)
