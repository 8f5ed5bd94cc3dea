"""CPU-side checks of the C ABI: the library builds, loads, exports every
function include/kn.h declares, and rejects bad arguments with status codes
(no GPU work is launched here)."""
import ctypes as C
import os

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def knmod():
    from paper_1409_5826_gb300 import build, kn
    build.build()
    return kn


def test_exports_every_declared_function(knmod):
    L = knmod.lib()
    names = knmod.header_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(L, n), n


def test_default_opts_match_header(knmod):
    o = knmod.default_opts()
    assert o.precision == knmod.PREC_MIXED
    assert o.kappa == 1.0  # Sec. 3: kappa = 1
    assert (o.eps_r, o.eps_c, o.y_min) == (0.05, 1e-6, 1e-10)
    assert (o.grow_max, o.safety, o.shrink, o.max_reject) == (1.5, 0.9, 0.5, 60)


def test_struct_sizes_match_header(knmod):
    # the binding's ctypes mirrors must match the C layouts byte for byte
    assert C.sizeof(knmod._Opts) == 4 * 2 + 8 * 8 + 8 + 4 * 4 + 8 * 3 + 8 + 8 * 5 + 8 * 5 + 4 * 2 + 8
    assert C.sizeof(knmod._Desc) == 8 + 5 * 8
    assert C.sizeof(knmod._Zones) == 7 * 8


def test_bad_arguments_return_codes(knmod):
    L = knmod.lib()
    assert L.kn_create_network(None, None) == knmod.KN_ERR_INVALID_ARG
    assert b"NULL" in L.kn_last_error()
    d = knmod._Desc(0, 0, None, None, None, None, None)
    h = C.c_void_p()
    assert L.kn_create_network(C.byref(d), C.byref(h)) == knmod.KN_ERR_INVALID_ARG
    # a reaction with a species id out of range is rejected before any GPU call
    A = np.ones(2)
    reac = np.array([[0, -1, -1]], np.int32)
    prod = np.array([[5, -1, -1]], np.int32)
    lk = np.zeros(1)
    d = knmod._Desc(2, 1, A.ctypes.data, reac.ctypes.data, prod.ctypes.data, lk.ctypes.data, lk.ctypes.data)
    assert L.kn_create_network(C.byref(d), C.byref(h)) == knmod.KN_ERR_INVALID_ARG
    assert b"product" in L.kn_last_error()
    # reactant list with a gap
    reac = np.array([[-1, 0, -1]], np.int32)
    prod = np.array([[1, -1, -1]], np.int32)
    d = knmod._Desc(2, 1, A.ctypes.data, reac.ctypes.data, prod.ctypes.data, lk.ctypes.data, lk.ctypes.data)
    assert L.kn_create_network(C.byref(d), C.byref(h)) == knmod.KN_ERR_INVALID_ARG
    assert L.kn_destroy_network(None) == knmod.KN_OK
    assert L.kn_integrate_batch(None, 0, None, None) == knmod.KN_ERR_INVALID_ARG


def test_struct_fields_match_header_offsets(knmod, tmp_path):
    """Every field of the binding's ctypes mirrors sits at the offset the C
    compiler gives the same-named member of the header's struct (a host-only
    C program including include/kn.h prints offsetof and sizeof)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    pairs = [("kn_network_desc", knmod._Desc), ("kn_zone_conditions", knmod._Zones),
             ("kn_opts", knmod._Opts), ("kn_batch_stats", knmod._Stats), ("kn_tiling", knmod._Tiling)]
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "kn.h"', "int main(void) {"]
    for cname, py in pairs:
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f in py._fields_:
            lines.append(f'  printf("{cname} {f[0]} %zu\\n", offsetof({cname}, {f[0]}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "offsets.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "offsets"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in pairs:
        assert got[(cname, "sizeof")] == C.sizeof(py), cname
        for f in py._fields_:
            assert got[(cname, f[0])] == getattr(py, f[0]).offset, (cname, f[0])
