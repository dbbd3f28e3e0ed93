"""C-ABI checks that need no GPU: libtopo.so loads, exports every entry point declared in
include/topo.h, the ctypes structures match the C layout, and invalid problem descriptions
are rejected on the host before any CUDA call."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2004_05756_gb300 import build, native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "topo.h")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return native.load()


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(topo_[A-Za-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    declared = _declared()
    assert set(declared) == set(native.EXPORTS)
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (topo_\w+)", out))
    for name in declared:
        assert name in exported, name
        assert hasattr(lib, name)


def test_struct_layout_matches_header(tmp_path):
    c = tmp_path / "sz.c"
    c.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "topo.h"\nint main(void){printf("%zu %zu %zu %zu\\n",'
                 'sizeof(topo_problem), offsetof(topo_problem, fixed_dof_mask), sizeof(topo_solve_info),'
                 'offsetof(topo_solve_info, status)); printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(topo_tr_state),'
                 'offsetof(topo_tr_state, ratio), offsetof(topo_tr_state, sel), offsetof(topo_tr_state, iter),'
                 'sizeof(topo_tr_params), offsetof(topo_tr_params, c1)); return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    assert vals == [ctypes.sizeof(native.topo_problem), native.topo_problem.fixed_dof_mask.offset,
                    ctypes.sizeof(native.topo_solve_info), native.topo_solve_info.status.offset,
                    ctypes.sizeof(native.topo_tr_state), native.topo_tr_state.ratio.offset,
                    native.topo_tr_state.sel.offset, native.topo_tr_state.iter.offset,
                    ctypes.sizeof(native.topo_tr_params), native.topo_tr_params.c1.offset]
    assert native.TR_STATE_BYTES == 128


@pytest.mark.parametrize("bad", [
    dict(dim=4), dict(nx=0), dict(E0=1e-9, Emin=1e-9), dict(nu=0.5), dict(penal=2.5), dict(penal=7.0),
    dict(rmin=0.0), dict(rmin=7.0), dict(mask=False)])
def test_create_rejects_invalid(lib, bad):
    N = 2 * 3 * 3
    mask = np.zeros(N, np.uint8)
    kw = dict(dim=2, nx=2, ny=2, nz=1, E0=1.0, Emin=1e-9, nu=0.3, penal=3.0, rmin=1.5)
    use_mask = bad.pop("mask", True)
    kw.update(bad)
    pr = native.topo_problem(kw["dim"], kw["nx"], kw["ny"], kw["nz"], kw["E0"], kw["Emin"], kw["nu"], kw["penal"],
                             kw["rmin"], mask.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)) if use_mask else None)
    h = ctypes.c_void_p()
    assert lib.topo_create(ctypes.byref(pr), None, ctypes.byref(h)) == native.TOPO_ERR_INVALID
    assert not h.value
    assert lib.topo_create(None, None, ctypes.byref(h)) == native.TOPO_ERR_INVALID
