"""Host-side checks of the C ABI (no GPU needed): the library builds for sm_103a,
loads, exports every entry point include/vd.h declares, its structs match the
binding's, and argument validation answers without touching a device."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "vd.h")


@pytest.fixture(scope="module")
def vd():
    from paper_1603_08161_b300 import build
    build.build()
    from paper_1603_08161_b300 import vd as mod
    return mod


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(vd_[a-z_0-9]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(vd):
    names = declared_functions()
    assert len(names) >= 20
    out = subprocess.check_output(["nm", "-D", "--defined-only", vd.LIB_PATH], text=True)
    exported = set(re.findall(r" T (vd_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert hasattr(vd.lib, n)
        assert n in vd._SIGS, f"binding lacks {n}"


def test_structs_match_header(vd):
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "vd.h"
int main(void) {
  printf("%zu %zu %zu\n", sizeof(vd_lattice_desc), sizeof(vd_solve_params), sizeof(vd_solve_report));
  printf("%zu %zu %zu\n", offsetof(vd_lattice_desc, cuda_stream), offsetof(vd_solve_params, cg_tol),
         offsetof(vd_solve_report, gn_done));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "t")
        subprocess.check_call(["gcc", "-std=c99", "-I", os.path.dirname(HEADER), c, "-o", exe])
        sizes, offs = subprocess.check_output([exe], text=True).split("\n")[:2]
    assert [int(v) for v in sizes.split()] == [ctypes.sizeof(vd.vd_lattice_desc), ctypes.sizeof(vd.vd_solve_params),
                                               ctypes.sizeof(vd.vd_solve_report)]
    assert [int(v) for v in offs.split()] == [vd.vd_lattice_desc.cuda_stream.offset, vd.vd_solve_params.cg_tol.offset,
                                              vd.vd_solve_report.gn_done.offset]


def test_invalid_arguments_rejected_on_host(vd):
    h = ctypes.c_void_p()
    bad = [vd.vd_lattice_desc(1, 4, 4, (ctypes.c_float * 3)(0, 0, 0), 0.1, 1, 0, None),
           vd.vd_lattice_desc(4, 4, 4, (ctypes.c_float * 3)(0, 0, 0), 0.0, 1, 0, None),
           vd.vd_lattice_desc(4, 4, 4, (ctypes.c_float * 3)(0, 0, 0), 0.1, 7, 0, None),
           vd.vd_lattice_desc(4, 4, 4, (ctypes.c_float * 3)(0, 0, 0), 0.1, 1, 9, None)]
    for d in bad:
        assert vd.vd_create_lattice(ctypes.byref(d), ctypes.byref(h)) == vd.VD_ERR_INVALID_ARG
    assert vd.vd_create_lattice(None, ctypes.byref(h)) == vd.VD_ERR_INVALID_ARG
    assert vd.vd_destroy_lattice(None) == vd.VD_OK
    assert vd.vd_solve(None, None, None) == vd.VD_ERR_INVALID_ARG
    assert vd.vd_set_frame(None, None, 0, 0, None, None, None, None, 0, 0) == vd.VD_ERR_INVALID_ARG
    assert vd.vd_get_warp(None, None, None, 0) == vd.VD_ERR_INVALID_ARG
    assert vd.vd_last_error(None) == b"null lattice"
    # the allocation-free rotation step bounds every dimension before forming the
    # product: 2^22 nodes per axis wraps a 64-bit product to 4, and must still be refused
    one = ctypes.c_void_p(16)
    big = 1 << 22
    for dims in [(big, big, big), (vd.VD_NOALLOC_MAX_NODES + 1, 2, 2), (41, 40, 40), (1, 4, 4)]:
        assert vd.vd_fit_rotations_noalloc(*dims, ctypes.c_float(0.01), one, one, one, None, None,
                                           None) == vd.VD_ERR_INVALID_ARG


def test_oracle_builds_and_is_independent():
    import oracle
    oracle.build()
    # the oracle and the CUDA sources share no file and include nothing of each other
    csrc = os.path.join(ROOT, "paper_1603_08161_b300", "csrc")
    for f in os.listdir(csrc):
        txt = open(os.path.join(csrc, f)).read()
        assert "oracle" not in txt.lower()
    txt = open(os.path.join(ROOT, "oracle", "vd_oracle.c")).read()
    assert "vd_kernels" not in txt and '#include "vd.h"' not in txt
    for f in ("vd.py", "build.py", "__init__.py", "synth.py"):
        t = open(os.path.join(ROOT, "paper_1603_08161_b300", f)).read()
        assert "import oracle" not in t and "from oracle" not in t


def test_marching_cubes_table_matches_the_oracle(vd):
    """The library and the oracle generate their case tables independently from the same
    rule; all 256 cases must agree triangle by triangle (host code, no device needed)."""
    import numpy as np

    import oracle
    e = (ctypes.c_int * 30)()
    for cs in range(256):
        n = vd.vd_mc_case(cs, e)
        ref = oracle.mc_case(cs)
        assert n == len(ref), cs
        assert list(e)[:3 * n] == ref.ravel().tolist(), cs
    assert vd.vd_mc_case(256, None) == -1
