"""The C ABI without a GPU: libpff.so loads, exports every function that
include/pff.h declares, the Python binding declares a signature for each of
them, and argument checks that need no device return PFF_ERR_ARG."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pff.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(pff_[a-z0-9_]+)\s*\(",
                       src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2606_23458_b300 import build
    path = build.build()
    return C.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("pff_mesh_create", "pff_mesh_set_material", "pff_step_explicit", "pff_damage_solve",
              "pff_run", "pff_run_ckpt", "pff_backward", "pff_batch_create", "pff_batch_run",
              "pff_mesh_destroy", "pff_last_error", "pff_damage_solve_noalloc"):
        assert n in names, n


def test_library_exports_every_declared_function(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_function(lib):
    import paper_2606_23458_b300 as pff
    bound = set(pff._sig) | {"pff_last_error", "pff_version"}
    assert set(_declared()) <= bound, sorted(set(_declared()) - bound)


def test_host_side_argument_checks(lib):
    lib.pff_last_error.restype = C.c_char_p
    lib.pff_version.restype = C.c_char_p
    assert lib.pff_version().decode()
    out = C.c_void_p()
    # null inputs are refused before any device work
    assert lib.pff_mesh_create(C.c_int64(0), None, C.c_int64(0), None, None, C.c_int64(0), None, None,
                               C.c_int32(0), C.byref(out)) == 1
    assert lib.pff_last_error().decode()
    assert lib.pff_mesh_set_material(None, None, C.c_double(0.5), None) == 1
    assert lib.pff_mesh_cg_choice(None, None, None, None) == 1
    assert lib.pff_mesh_fused_schedule(None, None, None) == 1
    assert lib.pff_ckpt_create(None, C.c_int64(10), C.c_int32(0), C.byref(out)) == 1
    assert lib.pff_backward(None, None, None, None, None, None) == 1
    lib.pff_mesh_destroy(None)  # a no-op


def test_subcycling_limit_matches_oracle(orc):
    """pff_subcycling_limit (host-only) against the oracle's check."""
    import paper_2606_23458_b300 as pff
    import pff_synth as S
    for plane in ("strain", "stress"):
        for nu in (0.1, 0.2, 0.25, 0.35, 0.45):
            mat = S.material(1e-3, nu=nu, plane=plane)
            r, n = pff.subcycling_limit(mat)
            ro, no = orc.subcycling_limit(mat)
            assert abs(r - ro) <= 1e-10 * ro and n == no, (plane, nu, r, ro)
    bad = pff.pff_material(0.0, 0.2, 2450.0, 3.0, 1e-3, 1e-7, 2, 0, 0, 0)
    assert pff._lib.pff_subcycling_limit(C.byref(bad), None, None) == 1



def test_struct_layouts_match_the_header(tmp_path):
    """Every struct the binding passes by pointer has the header's size and
    field offsets (a C program compiled against include/pff.h prints them)."""
    import shutil
    import subprocess
    import paper_2606_23458_b300 as pff
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"pff_material": pff.pff_material, "pff_options": pff.pff_options,
               "pff_state": pff.pff_state, "pff_qs_options": pff.pff_qs_options,
               "pff_plate": pff.pff_plate}
    lines = ['#include <stdio.h>', '#include "pff.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for ln in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        s, f, v = ln.split()
        got[(s, f)] = int(v)
    for name, cls in structs.items():
        assert got[(name, "size")] == C.sizeof(cls), name
        for f, _ in cls._fields_:
            assert got[(name, f)] == getattr(cls, f).offset, (name, f)
