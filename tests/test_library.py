"""Host-side checks of the C-ABI library (no GPU compute)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2207_08481_gb300 import build
    build.build()
    import paper_2207_08481_gb300.mcs as mcs
    return mcs


def _declared():
    txt = open(os.path.join(ROOT, "include", "mcs.h")).read()
    return sorted(set(re.findall(r"\b(mcs_[a-z_0-9]+)\s*\(", txt)))


def test_header_declares_exactly_the_binding(lib):
    assert _declared() == sorted(lib.EXPORTED)


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH], capture_output=True, text=True).stdout
    syms = {l.split()[-1] for l in out.splitlines() if l.strip()}
    for name in _declared():
        assert name in syms, name
        assert hasattr(lib.lib(), name)


def test_host_entry_points(lib):
    L = lib.lib()
    assert L.mcs_version() >= 100
    o = lib.default_options()
    assert o.precision == lib.MCS_MIXED and o.smooth_steps == 2 and o.rtol == 1e-8
    assert L.mcs_default_options(None) == lib.MCS_ERR_INVALID_ARG
    assert isinstance(L.mcs_last_error(), bytes)
    assert lib.launch_count() >= 0
    assert L.mcs_launch_count(None) == lib.MCS_ERR_INVALID_ARG


def test_invalid_arguments_are_reported_not_raised(lib):
    L = lib.lib()
    h = ctypes.c_void_p()
    o = lib.default_options()
    # bad dimension / degree / viscosity are rejected before any device work
    assert L.mcs_setup_structured(4, 8, 2, 1.0, ctypes.byref(o), None, ctypes.byref(h)) == lib.MCS_ERR_UNSUPPORTED
    assert L.mcs_setup_structured(2, 8, 1, 1.0, ctypes.byref(o), None, ctypes.byref(h)) == lib.MCS_ERR_UNSUPPORTED
    assert L.mcs_setup_structured(2, 8, 2, -1.0, ctypes.byref(o), None, ctypes.byref(h)) == lib.MCS_ERR_INVALID_ARG
    assert L.mcs_setup_structured(2, 8, 2, 1.0, ctypes.byref(o), None, None) == lib.MCS_ERR_INVALID_ARG
    assert b"NULL" in L.mcs_last_error()
    assert L.mcs_setup_structured(3, 4, 7, 1.0, ctypes.byref(o), None, ctypes.byref(h)) == lib.MCS_ERR_UNSUPPORTED
    assert L.mcs_setup_structured(2, 4, 0, 1.0, ctypes.byref(o), None, ctypes.byref(h)) == lib.MCS_ERR_UNSUPPORTED
    bad = lib.default_options(etol=-1.0)
    assert L.mcs_setup_structured(2, 8, 2, 1.0, ctypes.byref(bad), None, ctypes.byref(h)) == lib.MCS_ERR_INVALID_ARG
    assert b"etol" in L.mcs_last_error()
    bad = lib.default_options(tune=2)
    assert L.mcs_setup_structured(2, 8, 2, 1.0, ctypes.byref(bad), None, ctypes.byref(h)) == lib.MCS_ERR_INVALID_ARG
    assert b"tune" in L.mcs_last_error()
    assert lib.default_options().etol == 0.0 and lib.default_options().tune == 0
    bad = lib.default_options(residual_dd=3)
    assert L.mcs_setup_structured(2, 8, 2, 1.0, ctypes.byref(bad), None, ctypes.byref(h)) == lib.MCS_ERR_INVALID_ARG
    assert b"residual_dd" in L.mcs_last_error()
    bad = lib.default_options(asp=2)
    assert L.mcs_setup_structured(2, 8, 2, 1.0, ctypes.byref(bad), None, ctypes.byref(h)) == lib.MCS_ERR_INVALID_ARG
    assert lib.default_options().asp == 0
    bad = lib.default_options(lo_stab=2)
    assert L.mcs_setup_structured(3, 2, 1, 1.0, ctypes.byref(bad), None, ctypes.byref(h)) == lib.MCS_ERR_INVALID_ARG
    assert b"lo_stab" in L.mcs_last_error()
    assert lib.default_options().lo_stab == 0
    bad = lib.default_options(outflow=2)
    assert L.mcs_setup_structured(2, 4, 2, 1.0, ctypes.byref(bad), None, ctypes.byref(h)) == lib.MCS_ERR_INVALID_ARG
    bad = lib.default_options(outflow=1)
    assert L.mcs_setup_structured(3, 2, 1, 1.0, ctypes.byref(bad), None, ctypes.byref(h)) == lib.MCS_ERR_UNSUPPORTED
    assert b"outflow" in L.mcs_last_error()
    assert lib.default_options().outflow == 0
    assert L.mcs_apply(None, None, None) == lib.MCS_ERR_INVALID_ARG
    assert L.mcs_recover_stress(None, None, 1, None, None, None) == lib.MCS_ERR_INVALID_ARG
    assert L.mcs_residual(None, None, None, None) == lib.MCS_ERR_INVALID_ARG
    assert L.mcs_condense_batch(None, 0) == lib.MCS_ERR_INVALID_ARG
    assert L.mcs_destroy(None) == lib.MCS_OK


def test_binding_structs_match_the_header(lib, tmp_path):
    """The ctypes mirrors of the C structs have the header's size and field offsets (a mismatch would
    corrupt every call silently); checked against a C program compiled from include/mcs.h."""
    structs = {"mcs_options": lib.Options, "mcs_sizes_t": lib.Sizes, "mcs_solve_info": lib.SolveInfo,
               "mcs_kernel_stat": lib.KernelStat}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "mcs.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    cc = subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                        capture_output=True, text=True)
    assert cc.returncode == 0, cc.stderr
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        cname, fname, val = line.split()
        got[(cname, fname)] = int(val)
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
