"""The C-ABI library builds, loads and exports every symbol include/crash.h
declares; struct layouts agree between the header and the binding; argument
errors come back as status codes.  CPU only: no compute call needs a GPU."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_1101_4127_gb300 import build, native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "include", "crash.h")


def declared_symbols():
    src = open(HDR).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(crash_[a-z_]+)\s*\(", src)))


def test_library_builds_and_exports_every_declared_symbol():
    so = build.build()
    L = C.CDLL(so)
    syms = declared_symbols()
    assert len(syms) >= 20
    for s in syms:
        assert hasattr(L, s), s
    assert set(syms) == set(native.EXPORTED)


def test_struct_layouts_match_header(tmp_path):
    probe = tmp_path / "probe.c"
    probe.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "crash.h"\n'
                     'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu\\n", sizeof(crash_grid_desc),'
                     ' sizeof(crash_run_opts), offsetof(crash_grid_desc, f_rec),'
                     ' offsetof(crash_run_opts, sort_curve), offsetof(crash_grid_desc, periodic),'
                     ' offsetof(crash_run_opts, chunk_packets), offsetof(crash_grid_desc, uv_heat_eV));return 0;}\n')
    exe = tmp_path / "probe"
    subprocess.check_call(["gcc", "-I", os.path.dirname(HDR), str(probe), "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    assert got == [C.sizeof(native.crash_grid_desc), C.sizeof(native.crash_run_opts),
                   native.crash_grid_desc.f_rec.offset, native.crash_run_opts.sort_curve.offset,
                   native.crash_grid_desc.periodic.offset, native.crash_run_opts.chunk_packets.offset,
                   native.crash_grid_desc.uv_heat_eV.offset]


def test_argument_errors_are_status_codes():
    L = native.lib()
    ctx = C.c_void_p()
    assert L.crash_init_grid(None, C.byref(ctx)) == native.CRASH_ERR_ARG
    assert b"NULL" in L.crash_last_error(None)
    d = native.crash_grid_desc()
    d.nx = 0
    d.ny = d.nz = 4
    d.box_cm = 1.0
    d.T0 = 1e4
    assert L.crash_init_grid(C.byref(d), C.byref(ctx)) == native.CRASH_ERR_ARG
    d.nx = 4
    d.box_cm = -1.0
    assert L.crash_init_grid(C.byref(d), C.byref(ctx)) == native.CRASH_ERR_ARG
    d.box_cm = 1.0
    d.f_rec = 1.5                     # the re-emission threshold is a fraction
    assert L.crash_init_grid(C.byref(d), C.byref(ctx)) == native.CRASH_ERR_ARG
    d.f_rec = 0.0
    d.coupling = 2                    # 0 or 1
    assert L.crash_init_grid(C.byref(d), C.byref(ctx)) == native.CRASH_ERR_ARG
    d.coupling, d.periodic = 0, 3
    assert L.crash_init_grid(C.byref(d), C.byref(ctx)) == native.CRASH_ERR_ARG
    d.periodic = 0
    d.uv_rate[1] = -1e-13             # a background rate is >= 0
    assert L.crash_init_grid(C.byref(d), C.byref(ctx)) == native.CRASH_ERR_ARG
    d.uv_rate[1], d.uv_heat_eV[2] = 0.0, float("inf")
    assert L.crash_init_grid(C.byref(d), C.byref(ctx)) == native.CRASH_ERR_ARG
    d.uv_heat_eV[2] = 0.0
    assert L.crash_step(None, 1.0, 1) == native.CRASH_ERR_ARG
    assert L.crash_chemistry(None, 1.0) == native.CRASH_ERR_ARG
    p = C.c_void_p()
    assert L.crash_deposits_device(None, 0, C.byref(p), None) == native.CRASH_ERR_ARG
    assert L.crash_free(None) == native.CRASH_ERR_ARG
    o = native.default_opts()
    assert o.chemistry == 1 and o.pkt_end == 0xFFFFFFFF and o.cool_mask == 63
