"""The C-ABI library builds for sm_103a, loads, and exports what include/mcmi.h
declares; the ctypes mirrors of its structs match the C layout.  No GPU
compute here: without a device, entry points must fail with a status."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mcmi.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2409_03095_b300 import build
    build.build()
    import paper_2409_03095_b300 as mc
    return mc.load()


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mcmi_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("mcmi_build", "mcmi_build_ex", "mcmi_apply", "mcmi_matrix_csr", "mcmi_free",
                 "mcmi_last_error", "mcmi_walk_dump", "mcmi_debug_tables"):
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", os.path.join(ROOT, "paper_2409_03095_b300", "libmcmi.so")],
                         capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (mcmi_\w+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    for n in _declared():
        getattr(lib, n)


def test_library_targets_sm103a_only():
    out = subprocess.run(["/usr/local/cuda/bin/cuobjdump", "--list-elf",
                          os.path.join(ROOT, "paper_2409_03095_b300", "libmcmi.so")],
                         capture_output=True, text=True).stdout
    arches = set(re.findall(r"sm_(\d+a?)", out))
    assert arches == {"103a"}, arches


def test_struct_layout_matches_c(lib, tmp_path):
    import paper_2409_03095_b300 as mc
    prog = tmp_path / "layout.c"
    fields = {"mcmi_params": [f for f, _ in mc.mcmi_params._fields_],
              "mcmi_stats": [f for f, _ in mc.mcmi_stats._fields_],
              "mcmi_csr": [f for f, _ in mc.mcmi_csr._fields_]}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "mcmi.h"', "int main(void){"]
    for s, fs in fields.items():
        lines.append(f'printf("{s} %zu\\n", sizeof({s}));')
        for f in fs:
            lines.append(f'printf("{s}.{f} %zu\\n", offsetof({s}, {f}));')
    lines.append("return 0;}")
    prog.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n") if l)
    for s, fs in fields.items():
        cls = getattr(mc, s)
        assert int(got[s]) == ctypes.sizeof(cls), s
        for f in fs:
            assert int(got[f"{s}.{f}"]) == getattr(cls, f).offset, (s, f)


def test_defaults_and_version(lib):
    import paper_2409_03095_b300 as mc
    p = mc.params()
    assert p.precision == 32 and p.table == -1 and p.chains == 128 and p.max_len == 256
    assert "sm_103a" in mc.version()


def test_compute_without_device_fails_with_status(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    import paper_2409_03095_b300 as mc
    csr = mc.mcmi_csr(4, 4, 0, 0, 0)
    h = ctypes.c_void_p()
    p = mc.params()
    st = lib.mcmi_build_ex(ctypes.byref(csr), ctypes.byref(p), None, ctypes.byref(h), None)
    assert st != 0 and not h.value


def test_product_and_oracle_share_no_code():
    pkg = os.path.join(ROOT, "paper_2409_03095_b300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"\boracle\b|orc_", txt), f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c", ".h")):
            txt = open(os.path.join(ROOT, "oracle", f)).read()
            assert "paper_2409_03095_b300" not in txt and "mcmi.h" not in txt, f
