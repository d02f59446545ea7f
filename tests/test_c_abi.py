"""The C ABI from C: include/prost.h compiles as strict C99, a C program links
libprost and calls its host-only entry points, and the struct layouts it
prints are the ones the ctypes binding marshals (no GPU needed)."""

import ctypes as C
import os
import shutil
import subprocess

import pytest

import paper_1302_2073_gb300 as pg
from paper_1302_2073_gb300 import build as pb

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def c_run(request):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lib = pg.lib()._name
    out_dir = os.path.join(HERE, "_scratch", "c_abi")
    os.makedirs(out_dir, exist_ok=True)
    exe = os.path.join(out_dir, "abi_host")
    cmd = [cc, "-std=c99", "-pedantic", "-Wall", "-Wextra", "-Werror", "-I", pb.INCLUDE,
           os.path.join(HERE, "c", "abi_host.c"), "-o", exe,
           "-L", os.path.dirname(lib), "-lprost", "-Wl,-rpath," + os.path.dirname(lib)]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    return r


def test_c_program_builds_and_its_checks_pass(c_run):
    assert c_run.returncode == 0, c_run.stdout + c_run.stderr
    assert "failures 0" in c_run.stdout


def _layout(text):
    sizes, fields = {}, {}
    for line in text.splitlines():
        parts = line.split()
        if parts[:1] == ["sizeof"]:
            sizes[parts[1]] = int(parts[2])
        elif len(parts) == 4 and parts[0].startswith("prost_"):
            fields[(parts[0], parts[1])] = (int(parts[2]), int(parts[3]))
    return sizes, fields


@pytest.mark.parametrize("struct", [pg.prost_params, pg.prost_stats])
def test_ctypes_layout_matches_the_c_compiler(c_run, struct):
    sizes, fields = _layout(c_run.stdout)
    name = struct.__name__
    assert C.sizeof(struct) == sizes[name]
    names = [f[0] for f in struct._fields_]
    assert sorted(names) == sorted(f for (s, f) in fields if s == name)
    for f in names:
        desc = getattr(struct, f)
        assert (desc.offset, desc.size) == fields[(name, f)], f
