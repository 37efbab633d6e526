"""The C-ABI library builds for sm_103a, loads, and exports every function include/pms.h declares (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2403_00306_gb300 as pms

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "pms.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pms_[a-z_]+)\s*\(", src)))


def test_library_builds_and_loads():
    lib = pms.load()
    assert os.path.exists(pms.library_path())
    assert lib is not None


def test_every_declared_function_is_exported():
    declared = header_functions()
    assert "pms_solve" in declared and "pms_create" in declared and "pms_destroy" in declared
    lib = pms.load()
    for name in declared:
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", pms.library_path()], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (pms_[a-z_]+)", out))
    assert set(declared) <= exported, set(declared) - exported
    assert set(declared) == set(pms.ABI_FUNCTIONS)


def test_build_targets_sm_103a_only():
    from paper_2403_00306_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


@pytest.mark.gpu
def test_device_code_is_sm_103():
    # what the CUDA runtime reports for the library's own kernels on this GPU
    assert pms.pms_kernel_binary_version(0) == 103


def test_decode_is_host_only():
    assert pms.pms_decode(0, 3) == "AAA"
    assert pms.pms_decode(0b00_01_10_11, 4) == "ACGT"
    assert pms.pms_decode((1 << 64) - 1, 32) == "T" * 32
    with pytest.raises(pms.PMSError):
        pms.pms_decode(0, 33)


def test_no_gpu_means_a_loud_error():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(pms.PMSError):
        pms.Context(0)


STRUCTS = ["pms_instance", "pms_result", "pms_options", "pms_tuning", "pms_stats"]


def test_binding_structs_match_the_header_layout(tmp_path):
    # offsetof and sizeof of every field as a C compiler lays out include/pms.h,
    # against the ctypes structures of the binding
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "pms.h"', "int main(void) {"]
    for name in STRUCTS:
        cls = getattr(pms, name)
        lines.append(f'    printf("{name} sizeof %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'    printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    cc = subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                        capture_output=True, text=True)
    assert cc.returncode == 0, cc.stderr      # also fails if a binding field is missing from the header
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        struct, field, value = line.split()
        got[(struct, field)] = int(value)
    for name in STRUCTS:
        cls = getattr(pms, name)
        assert got[(name, "sizeof")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)


def test_header_structs_have_no_field_the_binding_lacks():
    src = open(os.path.join(ROOT, "include", "pms.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    for body, name in re.findall(r"typedef struct \{(.*?)\}\s*(pms_[a-z]+);", src, flags=re.S):
        fields = []
        for decl in body.split(";"):
            decl = decl.strip()
            if not decl:
                continue
            # "int n, m, l, d" or "const uint64_t *motifs"
            names = [t.strip().lstrip("*").split()[-1].lstrip("*") for t in decl.split(",")]
            fields += names
        assert [f for f, _ in getattr(pms, name)._fields_] == fields, name
