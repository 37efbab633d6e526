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


def test_built_for_sm_103a():
    out = subprocess.run(["cuobjdump", "--list-elf", pms.library_path()], capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    assert "sm_103a" in out.stdout


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
