"""The C ABI library builds, loads and exports every symbol the header declares
(no compute calls: these run without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2108_02259_gb300 import apic, build

    build.build()
    return apic.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "apiccontact.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(apic_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_expected(lib):
    from paper_2108_02259_gb300 import apic

    assert set(_declared()) == set(apic.EXPORTED)


def test_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_version_and_last_error(lib):
    assert b"sm_103a" in lib.apic_version()
    assert lib.apic_last_error() is not None


def test_flags_match_header():
    from paper_2108_02259_gb300 import apic

    hdr = open(os.path.join(ROOT, "include", "apiccontact.h")).read()
    for name in ("APIC_FP64", "APIC_HOST_PTRS", "APIC_VARIANT_PIC", "APIC_VARIANT_SEP23", "APIC_AUGURY_INIT",
                 "APIC_DETERMINISTIC", "APIC_CHECK", "APIC_MASS_NORMALS", "APIC_PARTITIONED"):
        m = re.search(rf"#define {name} \(1u << (\d+)\)", hdr)
        assert m, name
        assert getattr(apic, name) == 1 << int(m.group(1))
    for name in ("APIC_OK", "APIC_ERR_INVALID_ARG", "APIC_ERR_OUT_OF_MEMORY", "APIC_ERR_CUDA", "APIC_ERR_TIMEOUT"):
        m = re.search(rf"#define {name} \(?(-?\d+)\)?", hdr)
        assert m and getattr(apic, name) == int(m.group(1)), name


def test_flag_bits_are_distinct():
    hdr = open(os.path.join(ROOT, "include", "apiccontact.h")).read()
    bits = [int(b) for b in re.findall(r"#define APIC_[A-Z0-9_]+ \(1u << (\d+)\)", hdr)]
    assert len(bits) >= 7 and len(bits) == len(set(bits))


def test_struct_layout_matches_header(lib):
    """The ctypes mirror of apic_step_args / apic_stats has the C sizes."""
    from paper_2108_02259_gb300 import apic

    assert ctypes.sizeof(apic.StepArgs) == 8 + 4 + 4 + 8 * 8 + 8 + 8 + 8 + 8  # 112 with padding
    assert ctypes.sizeof(apic.Stats) == 12 * 8 + 3 * 8 + 2 * 8


def test_oracle_flags_match_library():
    import oracle
    from oracle.oracle import _load

    lib = _load()
    assert lib.oracle_flag_pic() == oracle.FLAG_PIC
    assert lib.oracle_flag_sep23() == oracle.FLAG_SEP23


def test_no_gpu_call_fails_cleanly_without_device(lib):
    """Without a GPU, apic_create reports an error instead of crashing."""
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    rc = lib.apic_create(ctypes.byref(h), 0, 0)
    assert rc != 0
    assert lib.apic_last_error()


def test_binding_pointer_of_numpy_arrays():
    """The binding's data pointers of host arrays (writable or not, views
    that start inside a buffer, empty) equal numpy's own."""
    import numpy as np

    from paper_2108_02259_gb300.apic import _ptr

    base = np.zeros((10, 3, 3), np.float32)
    ro = np.zeros(7)
    ro.setflags(write=False)
    for a in (base, base[3:], base.reshape(-1)[5:], np.arange(9, dtype=np.int32), ro, np.zeros((0, 3))):
        assert _ptr(a) == a.ctypes.data
    assert _ptr(None) is None
