"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, and
exports every entry point include/qarray.h declares (no compute calls)."""
import ctypes
import os
import re

from paper_2404_04994_gb300 import build as qbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    text = open(os.path.join(ROOT, "include", "qarray.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qa_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_entry_points()
    for must in ("qa_model_create", "qa_model_destroy", "qa_ground_state_open",
                 "qa_ground_state_closed", "qa_soft_occupation",
                 "qa_soft_occupation_backward", "qa_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(qbuild.build())
    for name in declared_entry_points():
        assert hasattr(lib, name), name


def test_binding_covers_every_symbol():
    from paper_2404_04994_gb300 import api
    for name in declared_entry_points():
        assert hasattr(api, name), name
    assert set(declared_entry_points()) <= set(api.exported_symbols())


def test_last_error_without_gpu():
    from paper_2404_04994_gb300 import api
    # host-side validation runs before any device call
    import numpy as np
    try:
        api.qa_model_create(np.array([[1.0, 2.0], [2.0, 1.0]]), np.eye(2))
    except api.QAError as e:
        assert e.code in (-4, -7)


def test_static_limit_matches_the_header():
    # the binding's copy of QA_STATIC_MAX_PIXELS follows include/qarray.h
    from paper_2404_04994_gb300 import api
    text = open(os.path.join(ROOT, "include", "qarray.h")).read()
    m = re.search(r"#define\s+QA_STATIC_MAX_PIXELS\s+(\d+)", text)
    assert m is not None
    assert int(m.group(1)) == api.STATIC_MAX_PIXELS
