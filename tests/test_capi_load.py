"""The C-ABI library loads on a host without a GPU and exports every symbol that
include/moqaia.h declares (no compute call is made here)."""
import ctypes
import os
import re

import pytest

from conftest import ROOT


def _declared():
    text = open(os.path.join(ROOT, "include", "moqaia.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(moq_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_pipeline():
    names = _declared()
    for n in ["moq_create_instance", "moq_sample", "moq_evaluate_cuts", "moq_pareto_front", "moq_hypervolume",
              "moq_archive_create", "moq_lambda_das_dennis", "moq_lambda_dirichlet", "moq_strerror"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2604_26477_b300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_wraps_every_symbol_and_strerror_works():
    from paper_2604_26477_b300 import build
    build.build()
    from paper_2604_26477_b300 import moqaia as M
    assert set(_declared()) <= set(M.EXPORTED)
    assert M.moq_strerror(M.MOQ_ERR_CAPACITY) == "capacity exceeded"
    p = M.moq_default_params(variant="bsb", steps=7, dt=0.5)
    assert (p.variant, p.steps, p.dt, p.a0, p.init_amp) == (M.MOQ_BSB, 7, 0.5, 1.0, pytest.approx(0.1))


def test_last_status_and_message_follow_a_rejected_call():
    # argument checks run before any device work, so this needs no GPU
    from paper_2604_26477_b300 import build
    lib = ctypes.CDLL(build.build())
    lib.moq_last_error_message.restype = ctypes.c_char_p
    out = ctypes.c_void_p()
    rc = lib.moq_create_instance(1, 3, 0, None, None, None, None, ctypes.byref(out))
    assert rc == -1 and lib.moq_last_status() == -1
    assert b"n" in lib.moq_last_error_message()
    lib.moq_default_params(None)  # a call that cannot fail leaves the status as it was
    assert lib.moq_last_status() == -1


def test_layout_argument_is_checked_before_device_work():
    # moq_create_instance_layout rejects a layout below MOQ_LAYOUT_PLAIN before any CUDA call
    from paper_2604_26477_b300 import build
    lib = ctypes.CDLL(build.build())
    lib.moq_last_error_message.restype = ctypes.c_char_p
    out = ctypes.c_void_p(1)
    ei = (ctypes.c_int32 * 1)(0)
    ej = (ctypes.c_int32 * 1)(1)
    w = (ctypes.c_int32 * 2)(1, 1)
    rc = lib.moq_create_instance_layout(2, 2, 1, ei, ej, w, -2, None, ctypes.byref(out))
    assert rc == -1 and out.value is None
    assert b"layout" in lib.moq_last_error_message()
