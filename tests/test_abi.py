"""The C ABI library: it loads, exports every entry point that include/wq.h
declares, and rejects bad arguments on the host (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "wq.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(wq_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1605_01238_gb300 import build, _lib
    build.build()
    return _lib.load()


def test_header_declares_the_core_entry_points():
    names = declared_functions()
    for core in ("wq_plan_create", "wq_assemble_stiffness", "wq_assemble_mass", "wq_plan_destroy"):
        assert core in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_1605_01238_gb300 import _lib
    assert set(declared_functions()) <= set(_lib.SIGNATURES)


def test_binding_enums_match_the_header():
    """Precision, value-type and algorithm constants of the binding equal the header's."""
    import paper_1605_01238_gb300 as wq
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    enum = {k: int(v) for k, v in re.findall(r"\b(WQ_(?:PREC|VALUES|ALGO)_[A-Z0-9]+)\s*=\s*(\d+)", text)}
    assert {k for k in enum if k.startswith("WQ_PREC_")} == {"WQ_PREC_FP64", "WQ_PREC_FP32", "WQ_PREC_MIXED",
                                                            "WQ_PREC_F32X2"}
    assert wq._PREC == {"fp64": enum["WQ_PREC_FP64"], "fp32": enum["WQ_PREC_FP32"],
                        "mixed": enum["WQ_PREC_MIXED"], "f32x2": enum["WQ_PREC_F32X2"]}


def _create(lib, p, knots, ctrl, d=3):
    kn = [np.ascontiguousarray(k, dtype=np.float64) for k in knots]
    n_knots = (ctypes.c_int64 * 3)(*[len(k) for k in kn])
    kp = (ctypes.c_void_p * 3)(*[k.ctypes.data for k in kn])
    h = ctypes.c_void_p()
    ctrl = np.ascontiguousarray(ctrl, dtype=np.float64)
    st = lib.wq_plan_create(ctypes.byref(h), d, p, n_knots, kp, ctypes.c_void_p(ctrl.ctypes.data), None)
    return st, h


def test_host_validation(lib):
    from wq_synth import perturbed_cube
    patch = perturbed_cube(2, 3, seed=1)
    assert _create(lib, 2, patch.knots, patch.ctrl, d=2)[0] == 2          # unsupported d
    assert _create(lib, 1, patch.knots, patch.ctrl)[0] == 1               # p out of range
    assert _create(lib, 9, patch.knots, patch.ctrl)[0] == 1
    bad = [k.copy() for k in patch.knots]
    bad[1][4] = bad[1][3]                                                  # repeated interior knot
    assert _create(lib, 2, bad, patch.ctrl)[0] == 1
    bad = [k.copy() for k in patch.knots]
    bad[0][1] = 0.01                                                       # not open
    assert _create(lib, 2, bad, patch.ctrl)[0] == 1
    nan_ctrl = patch.ctrl.copy()
    nan_ctrl[3, 1] = np.nan
    assert _create(lib, 2, patch.knots, nan_ctrl)[0] == 1
    assert b"finite" in lib.wq_last_error()


def test_status_strings_and_null_safety(lib):
    assert lib.wq_status_string(0) == b"WQ_OK"
    assert lib.wq_status_string(4) == b"WQ_ERR_BAD_GEOMETRY"
    assert lib.wq_plan_destroy(None) == 0
    assert lib.wq_assemble_stiffness(None, None, None, 0, 0, None) == 1
    assert lib.wq_plan_info(None, None, None, None, None, None) == 1


def test_no_device_is_an_error_not_a_fallback(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from wq_synth import perturbed_cube
    patch = perturbed_cube(2, 3, seed=1)
    st, h = _create(lib, 2, patch.knots, patch.ctrl)
    assert st == 6 and not h.value                                        # WQ_ERR_CUDA


def test_python_plan_fails_loudly_without_device():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_1605_01238_gb300 as wq
    from wq_synth import perturbed_cube
    patch = perturbed_cube(2, 3, seed=1)
    with pytest.raises((wq.WqError, RuntimeError)):
        wq.Plan(2, patch.knots, patch.ctrl)
