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
                                                            "WQ_PREC_F32X2", "WQ_PREC_TF32X3"}
    assert wq._PREC == {"fp64": enum["WQ_PREC_FP64"], "fp32": enum["WQ_PREC_FP32"],
                        "mixed": enum["WQ_PREC_MIXED"], "f32x2": enum["WQ_PREC_F32X2"],
                        "tf32x3": enum["WQ_PREC_TF32X3"]}


def _create(lib, p, knots, ctrl, d=3):
    kn = [np.ascontiguousarray(k, dtype=np.float64) for k in knots]
    n_knots = (ctypes.c_int64 * 3)(*[len(k) for k in kn])
    kp = (ctypes.c_void_p * 3)(*[k.ctypes.data for k in kn])
    h = ctypes.c_void_p()
    ctrl = np.ascontiguousarray(ctrl, dtype=np.float64)
    st = lib.wq_plan_create(ctypes.byref(h), d, p, n_knots, kp, ctypes.c_void_p(ctrl.ctypes.data), None, None)
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


def test_interface_names_of_the_boundary():
    """The entry points the library's interface description names are declared."""
    names = declared_functions()
    for name in ("wq_options_init", "wq_plan_create", "wq_plan_info", "wq_plan_pattern", "wq_assemble_stiffness",
                 "wq_assemble_mass", "wq_adjoint", "wq_batch_create", "wq_batch_assemble", "wq_sync_check",
                 "wq_last_error", "wq_destroy", "wq_plan_reserve"):
        assert name in names, name


def test_options_init_fills_the_defaults(lib):
    from paper_1605_01238_gb300._lib import Options
    o = Options()
    assert lib.wq_options_init(ctypes.byref(o)) == 0
    assert o.size == ctypes.sizeof(Options)
    assert (o.value_dtype, o.precision, o.algorithm, o.tile[0], o.tile[1], o.checked) == (0, 0, 2, 0, 0, 0)
    assert not o.alloc and not o.free and not o.tune_cache
    assert lib.wq_options_init(None) == 1


def _create_opt(lib, opt):
    from wq_synth import perturbed_cube
    patch = perturbed_cube(2, 3, seed=1)
    kn = [np.ascontiguousarray(k, dtype=np.float64) for k in patch.knots]
    n_knots = (ctypes.c_int64 * 3)(*[len(k) for k in kn])
    kp = (ctypes.c_void_p * 3)(*[k.ctypes.data for k in kn])
    h = ctypes.c_void_p()
    ctrl = np.ascontiguousarray(patch.ctrl)
    return lib.wq_plan_create(ctypes.byref(h), 3, 2, n_knots, kp, ctypes.c_void_p(ctrl.ctypes.data),
                              ctypes.byref(opt), None)


@pytest.mark.parametrize("field,value,needle", [
    ("size", 8, b"size"), ("value_dtype", 5, b"value_dtype"), ("precision", 9, b"precision"),
    ("algorithm", 7, b"algorithm"), ("checked", 2, b"checked")])
def test_invalid_options_are_rejected_before_any_device_work(lib, field, value, needle):
    from paper_1605_01238_gb300._lib import Options
    o = Options()
    lib.wq_options_init(ctypes.byref(o))
    setattr(o, field, value)
    assert _create_opt(lib, o) == 1
    assert needle in lib.wq_last_error()


def test_options_reject_fp32_values_under_fp64_and_lone_allocators(lib):
    from paper_1605_01238_gb300._lib import ALLOC_FN, Options
    o = Options()
    lib.wq_options_init(ctypes.byref(o))
    o.value_dtype = 1
    assert _create_opt(lib, o) == 1
    o = Options()
    lib.wq_options_init(ctypes.byref(o))
    o.tile[0] = 8                                                     # the other extent left at 0
    assert _create_opt(lib, o) == 1
    o = Options()
    lib.wq_options_init(ctypes.byref(o))
    o.alloc = ALLOC_FN(lambda size, stream, ctx: None)                # alloc without free
    assert _create_opt(lib, o) == 1
    assert b"alloc" in lib.wq_last_error()


def test_tune_cache_round_trip(tmp_path):
    from paper_1605_01238_gb300 import tune
    path = str(tmp_path / "tiles.txt")
    tune.save_tiles({4: (12, 4), 2: (16, 2)}, path)
    text = open(path).read()
    assert "4 12 4" in text and "2 16 2" in text
    assert tune.load_tiles(path) == {2: (16, 2), 4: (12, 4)}
