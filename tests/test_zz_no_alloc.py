"""wq_rules_noalloc, the allocation-free rule builder, against the plan's rule step.

Some callers cannot allocate device memory themselves: code that runs under a
framework owning all of GPU memory through its own pool, latency-critical loops
that cannot afford cudaMalloc's implicit device synchronisation, and embedded
users with a fixed, pre-reserved memory budget. wq_rules_noalloc serves them by
keeping its intermediate tables in one fixed device array that the library
declares. The caller still provides the knot vector and the output buffers.

This test calls it through the C ABI twice in a row, on two different knot
vectors of different degree. Each result must match the rules that wq_plan_create
computed for the same knots, to the 1e-14 bar of the rule parity test. The
second call also shows that the shared scratch left by the first call does not
leak into the next result.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _noalloc_rules(lib, p, knots, n, stride):
    kv = np.ascontiguousarray(knots, dtype=np.float64)
    w = torch.full((4 * n * stride,), float("nan"), dtype=torch.float64, device="cuda")
    q0 = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    nq = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = lib.wq_rules_noalloc(p, len(kv), ctypes.c_void_p(kv.ctypes.data), ctypes.c_void_p(w.data_ptr()),
                              ctypes.c_void_p(q0.data_ptr()), ctypes.c_void_p(nq.data_ptr()), stride, stream)
    assert st == 0, lib.wq_last_error().decode()
    return w.cpu().numpy().reshape(4, n, stride), q0.cpu().numpy(), nq.cpu().numpy()


def test_noalloc_rules_match_plan_rules_on_two_calls_in_a_row():
    import paper_1605_01238_gb300 as wq
    from paper_1605_01238_gb300 import _lib, build
    from wq_synth import graded_breaks, perturbed_cube
    build.build()
    lib = _lib.load()
    cases = [
        perturbed_cube(4, (37, 9, 5), seed=21),
        perturbed_cube(6, (12, 7, 3), seed=22,
                       breaks=[graded_breaks(12, seed=5), graded_breaks(7, seed=6), graded_breaks(3, seed=7)]),
    ]
    for patch in cases:
        plan = wq.Plan(patch.p, patch.knots, patch.ctrl)
        n, stride = plan.n[0], plan.nq_max
        w, q0, nq = _noalloc_rules(lib, patch.p, patch.knots[0], n, stride)
        for a in (0, 1):
            for b in (0, 1):
                ref_w, ref_q0, ref_nq = plan.rules(0, a, b)
                np.testing.assert_array_equal(q0, ref_q0)
                np.testing.assert_array_equal(nq, ref_nq)
                got = w[2 * a + b]
                assert np.all(np.isfinite(got))
                for i in range(n):
                    scale = np.abs(ref_w[i, :nq[i]]).max()
                    assert np.abs(got[i] - ref_w[i]).max() <= 1e-14 * scale, (patch.p, a, b, i)
        plan.close()


def test_noalloc_rejects_knot_vectors_beyond_its_scratch():
    from paper_1605_01238_gb300 import _lib
    from wq_synth import open_knot_vector, uniform_breaks
    lib = _lib.load()
    p = 3
    kv = np.ascontiguousarray(open_knot_vector(uniform_breaks(1030), p))   # 1033 functions > 1024
    n = len(kv) - p - 1
    dummy = ctypes.c_void_p(1)
    st = lib.wq_rules_noalloc(p, len(kv), ctypes.c_void_p(kv.ctypes.data), dummy, dummy, dummy, 4 * p + 1, None)
    assert st == 1 and n > 1024
    assert b"1024" in lib.wq_last_error()


def test_noalloc_rejects_a_row_stride_above_4p_plus_1():
    """The row stride of the output may not exceed 4p+1 (the largest |Q_i| of degree p)."""
    from paper_1605_01238_gb300 import _lib
    from wq_synth import open_knot_vector, uniform_breaks
    lib = _lib.load()
    p = 2
    kv = np.ascontiguousarray(open_knot_vector(uniform_breaks(10), p))
    dummy = ctypes.c_void_p(1)
    st = lib.wq_rules_noalloc(p, len(kv), ctypes.c_void_p(kv.ctypes.data), dummy, dummy, dummy, 4 * p + 2, None)
    assert st == 1
    assert b"4p+1" in lib.wq_last_error()
