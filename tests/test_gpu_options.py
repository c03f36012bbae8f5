"""Plan options (wq_options) on the GPU: the caller's allocator, host-side fault
injection without leaks, checked mode, wq_plan_reserve and the tune cache.

Every failure here is made on the host (WQ_FAULT, or a buffer the checked mode
rejects before anything is launched); no kernel is given an invalid input."""
import ctypes
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wq():
    import paper_1605_01238_gb300 as wq
    from paper_1605_01238_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    return wq


@pytest.fixture
def patch():
    from wq_synth import perturbed_cube
    return perturbed_cube(3, (7, 5, 6), seed=71)


def test_caller_allocator_gives_identical_values_and_frees_everything(wq, patch):
    ref = wq.Plan(patch.p, patch.knots, patch.ctrl)
    S0, M0 = ref.stiffness(), ref.mass()
    A0 = ref.stiffness(precision="mixed", dtype=torch.float32)
    ref.close()
    alloc = wq.TorchAllocator()
    plan = wq.Plan(patch.p, patch.knots, patch.ctrl, allocator=alloc)
    assert len(alloc.live) > 10
    S, M = plan.stiffness(), plan.mass()
    A = plan.stiffness(precision="mixed", dtype=torch.float32)
    torch.cuda.synchronize()
    assert torch.equal(S, S0) and torch.equal(M, M0) and torch.equal(A, A0)
    plan.close()
    assert alloc.live == {}


@pytest.mark.parametrize("step", ["alloc", "h2d", "solve", "geometry"])
def test_injected_failures_at_plan_creation_leak_nothing(wq, patch, step, monkeypatch):
    alloc = wq.TorchAllocator()
    monkeypatch.setenv("WQ_FAULT", step)
    with pytest.raises(wq.WqError) as e:
        wq.Plan(patch.p, patch.knots, patch.ctrl, allocator=alloc)
    assert e.value.status == 8                                         # WQ_ERR_INJECTED
    assert alloc.live == {}
    monkeypatch.delenv("WQ_FAULT")
    plan = wq.Plan(patch.p, patch.knots, patch.ctrl, allocator=alloc)   # the library is still usable
    plan.stiffness()
    torch.cuda.synchronize()
    plan.close()
    assert alloc.live == {}


def test_injected_failure_of_a_refresh_leaves_the_plan_usable(wq, patch, monkeypatch):
    plan = wq.Plan(patch.p, patch.knots, patch.ctrl)
    S0 = plan.stiffness()
    for step in ("geometry", "solve", "h2d"):
        monkeypatch.setenv("WQ_FAULT", step)
        with pytest.raises(wq.WqError) as e:
            plan.refresh(patch.ctrl)                                   # host control points: h2d applies
        assert e.value.status == 8
        monkeypatch.delenv("WQ_FAULT")
    plan.refresh(patch.ctrl)
    S = plan.stiffness()
    torch.cuda.synchronize()
    assert torch.equal(S, S0)
    plan.close()


def test_checked_mode_rejects_a_buffer_that_runs_past_its_allocation(wq):
    from wq_synth import perturbed_cube
    patch = perturbed_cube(3, (16, 14, 12), seed=72)
    plan = wq.Plan(patch.p, patch.knots, patch.ctrl, checked=True)
    lib = wq.load()
    _, col = plan.pattern()                    # a plan-owned allocation of nnz int32 (4.8 MB)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for offset in (0, 4 * plan.nnz - 64):      # nnz doubles from there run past its end
        st = lib.wq_assemble_stiffness(plan.handle, None, ctypes.c_void_p(col.data_ptr() + offset), 0, 0, stream)
        assert st == 1 and b"allocation" in lib.wq_last_error()
    host = np.zeros(plan.nnz)
    st = lib.wq_assemble_stiffness(plan.handle, None, ctypes.c_void_p(host.ctypes.data), 0, 0, stream)
    assert st == 1 and b"device" in lib.wq_last_error()
    S = plan.stiffness()                                              # a correct buffer passes
    ref = wq.Plan(patch.p, patch.knots, patch.ctrl)
    assert torch.equal(S, ref.stiffness())
    ref.close()
    plan.close()


def test_checked_mode_reports_non_finite_values(wq, patch):
    plan = wq.Plan(patch.p, patch.knots, patch.ctrl, checked=True)
    kappa = torch.ones(int(np.prod(plan.n_qp)), dtype=torch.float64, device="cuda")
    kappa[17] = float("nan")
    with pytest.raises(wq.WqError) as e:
        plan.stiffness(kappa=kappa)
    assert e.value.status == 9                                         # WQ_ERR_NONFINITE
    kappa[17] = 1.0
    plan.stiffness(kappa=kappa)
    plan.close()


def test_reserve_makes_the_first_assembly_allocate_nothing(wq, patch):
    alloc = wq.TorchAllocator()
    plan = wq.Plan(patch.p, patch.knots, patch.ctrl, allocator=alloc)
    n0 = len(alloc.live)
    plan.reserve("mixed", torch.float32, adjoint=True)
    n1 = len(alloc.live)
    assert n1 > n0
    plan.stiffness(precision="mixed", dtype=torch.float32)
    plan.mass(precision="mixed", dtype=torch.float32)
    lam = torch.randn(plan.n_rows, dtype=torch.float64, device="cuda")
    plan.adjoint(lam, lam)
    torch.cuda.synchronize()
    assert len(alloc.live) == n1
    plan.close()
    assert alloc.live == {}


def test_option_defaults_drive_the_assembly_calls(wq, patch):
    plan = wq.Plan(patch.p, patch.knots, patch.ctrl, precision="mixed", dtype=torch.float32)
    A = plan.stiffness()
    assert A.dtype == torch.float32
    ref = wq.Plan(patch.p, patch.knots, patch.ctrl)
    B = ref.stiffness(precision="mixed", dtype=torch.float32)
    torch.cuda.synchronize()
    assert torch.equal(A, B)
    plan.close()
    ref.close()


def test_tune_cache_sets_the_tiles_of_the_plans_degree(wq, patch, tmp_path):
    from paper_1605_01238_gb300 import tune
    path = str(tmp_path / "tiles.txt")
    tune.save_tiles({patch.p: (12, 2), patch.p + 1: (8, 4)}, path)
    plan = wq.Plan(patch.p, patch.knots, patch.ctrl, algorithm="fused", tune_cache=path)
    assert plan.tiles() == (12, 2)
    plan.close()
    plan = wq.Plan(patch.p, patch.knots, patch.ctrl, algorithm="fused", tune_cache=path, tiles=(16, 4))
    assert plan.tiles() == (16, 4)                                    # explicit tiles win
    plan.close()


def test_slabs_of_direction_3_give_identical_values(wq):
    """A scratch limit that forces one or two rows i3 per slab changes nothing in the
    values (every mode product computes the same sums, slab by slab), and the scratch
    the plan holds shrinks accordingly."""
    from wq_synth import perturbed_cube
    patch = perturbed_cube(4, (9, 7, 11), seed=73)
    ref = wq.Plan(patch.p, patch.knots, patch.ctrl)
    want = {m: ref.stiffness(precision=m, dtype=torch.float32 if m in ("mixed", "tf32x3", "fp32") else None)
            for m in ("fp64", "mixed", "tf32x3", "f32x2", "fp32")}
    want["mass"] = ref.mass()
    ref.close()
    for limit in (1, 3 << 20):
        alloc = wq.TorchAllocator()
        plan = wq.Plan(patch.p, patch.knots, patch.ctrl, scratch_limit=limit, allocator=alloc)
        for m, v in want.items():
            if m == "mass":
                got = plan.mass()
            else:
                got = plan.stiffness(precision=m, dtype=v.dtype)
            torch.cuda.synchronize()
            assert torch.equal(got, v), (limit, m)
        plan.close()


@pytest.mark.parametrize("p,nel", [(3, (8, 6, 19)), (8, (9, 11, 10))])
def test_end_to_end_call_into_host_memory(wq, p, nel):
    """wq_assemble_host returns the device path's values bit for bit: stored straight
    into page-locked memory by the last mode product (wq_host_alloc, with or without a
    staging array), and slab by slab through the staging array and a copy stream into
    pageable memory. n_el = 11 in direction 2 leaves a partial last warp of band pairs."""
    from wq_synth import perturbed_cube
    patch = perturbed_cube(p, nel, seed=74)
    plan = wq.Plan(patch.p, patch.knots, patch.ctrl)
    S = plan.stiffness().cpu().numpy()
    M = plan.mass().cpu().numpy()
    d = torch.empty(plan.nnz, dtype=torch.float64, device="cuda")
    hb = wq.HostBuffer(plan.nnz)
    for which, want in (("stiffness", S), ("mass", M)):
        for stage in (d, None):
            hb.array[:] = np.nan
            plan.assemble_host(which, patch.ctrl.reshape(-1), stage, hb.array)
            np.testing.assert_array_equal(hb.array, want)
        pageable = np.full(plan.nnz, np.nan)
        plan.assemble_host(which, None, d, pageable)
        np.testing.assert_array_equal(pageable, want)
    with pytest.raises(wq.WqError):
        plan.assemble_host("stiffness", None, None, np.zeros(plan.nnz))   # pageable needs staging
    hb.close()
    plan.close()
