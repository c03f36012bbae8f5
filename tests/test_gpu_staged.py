"""The staged assembly (three kernels, one per mode product, intermediates in device
memory) against the oracle, and against the fused kernel."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import Oracle3D  # noqa: E402
from test_gpu_parity import TOL_F64, TOL_F64_P8, check_rows  # noqa: E402
from wq_synth import (graded_breaks, perturbed_cube, random_field, sample_rows, workload_p4_64,  # noqa: E402
                      workload_sweep)


@pytest.fixture(scope="module")
def wq():
    import paper_1605_01238_gb300 as wq
    from paper_1605_01238_gb300 import build
    build.build()
    wq.load()
    return wq


SMALL = [
    ("p2_2x2x2", lambda: perturbed_cube(2, (2, 2, 2), seed=3)),
    ("p3_2x3x7", lambda: perturbed_cube(3, (2, 3, 7), seed=4)),
    ("p4_3x9x5", lambda: perturbed_cube(4, (3, 9, 5), seed=5)),
    ("p5_12x7x4", lambda: perturbed_cube(5, (12, 7, 4), seed=6)),
    ("p3_graded", lambda: perturbed_cube(3, (9, 11, 7), seed=7,
                                         breaks=[graded_breaks(e, seed=40 + k) for k, e in enumerate((9, 11, 7))])),
    ("p2_ragged_37x5x3", lambda: perturbed_cube(2, (37, 5, 3), seed=8)),
]


@pytest.mark.parametrize("name,factory", SMALL, ids=[s[0] for s in SMALL])
def test_staged_every_row(wq, name, factory):
    patch = factory()
    plan = wq.Plan(patch.p, patch.knots, patch.ctrl)
    plan.set_algorithm("staged")
    orc = Oracle3D(patch.p, patch.knots, patch.ctrl)
    kappa = random_field(int(np.prod(plan.n_qp)), seed=9, kind="positive")
    kd = torch.as_tensor(kappa, device="cuda")
    S, M = plan.stiffness(), plan.mass(kappa=kd)
    torch.cuda.synchronize()
    rows = np.arange(plan.n_rows)
    check_rows(orc, plan, S, "stiffness", rows)
    check_rows(Oracle3D(patch.p, patch.knots, patch.ctrl, kappa=kappa), plan, M, "mass", rows)
    plan.set_algorithm("fused")
    S2 = plan.stiffness()
    torch.cuda.synchronize()
    assert float((S - S2).abs().max()) <= 1e-13 * float(S2.abs().max())


@pytest.mark.parametrize("p,count", [(4, 120), (5, 48), (8, 12)])
def test_staged_full_size_sampled_rows(wq, p, count):
    patch = workload_p4_64() if p == 4 else workload_sweep(p)
    plan = wq.Plan(patch.p, patch.knots, patch.ctrl)
    plan.set_algorithm("staged")
    S = plan.stiffness()
    torch.cuda.synchronize()
    orc = Oracle3D(patch.p, patch.knots, patch.ctrl)
    rows = sample_rows(plan.n, plan.p, count, seed=7000 + p)
    check_rows(orc, plan, S, "stiffness", rows, tol=TOL_F64_P8 if p == 8 else TOL_F64)
    del S
    plan.close()
    torch.cuda.empty_cache()


def test_staged_fp32(wq):
    patch = perturbed_cube(4, (12, 10, 9), seed=12)
    plan = wq.Plan(patch.p, patch.knots, patch.ctrl)
    plan.set_algorithm("staged")
    S = plan.stiffness(precision="fp32", dtype=torch.float32)
    torch.cuda.synchronize()
    orc = Oracle3D(patch.p, patch.knots, patch.ctrl)
    rows = sample_rows(plan.n, plan.p, 120, seed=5)
    worst = check_rows(orc, plan, S, "stiffness", rows, tol=2e-6)
    print(f"staged fp32: worst row-relative error {worst:.3e}")


@pytest.mark.parametrize("p", [2, 3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("which", ["stiffness", "mass"])
@pytest.mark.parametrize("precision", ["mixed", "tf32x3"])
def test_staged_mixed_precision(wq, p, which, precision):
    """Mixed precision: double-float for the q3 mode product; for the q2 one double-float on
    the first and last p+1 rows of direction 2 and on the points q1 that the first and last
    p+1 rows of direction 1 read, FP32 elsewhere; FP32 for the q1 one (FFMA, or 3xTF32 on
    the tensor cores) with its first and last p+1 rows of direction 1 in FP64: 1e-6
    row-relative."""
    patch = perturbed_cube(p, (2 * p + 5, p + 4, p + 3), seed=40 + p)
    plan = wq.Plan(patch.p, patch.knots, patch.ctrl)
    kappa = random_field(int(np.prod(plan.n_qp)), seed=90 + p, kind="positive")
    fn = plan.stiffness if which == "stiffness" else plan.mass
    S = fn(kappa=torch.as_tensor(kappa, device="cuda"), precision=precision, dtype=torch.float32)
    torch.cuda.synchronize()
    orc = Oracle3D(patch.p, patch.knots, patch.ctrl, kappa=kappa)
    rows = sample_rows(plan.n, plan.p, 80, seed=600 + p)
    worst = check_rows(orc, plan, S, which, rows, tol=1e-6)
    print(f"{precision} p={p} {which}: worst row-relative error {worst:.3e}")
    plan.close()


@pytest.mark.parametrize("p", [3, 5, 8])
@pytest.mark.parametrize("which", ["stiffness", "mass"])
def test_tensor_core_stage1_tiles_chunks_and_tails(wq, p, which):
    """The 3xTF32 tensor-core stage 1 over several 32-row chunks of direction 1 and
    several 128-pair tiles of direction 2 with a ragged last tile: every regular row of
    direction 1 it writes matches the oracle at 1e-6, and the FFMA mixed path to FP32
    rounding; FP64 values too."""
    patch = perturbed_cube(p, (p + 70, 2 * p + 9, 3), seed=130 + p)
    plan = wq.Plan(patch.p, patch.knots, patch.ctrl)
    n1, n2, n3 = plan.n
    fn = plan.stiffness if which == "stiffness" else plan.mass
    T = fn(precision="tf32x3", dtype=torch.float32)
    T64 = fn(precision="tf32x3", dtype=torch.float64)
    F = fn(precision="mixed", dtype=torch.float32)
    torch.cuda.synchronize()
    rp = plan.pattern()[0].cpu().numpy()
    i1s = [p + 1, p + 2, 33, 40 + p, n1 - p - 2]
    rows = np.array([i1 + n1 * (i2 + n2 * i3) for i3 in (0, n3 - 1) for i2 in (0, n2 // 2, n2 - 1) for i1 in i1s])
    orc = Oracle3D(patch.p, patch.knots, patch.ctrl)
    check_rows(orc, plan, T, which, rows, tol=1e-6)
    t, t64, f = T.double().cpu().numpy(), T64.cpu().numpy(), F.double().cpu().numpy()
    for r in rows:
        a, b = t[rp[r]:rp[r + 1]], f[rp[r]:rp[r + 1]]
        np.testing.assert_array_equal(a, t64[rp[r]:rp[r + 1]])   # FP32 accumulators, either value type
        assert np.abs(a - b).max() <= 2e-6 * np.abs(b).max(), r
    plan.close()


def _edge_rows(n, p):
    """Every row whose direction-2 index is within p+1 of an end, crossed with a
    few direction-1 and direction-3 indices (ends, p, n-p-1, middle)."""
    def picks(m):
        return sorted({0, min(p, m - 1), m // 2, max(0, m - p - 1), m - 1})
    e2 = [i for i in range(n[1]) if i <= p or i >= n[1] - p - 1]
    return np.array([(i3 * n[1] + i2) * n[0] + i1 for i3 in picks(n[2]) for i2 in e2 for i1 in picks(n[0])])


@pytest.mark.parametrize("p", [2, 3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("extra", [0, 1])
def test_staged_edge_rows_compile_time_patterns(wq, p, extra):
    """Direction 2 with n_el = 2p+2 (+1): the first and last p+1 rows take the
    kernels with compile-time point patterns; FP64 stiffness, FP64 mass with a
    coefficient field, and mixed-precision stiffness against the oracle."""
    patch = perturbed_cube(p, (3, 2 * p + 2 + extra, 2), seed=70 + p + extra)
    plan = wq.Plan(patch.p, patch.knots, patch.ctrl)
    kappa = random_field(int(np.prod(plan.n_qp)), seed=80 + p, kind="positive")
    rows = _edge_rows(plan.n, p)
    S = plan.stiffness()
    M = plan.mass(kappa=torch.as_tensor(kappa, device="cuda"))
    X = plan.stiffness(precision="mixed", dtype=torch.float32)
    torch.cuda.synchronize()
    tol = TOL_F64_P8 if p == 8 else TOL_F64
    check_rows(Oracle3D(patch.p, patch.knots, patch.ctrl), plan, S, "stiffness", rows, tol=tol)
    check_rows(Oracle3D(patch.p, patch.knots, patch.ctrl, kappa=kappa), plan, M, "mass", rows, tol=tol)
    check_rows(Oracle3D(patch.p, patch.knots, patch.ctrl), plan, X, "stiffness", rows, tol=1e-6)
    plan.close()


@pytest.mark.parametrize("p", [2, 3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("which", ["stiffness", "mass"])
def test_staged_double_float(wq, p, which):
    """WQ_PREC_F32X2 (double-float on the FP32 pipe) holds the FP64 parity bar."""
    patch = perturbed_cube(p, (2 * p + 5, 2 * p + 4, p + 3), seed=50 + p)
    plan = wq.Plan(patch.p, patch.knots, patch.ctrl)
    kappa = random_field(int(np.prod(plan.n_qp)), seed=60 + p, kind="positive")
    fn = plan.stiffness if which == "stiffness" else plan.mass
    S = fn(kappa=torch.as_tensor(kappa, device="cuda"), precision="f32x2")
    torch.cuda.synchronize()
    orc = Oracle3D(patch.p, patch.knots, patch.ctrl, kappa=kappa)
    rows = sample_rows(plan.n, plan.p, 80, seed=900 + p)
    worst = check_rows(orc, plan, S, which, rows, tol=TOL_F64_P8 if p == 8 else TOL_F64)
    print(f"f32x2 p={p} {which}: worst row-relative error {worst:.3e}")
    plan.close()
