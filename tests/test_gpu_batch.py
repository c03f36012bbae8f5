"""Batched assembly (one graph launch for many patches: the staged kernels of every
patch on parallel branches, or the persistent fused kernel) against the per-plan
assembly and the oracle; the seeded 64-patch workload on sampled rows of every patch,
and the adjoint of three of its patches against finite differences."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import Oracle3D, rows_c  # noqa: E402
from wq_synth import perturbed_cube, sample_rows, workload_batch  # noqa: E402


@pytest.fixture(scope="module")
def wq():
    import paper_1605_01238_gb300 as wq
    from paper_1605_01238_gb300 import build
    build.build()
    wq.load()
    return wq


@pytest.mark.parametrize("form", ["staged", "fused"])
def test_batch_matches_single_plan_assembly_and_oracle(wq, form):
    patches = [perturbed_cube(2, (9, 12, 8), seed=31), perturbed_cube(3, (14, 8, 10), seed=32),
               perturbed_cube(4, (8, 11, 9), seed=33), perturbed_cube(5, (10, 9, 8), seed=34),
               perturbed_cube(2, (20, 6, 7), seed=35)]
    plans = [wq.Plan(pt.p, pt.knots, pt.ctrl) for pt in patches]
    plans[1].set_tiles(8, 2)                       # a per-plan tile choice is honoured
    if form == "fused":
        plans[0].set_algorithm("fused")            # one fused plan selects the persistent kernel
    S = [torch.full((pl.nnz,), float("nan"), dtype=torch.float64, device="cuda") for pl in plans]
    M = [torch.full((pl.nnz,), float("nan"), dtype=torch.float64, device="cuda") if k % 2 == 0 else None
         for k, pl in enumerate(plans)]
    batch = wq.Batch(plans, stiffness=S, mass=M)
    for _ in range(2):                              # replaying the graph gives the same values
        batch.launch()
    torch.cuda.synchronize()
    for k, (pl, pt) in enumerate(zip(plans, patches)):
        pl.set_algorithm(form)                      # the per-plan kernels the batch ran
        ref = pl.stiffness()
        torch.cuda.synchronize()
        assert torch.equal(S[k], ref), k
        if M[k] is not None:
            assert torch.equal(M[k], pl.mass())
        orc = Oracle3D(pt.p, pt.knots, pt.ctrl)
        rows = sample_rows(pl.n, pl.p, 30, seed=k)
        rp = pl.pattern()[0].cpu().numpy()
        got = S[k].cpu().numpy()
        for r, rv in zip(rows, rows_c(orc, rows, "stiffness", threads=8)):
            assert np.abs(got[rp[r]:rp[r + 1]] - rv).max() <= 1e-12 * np.abs(rv).max()
    batch.close()


def test_batch_workload_generator_spans_degrees_and_sizes():
    patches = workload_batch(64)
    assert len(patches) == 64
    assert {pt.p for pt in patches} == {2, 3, 4, 5}
    nel = np.array([pt.n_el for pt in patches])
    assert nel.min() >= 8 and nel.max() <= 48


@pytest.fixture(scope="module")
def batch64(wq):
    """The seeded 64-patch workload (n_el in [8, 48]^3, p in {2, 3, 4, 5}), stiffness
    and mass of every patch in one staged graph launch."""
    patches = workload_batch(64)
    plans = [wq.Plan(pt.p, pt.knots, pt.ctrl) for pt in patches]
    S = [torch.empty(pl.nnz, dtype=torch.float64, device="cuda") for pl in plans]
    M = [torch.empty(pl.nnz, dtype=torch.float64, device="cuda") for pl in plans]
    batch = wq.Batch(plans, stiffness=S, mass=M)
    batch.launch()
    torch.cuda.synchronize()
    yield patches, plans, S, M
    batch.close()
    for pl in plans:
        pl.close()
    torch.cuda.empty_cache()


def test_every_patch_of_the_64_patch_batch_matches_the_oracle(batch64):
    patches, plans, S, M = batch64
    worst = 0.0
    for k, (pt, pl) in enumerate(zip(patches, plans)):
        orc = Oracle3D(pt.p, pt.knots, pt.ctrl)
        rows = sample_rows(pl.n, pl.p, 6, seed=500 + k)[::5]       # a boundary row, an interior one, ...
        rp = pl.pattern()[0].cpu().numpy()
        idx = np.concatenate([np.arange(rp[r], rp[r + 1]) for r in rows])
        idx_d = torch.as_tensor(idx, device="cuda")
        for vals, which in ((S[k], "stiffness"), (M[k], "mass")):
            got = vals[idx_d].cpu().numpy()
            off = 0
            for rv in rows_c(orc, rows, which, threads=8):
                err = np.abs(got[off:off + len(rv)] - rv).max() / np.abs(rv).max()
                worst = max(worst, err)
                assert err <= 1e-12, (k, which, err)
                off += len(rv)
    print(f"64-patch batch: worst row-relative error {worst:.2e}")


@pytest.mark.parametrize("k", [3, 17, 42])
def test_adjoint_of_batch_patches_against_finite_differences(batch64, k):
    """dJ/dC of J = lam^T (S + M) u for three of the seeded patches, seeded N(0,1) lam, u."""
    from wq_synth import random_field
    patches, plans, _, _ = batch64
    pt, pl = patches[k], plans[k]
    dev = lambda a: torch.as_tensor(a, device="cuda")  # noqa: E731
    lam, u = random_field(pl.n_rows, seed=700 + k), random_field(pl.n_rows, seed=800 + k)
    J, _, gc = pl.adjoint(dev(lam), dev(u), None, "both", grad_kappa=False)
    gc = gc.cpu().numpy()
    eps = 1e-6
    ctrl = pt.ctrl.copy()
    N = pl.n_rows
    for (i, r) in [(N // 5, 0), (N // 2, 1), (N - 2, 2)]:
        vals = []
        for sgn in (1, -1):
            c2 = ctrl.copy()
            c2[i, r] += sgn * eps
            pl.set_geometry(dev(c2.reshape(-1)))
            vals.append(pl.adjoint(dev(lam), dev(u), None, "both", False, False)[0])
        fd = (vals[0] - vals[1]) / (2 * eps)
        assert abs(fd - gc[i, r]) <= 1e-6 * max(1.0, abs(fd)), (k, i, r, fd, gc[i, r])
    pl.set_geometry(dev(ctrl.reshape(-1)))
