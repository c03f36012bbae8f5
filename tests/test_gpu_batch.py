"""Batched assembly (one persistent, graph-captured launch for many patches)
against the per-plan assembly and the oracle."""
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


def test_batch_matches_single_plan_assembly_and_oracle(wq):
    patches = [perturbed_cube(2, (9, 12, 8), seed=31), perturbed_cube(3, (14, 8, 10), seed=32),
               perturbed_cube(4, (8, 11, 9), seed=33), perturbed_cube(5, (10, 9, 8), seed=34),
               perturbed_cube(2, (20, 6, 7), seed=35)]
    plans = [wq.Plan(pt.p, pt.knots, pt.ctrl) for pt in patches]
    plans[1].set_tiles(8, 2)                       # a per-plan tile choice is honoured
    S = [torch.full((pl.nnz,), float("nan"), dtype=torch.float64, device="cuda") for pl in plans]
    M = [torch.full((pl.nnz,), float("nan"), dtype=torch.float64, device="cuda") if k % 2 == 0 else None
         for k, pl in enumerate(plans)]
    batch = wq.Batch(plans, stiffness=S, mass=M)
    for _ in range(2):                              # replaying the graph gives the same values
        batch.launch()
    torch.cuda.synchronize()
    for k, (pl, pt) in enumerate(zip(plans, patches)):
        pl.set_algorithm("fused")                   # the batch runs the fused tile kernel
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
