"""The algorithmic operation count that bench.py divides by the assembly time (the
roofline's "achieved" figure), and the key that ties a stored ncu traffic capture to
the kernel code.

- The census's per-direction sets (points, Q_i, band I_i, overlaps |Q_i n Q_j|) agree
  with the oracle's, which come from the point grid of the Remark on the choice of
  points and the open supports of Eq. (support).
- Per nonzero, the census tends to the interior closed form of the sum factorisation
  as the mesh grows: for interior rows, |Q_i| = 2p+1 and sum_j |Q_i n Q_j| = 2p^2+2p+1.
- The source key ignores comments and blank space and changes with any code edit.
"""
import numpy as np
import pytest

import bench
from oracle.wq_oracle import Direction
from wq_synth import graded_breaks, open_knot_vector, uniform_breaks


@pytest.mark.parametrize("p,ne", [(2, 5), (3, 9), (4, 11), (5, 13)])
def test_census_sets_match_the_oracle(p, ne):
    for breaks in (uniform_breaks(ne), graded_breaks(ne, seed=3)):
        d = Direction(open_knot_vector(breaks, p), p)
        nqp, nq, ov, bw = bench._dir_census(ne + p, p)
        assert nqp == len(d.x)
        assert nq == [len(q) for q in d.Q]
        assert bw == [len(i) for i in d.I]
        assert ov == [sum(len(np.intersect1d(d.Q[i], d.Q[j])) for j in d.I[i]) for i in range(d.n)]


def interior_flops_per_nnz(p: int, mass: bool) -> float:
    b, o = 2 * p + 1, 2 * p * p + 2 * p + 1
    if mass:
        return 2 * ((b + o) / b + 2 * (b + o) / b ** 2 + 4 * o / b ** 3)
    return 2 * ((4 * b + 2 * o) / b + 2 * (9 * b + 6 * o) / b ** 2 + 36 * o / b ** 3)


@pytest.mark.parametrize("p", [2, 3, 4, 5, 6, 8])
@pytest.mark.parametrize("mass", [False, True])
def test_census_tends_to_the_interior_closed_form(p, mass):
    target = interior_flops_per_nnz(p, mass)
    errs = []
    for n in (200, 1600):
        nnz = float(sum(bench._dir_census(n, p)[3])) ** 3
        errs.append(abs(bench.algorithmic_flops((n, n, n), p, mass) / nnz - target) / target)
    assert errs[1] < errs[0] and errs[1] < 0.01


def test_census_of_the_bench_workload():
    """p = 4, 64^3: 48.9 flop per nonzero (the figure the bench line quotes)."""
    n = (68, 68, 68)
    nnz = float(sum(bench._dir_census(68, 4)[3])) ** 3
    assert nnz == 207474688
    assert abs(bench.algorithmic_flops(n, 4) / nnz - 48.906) < 1e-3


def test_source_key_ignores_comments_and_sees_code(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("// kernel\n__global__ void k(float* a) { a[0] = 1.0f; }\n")
    monkeypatch.setitem(bench.TRAFFIC_CAPTURE, "files", (str(src),))
    key = bench.kernel_source_hash()
    src.write_text("/* a longer\n   comment */\n__global__ void k(float* a) {\n  a[0] = 1.0f;  // store\n}\n")
    assert bench.kernel_source_hash() == key
    src.write_text("__global__ void k(float* a) { a[0] = 2.0f; }\n")
    assert bench.kernel_source_hash() != key



def test_traffic_capture_scales_by_nonzeros_and_follows_the_sources(monkeypatch):
    """The captured bytes of the small case are scaled to the bench workload by the nonzeros
    assembled, for the captured degree only, and dropped once the kernel code changes."""
    monkeypatch.setitem(bench.TRAFFIC_CAPTURE, "bytes", 1.0e9)
    monkeypatch.setitem(bench.TRAFFIC_CAPTURE, "nnz", 1.0e8)
    monkeypatch.setitem(bench.TRAFFIC_CAPTURE, "sources", bench.kernel_source_hash())
    assert bench.captured_traffic(bench.TRAFFIC_CAPTURE["p"], 4e8) == 4.0e9
    assert bench.captured_traffic(bench.TRAFFIC_CAPTURE["p"] - 1, 4e8) is None
    monkeypatch.setitem(bench.TRAFFIC_CAPTURE, "sources", "0" * 16)
    assert bench.captured_traffic(bench.TRAFFIC_CAPTURE["p"], 4e8) is None


def test_bench_arguments():
    """The default run measures the FP64 step and keeps the precision study; --precision
    selects the step's mode for --steps-only captures only."""
    a = bench.parse_args([])
    assert a.step_precision == "fp64" and a.precision is True and a.workload == "sweep8" and a.warmup >= 3
    b = bench.parse_args(["--steps-only", "--precision", "mixed", "--workload", "p5_128"])
    assert b.step_precision == "mixed" and bench.PRECISION_MODES[b.step_precision][:2] == ("mixed", "f32")
    assert bench.parse_args(["--no-precision"]).precision is False
    with pytest.raises(SystemExit):
        bench.parse_args(["--precision", "fp32"])
