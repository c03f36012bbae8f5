"""Pins of the oracle's adjoint: the point-wise form of J equals lambda^T A u with
the assembled oracle matrices, dJ/dkappa is exact for the linear dependence on
kappa, and dJ/dC matches central finite differences of the assembled J."""
import numpy as np
import pytest

from oracle import wq_oracle as wo
from wq_synth import perturbed_cube, random_field


def _J_dense(p, knots, ctrl, kappa, lam, u, which):
    orc = wo.Oracle3D(p, knots, ctrl, kappa=kappa)
    A = 0
    if which in ("stiffness", "both"):
        A = A + orc.dense("stiffness")
    if which in ("mass", "both"):
        A = A + orc.dense("mass")
    return float(lam @ A @ u)


@pytest.mark.parametrize("which", ["stiffness", "mass", "both"])
def test_oracle_adjoint_pointwise_form_and_gradients(which):
    patch = perturbed_cube(2, (3, 2, 3), seed=51, amp=0.05)
    orc = wo.Oracle3D(2, patch.knots, patch.ctrl)
    N = int(np.prod(orc.n))
    lam = random_field(N, seed=1)
    u = random_field(N, seed=2)
    kappa = random_field(int(np.prod(orc.nqp)), seed=3, kind="positive")
    J, gk, gc = wo.adjoint(orc, lam, u, which, kappa=kappa)
    J_dense = _J_dense(2, patch.knots, patch.ctrl, kappa, lam, u, which)
    assert abs(J - J_dense) <= 1e-12 * abs(J_dense)
    # J is linear in kappa: J(kappa + e_q) - J(kappa) = gk[q]
    rng = np.random.default_rng(0)
    for q in rng.integers(0, kappa.size, 3):
        k2 = kappa.copy()
        k2[q] += 0.25
        dJ = _J_dense(2, patch.knots, patch.ctrl, k2, lam, u, which) - J_dense
        assert abs(dJ - 0.25 * gk.ravel()[q]) <= 1e-10 * max(abs(dJ), 1e-12) + 1e-14
    # control points: central differences
    eps = 1e-6
    for (i, r) in [(0, 0), (5, 1), (N - 1, 2), (N // 2, 0)]:
        cp, cm = patch.ctrl.copy(), patch.ctrl.copy()
        cp[i, r] += eps
        cm[i, r] -= eps
        fd = (_J_dense(2, patch.knots, cp, kappa, lam, u, which) - _J_dense(2, patch.knots, cm, kappa, lam, u, which)) / (2 * eps)
        assert abs(fd - gc[i, r]) <= 1e-6 * max(1.0, abs(fd)), (i, r, fd, gc[i, r])
