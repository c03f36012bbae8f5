"""The adjoint kernels (wq_adjoint) against the oracle's adjoint, the assembled
matrices and finite differences; the autograd Function against the direct call."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import wq_oracle as wo  # noqa: E402
from wq_synth import perturbed_cube, random_field  # noqa: E402


@pytest.fixture(scope="module")
def wq():
    import paper_1605_01238_gb300 as wq
    from paper_1605_01238_gb300 import build
    build.build()
    wq.load()
    return wq


def _setup(wq, p, nel, seed):
    patch = perturbed_cube(p, nel, seed=seed)
    plan = wq.Plan(p, patch.knots, patch.ctrl)
    N, nqp = plan.n_rows, int(np.prod(plan.n_qp))
    lam = random_field(N, seed=seed + 1)
    u = random_field(N, seed=seed + 2)
    kappa = random_field(nqp, seed=seed + 3, kind="positive")
    dev = lambda a: torch.as_tensor(a, device="cuda")
    return patch, plan, lam, u, kappa, dev


@pytest.mark.parametrize("which", ["stiffness", "mass", "both"])
def test_adjoint_matches_oracle_and_matrix(wq, which):
    patch, plan, lam, u, kappa, dev = _setup(wq, 3, (6, 5, 4), 61)
    J, gk, gc = plan.adjoint(dev(lam), dev(u), dev(kappa), which)
    orc = wo.Oracle3D(3, patch.knots, patch.ctrl)
    Jo, gko, gco = wo.adjoint(orc, lam, u, which, kappa=kappa)
    assert abs(J - Jo) <= 1e-12 * abs(Jo)
    assert np.abs(gk.cpu().numpy() - gko.ravel()).max() <= 1e-11 * np.abs(gko).max()
    assert np.abs(gc.cpu().numpy() - gco).max() <= 1e-11 * np.abs(gco).max()
    # J = lam^T A u with the GPU-assembled CSR matrices
    A = 0
    if which in ("stiffness", "both"):
        A = A + plan.csr(plan.stiffness(kappa=dev(kappa))).to_dense()
    if which in ("mass", "both"):
        A = A + plan.csr(plan.mass(kappa=dev(kappa))).to_dense()
    Jm = float(dev(lam) @ (A @ dev(u)))
    assert abs(J - Jm) <= 1e-12 * abs(Jm)


def test_adjoint_control_gradient_finite_differences(wq):
    patch, plan, lam, u, kappa, dev = _setup(wq, 4, (7, 6, 8), 71)
    J, _, gc = plan.adjoint(dev(lam), dev(u), dev(kappa), "both", grad_kappa=False)
    gc = gc.cpu().numpy()
    eps = 1e-6
    ctrl = patch.ctrl.copy()
    N = plan.n_rows
    for (i, r) in [(0, 0), (N // 3, 1), (N // 2, 2), (N - 1, 0), (123, 1)]:
        vals = []
        for sgn in (1, -1):
            c2 = ctrl.copy()
            c2[i, r] += sgn * eps
            plan.set_geometry(dev(c2.reshape(-1)))
            vals.append(plan.adjoint(dev(lam), dev(u), dev(kappa), "both", False, False)[0])
        fd = (vals[0] - vals[1]) / (2 * eps)
        assert abs(fd - gc[i, r]) <= 1e-6 * max(1.0, abs(fd)), (i, r, fd, gc[i, r])
    plan.set_geometry(dev(ctrl.reshape(-1)))


def test_autograd_function_matches_direct_adjoint(wq):
    patch, plan, lam, u, kappa, dev = _setup(wq, 2, (5, 6, 4), 81)
    ctrl = dev(patch.ctrl).clone().requires_grad_(True)
    kap = dev(kappa).clone().requires_grad_(True)
    J = wq.bilinear(plan, ctrl, dev(lam), dev(u), kappa=kap, which="stiffness")
    (2.0 * J).backward()
    J2, gk, gc = plan.adjoint(dev(lam), dev(u), dev(kappa), "stiffness")
    assert abs(float(J) - J2) <= 1e-14 * abs(J2)
    assert torch.allclose(ctrl.grad, 2.0 * gc, rtol=0, atol=1e-14 * float(gc.abs().max()))
    assert torch.allclose(kap.grad, 2.0 * gk, rtol=0, atol=1e-14 * float(gk.abs().max()))
