"""NURBS geometry, NURBS-basis mass and a coefficient tensor on the GPU against the
oracle (the sentence after Eq. (mass2) and Eq. (coef_stiff) with a tensor K).

FP64 bar as the other parity tests: every value within 1e-12 of its row's largest
|entry|, pattern bit-exact; every row of small meshes."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import Oracle3D  # noqa: E402
from test_gpu_parity import TOL_F64, check_rows  # noqa: E402
from wq_synth import (perturbed_cube, perturbed_nurbs_cube, quarter_annulus, random_field,  # noqa: E402
                      random_spd_field)


@pytest.fixture(scope="module")
def wq():
    import paper_1605_01238_gb300 as wq
    from paper_1605_01238_gb300 import build
    build.build()
    return wq


def _all_rows(plan):
    return np.arange(plan.n_rows)


@pytest.mark.parametrize("p", [2, 3, 4, 5])
def test_rational_map_matches_the_oracle(wq, p):
    patch = perturbed_nurbs_cube(p, (p + 3, p + 2, 4), seed=200 + p)
    plan = wq.Plan(patch.p, patch.knots, patch.ctrl)
    plan.set_weights(patch.weights)
    kappa = random_field(int(np.prod(plan.n_qp)), seed=210 + p, kind="positive")
    S = plan.stiffness()
    M = plan.mass(kappa=torch.as_tensor(kappa, device="cuda"))
    torch.cuda.synchronize()
    plan.sync_check()
    orc = Oracle3D(patch.p, patch.knots, patch.ctrl, weights=patch.weights)
    check_rows(orc, plan, S, "stiffness", _all_rows(plan), tol=TOL_F64)
    orck = Oracle3D(patch.p, patch.knots, patch.ctrl, kappa=kappa, weights=patch.weights)
    check_rows(orck, plan, M, "mass", _all_rows(plan), tol=TOL_F64)
    c = plan.coefficients()
    assert np.abs(c - orc.coef).max() <= 1e-13 * np.abs(orc.coef).max()
    plan.close()


@pytest.mark.parametrize("p", [2, 3])
def test_quarter_annulus_stiffness_mass_and_nurbs_basis_mass(wq, p):
    patch = quarter_annulus(p, (3, 4, 2))
    plan = wq.Plan(patch.p, patch.knots, patch.ctrl)
    plan.set_weights(patch.weights)
    S, M = plan.stiffness(), plan.mass()
    plan.set_weights(patch.weights, nurbs_basis=True)
    Mn = plan.mass()
    Mn32 = plan.mass(precision="mixed", dtype=torch.float32)
    with pytest.raises(wq.WqError) as e:
        plan.stiffness()
    assert e.value.status == 2                                      # WQ_ERR_UNSUPPORTED
    torch.cuda.synchronize()
    rows = _all_rows(plan)
    orc = Oracle3D(patch.p, patch.knots, patch.ctrl, weights=patch.weights)
    check_rows(orc, plan, S, "stiffness", rows, tol=TOL_F64)
    check_rows(orc, plan, M, "mass", rows, tol=TOL_F64)
    orn = Oracle3D(patch.p, patch.knots, patch.ctrl, weights=patch.weights, nurbs_basis=True)
    check_rows(orn, plan, Mn, "mass", rows, tol=TOL_F64)
    check_rows(orn, plan, Mn32, "mass", rows, tol=1e-6)
    # partition of unity of the NURBS basis: the WQ total approaches the volume
    assert abs(float(Mn.sum()) - patch.meta["volume"]) < 1e-2 * patch.meta["volume"]
    plan.close()


@pytest.mark.parametrize("p", [2, 4])
@pytest.mark.parametrize("nurbs", [False, True])
def test_tensor_coefficient_matches_the_oracle(wq, p, nurbs):
    patch = (perturbed_nurbs_cube if nurbs else perturbed_cube)(p, (p + 3, 4, p + 2), seed=220 + p)
    plan = wq.Plan(patch.p, patch.knots, patch.ctrl)
    if nurbs:
        plan.set_weights(patch.weights)
    nq = int(np.prod(plan.n_qp))
    K = random_spd_field(nq, seed=230 + p)
    plan.set_tensor(torch.as_tensor(K, device="cuda"))
    S = plan.stiffness()
    S32 = plan.stiffness(precision="mixed", dtype=torch.float32)
    torch.cuda.synchronize()
    orc = Oracle3D(patch.p, patch.knots, patch.ctrl, weights=patch.weights if nurbs else None, K=K)
    rows = _all_rows(plan)
    check_rows(orc, plan, S, "stiffness", rows, tol=TOL_F64)
    check_rows(orc, plan, S32, "stiffness", rows, tol=1e-6)
    plan.close()


def test_identity_tensor_and_unit_weights_give_back_the_spline_path(wq):
    patch = perturbed_cube(3, (6, 5, 4), seed=240)
    plan = wq.Plan(patch.p, patch.knots, patch.ctrl)
    S0, M0 = plan.stiffness(), plan.mass()
    nq = int(np.prod(plan.n_qp))
    K = np.zeros((6, nq))
    K[0] = K[3] = K[5] = 1.0
    plan.set_tensor(torch.as_tensor(K, device="cuda"))
    S1 = plan.stiffness()
    plan.set_tensor(None)
    plan.set_weights(np.ones(plan.n_rows))
    S2, M2 = plan.stiffness(), plan.mass()
    plan.set_weights(None)
    S3 = plan.stiffness()
    torch.cuda.synchronize()
    scale = S0.abs().max()
    assert float((S1 - S0).abs().max() / scale) < 1e-15
    assert float((S2 - S0).abs().max() / scale) < 1e-13
    assert float((M2 - M0).abs().max() / M0.abs().max()) < 1e-13
    assert torch.equal(S3, S0)
    plan.close()


def test_adjoint_and_batch_refuse_what_they_do_not_handle(wq):
    patch = perturbed_nurbs_cube(2, (4, 4, 4), seed=250)
    plan = wq.Plan(patch.p, patch.knots, patch.ctrl)
    plan.set_weights(patch.weights)
    lam = torch.ones(plan.n_rows, dtype=torch.float64, device="cuda")
    with pytest.raises(wq.WqError) as e:
        plan.adjoint(lam, lam)
    assert e.value.status == 2
    plan.set_weights(patch.weights, nurbs_basis=True)
    M = torch.empty(plan.nnz, dtype=torch.float64, device="cuda")
    with pytest.raises(wq.WqError) as e:
        wq.Batch([plan], mass=[M])
    assert e.value.status == 2
    plan.close()
