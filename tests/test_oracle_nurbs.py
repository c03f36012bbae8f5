"""Pins of the oracle's NURBS geometry, coefficient tensor and NURBS-basis mass
(after Eq. (mass2) the paper lets c take in the PDE coefficient and, for NURBS
functions, the denominator polynomial; Eq. (coef_stiff) with a tensor K).

- unit (and constant) weights give back the spline map, and constant weights give
  NURBS basis functions equal to the B-splines;
- the rational Jacobian agrees with central differences of the map evaluated with
  scipy's B-splines (an independent basis), on a map with seeded non-tensor weights;
- the degree-p quarter annulus maps every point onto its circle, its Jacobian has
  the radial, tangential and vertical structure of the exact map, and the Galerkin
  mass of either basis sums to the exact volume (partition of unity);
- K = I gives back Eq. (coef_stiff); the entries are linear in K; with a constant
  SPD K on a sheared affine map WQ equals the Galerkin matrix (exactness, Section 4).
"""
import math

import numpy as np
import pytest
from scipy.interpolate import BSpline

from oracle import Oracle3D, galerkin_dense
from oracle.wq_oracle import coefficients, jacobians, rational_jacobians
from wq_synth import (affine_cube, perturbed_cube, perturbed_nurbs_cube, quarter_annulus, random_spd_field,
                      sample_rows)

SHEAR = np.array([[1.2, 0.3, 0.1], [-0.2, 0.8, 0.25], [0.15, -0.1, 1.05]])


def _rows_rel(a, b):
    return max(np.abs(x - y).max() / np.abs(y).max() for x, y in zip(a, b))


@pytest.mark.parametrize("w0", [1.0, 2.5])
def test_constant_weights_give_back_the_spline_map_and_basis(w0):
    patch = perturbed_cube(3, (4, 3, 5), seed=31)
    o = Oracle3D(patch.p, patch.knots, patch.ctrl)
    J0 = jacobians(o.dirs, patch.ctrl)
    J1, W = rational_jacobians(o.dirs, patch.ctrl, np.full(patch.n_dof, w0))
    assert np.abs(J1 - J0).max() < 1e-14
    assert np.abs(W - w0).max() < 1e-14 * w0
    on = Oracle3D(patch.p, patch.knots, patch.ctrl, weights=np.full(patch.n_dof, w0), nurbs_basis=True)
    rows = sample_rows(o.n, o.p, 40, seed=2)
    assert _rows_rel(on.rows(rows, "mass"), o.rows(rows, "mass")) < 1e-13
    on2 = Oracle3D(patch.p, patch.knots, patch.ctrl, weights=np.full(patch.n_dof, w0))
    assert _rows_rel(on2.rows(rows, "stiffness"), o.rows(rows, "stiffness")) < 1e-13


def _nurbs_map(patch, z):
    """F(z) = sum w C B / sum w B with scipy's B-splines, at parametric points z (m, 3)."""
    p = patch.p
    n1, n2, n3 = patch.n
    cols = []
    for l, kv in enumerate(patch.knots):
        n = len(kv) - p - 1
        cols.append(np.stack([BSpline(kv, np.eye(n)[j], p, extrapolate=False)(z[:, l]) for j in range(n)], -1))
    C = patch.ctrl.reshape(n3, n2, n1, 3)
    w = patch.weights.reshape(n3, n2, n1)
    Bt = np.einsum("ma,mb,mc->mcba", cols[0], cols[1], cols[2])
    W = np.einsum("mcba,cba->m", Bt, w)
    return np.einsum("mcba,cba,cbar->mr", Bt, w, C) / W[:, None]


def test_rational_jacobian_matches_differences_of_an_independent_map():
    patch = perturbed_nurbs_cube(3, (4, 3, 5), seed=32, wspread=0.4)
    o = Oracle3D(patch.p, patch.knots, patch.ctrl)
    J, _ = rational_jacobians(o.dirs, patch.ctrl, patch.weights)
    x = [d.x for d in o.dirs]
    rng = np.random.default_rng(5)
    picks = [(rng.integers(len(x[0])), rng.integers(len(x[1])), rng.integers(len(x[2]))) for _ in range(40)]
    h = 1e-6
    worst = 0.0
    for (a, b, c) in picks:
        z0 = np.array([x[0][a], x[1][b], x[2][c]])
        zs = []
        for k in range(3):
            e = np.zeros(3)
            e[k] = h
            zs += [np.clip(z0 + e, 0, 1 - 1e-15), np.clip(z0 - e, 0, 1)]
        Fz = _nurbs_map(patch, np.array(zs))
        fd = np.stack([(Fz[2 * k] - Fz[2 * k + 1]) / ((zs[2 * k] - zs[2 * k + 1])[k]) for k in range(3)], -1)
        worst = max(worst, np.abs(fd - J[c, b, a]).max() / np.abs(J[c, b, a]).max())
    assert worst < 1e-7


@pytest.mark.parametrize("p", [2, 3, 4])
def test_quarter_annulus_is_exact(p):
    patch = quarter_annulus(p, (2, 3, 2))
    m = patch.meta
    o = Oracle3D(patch.p, patch.knots, patch.ctrl)
    J, W, F = rational_jacobians(o.dirs, patch.ctrl, patch.weights, with_map=True)
    x1 = o.dirs[0].x[None, None, :]
    r = m["r_in"] + (m["r_out"] - m["r_in"]) * x1
    rho = np.hypot(F[..., 0], F[..., 1])
    assert np.abs(rho - r).max() < 1e-14 * m["r_out"]
    assert np.abs(F[..., 2] - m["height"] * o.dirs[2].x[:, None, None]).max() < 1e-15
    u = F[..., :2] / rho[..., None]                                   # unit radial direction
    assert np.abs(J[..., :2, 0] - (m["r_out"] - m["r_in"]) * u).max() < 1e-13
    assert np.abs(np.einsum("...r,...r->...", J[..., :2, 1], u)).max() < 1e-13   # tangential
    assert np.abs(J[..., 2, :2]).max() < 1e-15 and np.abs(J[..., :2, 2]).max() < 1e-15
    assert np.abs(J[..., 2, 2] - m["height"]).max() < 1e-14
    assert np.all(np.linalg.det(J) > 0)


@pytest.mark.parametrize("nurbs_basis", [False, True])
def test_annulus_galerkin_mass_sums_to_the_volume(nurbs_basis):
    patch = quarter_annulus(2, (2, 2, 2))
    _, M = galerkin_dense(2, patch.knots, patch.ctrl, ng=12, weights=patch.weights, nurbs_basis=nurbs_basis)
    assert abs(M.sum() - patch.meta["volume"]) < 1e-12 * patch.meta["volume"]


def test_wq_nurbs_mass_total_converges_to_the_volume():
    errs = []
    for ne in (2, 4, 8):
        patch = quarter_annulus(2, (2, ne, 2))
        o = Oracle3D(2, patch.knots, patch.ctrl, weights=patch.weights, nurbs_basis=True)
        N = int(np.prod(o.n))
        total = sum(v.sum() for v in o.rows(np.arange(N), "mass"))
        errs.append(abs(total - patch.meta["volume"]) / patch.meta["volume"])
    assert errs[0] > 4 * errs[1] > 16 * errs[2]


def test_identity_tensor_gives_back_the_coefficients():
    patch = perturbed_cube(2, (3, 4, 3), seed=33)
    o = Oracle3D(patch.p, patch.knots, patch.ctrl)
    nq = int(np.prod(o.nqp))
    K = np.zeros((6, nq))
    K[0] = K[3] = K[5] = 1.0
    c = coefficients(o.dirs, patch.ctrl, K=K)
    assert np.abs(c - o.coef).max() < 1e-15 * np.abs(o.coef).max()


def test_entries_are_linear_in_the_tensor():
    patch = perturbed_nurbs_cube(2, (3, 3, 4), seed=34)
    base = Oracle3D(patch.p, patch.knots, patch.ctrl)
    nq = int(np.prod(base.nqp))
    Ka, Kb = random_spd_field(nq, seed=3), random_spd_field(nq, seed=4)
    rows = sample_rows(base.n, base.p, 30, seed=6)
    va = Oracle3D(patch.p, patch.knots, patch.ctrl, weights=patch.weights, K=Ka).rows(rows, "stiffness")
    vb = Oracle3D(patch.p, patch.knots, patch.ctrl, weights=patch.weights, K=Kb).rows(rows, "stiffness")
    vab = Oracle3D(patch.p, patch.knots, patch.ctrl, weights=patch.weights, K=Ka + Kb).rows(rows, "stiffness")
    assert _rows_rel([a + b for a, b in zip(va, vb)], vab) < 1e-13


@pytest.mark.parametrize("p", [2, 3])
def test_constant_tensor_on_an_affine_map_equals_galerkin(p):
    patch = affine_cube(p, (2, 3, 2), SHEAR, np.array([0.1, -0.2, 0.3]))
    Kc = np.array([[2.0, 0.3, -0.2], [0.3, 1.0, 0.4], [-0.2, 0.4, 1.5]])
    o = Oracle3D(p, patch.knots, patch.ctrl)
    nq = int(np.prod(o.nqp))
    K = np.repeat(np.array([Kc[0, 0], Kc[0, 1], Kc[0, 2], Kc[1, 1], Kc[1, 2], Kc[2, 2]])[:, None], nq, axis=1)
    ok = Oracle3D(p, patch.knots, patch.ctrl, K=K)
    S_g, _ = galerkin_dense(p, patch.knots, patch.ctrl, K=Kc)
    S = ok.dense("stiffness")
    assert np.abs(S - S_g).max() < 1e-12 * np.abs(S_g).max()
    S_i, _ = galerkin_dense(p, patch.knots, patch.ctrl)
    assert np.abs(S_g - S_i).max() > 1e-2 * np.abs(S_i).max()         # the tensor matters
