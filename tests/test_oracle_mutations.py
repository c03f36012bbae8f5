"""Plant plausible mistakes in the oracle (on the CPU) and check that its pins fail.

Each mutation monkeypatches one step of oracle/wq_oracle.py; the check that
follows is one of the pins of test_oracle_pins.py written as a function that
returns an error measure. A pin that still passed under a mutation would not
be pinning that step.
"""
from fractions import Fraction

import numpy as np
import pytest

from conftest import read_golden
from oracle import wq_oracle as wo
from wq_synth import affine_cube, open_knot_vector, uniform_breaks

SHEAR = np.array([[1.2, 0.3, 0.1], [-0.2, 0.8, 0.25], [0.15, -0.1, 1.05]])


def galerkin_gap():
    patch = affine_cube(2, (2, 3, 2), SHEAR, np.zeros(3))
    orc = wo.Oracle3D(2, patch.knots, patch.ctrl)
    S_g, M_g = wo.galerkin_dense(2, patch.knots, patch.ctrl)
    return max(np.abs(orc.dense("stiffness") - S_g).max() / np.abs(S_g).max(),
               np.abs(orc.dense("mass") - M_g).max() / np.abs(M_g).max())


def printed_weight_gap():
    gold = read_golden("interior_weights.txt")["p=2"]
    chi = np.arange(-12, 13, 1.0)
    d = wo.Direction(open_knot_vector(chi, 2), 2)
    i = [k for k in range(d.n) if d.xi[k] == 0.0][-1]
    w = d.W[0, 0, i, d.Q[i]]
    return np.abs(w - gold).max() if len(w) == len(gold) else 1.0


def min_norm_gap():
    d = wo.Direction(open_knot_vector(uniform_breaks(7), 3), 3)
    worst = 0.0
    for b in (0, 1):
        for i in range(d.n):
            M = d.B[b][np.ix_(d.I[i], d.Q[i])]
            M = M / np.linalg.norm(M, axis=1, keepdims=True)
            _, s, Vt = np.linalg.svd(M)
            rank = int(np.sum(s > 1e-12 * s[0]))
            w = d.W[0, b, i, d.Q[i]]
            worst = max(worst, np.linalg.norm(Vt[rank:] @ w) / np.linalg.norm(w))
    return worst


def coef_gap():
    patch = affine_cube(2, (2, 2, 3), SHEAR, np.zeros(3))
    orc = wo.Oracle3D(2, patch.knots, patch.ctrl)
    Ai = np.linalg.inv(SHEAR)
    P = np.linalg.det(SHEAR) * Ai @ Ai.T
    return max(np.abs(orc.coef[s] - P[l, m]).max() for s, (l, m) in enumerate(wo.COEF_LM))


BASELINE = {"galerkin": 1e-11, "weights": 1e-13, "min_norm": 1e-9, "coef": 1e-12}
CHECKS = {"galerkin": galerkin_gap, "weights": printed_weight_gap,
          "min_norm": min_norm_gap, "coef": coef_gap}


@pytest.fixture(autouse=True)
def fresh_cache():
    wo._direction_exact.cache_clear()
    yield
    if hasattr(wo._direction_exact, "cache_clear"):
        wo._direction_exact.cache_clear()


def test_unmutated_oracle_passes_every_check():
    for name, fn in CHECKS.items():
        assert fn() < BASELINE[name], name


_ORIG_DIRECTION_EXACT = wo._direction_exact.__wrapped__


def _mut_rhs_kind_swapped(monkeypatch):
    # right-hand side int B^{(b)}_i B^{(a)}_j instead of int B^{(a)}_i B^{(b)}_j
    monkeypatch.setattr(wo, "_direction_exact", _direction_exact_swapped)


def _direction_exact_swapped(xi_t, p):
    x, B, I, W = _ORIG_DIRECTION_EXACT(xi_t, p)
    xi = [Fraction(v) for v in xi_t]
    n = len(xi) - p - 1
    W2 = {}
    for i in range(n):
        Q = [q for q, xq in enumerate(x) if xi[i] < xq < xi[i + p + 1]]
        Iset = list(range(max(0, i - p), min(n, i + p + 1)))
        for a in (0, 1):
            for b in (0, 1):
                M = [[B.get((b, j, q), Fraction(0)) for q in Q] for j in Iset]
                r = [I.get((b, a, i, j), Fraction(0)) for j in Iset]
                W2[(a, b, i)] = wo.min_norm_exact(M, r, drop_last=(b == 1))
    return x, B, I, W2


def _mut_drop_term(monkeypatch):
    orig = wo.Oracle3D.row_values
    def row_values(self, r, which):
        full = orig(self, r, which)
        if which == "mass":
            return full
        # remove the (l, m) = (1, 2) term by recomputing it alone and subtracting
        i = self.row_multi(r)
        Qs = [d.Q[ik] for d, ik in zip(self.dirs, i)]
        Is = [d.I[ik] for d, ik in zip(self.dirs, i)]
        c = self.coef[:, Qs[2]][:, :, Qs[1]][:, :, :, Qs[0]][wo.coef_index(0, 1)]
        kinds = [(int(k == 0), int(k == 1)) for k in range(3)]
        A = [d.W[a, b, ik][Qs[k]][None, :] * d.B[b][np.ix_(Is[k], Qs[k])]
             for k, (d, ik, (a, b)) in enumerate(zip(self.dirs, i, kinds))]
        return full - np.einsum("xc,yb,za,cba->xyz", A[2], A[1], A[0], c).ravel()
    monkeypatch.setattr(wo.Oracle3D, "row_values", row_values)


def _mut_transposed_jacobian(monkeypatch):
    orig = wo.jacobians
    monkeypatch.setattr(wo, "jacobians", lambda dirs, ctrl: np.swapaxes(orig(dirs, ctrl), -1, -2))


def _mut_derivative_sign(monkeypatch):
    orig = wo.basis_on_span
    def flipped(xi, p, s, x):
        v, d = orig(xi, p, s, x)
        return v, [-t for t in d]
    monkeypatch.setattr(wo, "basis_on_span", flipped)


def _mut_endpoint_points(monkeypatch):
    # boundary spans sampled at k = 0..p (the left end knot included)
    def pts(chi, p, exact=False):
        chi = [wo._fr(c) for c in chi]
        n_el = len(chi) - 1
        out = list(chi[1:-1]) + [(chi[k] + chi[k + 1]) / 2 for k in range(1, n_el - 1)]
        for (a, b) in ((chi[0], chi[1]), (chi[-2], chi[-1])):
            out += [a + k * (b - a) / (p + 2) for k in range(0, p + 1)]
        out = sorted(out)
        return out if exact else np.array([float(v) for v in out])
    monkeypatch.setattr(wo, "quadrature_points", pts)


def _mut_not_min_norm(monkeypatch):
    orig = wo.min_norm_exact
    def basic(M, r, drop_last, digits=80):
        w = orig(M, r, drop_last, digits)
        # add a null-space vector of the (square part of the) system when one exists
        Mm = M[:-1] if drop_last else M
        if len(Mm[0]) > len(Mm):
            A = np.array([[float(v) for v in row] for row in Mm])
            _, _, Vt = np.linalg.svd(A)
            z = Vt[-1]
            return [wk + Fraction(float(0.1 * zk)) for wk, zk in zip(w, z)]
        return w
    monkeypatch.setattr(wo, "min_norm_exact", basic)


MUTATIONS = {
    "rhs_kind_swapped": _mut_rhs_kind_swapped,
    "dropped_stiffness_term": _mut_drop_term,
    "transposed_jacobian": _mut_transposed_jacobian,
    "derivative_sign": _mut_derivative_sign,
    "endpoint_boundary_points": _mut_endpoint_points,
    "not_minimum_norm": _mut_not_min_norm,
}


@pytest.mark.parametrize("name", list(MUTATIONS))
def test_mutation_is_caught(name, monkeypatch):
    MUTATIONS[name](monkeypatch)
    failed = []
    for check, fn in CHECKS.items():
        try:
            gap = fn()
        except (ValueError, ArithmeticError, np.linalg.LinAlgError, StopIteration, IndexError):
            gap = np.inf
        if not gap < BASELINE[check]:
            failed.append(check)
    assert failed, f"mutation {name} passed every pin"
