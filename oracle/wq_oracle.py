"""Plain FP64 CPU oracle for weighted-quadrature (WQ) assembly of isogeometric
stiffness and mass matrices (Calabro, Sangalli, Tani, "Fast formation of
isogeometric Galerkin matrices by weighted quadrature").

TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and the
cpu_baseline / reference legs of bench.py may import or run anything under
oracle/. The product path (paper_1605_01238_gb300) never calls it and shares no
code with it.

Every quantity is computed from its definition in the paper, in float64, with
numpy primitives (einsum, lstsq, inv, det, Gauss-Legendre nodes) as the only
library steps:

* open knot vectors and maximal regularity ........ Section 3 (Xi, n_KNT)
* quadrature points ............................... Remark "choice of quadrature points" (Section 4)
* univariate B-splines and derivatives ............ Cox-de Boor recursion (Section 3 refers to
                                                    the textbook definition)
* exact univariate integrals I^{(a,b)} ............ Eq. (integrals); element-wise Gauss (Algorithm 1)
* WQ rules, four kinds, minimum Euclidean norm .... Eqs. (quadrule), (exact), (support); Algorithm 2;
                                                    Remark "computation of quadrature weights"
* coefficients c_lm and c ......................... Eq. (coef_stiff) and Eq. (mass2); a
                                                    coefficient tensor K in c_lm =
                                                    det DF (DF^{-1} K DF^{-T})_lm and NURBS
                                                    geometry / basis denominators (the
                                                    sentence after Eq. (mass2))
* WQ mass / stiffness entries ..................... Eq. (Mass_approx), Eq. (massquadrature) and
                                                    Eq. (stiff) with the term (l, m) integrated by
                                                    the rule (delta_kl, delta_km) in direction k
* brute-force Galerkin (element-wise Gauss) ....... Eqs. (stiffness-3d), (mass-3d), used by the pins

Readings where the paper is ambiguous:

* Rule kinds (a, b): a = derivative order on the test function (folded into the
  weight), b = derivative order on the trial function evaluated at the point.
  The system matrix holds B^{(b)}_j(x_q) and the right-hand side is
  int B^{(a)}_i B^{(b)}_j. This is the only assignment for which WQ is exact for
  constant coefficients (Section 4 states that requirement).
* Boundary spans get p+1 points strictly inside: x = a + k (b - a)/(p + 2),
  k = 1..p+1. Supports are open sets, so knots 0 and 1 are never points.
* For b = 1 the rows of the system sum to zero (sum_j B'_j = 0 on supp B_i) and
  the right-hand side is consistent, so the last equation is dropped and the
  minimum-norm solution of the remaining full-row-rank system is taken.
* det DF must be positive at every quadrature point (Eq. (mass2) uses det DF).
* NURBS: with weights w_i the geometry is F = sum_i w_i C_i B_i / W, W = sum_i w_i B_i.
  The basis functions stay R_i = B_i o F^{-1} (Section 3 defines them so), so only
  DF changes. With NURBS basis functions R_i = (w_i B_i / W) o F^{-1} the mass entry
  is w_i w_j times the B-spline entry with c = det DF / W^2: the denominator is
  absorbed by c, as the sentence after Eq. (mass2) states. (The stiffness with NURBS
  basis functions would need the lower-order terms of the quotient rule, which the
  paper does not treat; it is not provided.)

Parity unpinned: none of the functions below lacks a pin; entries on curved
(perturbed) geometry are pinned only through the invariants (row sums of the
stiffness matrix, exactness of the rules, Galerkin equality on affine maps).
"""
from __future__ import annotations

import math
from decimal import Decimal, localcontext
from fractions import Fraction
from functools import lru_cache

import numpy as np


# ---------------------------------------------------------------------------
# Knot vectors (Section 3)

def distinct_knots(knot_vector: np.ndarray, p: int) -> np.ndarray:
    """Distinct knots chi_0 < ... < chi_{n_el} of an open knot vector of degree p."""
    xi = np.asarray(knot_vector, dtype=np.float64)
    return xi[p:len(xi) - p].copy()


def check_open_knot_vector(knot_vector: np.ndarray, p: int) -> None:
    """Raise ValueError unless the end knots repeat p+1 times and interior knots are simple."""
    xi = np.asarray(knot_vector, dtype=np.float64)
    if len(xi) < 2 * (p + 1) + 1:
        raise ValueError("need at least two spans")
    if np.any(xi[:p + 1] != xi[0]) or np.any(xi[-(p + 1):] != xi[-1]):
        raise ValueError("end knots must repeat p+1 times")
    chi = xi[p:len(xi) - p]
    if np.any(np.diff(chi) <= 0.0):
        raise ValueError("interior knots must be simple and increasing")


# ---------------------------------------------------------------------------
# B-splines by the Cox-de Boor recursion

def bspline_all(knot_vector: np.ndarray, p: int, x: np.ndarray, deriv: int = 0) -> np.ndarray:
    """Values B^{(deriv)}_{j,p}(x) of every basis function: array (len(x), n).

    Degree 0 uses half-open spans [xi_j, xi_{j+1}); the right end of the
    parameter domain belongs to the last non-empty span. Degree k follows
    B_{j,k} = (x - xi_j)/(xi_{j+k} - xi_j) B_{j,k-1}
            + (xi_{j+k+1} - x)/(xi_{j+k+1} - xi_{j+1}) B_{j+1,k-1}
    with 0/0 read as 0; the derivative is
    B'_{j,p} = p/(xi_{j+p} - xi_j) B_{j,p-1} - p/(xi_{j+p+1} - xi_{j+1}) B_{j+1,p-1}.
    """
    xi = np.asarray(knot_vector, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    m = len(xi) - 1                      # number of degree-0 functions
    N = np.zeros((len(x), m))
    for j in range(m):
        if xi[j] < xi[j + 1]:
            N[:, j] = (x >= xi[j]) & (x < xi[j + 1])
    last = max(j for j in range(m) if xi[j] < xi[j + 1])
    N[x == xi[-1], last] = 1.0

    def raise_degree(N, k):
        out = np.zeros((len(x), N.shape[1] - 1))
        for j in range(N.shape[1] - 1):
            d1 = xi[j + k] - xi[j]
            d2 = xi[j + k + 1] - xi[j + 1]
            if d1 > 0:
                out[:, j] += (x - xi[j]) / d1 * N[:, j]
            if d2 > 0:
                out[:, j] += (xi[j + k + 1] - x) / d2 * N[:, j + 1]
        return out

    for k in range(1, p - deriv + 1):
        N = raise_degree(N, k)
    # derivative orders: differentiate from degree p - deriv up to p
    for k in range(p - deriv + 1, p + 1):
        out = np.zeros((len(x), N.shape[1] - 1))
        for j in range(N.shape[1] - 1):
            d1 = xi[j + k] - xi[j]
            d2 = xi[j + k + 1] - xi[j + 1]
            if d1 > 0:
                out[:, j] += k / d1 * N[:, j]
            if d2 > 0:
                out[:, j] -= k / d2 * N[:, j + 1]
        N = out
    return N


# ---------------------------------------------------------------------------
# One direction: points, tables, integrals, rules, in exact rational arithmetic
#
# The rule systems of Algorithm 2 are badly conditioned near the boundary at high
# degree (row-scaled condition numbers reach ~1e7 at p = 8), so a float64 solve
# would carry errors far above the 1e-12 parity bar. Points, B-spline values and
# integrals are therefore computed exactly with fractions.Fraction (float knots
# are binary rationals, so they convert exactly), the solves run in 80-digit
# decimal arithmetic, and every result is rounded to float64 once at the end.

def _fr(v) -> Fraction:
    return v if isinstance(v, Fraction) else Fraction(float(v))


def find_span(xi: list, p: int, x: Fraction) -> int:
    """Index s with xi_s <= x < xi_{s+1} among the non-empty spans p..n-1
    (the last span also takes x = xi_{n})."""
    n = len(xi) - p - 1
    if x >= xi[n]:
        return n - 1
    lo, hi = p, n
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if x < xi[mid]:
            hi = mid
        else:
            lo = mid
    return lo


def basis_on_span(xi: list, p: int, s: int, x: Fraction) -> tuple:
    """Cox-de Boor on span s: values and first derivatives of the p+1 functions
    B_{s-p..s} that are non-zero there, as polynomials of that span evaluated at x
    (x may be any number; the span's polynomial pieces are used)."""
    N = [Fraction(1)]                                  # degree 0: B_s
    lower = None
    for k in range(1, p + 1):
        new = []
        for t in range(k + 1):                         # function j = s - k + t
            j = s - k + t
            v = Fraction(0)
            if t >= 1:                                 # term with B_{j,k-1} = N[t-1]
                v += (x - xi[j]) / (xi[j + k] - xi[j]) * N[t - 1]
            if t <= k - 1:                             # term with B_{j+1,k-1} = N[t]
                v += (xi[j + k + 1] - x) / (xi[j + k + 1] - xi[j + 1]) * N[t]
            new.append(v)
        if k == p:
            lower = N                                  # degree p-1 values
        N = new
    dN = []
    for t in range(p + 1):                             # derivative of B_{s-p+t}
        j = s - p + t
        v = Fraction(0)
        if t >= 1:
            v += p / (xi[j + p] - xi[j]) * lower[t - 1]
        if t <= p - 1:
            v -= p / (xi[j + p + 1] - xi[j + 1]) * lower[t]
        dN.append(v)
    return N, dN


@lru_cache(maxsize=None)
def open_newton_cotes(m: int) -> tuple:
    """Nodes k/(m+1), k = 1..m, and weights of the open Newton-Cotes rule on [0, 1]
    with m points, from the exact moment equations sum_k w_k t_k^e = 1/(e+1),
    e = 0..m-1. With m odd the rule is exact for degree m."""
    t = [Fraction(k, m + 1) for k in range(1, m + 1)]
    A = [[tk ** e for tk in t] + [Fraction(1, e + 1)] for e in range(m)]
    w = _solve_exact(A)
    return tuple(t), tuple(w)


def _solve_exact(aug: list) -> list:
    """Gauss-Jordan elimination with non-zero pivots on an augmented rational matrix."""
    m = len(aug)
    A = [row[:] for row in aug]
    for c in range(m):
        piv = next(r for r in range(c, m) if A[r][c] != 0)
        A[c], A[piv] = A[piv], A[c]
        inv = 1 / A[c][c]
        A[c] = [v * inv for v in A[c]]
        for r in range(m):
            if r != c and A[r][c] != 0:
                f = A[r][c]
                A[r] = [vr - f * vc for vr, vc in zip(A[r], A[c])]
    return [A[r][m] for r in range(m)]


class Direction:
    """All univariate data of one direction (Algorithms 1 and 2 for fixed l).

    Exact rational values are kept in *_exact attributes; the float64 arrays
    x, B[deriv, j, q], integrals[a, b, i, j] and W[a, b, i, q] are their roundings.
    """

    def __init__(self, knot_vector, p: int):
        check_open_knot_vector(knot_vector, p)
        self.p = p
        self.xi = np.asarray(knot_vector, dtype=np.float64)
        self.chi = distinct_knots(self.xi, p)
        self.n_el = len(self.chi) - 1
        self.n = len(self.xi) - p - 1
        data = _direction_exact(tuple(float(v) for v in self.xi), p)
        self.x_exact, self.B_exact, self.I_exact, self.W_exact = data
        self.x = np.array([float(v) for v in self.x_exact])
        self.nqp = len(self.x)
        # Q_i: points inside the open support (xi_i, xi_{i+p+1}) of B_i (Eq. (support))
        self.Q = [np.nonzero((self.x > self.xi[i]) & (self.x < self.xi[i + p + 1]))[0]
                  for i in range(self.n)]
        # I_i: trial functions with B_i B_j not identically zero
        self.I = [np.arange(max(0, i - p), min(self.n, i + p + 1)) for i in range(self.n)]
        self.B = np.zeros((2, self.n, self.nqp))
        for (b, j, q), v in self.B_exact.items():
            self.B[b, j, q] = float(v)
        self.integrals = np.zeros((2, 2, self.n, self.n))
        for (a, b, i, j), v in self.I_exact.items():
            self.integrals[a, b, i, j] = float(v)
        self.W = np.zeros((2, 2, self.n, self.nqp))
        for (a, b, i), w in self.W_exact.items():
            self.W[a, b, i, self.Q[i]] = [float(v) for v in w]

    def q_range(self, i: int) -> tuple:
        q = self.Q[i]
        return int(q[0]), int(q[-1]) + 1


def quadrature_points(chi, p: int, exact: bool = False):
    """Global point grid: interior knots, midpoints of internal spans, and p+1
    equally spaced points strictly inside each of the two boundary spans
    (Remark on the choice of quadrature points; boundary reading in the header)."""
    chi = [_fr(c) for c in chi]
    n_el = len(chi) - 1
    pts = list(chi[1:-1])
    pts += [(chi[k] + chi[k + 1]) / 2 for k in range(1, n_el - 1)]
    for (a, b) in ((chi[0], chi[1]), (chi[-2], chi[-1])):
        pts += [a + k * (b - a) / (p + 2) for k in range(1, p + 2)]
    pts = sorted(pts)
    return pts if exact else np.array([float(v) for v in pts])


@lru_cache(maxsize=None)
def _direction_exact(xi_t: tuple, p: int) -> tuple:
    xi = [Fraction(v) for v in xi_t]
    n = len(xi) - p - 1
    chi = xi[p:len(xi) - p]
    x = quadrature_points(chi, p, exact=True)
    # B^{(0)}, B^{(1)} of every function at every point: only the p+1 functions of
    # the point's span can be non-zero, the rest are zero (stored sparsely)
    B = {}
    for q, xq in enumerate(x):
        s = find_span(xi, p, xq)
        vals, ders = basis_on_span(xi, p, s, xq)
        for t in range(p + 1):
            B[(0, s - p + t, q)] = vals[t]
            B[(1, s - p + t, q)] = ders[t]
    # exact integrals, span by span, with the open Newton-Cotes rule of 2p+1 points
    tq, wq = open_newton_cotes(2 * p + 1)
    I = {}
    for s in range(p, n):
        a0, h = xi[s], xi[s + 1] - xi[s]
        for tk, wk in zip(tq, wq):
            vals, ders = basis_on_span(xi, p, s, a0 + tk * h)
            both = (vals, ders)
            for ti in range(p + 1):
                for tj in range(p + 1):
                    i, j = s - p + ti, s - p + tj
                    for a in (0, 1):
                        for b in (0, 1):
                            key = (a, b, i, j)
                            I[key] = I.get(key, 0) + wk * h * both[a][ti] * both[b][tj]
    # rules: minimum-norm solutions (Algorithm 2)
    W = {}
    for i in range(n):
        Q = [q for q, xq in enumerate(x) if xi[i] < xq < xi[i + p + 1]]
        Iset = list(range(max(0, i - p), min(n, i + p + 1)))
        for a in (0, 1):
            for b in (0, 1):
                M = [[B.get((b, j, q), Fraction(0)) for q in Q] for j in Iset]
                r = [I.get((a, b, i, j), Fraction(0)) for j in Iset]
                W[(a, b, i)] = min_norm_exact(M, r, drop_last=(b == 1))
    return x, B, I, W


def min_norm_exact(M: list, r: list, drop_last: bool, digits: int = 80) -> list:
    """Minimum Euclidean-norm solution w = M^T (M M^T)^{-1} r of M w = r.

    M and r are exact rationals. The solve runs in `digits`-digit decimal
    arithmetic (Gaussian elimination with partial pivoting on the normal
    equations): with condition numbers below 1e30 its error stays under 1e-50,
    far below the float64 rounding of the result. For the derivative-trial
    kinds the rows of M sum to zero and the right-hand side is consistent, so
    the last row is dropped first."""
    if drop_last:
        M, r = M[:-1], r[:-1]
    m, nq = len(M), len(M[0])
    if m > nq:
        raise ValueError("fewer points than exactness conditions")
    with localcontext() as ctx:
        ctx.prec = digits
        D = lambda f: Decimal(f.numerator) / Decimal(f.denominator)
        Md = [[D(v) for v in row] for row in M]
        A = [[sum((Md[a][k] * Md[b][k] for k in range(nq)), Decimal(0)) for b in range(m)] + [D(r[a])]
             for a in range(m)]
        for c in range(m):
            piv = max(range(c, m), key=lambda rr: abs(A[rr][c]))
            A[c], A[piv] = A[piv], A[c]
            for rr in range(c + 1, m):
                f = A[rr][c] / A[c][c]
                if f:
                    A[rr] = [vr - f * vc for vr, vc in zip(A[rr], A[c])]
        y = [Decimal(0)] * m
        for c in range(m - 1, -1, -1):
            y[c] = (A[c][m] - sum((A[c][k] * y[k] for k in range(c + 1, m)), Decimal(0))) / A[c][c]
        w = [sum((Md[a][k] * y[a] for a in range(m)), Decimal(0)) for k in range(nq)]
        return [Fraction(v) for v in w]


def wq_rule(d: Direction, i: int, a: int, b: int) -> np.ndarray:
    """Float64 weights w^{(a,b)}_{i,q}, q in Q_i (Eq. (exact), Algorithm 2)."""
    return d.W[a, b, i, d.Q[i]].copy()


def exact_integrals(knot_vector, p: int, ng: int) -> np.ndarray:
    """I[a, b, i, j] = int_0^1 B^{(a)}_i B^{(b)}_j in float64 by ng-point
    Gauss-Legendre per span (exact when 2 ng - 1 >= 2p); used to cross-check the
    rational Newton-Cotes integrals of Direction."""
    xi = np.asarray(knot_vector, dtype=np.float64)
    chi = distinct_knots(xi, p)
    t, wt = np.polynomial.legendre.leggauss(ng)
    xs, ws = [], []
    for k in range(len(chi) - 1):
        a, b = chi[k], chi[k + 1]
        xs.append(0.5 * (a + b) + 0.5 * (b - a) * t)
        ws.append(0.5 * (b - a) * wt)
    xs = np.concatenate(xs)
    ws = np.concatenate(ws)
    B = [bspline_all(xi, p, xs, 0), bspline_all(xi, p, xs, 1)]     # (ngauss, n)
    out = np.zeros((2, 2) + (B[0].shape[1],) * 2)
    for a in (0, 1):
        for b in (0, 1):
            out[a, b] = np.einsum("g,gi,gj->ij", ws, B[a], B[b])
    return out


# ---------------------------------------------------------------------------
# Geometry and coefficients (Eqs. (coef_stiff), (mass2))

# storage order of the six symmetric components, then c = det DF
COEF_LM = ((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2))


def greville_exact(knot_vector, p: int) -> list:
    """Greville abscissae g_i = (xi_{i+1} + ... + xi_{i+p}) / p as exact rationals."""
    xi = [Fraction(float(v)) for v in knot_vector]
    n = len(xi) - p - 1
    return [sum(xi[i + 1:i + p + 1], Fraction(0)) / p for i in range(n)]


def control_offsets(dirs: list, ctrl: np.ndarray) -> np.ndarray:
    """C_i - g_i, g_i = (g_{1,i1}, g_{2,i2}, g_{3,i3}) the Greville point of i:
    array (n3, n2, n1, 3). Each Greville abscissa is split exactly into
    hi + lo doubles; C - hi is formed exactly by two-sum, and the result is
    rounded once more (within one ulp of the exact difference)."""
    n1, n2, n3 = (d.n for d in dirs)
    C = np.asarray(ctrl, dtype=np.float64).reshape(n3, n2, n1, 3)
    out = np.empty_like(C)
    shapes = [(1, 1, n1), (1, n2, 1), (n3, 1, 1)]
    for r, d in enumerate(dirs):
        g = greville_exact(d.xi, d.p)
        hi = np.array([float(v) for v in g])
        lo = np.array([float(v - Fraction(float(v))) for v in g])
        hi, lo = hi.reshape(shapes[r]), lo.reshape(shapes[r])
        c = C[..., r]
        s = c - hi                                   # two-sum: s + e = c - hi exactly
        bb = s - c
        e = (c - (s - bb)) + (-hi - bb)
        out[..., r] = s + (e - lo)
    return out


def jacobians(dirs: list, ctrl: np.ndarray) -> np.ndarray:
    """DF at every point of the tensor grid: array (nqp3, nqp2, nqp1, 3, 3),
    DF[r, c] = d/dzeta_c of F_r, F = sum_i C_i B_i (Section 3).

    B-splines reproduce linear functions with the Greville points as
    coefficients, zeta = sum_i g_i B_i(zeta), so F(zeta) = zeta + sum_i (C_i - g_i) B_i(zeta)
    and DF = I + sum_i (C_i - g_i) x grad B_i: the same matrix, without summing the
    O(1/h) terms C_i x grad B_i that cancel to O(1) (their rounding would reach
    the stiffness entries amplified by the rules' conditioning at high degree).
    The sums are einsums over the dense univariate tables."""
    D = control_offsets(dirs, ctrl)
    B = [d.B for d in dirs]                          # (2, n, nqp) each
    out = np.empty((dirs[2].nqp, dirs[1].nqp, dirs[0].nqp, 3, 3))
    for c in range(3):
        D1 = B[0][1 if c == 0 else 0]
        D2 = B[1][1 if c == 1 else 0]
        D3 = B[2][1 if c == 2 else 0]
        out[..., :, c] = np.einsum("kjir,ia,jb,kc->cbar", D, D1, D2, D3, optimize=True)
    out[..., 0, 0] += 1.0
    out[..., 1, 1] += 1.0
    out[..., 2, 2] += 1.0
    return out


def _active(d) -> tuple:
    """First basis function s - p of the span s holding each point (x in [xi_s, xi_{s+1}),
    the last span for the right end) and the p+1 values B^{(b)}_{s-p+t}(x_q): (first[nqp],
    vals[2, nqp, p+1])."""
    p = d.p
    s = np.clip(np.searchsorted(d.xi, d.x, side="right") - 1, p, d.n - 1)
    first = s - p
    cols = first[:, None] + np.arange(p + 1)[None, :]
    vals = np.stack([d.B[b][cols, np.arange(d.nqp)[:, None]] for b in (0, 1)])
    return first, vals


def rational_jacobians(dirs: list, ctrl: np.ndarray, weights: np.ndarray, with_map: bool = False) -> tuple:
    """DF and W at every point of the tensor grid for the NURBS map
    F = sum_i w_i C_i B_i / W, W = sum_i w_i B_i: arrays (nqp3, nqp2, nqp1, 3, 3) and
    (nqp3, nqp2, nqp1). Point by point over the (p+1)^3 functions active there,
    F first and then DF = sum_i w_i (C_i - F) x grad B_i / W (the quotient rule with
    sum_i w_i grad B_i = grad W); the differences C_i - F stay small, so the O(1/h)
    gradients do not cancel in the sum."""
    p = dirs[0].p
    n1, n2, n3 = (d.n for d in dirs)
    C = np.asarray(ctrl, dtype=np.float64).reshape(n3, n2, n1, 3)
    w = np.asarray(weights, dtype=np.float64).reshape(n3, n2, n1)
    (f1, v1), (f2, v2), (f3, v3) = (_active(d) for d in dirs)
    t = np.arange(p + 1)
    I3 = (f3[:, None] + t)[:, None, None, :, None, None]
    I2 = (f2[:, None] + t)[None, :, None, None, :, None]
    I1 = (f1[:, None] + t)[None, None, :, None, None, :]
    Cw = C[I3, I2, I1]                                   # (q3, q2, q1, t3, t2, t1, 3)
    ww = w[I3, I2, I1]                                   # (q3, q2, q1, t3, t2, t1)
    def tens(b1, b2, b3):
        return (v3[b3][:, None, None, :, None, None] * v2[b2][None, :, None, None, :, None] *
                v1[b1][None, None, :, None, None, :])
    B0 = tens(0, 0, 0)
    Wq = np.einsum("abcxyz,abcxyz->abc", ww, B0)
    F = np.einsum("abcxyz,abcxyzr->abcr", ww * B0, Cw) / Wq[..., None]
    D = Cw - F[:, :, :, None, None, None, :]
    grads = [tens(1, 0, 0), tens(0, 1, 0), tens(0, 0, 1)]
    J = np.empty(Wq.shape + (3, 3))
    for c in range(3):
        J[..., :, c] = np.einsum("abcxyz,abcxyzr->abcr", ww * grads[c], D) / Wq[..., None]
    return (J, Wq, F) if with_map else (J, Wq)


def coefficients(dirs: list, ctrl: np.ndarray, kappa: np.ndarray | None = None,
                 weights: np.ndarray | None = None, K: np.ndarray | None = None,
                 nurbs_basis: bool = False) -> np.ndarray:
    """coef[7, nqp3, nqp2, nqp1]: c_11, c_12, c_13, c_22, c_23, c_33 of
    det DF * DF^{-1} K DF^{-T} (Eq. (coef_stiff), K = I unless the symmetric tensor
    field K[6, ...] = K11 K12 K13 K22 K23 K33 is given) and c = det DF (Eq. (mass2);
    det DF / W^2 for NURBS basis functions), each times kappa when kappa (same grid)
    is given. weights: NURBS weights of the control points (rational map)."""
    if weights is not None:
        J, Wq = rational_jacobians(dirs, ctrl, weights)
    else:
        J, Wq = jacobians(dirs, ctrl), None
    det = np.linalg.det(J)
    if not np.all(np.isfinite(det)) or np.any(det <= 0.0):
        raise ValueError("det DF must be positive at every quadrature point")
    Jinv = np.linalg.inv(J)
    if K is None:
        P = np.einsum("...ik,...jk->...ij", Jinv, Jinv) * det[..., None, None]
    else:
        Kf = np.asarray(K, dtype=np.float64).reshape((6,) + det.shape)
        Km = np.empty(det.shape + (3, 3))
        for s, (l, m) in enumerate(COEF_LM):
            Km[..., l, m] = Km[..., m, l] = Kf[s]
        P = np.einsum("...ia,...ab,...jb->...ij", Jinv, Km, Jinv) * det[..., None, None]
    out = np.empty((7,) + det.shape)
    for s, (l, m) in enumerate(COEF_LM):
        out[s] = P[..., l, m]
    out[6] = det
    if nurbs_basis:
        if Wq is None:
            raise ValueError("NURBS basis functions need weights")
        out[6] = det / Wq ** 2
    if kappa is not None:
        out *= np.asarray(kappa, dtype=np.float64).reshape(det.shape)[None]
    return out


def coef_index(l: int, m: int) -> int:
    return COEF_LM.index((min(l, m), max(l, m)))


# ---------------------------------------------------------------------------
# The assembled operator

class Oracle3D:
    """Oracle for one 3D patch: univariate rules, coefficients, and entries."""

    def __init__(self, p: int, knots: list, ctrl: np.ndarray, kappa: np.ndarray | None = None,
                 weights: np.ndarray | None = None, K: np.ndarray | None = None, nurbs_basis: bool = False):
        self.p = p
        self.dirs = [Direction(k, p) for k in knots]
        self.n = tuple(d.n for d in self.dirs)
        self.nqp = tuple(d.nqp for d in self.dirs)
        self.ctrl = np.asarray(ctrl, dtype=np.float64).reshape(-1, 3)
        self.weights = None if weights is None else np.asarray(weights, dtype=np.float64).reshape(-1)
        self.nurbs_basis = bool(nurbs_basis)
        self.coef = coefficients(self.dirs, self.ctrl, kappa, self.weights, K, self.nurbs_basis)

    def basis_scale(self, r: int, which: str):
        """w_i w_j of row r for NURBS basis functions (mass only), else None."""
        if not self.nurbs_basis:
            return None
        if which != "mass":
            raise ValueError("the stiffness with NURBS basis functions is not provided")
        return self.weights[r] * self.weights[self.row_cols(r)]

    # -- pattern (Section 3: I_i = prod I_{l,i_l}; linear index i1 + n1(i2 + n2 i3))
    def row_multi(self, r: int) -> tuple:
        n1, n2, _ = self.n
        return r % n1, (r // n1) % n2, r // (n1 * n2)

    def row_cols(self, r: int) -> np.ndarray:
        n1, n2, _ = self.n
        i1, i2, i3 = self.row_multi(r)
        I1, I2, I3 = (d.I[i] for d, i in zip(self.dirs, (i1, i2, i3)))
        return (I1[None, None, :] + n1 * (I2[None, :, None] + n2 * I3[:, None, None])).ravel()

    def row_ptr(self) -> np.ndarray:
        n1, n2, n3 = self.n
        counts = np.array([len(self.row_cols(r)) for r in range(n1 * n2 * n3)], dtype=np.int64)
        return np.concatenate([[0], np.cumsum(counts)])

    # -- entries by the nested sums of Eq. (massquadrature), extended to Eq. (stiff)
    def row_values(self, r: int, which: str) -> np.ndarray:
        """All nonzeros of row r in ascending column order, by the nested WQ sums."""
        i = self.row_multi(r)
        Qs = [d.Q[ik] for d, ik in zip(self.dirs, i)]
        Is = [d.I[ik] for d, ik in zip(self.dirs, i)]
        c = self.coef[:, Qs[2]][:, :, Qs[1]][:, :, :, Qs[0]]       # (7, q3, q2, q1)
        out = np.zeros((len(Is[2]), len(Is[1]), len(Is[0])))
        terms = [(None, None)] if which == "mass" else [(l, m) for l in range(3) for m in range(3)]
        for (l, m) in terms:
            if l is None:
                kinds = [(0, 0)] * 3
                cc = c[6]
            else:
                kinds = [(int(k == l), int(k == m)) for k in range(3)]
                cc = c[coef_index(l, m)]
            # A_k[j, q] = w^{(a,b)}_{k, i_k, q} B^{(b)}_{k, j}(x_q) over q in Q_{i_k}
            A = [d.W[a, b, ik][Qs[k]][None, :] * d.B[b][np.ix_(Is[k], Qs[k])]
                 for k, (d, ik, (a, b)) in enumerate(zip(self.dirs, i, kinds))]
            # nested sum: innermost over q3, then q2, then q1
            out += np.einsum("xc,yb,za,cba->xyz", A[2], A[1], A[0], cc, optimize=False)
        scale = self.basis_scale(r, which)
        return out.ravel() if scale is None else out.ravel() * scale

    def load(self, f: np.ndarray) -> np.ndarray:
        """WQ load vector b_i = sum_{q in Q_i} prod_k w^{(0,0)}_{k,i_k,q_k} f(x_q) c(x_q)
        (Eq. (quadrule) with the test function's (0,0) rules, c = det DF): array (N_DOF,)
        with i1 fastest. f: values at the point grid (q1 fastest)."""
        if self.nurbs_basis:
            raise ValueError("the load vector with NURBS basis functions is not provided")
        g = np.asarray(f, dtype=np.float64).reshape(self.coef[6].shape) * self.coef[6]   # (q3, q2, q1)
        W = [d.W[0, 0] for d in self.dirs]                                             # (n, nqp) each
        return np.einsum("xc,yb,za,cba->xyz", W[2], W[1], W[0], g, optimize=True).ravel()

    def rows(self, rows, which: str) -> list:
        return [self.row_values(int(r), which) for r in rows]

    def dense(self, which: str) -> np.ndarray:
        """Full matrix (tiny meshes only)."""
        N = self.n[0] * self.n[1] * self.n[2]
        A = np.zeros((N, N))
        for r in range(N):
            A[r, self.row_cols(r)] = self.row_values(r, which)
        return A


# ---------------------------------------------------------------------------
# Brute-force Galerkin matrices (Eqs. (stiffness-3d), (mass-3d)) for the pins

def galerkin_dense(p: int, knots: list, ctrl: np.ndarray, ng: int | None = None,
                   kappa_fn=None, weights: np.ndarray | None = None, K: np.ndarray | None = None,
                   nurbs_basis: bool = False) -> tuple:
    """Exact-as-Gauss Galerkin stiffness and mass on the parametric cube:
    s_ij = int grad B_i . (det DF DF^{-1} K DF^{-T}) grad B_j, m_ij = int R_i R_j det DF
    (R_i = B_i, or w_i B_i / W for NURBS basis functions), by ng^3-point Gauss on every
    element (tiny meshes only). weights: NURBS weights of the map F = sum w C B / W;
    K: constant symmetric 3x3 coefficient tensor (default I)."""
    ng = ng if ng is not None else p + 2
    t, wt = np.polynomial.legendre.leggauss(ng)
    gx, gw = [], []
    for kv in knots:
        chi = distinct_knots(kv, p)
        xs = np.concatenate([0.5 * (chi[e] + chi[e + 1]) + 0.5 * (chi[e + 1] - chi[e]) * t
                             for e in range(len(chi) - 1)])
        ws = np.concatenate([0.5 * (chi[e + 1] - chi[e]) * wt for e in range(len(chi) - 1)])
        gx.append(xs)
        gw.append(ws)
    B = [[bspline_all(kv, p, gx[k], dd) for dd in (0, 1)] for k, kv in enumerate(knots)]
    n1, n2, n3 = (b[0].shape[1] for b in B)
    C = np.asarray(ctrl).reshape(n3, n2, n1, 3)
    # basis gradients on the tensor Gauss grid: G[c][g3, g2, g1, i3, i2, i1]
    def tensor(d1, d2, d3):
        return np.einsum("ax,by,cz->cbazyx", B[0][d1], B[1][d2], B[2][d3])
    Bv = tensor(0, 0, 0)
    G = [tensor(1, 0, 0), tensor(0, 1, 0), tensor(0, 0, 1)]
    wgt = np.ones((n3, n2, n1)) if weights is None else np.asarray(weights, dtype=np.float64).reshape(n3, n2, n1)
    Wv = np.einsum("cbazyx,zyx->cba", Bv, wgt)
    Wd = [np.einsum("cbazyx,zyx->cba", G[c], wgt) for c in range(3)]
    Nv = [np.einsum("cbazyx,zyx->cba", Bv, wgt * C[..., r]) for r in range(3)]
    # DF_rc = (d_c N_r - F_r d_c W) / W with F = N / W (quotient rule)
    DF = np.stack([np.stack([(np.einsum("cbazyx,zyx->cba", G[c], wgt * C[..., r]) - Nv[r] / Wv * Wd[c]) / Wv
                             for c in range(3)], -1) for r in range(3)], -2)
    det = np.linalg.det(DF)
    Jinv = np.linalg.inv(DF)
    Km = np.eye(3) if K is None else np.asarray(K, dtype=np.float64)
    P = np.einsum("...ia,ab,...jb->...ij", Jinv, Km, Jinv) * det[..., None, None]
    w3 = np.einsum("c,b,a->cba", gw[2], gw[1], gw[0])
    if kappa_fn is not None:
        w3 = w3 * kappa_fn(gx)
    N = n1 * n2 * n3
    Bf = Bv.reshape(w3.shape + (N,))
    Gf = [g.reshape(w3.shape + (N,)) for g in G]
    if nurbs_basis:
        Rf = Bf * wgt.reshape(N)[None, None, None, :] / Wv[..., None]
        M = np.einsum("cba,cbai,cbaj->ij", w3 * det, Rf, Rf)
    else:
        M = np.einsum("cba,cbai,cbaj->ij", w3 * det, Bf, Bf)
    S = np.zeros((N, N))
    for l in range(3):
        for m in range(3):
            S += np.einsum("cba,cbai,cbaj->ij", w3 * P[..., l, m], Gf[l], Gf[m])
    return S, M


def cardinal_bspline(m: int, x) -> np.ndarray:
    """Uniform cardinal B-spline N_m of degree m on [0, m+1] by its truncated-power
    closed form N_m(x) = (1/m!) sum_k (-1)^k C(m+1, k) (x - k)_+^m. Integer
    arguments are summed exactly in rational arithmetic (the alternating sum
    cancels badly in floating point at high degree)."""
    from fractions import Fraction
    xs = np.atleast_1d(np.asarray(x))
    out = np.empty(xs.shape, dtype=np.float64)
    for idx, xv in np.ndenumerate(xs):
        xv = Fraction(int(xv)) if float(xv).is_integer() else Fraction(float(xv))
        acc = Fraction(0)
        for k in range(m + 2):
            if xv > k:
                acc += (-1) ** k * math.comb(m + 1, k) * (xv - k) ** m
        out[idx] = float(acc / math.factorial(m))
    return out


# ---------------------------------------------------------------------------
# Adjoint of the bilinear forms (derivative of the WQ matrices; the paper has no
# adjoint). J = lambda^T A u with A = S, M or S + M assembled with kappa at the
# points; the gradients follow from writing the WQ entries out point by point.

def adjoint_fields(orc: "Oracle3D", lam: np.ndarray, u: np.ndarray) -> tuple:
    """U[m] (m = 0 value, 1..3 parametric derivatives of sum_j u_j B_j) and
    Lam[t] (t = 3l + m: sum_i lambda_i prod_k w^{(delta_kl, delta_km)}_{k,i_k}; t = 9:
    the (0,0) rules) at every point, arrays (nqp3, nqp2, nqp1), by einsum over the
    dense univariate tables."""
    n1, n2, n3 = orc.n
    L3 = np.asarray(lam, dtype=np.float64).reshape(n3, n2, n1)
    U3 = np.asarray(u, dtype=np.float64).reshape(n3, n2, n1)
    d = orc.dirs
    U = []
    for m in range(4):
        der = [int(k == m - 1) for k in range(3)]
        U.append(np.einsum("kji,ia,jb,kc->cba", U3, d[0].B[der[0]], d[1].B[der[1]], d[2].B[der[2]], optimize=True))
    Lam = []
    for t in range(10):
        if t < 9:
            l, m = divmod(t, 3)
            kinds = [(int(k == l), int(k == m)) for k in range(3)]
        else:
            kinds = [(0, 0)] * 3
        W = [d[k].W[kinds[k][0], kinds[k][1]] for k in range(3)]     # (n, nqp)
        Lam.append(np.einsum("kji,ia,jb,kc->cba", L3, W[0], W[1], W[2], optimize=True))
    return U, Lam


def adjoint(orc: "Oracle3D", lam, u, which: str = "stiffness", kappa=None) -> tuple:
    """(J, dJ/dkappa (nqp3, nqp2, nqp1), dJ/dC (N_DOF, 3)) for the oracle's geometry.
    orc.coef must hold the coefficients without kappa (kappa is passed here)."""
    U, Lam = adjoint_fields(orc, lam, u)
    kap = np.ones(orc.coef.shape[1:]) if kappa is None else np.asarray(kappa, dtype=np.float64).reshape(orc.coef.shape[1:])
    gk = np.zeros(orc.coef.shape[1:])
    Kb = np.zeros(orc.coef.shape[1:] + (3, 3))
    cb = np.zeros(orc.coef.shape[1:])
    if which in ("stiffness", "both"):
        for l in range(3):
            for m in range(3):
                lu = Lam[3 * l + m] * U[m + 1]
                gk += orc.coef[coef_index(l, m)] * lu
                Kb[..., l, m] = kap * lu
    if which in ("mass", "both"):
        lu = Lam[9] * U[0]
        gk += orc.coef[6] * lu
        cb = kap * lu
    J = float(np.sum(kap * gk))
    G = jacobians(orc.dirs, orc.ctrl)
    det = np.linalg.det(G)
    Gi = np.linalg.inv(G)
    GiT = np.swapaxes(Gi, -1, -2)
    P = Gi @ GiT
    KP = np.einsum("...ij,...ij->...", Kb, P)
    Ks = Kb + np.swapaxes(Kb, -1, -2)
    Gbar = det[..., None, None] * ((KP + cb)[..., None, None] * GiT - GiT @ Ks @ P)
    n1, n2, n3 = orc.n
    d = orc.dirs
    gc = np.zeros((n3, n2, n1, 3))
    for c in range(3):
        der = [int(k == c) for k in range(3)]
        gc += np.einsum("cbar,ia,jb,kc->kjir", Gbar[..., :, c], d[0].B[der[0]], d[1].B[der[1]], d[2].B[der[2]],
                        optimize=True)
    return J, gk, gc.reshape(-1, 3)
