"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds input generation only: knot vectors, control nets and random
fields. It contains none of the weighted-quadrature arithmetic (no basis
evaluation, no quadrature, no solves, no assembly), so the CUDA path and the
CPU oracle can both draw their inputs from it without sharing method code.

Workloads follow the single-patch cube tests of the paper (Section 7.2): open
knot vectors with simple interior knots (maximal C^{p-1} regularity, Section 3)
on [0,1] in each direction, and a degree-p spline map whose control points sit
at the Greville abscissae of the knot vector, each coordinate perturbed by a
seeded uniform draw in [-amp*h, amp*h] with h = 1/n_el.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): state += 0x9E3779B97F4A7C15,
then two xor-shift-multiply rounds. Uniforms use the top 53 bits. Normals use
the Box-Muller transform.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 generator producing uint64 words, 53-bit uniforms and normals."""

    def __init__(self, seed: int):
        self.state = seed & _MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        return z ^ (z >> 31)

    def uniforms(self, count: int) -> np.ndarray:
        """`count` doubles in [0, 1): the top 53 bits of each word times 2^-53."""
        return _splitmix_uniform_block(self, count)

    def normals(self, count: int) -> np.ndarray:
        """`count` N(0,1) doubles by Box-Muller on pairs of uniforms."""
        m = (count + 1) // 2
        u = self.uniforms(2 * m)
        u1 = 1.0 - u[0::2]          # (0, 1]
        u2 = u[1::2]
        r = np.sqrt(-2.0 * np.log(u1))
        z = np.empty(2 * m)
        z[0::2] = r * np.cos(2.0 * math.pi * u2)
        z[1::2] = r * np.sin(2.0 * math.pi * u2)
        return z[:count]


def _splitmix_uniform_block(gen: SplitMix64, count: int) -> np.ndarray:
    # Vectorised SplitMix64: word k uses state s0 + (k+1)*gamma (mod 2^64).
    if count <= 0:
        return np.zeros(0)
    gamma = np.uint64(0x9E3779B97F4A7C15)
    k = np.arange(1, count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(gen.state) + k * gamma
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    gen.state = (gen.state + count * 0x9E3779B97F4A7C15) & _MASK64
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform_breaks(n_el: int, a: float = 0.0, b: float = 1.0) -> np.ndarray:
    """n_el + 1 equally spaced distinct knots on [a, b]."""
    return np.linspace(a, b, n_el + 1)


def open_knot_vector(breaks: np.ndarray, p: int) -> np.ndarray:
    """Full open knot vector: end knots repeated p+1 times, interior knots simple."""
    breaks = np.asarray(breaks, dtype=np.float64)
    return np.concatenate([np.full(p, breaks[0]), breaks, np.full(p, breaks[-1])])


def greville(knot_vector: np.ndarray, p: int) -> np.ndarray:
    """Greville abscissae (xi_{i+1} + ... + xi_{i+p}) / p of a full knot vector."""
    xi = np.asarray(knot_vector, dtype=np.float64)
    n = len(xi) - p - 1
    return np.array([xi[i + 1:i + p + 1].sum() / p for i in range(n)])


@dataclass
class Patch:
    """One single-patch spline cube: degree, three full knot vectors, control net.

    ctrl has shape (N_DOF, 3), xyz per control point, linear index
    i1 + n1*(i2 + n2*i3) (direction 1 fastest, as in Section 3).
    """
    p: int
    knots: list                      # three float64 arrays (full open knot vectors)
    ctrl: np.ndarray                 # (N_DOF, 3) float64
    name: str = ""
    meta: dict = field(default_factory=dict)
    weights: np.ndarray | None = None  # (N_DOF,) NURBS weights, or None for a B-spline map

    @property
    def n(self) -> tuple:
        return tuple(len(k) - self.p - 1 for k in self.knots)

    @property
    def n_el(self) -> tuple:
        return tuple(len(np.unique(k)) - 1 for k in self.knots)

    @property
    def n_dof(self) -> int:
        n1, n2, n3 = self.n
        return n1 * n2 * n3


def greville_net(knots: list, p: int) -> np.ndarray:
    """Control points at the Greville abscissae (the identity map of [0,1]^3)."""
    g = [greville(k, p) for k in knots]
    g3, g2, g1 = np.meshgrid(g[2], g[1], g[0], indexing="ij")
    return np.stack([g1.ravel(), g2.ravel(), g3.ravel()], axis=1)


def perturbed_cube(p: int, n_el, seed: int, amp: float = 0.05,
                   breaks: list | None = None) -> Patch:
    """Greville control net of [0,1]^3 plus seeded U[-amp*h, amp*h] per coordinate.

    n_el is an int or a 3-tuple. h = 1/n_el of the direction of each coordinate's
    own axis is not used: the perturbation of every coordinate uses
    h = 1/max(n_el), the smallest span of a uniform cube.
    """
    if isinstance(n_el, int):
        n_el = (n_el, n_el, n_el)
    if breaks is None:
        breaks = [uniform_breaks(e) for e in n_el]
    knots = [open_knot_vector(b, p) for b in breaks]
    ctrl = greville_net(knots, p)
    h = 1.0 / max(n_el)
    if amp != 0.0:
        gen = SplitMix64(seed)
        ctrl = ctrl + (2.0 * gen.uniforms(ctrl.size).reshape(ctrl.shape) - 1.0) * (amp * h)
    return Patch(p=p, knots=knots, ctrl=np.ascontiguousarray(ctrl),
                 name=f"cube_p{p}_nel{'x'.join(map(str, n_el))}_seed{seed}",
                 meta={"seed": seed, "amp": amp, "n_el": tuple(n_el)})


def affine_cube(p: int, n_el, A: np.ndarray, b: np.ndarray,
                breaks: list | None = None) -> Patch:
    """Affine image x -> A x + b of the Greville net (exact for any p >= 1)."""
    if isinstance(n_el, int):
        n_el = (n_el, n_el, n_el)
    if breaks is None:
        breaks = [uniform_breaks(e) for e in n_el]
    knots = [open_knot_vector(bb, p) for bb in breaks]
    ctrl = greville_net(knots, p) @ np.asarray(A, dtype=np.float64).T + np.asarray(b, dtype=np.float64)
    return Patch(p=p, knots=knots, ctrl=np.ascontiguousarray(ctrl),
                 name=f"affine_p{p}_nel{'x'.join(map(str, n_el))}", meta={"A": A, "b": b})


def graded_breaks(n_el: int, seed: int, spread: float = 0.5) -> np.ndarray:
    """Strictly increasing non-uniform distinct knots on [0,1] (seeded spans)."""
    gen = SplitMix64(seed)
    w = 1.0 + spread * (2.0 * gen.uniforms(n_el) - 1.0)
    x = np.concatenate([[0.0], np.cumsum(w)])
    return x / x[-1]


# ---------------------------------------------------------------------------
# Rational (NURBS) geometries. Control points and weights are built in
# homogeneous coordinates (w x, w y, w z, w), where degree elevation and knot
# insertion are the B-spline ones; they change the representation, not the map.

def _elevate_bezier(Pw: np.ndarray) -> np.ndarray:
    """One degree elevation of a Bezier curve (rows = homogeneous control points):
    Q_0 = P_0, Q_i = (i/(k+1)) P_{i-1} + (1 - i/(k+1)) P_i, Q_{k+1} = P_k."""
    k = len(Pw) - 1
    Q = np.empty((k + 2, Pw.shape[1]))
    Q[0], Q[k + 1] = Pw[0], Pw[k]
    for i in range(1, k + 1):
        a = i / (k + 1)
        Q[i] = a * Pw[i - 1] + (1.0 - a) * Pw[i]
    return Q


def _insert_knot(U: np.ndarray, Pw: np.ndarray, p: int, u: float) -> tuple:
    """Insert knot u once into knot vector U of degree p (Boehm): the points of the
    p spans around u become convex combinations of their neighbours."""
    k = int(np.searchsorted(U, u, side="right") - 1)        # U[k] <= u < U[k+1]
    n = len(Pw)
    Q = np.empty((n + 1, Pw.shape[1]))
    for i in range(n + 1):
        if i <= k - p:
            Q[i] = Pw[i]
        elif i >= k + 1:
            Q[i] = Pw[i - 1]
        else:
            a = (u - U[i]) / (U[i + p] - U[i])
            Q[i] = (1.0 - a) * Pw[i - 1] + a * Pw[i]
    return np.insert(U, k + 1, u), Q


def refined_curve(values, p: int, n_el: int) -> tuple:
    """A degree-p spline curve fixed on one span (Bezier control values `values`, p+1
    of them, shape (p+1,) or (p+1, k)) and refined by knot insertion to n_el uniform
    spans with simple knots: the same curve on every mesh. Returns (knots, control values)."""
    P = np.asarray(values, dtype=np.float64)
    P = P.reshape(p + 1, -1)
    U = np.concatenate([np.zeros(p + 1), np.ones(p + 1)])
    for e in range(1, n_el):
        U, P = _insert_knot(U, P, p, e / n_el)
    return U, P if np.asarray(values).ndim > 1 else P[:, 0]


def quarter_arc(p: int, n_el: int) -> tuple:
    """The quarter of the unit circle from (1, 0) to (0, 1) as a degree-p NURBS curve
    with n_el uniform spans and simple interior knots: the rational quadratic arc
    (control points (1,0), (1,1), (0,1), weights 1, 1/sqrt(2), 1), degree-elevated
    and refined. Returns (open knot vector, (n, 2) control points, (n,) weights)."""
    w1 = math.sqrt(0.5)
    Pw = np.array([[1.0, 0.0, 1.0], [w1, w1, w1], [0.0, 1.0, 1.0]])
    for _ in range(p - 2):
        Pw = _elevate_bezier(Pw)
    U = np.concatenate([np.zeros(p + 1), np.ones(p + 1)])
    for e in range(1, n_el):
        U, Pw = _insert_knot(U, Pw, p, e / n_el)
    return U, Pw[:, :2] / Pw[:, 2:3], Pw[:, 2].copy()


def quarter_annulus(p: int, n_el, r_in: float = 1.0, r_out: float = 2.0, height: float = 1.0) -> Patch:
    """Thick quarter annulus {r_in <= sqrt(x^2 + y^2) <= r_out, x, y >= 0, 0 <= z <= height}
    as a degree-p NURBS solid: direction 1 radial and direction 3 vertical (linear,
    Greville control points, weight 1), direction 2 the circular arc of quarter_arc.
    Every point of the map lies on the circle of radius r_in + (r_out - r_in) zeta_1."""
    if isinstance(n_el, int):
        n_el = (n_el, n_el, n_el)
    U, arc, wa = quarter_arc(p, n_el[1])
    k1 = open_knot_vector(uniform_breaks(n_el[0]), p)
    k3 = open_knot_vector(uniform_breaks(n_el[2]), p)
    r = r_in + (r_out - r_in) * greville(k1, p)
    z = height * greville(k3, p)
    n1, n2, n3 = len(r), len(wa), len(z)
    i3, i2, i1 = np.meshgrid(np.arange(n3), np.arange(n2), np.arange(n1), indexing="ij")
    ctrl = np.stack([r[i1] * arc[i2, 0], r[i1] * arc[i2, 1], z[i3]], axis=-1).reshape(-1, 3)
    weights = wa[i2].reshape(-1).astype(np.float64)
    return Patch(p=p, knots=[k1, U, k3], ctrl=np.ascontiguousarray(ctrl), weights=np.ascontiguousarray(weights),
                 name=f"annulus_p{p}_nel{'x'.join(map(str, n_el))}",
                 meta={"r_in": r_in, "r_out": r_out, "height": height,
                       "volume": 0.25 * math.pi * (r_out ** 2 - r_in ** 2) * height})


def perturbed_nurbs_cube(p: int, n_el, seed: int, amp: float = 0.05, wspread: float = 0.3) -> Patch:
    """perturbed_cube with seeded NURBS weights U[1 - wspread, 1 + wspread] on every
    control point (a general rational map, weights not of tensor-product form)."""
    patch = perturbed_cube(p, n_el, seed=seed, amp=amp)
    gen = SplitMix64(seed + 7919)
    patch.weights = 1.0 + wspread * (2.0 * gen.uniforms(patch.n_dof) - 1.0)
    patch.name = patch.name.replace("cube", "nurbs_cube")
    return patch


def random_spd_field(count: int, seed: int, spread: float = 0.5) -> np.ndarray:
    """(6, count) symmetric positive-definite 3x3 tensors K = L L^T + (1 - spread) I with
    L lower triangular, entries U[-spread, spread] (components K11 K12 K13 K22 K23 K33)."""
    gen = SplitMix64(seed)
    u = spread * (2.0 * gen.uniforms(6 * count).reshape(6, count) - 1.0)
    L = np.zeros((count, 3, 3))
    L[:, 0, 0], L[:, 1, 0], L[:, 2, 0], L[:, 1, 1], L[:, 2, 1], L[:, 2, 2] = u
    K = np.einsum("nik,njk->nij", L, L) + (1.0 - spread) * np.eye(3)[None]
    return np.stack([K[:, 0, 0], K[:, 0, 1], K[:, 0, 2], K[:, 1, 1], K[:, 1, 2], K[:, 2, 2]])


# ---------------------------------------------------------------------------
# Named workloads. Seed = 1605 + workload index.

def workload_small() -> Patch:
    """p=2, 16 elements per direction (N_DOF = 18^3 = 5832): stiffness + mass."""
    return perturbed_cube(2, 16, seed=1605 + 0)


def workload_p4_64() -> Patch:
    """p=4, 64 elements per direction (N_DOF = 68^3 = 314432): stiffness."""
    return perturbed_cube(4, 64, seed=1605 + 1)


def workload_sweep(p: int) -> Patch:
    """Degree sweep at about 1M DOF: n_el = 101 - p per direction."""
    return perturbed_cube(p, 101 - p, seed=1605 + 2)


def workload_p5_128() -> Patch:
    """p=5, 128 elements per direction (N_DOF = 133^3 = 2352637)."""
    return perturbed_cube(5, 128, seed=1605 + 3)


def workload_batch(count: int = 64, seed: int = 1605 + 4, nel_lo: int = 8,
                   nel_hi: int = 48, degrees=(2, 3, 4, 5)) -> list:
    """`count` cubes with seeded n_el in [nel_lo, nel_hi]^3 and p drawn from `degrees`."""
    gen = SplitMix64(seed)
    patches = []
    for k in range(count):
        u = gen.uniforms(4)
        p = int(degrees[min(int(u[0] * len(degrees)), len(degrees) - 1)])
        n_el = tuple(int(nel_lo + min(int(v * (nel_hi - nel_lo + 1)), nel_hi - nel_lo)) for v in u[1:])
        patches.append(perturbed_cube(p, n_el, seed=seed * 1000 + k))
    return patches


def sample_rows(n: tuple, p: int, count: int, seed: int) -> np.ndarray:
    """Seeded row indices (linear, i1 fastest), with one row of each of the 27
    boundary/interior classes forced in (per direction: i < p, p <= i < n-p, i >= n-p)."""
    n1, n2, n3 = n
    forced = []
    def pick(nl, cls):
        if cls == 0:
            return 0 if nl > 0 else 0
        if cls == 1:
            return nl // 2
        return nl - 1
    seen = set()
    for c3 in range(3):
        for c2 in range(3):
            for c1 in range(3):
                i1, i2, i3 = pick(n1, c1), pick(n2, c2), pick(n3, c3)
                r = i1 + n1 * (i2 + n2 * i3)
                if r not in seen:
                    seen.add(r)
                    forced.append(r)
    # near-boundary rows with partial bands (i = 1 .. p) in every direction
    for k in range(1, p + 1):
        for (i1, i2, i3) in ((k, k, k), (n1 - 1 - k, n2 - 1 - k, n3 - 1 - k)):
            if 0 <= i1 < n1 and 0 <= i2 < n2 and 0 <= i3 < n3:
                r = i1 + n1 * (i2 + n2 * i3)
                if r not in seen:
                    seen.add(r)
                    forced.append(r)
    n_rows = n1 * n2 * n3
    rest = max(0, count - len(forced))
    if rest:
        gen = SplitMix64(seed)
        extra = (gen.uniforms(rest) * n_rows).astype(np.int64)
        for r in extra.tolist():
            if r not in seen:
                seen.add(r)
                forced.append(r)
    return np.array(sorted(forced[:max(count, 27)]), dtype=np.int64)


def random_field(count: int, seed: int, kind: str = "normal") -> np.ndarray:
    """Seeded N(0,1) (kind='normal') or U[0.5,1.5] (kind='positive') doubles."""
    gen = SplitMix64(seed)
    if kind == "normal":
        return gen.normals(count)
    if kind == "positive":
        return 0.5 + gen.uniforms(count)
    raise ValueError(kind)
