"""Seeded synthetic polynomial systems.

This module only draws inputs; it holds none of the method's arithmetic, and both the CUDA
path (tests, benchmark) and the CPU oracle's tests take their inputs from it.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014): state advances by the golden gamma 0x9E3779B97F4A7C15 and
each output is the state passed through the variant-13 finaliser of MurmurHash3.  Integers in
a range are drawn by rejection, and N(0,1) variates by the Box-Muller transform in FP64.

The workloads stand in for the paper's random polynomial experiments (Sec. 4.1, Table 1:
dense random polynomials of total degree 20 and 100 in 2-4 variables, whose coefficients the
paper does not publish), with the sizes, degrees, domains and coefficient laws listed in
``CONFIGS`` below.
"""
from __future__ import annotations

import hashlib
import math
from dataclasses import dataclass, field

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
BASE_SEED = 240609857


def splitmix64(seed: int, n: int, start: int = 0) -> np.ndarray:
    """Outputs start+1 .. start+n of the SplitMix64 stream seeded with ``seed`` (uint64)."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


class Stream:
    """Sequential draws from one SplitMix64 stream."""

    def __init__(self, seed: int):
        self.seed = seed
        self.pos = 0

    def raw(self, n: int) -> np.ndarray:
        out = splitmix64(self.seed, n, self.pos)
        self.pos += n
        return out

    def uniform_int(self, lo: int, hi: int, n: int) -> np.ndarray:
        """n integers uniform in [lo, hi] (inclusive), by rejection of the top partial range."""
        r = hi - lo + 1
        limit = (1 << 64) - ((1 << 64) % r)
        out = np.empty(0, dtype=np.int64)
        while out.size < n:
            z = self.raw(max(n - out.size, 16))
            ok = z[z < np.uint64(limit)] if limit < (1 << 64) else z
            vals = (ok % np.uint64(r)).astype(np.int64) + lo
            out = np.concatenate([out, vals])
        return out[:n]

    def unit(self, n: int) -> np.ndarray:
        """n doubles uniform in [0, 1): the top 53 bits of each output."""
        return (self.raw(n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)

    def normal(self, n: int) -> np.ndarray:
        """n N(0,1) doubles by Box-Muller (cosine branch), one pair of uniforms per variate."""
        u1 = 1.0 - self.unit(n)  # (0, 1]
        u2 = self.unit(n)
        return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


def dense_total_degree(k: int, d: int) -> np.ndarray:
    """All exponent tuples with sum <= d, lexicographic order: int32 [C(d+k,k), k]."""
    out = []

    def rec(prefix, left):
        if len(prefix) == k:
            out.append(prefix)
            return
        for a in range(left + 1):
            rec(prefix + [a], left - a)

    rec([], d)
    return np.asarray(out, dtype=np.int32).reshape(-1, k)


def dense_per_variable(k: int, d: int) -> np.ndarray:
    """All exponent tuples with every entry <= d, lexicographic order: int32 [(d+1)^k, k]."""
    grids = np.meshgrid(*[np.arange(d + 1, dtype=np.int32)] * k, indexing="ij")
    return np.stack([g.reshape(-1) for g in grids], axis=1).astype(np.int32)


def kostlan_scale(exps: np.ndarray, d: int) -> np.ndarray:
    """sqrt(multinomial(d; d-|a|, a_1, ..., a_k)) per exponent tuple a, as doubles.

    The multinomial is an exact integer; its conversion to a double and the square root
    are each correctly rounded, so the scale is the same on every machine."""
    fact = [math.factorial(i) for i in range(d + 1)]
    out = np.empty(exps.shape[0], dtype=np.float64)
    for i, a in enumerate(exps.tolist()):
        s = sum(a)
        den = fact[d - s]
        for x in a:
            den *= fact[x]
        out[i] = math.sqrt(float(fact[d] // den))
    return out


def seed_for(config: int, system: int = 0, poly: int = 0) -> int:
    return BASE_SEED + 1000003 * config + 1009 * system + poly


def sha256(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


@dataclass
class System:
    """A polynomial system on a box domain, with the subdivision depth it is run to."""
    name: str
    k: int
    polys: list  # [(exps int32 [T, k], coefs float64 [T])]
    domain: np.ndarray  # float64 [2k]: lo, hi per axis
    depth: int
    meta: dict = field(default_factory=dict)
    # interval coefficients: his[f] (float64 [T]) the upper ends of polynomial f's coefficients
    # (None: point coefficients); rel[f]: 0 F = 0, 1 F <= 0, 2 F >= 0, 3 F < 0, 4 F > 0
    his: list = None
    rel: list = None

    @property
    def npoly(self) -> int:
        return len(self.polys)

    def digest(self) -> str:
        h = hashlib.sha256()
        for e, c in self.polys:
            h.update(np.ascontiguousarray(e).tobytes())
            h.update(np.ascontiguousarray(c).tobytes())
        h.update(np.ascontiguousarray(self.domain).tobytes())
        return h.hexdigest()


def cube(k: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    return np.asarray([lo, hi] * k, dtype=np.float64)


def uniform_int_poly(k: int, d: int, lo: int, hi: int, seed: int):
    e = dense_total_degree(k, d)
    c = Stream(seed).uniform_int(lo, hi, e.shape[0]).astype(np.float64)
    return e, c


def kostlan_poly(k: int, d: int, seed: int):
    e = dense_total_degree(k, d)
    c = Stream(seed).normal(e.shape[0]) * kostlan_scale(e, d)
    return e, c


def gaussian_tensor_poly(k: int, d: int, seed: int):
    e = dense_per_variable(k, d)
    c = Stream(seed).normal(e.shape[0])
    return e, c


def plain(depth: int = 8) -> System:
    """One bivariate polynomial of total degree 20, integer coefficients uniform in
    [-1000, 1000] stored as FP64, on [-1,1]^2, depth 8 (256x256 finest grid)."""
    return System("plain-k2-d20", 2, [uniform_int_poly(2, 20, -1000, 1000, seed_for(1))],
                  cube(2), depth)


def surface(depth: int = 9, d: int = 50) -> System:
    """One trivariate Kostlan polynomial of total degree 50 on [-1,1]^3, depth 9."""
    return System("surface-k3-d%d" % d, 3, [kostlan_poly(3, d, seed_for(2))], cube(3), depth)


def curve(depth: int = 10, d: int = 100) -> System:
    """Two trivariate Kostlan polynomials of total degree 100 on [-1,1]^3, depth 10."""
    return System("curve-k3-d%d" % d, 3,
                  [kostlan_poly(3, d, seed_for(3, 0, p)) for p in range(2)], cube(3), depth)


def batch(nsys: int = 256):
    """Independent systems of uneven degree and depth: half bivariate (1 polynomial, degree
    uniform in 10..60), half trivariate (2 polynomials, degree uniform in 10..40), Kostlan
    coefficients, depth uniform in 8..10."""
    out = []
    for s in range(nsys):
        st = Stream(seed_for(4, s, 99))
        depth = int(st.uniform_int(8, 10, 1)[0])
        if s < nsys // 2:
            d = int(st.uniform_int(10, 60, 1)[0])
            polys = [kostlan_poly(2, d, seed_for(4, s, 0))]
            k = 2
        else:
            d = int(st.uniform_int(10, 40, 1)[0])
            polys = [kostlan_poly(3, d, seed_for(4, s, p)) for p in range(2)]
            k = 3
        out.append(System("batch-%d-k%d-d%d" % (s, k, d), k, polys, cube(k), depth,
                          {"degree": d}))
    return out


def dense_sweep(d: int = 32) -> System:
    """One trivariate polynomial of degree d in each variable ((d+1)^3 coefficients, iid
    N(0,1)) on [-1,1]^3; evaluated on a full grid with no pruning."""
    return System("dense-k3-d%d" % d, 3, [gaussian_tensor_poly(3, d, seed_for(5, d))], cube(3), 0)


def uniform_real_poly(k: int, d: int, lo: float, hi: float, seed: int):
    """Dense total degree d, binary64 coefficients uniform in [lo, hi) (lo + (hi - lo) u)."""
    e = dense_total_degree(k, d)
    c = lo + (hi - lo) * Stream(seed).unit(e.shape[0])
    return e, c


# Depths of the random-polynomial family: boxes of [-2,2]^k no larger than 2^-8 for points
# and curves, 2^-5 for hypersurfaces (exclusion only, no inclusion test).
TABLE1_DEPTH = {"points": 10, "curves": 10, "hypersurfaces": 7}


def table1(k: int, d: int, kind: str) -> System:
    """The random-polynomial family of the experiments (Sec. 4.1): k variables, total degree
    d, coefficients uniform in [-10, 10], on [-2,2]^k; points = k equations, curves = k-1,
    hypersurfaces = 1."""
    npoly = {"points": k, "curves": k - 1, "hypersurfaces": 1}[kind]
    cell = 100 * k + d + {"points": 0, "curves": 1, "hypersurfaces": 2}[kind] * 1000
    polys = [uniform_real_poly(k, d, -10.0, 10.0, seed_for(6, cell, p)) for p in range(npoly)]
    return System("table1-%s-k%d-d%d" % (kind, k, d), k, polys, cube(k, -2.0, 2.0),
                  TABLE1_DEPTH[kind])


def random_small(k: int, d: int, npoly: int, seed: int, lo: int = -9, hi: int = 9,
                 density: float = 1.0):
    """Small dense-or-sparse integer polynomials for exhaustive tests."""
    st = Stream(seed)
    polys = []
    for _ in range(npoly):
        e = dense_total_degree(k, d)
        if density < 1.0:
            keep = st.unit(e.shape[0]) < density
            keep[0] = True
            e = e[keep]
        c = st.uniform_int(lo, hi, e.shape[0]).astype(np.float64)
        polys.append((e, c))
    return polys


def random_tuples(k: int, level: int, n: int, seed: int) -> np.ndarray:
    """Up to n distinct lex-sorted box indices of the level grid, drawn uniformly."""
    side = 1 << level
    total = side ** k
    st = Stream(seed)
    raw = st.uniform_int(0, total - 1, n)
    flat = np.unique(raw)
    out = np.empty((flat.size, k), dtype=np.int32)
    r = flat.copy()
    for c in range(k - 1, -1, -1):
        out[:, c] = r % side
        r //= side
    return out


# ---------------------------------------------------------------------------------------
# The two systems of Sec. 4.2, transcribed from the paper's displayed equations.
# ---------------------------------------------------------------------------------------
REL_EQ, REL_LE, REL_GE, REL_LT, REL_GT = 0, 1, 2, 3, 4

# (R): the parallel singularities of the 3-PPPS manipulator in quaternion coordinates
# Q1..Q4.  Terms of the first equation as (integer factor, 1 if multiplied by sqrt(3),
# exponents of Q1, Q2, Q3, Q4); the second equation is Q1^2 + Q2^2 + Q3^2 + Q4^2 = 1.
ROBOTICS_F1 = [
    (-6, 0, (1, 2, 1, 0)), (6, 0, (0, 1, 2, 1)), (3, 1, (0, 2, 1, 1)), (-6, 0, (2, 1, 0, 1)),
    (6, 0, (1, 0, 1, 2)), (-3, 1, (1, 1, 0, 2)), (3, 1, (1, 1, 2, 0)), (-3, 1, (2, 0, 1, 1)),
    (1, 1, (1, 3, 0, 0)), (-1, 1, (3, 1, 0, 0)), (1, 1, (0, 0, 3, 1)), (-1, 1, (0, 0, 1, 3)),
]

# (A): a control-design system in three complex variables z1, z2, z3 (no solution with
# |z_j| <= 1 is expected).  Terms as (integer coefficient, exponents of z1, z2, z3).
AUTOMATIC_Z = [
    [(1, (1, 2, 0)), (-1, (1, 0, 1)), (-2, (0, 0, 0))],
    [(12, (0, 3, 3)), (-2, (2, 1, 2)), (1, (0, 3, 2)), (-2, (0, 2, 3)), (-12, (0, 1, 4)),
     (2, (2, 0, 2)), (-1, (0, 1, 3)), (-2, (1, 1, 1)), (-7, (0, 3, 0)), (-10, (0, 2, 1)),
     (14, (1, 0, 1)), (-8, (0, 2, 0)), (9, (0, 1, 1)), (12, (0, 0, 2)), (30, (0, 0, 1)),
     (2, (0, 0, 0))],
    [(1, (3, 0, 3)), (1, (1, 1, 4)), (-1, (3, 0, 2)), (1, (1, 0, 4)), (-12, (0, 2, 3)),
     (-6, (2, 1, 1)), (3, (2, 0, 2)), (-1, (1, 1, 2)), (-1, (0, 2, 2)), (-10, (0, 1, 3)),
     (-7, (2, 0, 1)), (-12, (1, 1, 1)), (-2, (1, 0, 2)), (-1, (0, 1, 2)), (2, (0, 0, 3)),
     (-1, (1, 1, 0)), (-9, (1, 0, 1)), (7, (0, 2, 0)), (10, (0, 1, 1)), (-1, (1, 0, 0)),
     (15, (0, 1, 0)), (8, (0, 0, 1)), (8, (0, 0, 0))],
    [(1, (3, 1, 2)), (-1, (3, 0, 2)), (1, (1, 0, 4)), (1, (2, 1, 1)), (-12, (0, 1, 3)),
     (-7, (2, 0, 1)), (-1, (1, 1, 1)), (-1, (1, 0, 2)), (-1, (0, 1, 2)), (2, (0, 0, 3)),
     (-11, (1, 0, 1)), (-1, (1, 0, 0)), (7, (0, 1, 0)), (10, (0, 0, 1)), (8, (0, 0, 0))],
]


def sqrt_bounds(n: int, c: int):
    """The binary64 numbers next to c * sqrt(n) below and above (equal when exact)."""
    from fractions import Fraction
    import math

    t = Fraction(c * c * n)  # (c sqrt(n))^2
    x = math.sqrt(c * c * n)
    lo = x
    while lo > 0 and Fraction(lo) ** 2 > t:
        lo = math.nextafter(lo, 0.0)
    while Fraction(math.nextafter(lo, math.inf)) ** 2 <= t:
        lo = math.nextafter(lo, math.inf)
    hi = lo if Fraction(lo) ** 2 == t else math.nextafter(lo, math.inf)
    if c < 0:
        lo, hi = -hi, -lo
    return lo, hi


def robotics(depth: int = 6) -> System:
    """System (R) of Sec. 4.2 on [-1,1]^4 (each quaternion coordinate of a unit quaternion):
    the first equation's sqrt(3) coefficients become binary64 intervals [RD, RU]."""
    e = np.array([t[2] for t in ROBOTICS_F1], dtype=np.int32)
    lo = np.empty(len(ROBOTICS_F1))
    hi = np.empty(len(ROBOTICS_F1))
    for i, (c, r3, _) in enumerate(ROBOTICS_F1):
        lo[i], hi[i] = sqrt_bounds(3, c) if r3 else (float(c), float(c))
    sphere = (np.array([[2, 0, 0, 0], [0, 2, 0, 0], [0, 0, 2, 0], [0, 0, 0, 2], [0, 0, 0, 0]],
                       dtype=np.int32), np.array([1.0, 1.0, 1.0, 1.0, -1.0]))
    return System("robotics-R", 4, [(e, lo), sphere], cube(4), depth, his=[hi, None],
                  rel=[REL_EQ, REL_EQ])


def complex_to_real(terms, nz: int):
    """Real and imaginary parts of sum c z^a with z_j = x_j + i y_j, as polynomials in
    (x_1, y_1, ..., x_nz, y_nz) with exact integer coefficients: two dicts exps -> int."""
    from math import comb

    re, im = {}, {}
    for c, a in terms:
        # prod_j (x_j + i y_j)^{a_j} = sum over b_j <= a_j of prod C(a_j, b_j) x^(a-b) (i y)^b
        parts = [[]]
        for j in range(nz):
            parts = [p + [b] for p in parts for b in range(a[j] + 1)]
        for bs in parts:
            coef = c
            ex = []
            for j in range(nz):
                coef *= comb(a[j], bs[j])
                ex += [a[j] - bs[j], bs[j]]
            ipow = sum(bs) % 4  # i^sum(b)
            sgn = 1 if ipow in (0, 1) else -1
            tgt = re if ipow % 2 == 0 else im
            key = tuple(ex)
            tgt[key] = tgt.get(key, 0) + sgn * coef
    clean = [{k: v for k, v in d.items() if v != 0} for d in (re, im)]
    return clean[0], clean[1]


def _poly_of(d: dict, k: int):
    keys = sorted(d)
    e = np.array(keys, dtype=np.int32).reshape(-1, k)
    c = np.array([float(d[t]) for t in keys])
    return e, c


def automatic(depth: int = 8) -> System:
    """System (A) of Sec. 4.2 with z_j = x_j + i y_j: eight real equations (real and
    imaginary parts) and the three inequalities x_j^2 + y_j^2 - 1 <= 0, variables
    (x1, y1, x2, y2, x3, y3) on [-1,1]^6."""
    polys, rel = [], []
    for terms in AUTOMATIC_Z:
        re, im = complex_to_real(terms, 3)
        polys += [_poly_of(re, 6), _poly_of(im, 6)]
        rel += [REL_EQ, REL_EQ]
    for j in range(3):
        disk = {tuple(2 if i == 2 * j else 0 for i in range(6)): 1,
                tuple(2 if i == 2 * j + 1 else 0 for i in range(6)): 1, (0,) * 6: -1}
        polys.append(_poly_of(disk, 6))
        rel.append(REL_LE)
    return System("automatic-A", 6, polys, cube(6), depth, his=[None] * len(polys), rel=rel)
