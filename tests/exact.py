"""Exact rational helpers for pinning the oracle (Python ``fractions``; no oracle code)."""
import math
from fractions import Fraction


def rd(q: Fraction) -> float:
    """Largest double <= q."""
    x = float(q)  # int / int true division is correctly rounded
    if Fraction(x) > q:
        x = math.nextafter(x, -math.inf)
    return x


def ru(q: Fraction) -> float:
    """Smallest double >= q."""
    x = float(q)
    if Fraction(x) < q:
        x = math.nextafter(x, math.inf)
    return x


def poly_value(exps, coefs, point):
    """Exact value of sum_t coefs[t] * prod_i point[i]^exps[t][i] (point: Fractions)."""
    s = Fraction(0)
    for e, c in zip(exps, coefs):
        term = Fraction(c)
        for x, a in zip(point, e):
            term *= x ** int(a)
        s += term
    return s


def grid_box(domain, level, tup):
    """Exact closed box [lo_i + t w_i, lo_i + (t+1) w_i] of the level grid (Fractions)."""
    out = []
    for i, t in enumerate(tup):
        lo, hi = Fraction(domain[2 * i]), Fraction(domain[2 * i + 1])
        w = (hi - lo) / (1 << level)
        out.append((lo + int(t) * w, lo + (int(t) + 1) * w))
    return out
