"""Correctly rounded sine / cosine of angles given in degrees (oracle side).

Test infrastructure only (see ``oracle/__init__.py``).

The paper builds the displacement arrays D_a[i][j] = i sin j and
D_b[i][j] = i cos j (§2 Methods, Fig. 2) without fixing the unit of j or how the
sine is evaluated.  The reading taken here: j is in degrees, and the table
entry is the double nearest to the real sin(j * pi/180) (resp. cos).  The angle
is reduced to [0, 90] with exact rational arithmetic, so sin(j + 180) is the
exact negation of sin(j) - the point symmetry of the pair (§2 Methods) then
holds bit for bit.  Values are computed with ``decimal`` at 80 digits and
rounded once; the rounding is certified by checking the distance to the nearest
rounding boundary.
"""
from __future__ import annotations

import math
from decimal import Decimal, localcontext
from fractions import Fraction

_PREC = 80


def _atan_inv(n: int) -> Decimal:
    """atan(1/n) by its alternating series."""
    x = Decimal(1) / n
    x2 = x * x
    term, total, k = x, x, 1
    eps = Decimal(10) ** -(_PREC + 5)
    while True:
        term *= -x2
        k += 2
        t = term / k
        if abs(t) < eps:
            return total
        total += t


def _pi() -> Decimal:
    """pi from Machin's formula: pi = 16 atan(1/5) - 4 atan(1/239)."""
    return 16 * _atan_inv(5) - 4 * _atan_inv(239)


def _sin_series(x: Decimal) -> Decimal:
    term, total, k = x, x, 1
    x2 = x * x
    eps = Decimal(10) ** -(_PREC + 5)
    while abs(term) > eps:
        term = -term * x2 / ((k + 1) * (k + 2))
        k += 2
        total += term
    return total


def _to_double_certified(v: Decimal) -> float:
    """Round a high-precision Decimal to the nearest double; fail if too close
    to a rounding boundary for the rounding to be certain."""
    fr = Fraction(v)
    d = fr.numerator / fr.denominator
    if v != 0:
        up, dn = math.nextafter(d, math.inf), math.nextafter(d, -math.inf)
        for nb in (up, dn):
            mid = (Fraction(d) + Fraction(nb)) / 2
            if abs(fr - mid) < abs(fr) * Fraction(1, 10 ** (_PREC - 10)):
                raise ArithmeticError("sine value too close to a rounding boundary")
    return d


def _sin_first_quadrant(theta: Fraction, pi: Decimal) -> float:
    """RN(sin(theta degrees)) for an exact rational theta in [0, 90]."""
    if theta == 0:
        return 0.0
    if theta == 90:
        return 1.0
    if theta == 30:
        return 0.5
    with localcontext() as ctx:
        ctx.prec = _PREC
        x = Decimal(theta.numerator) / Decimal(theta.denominator) * pi / 180
        return _to_double_certified(_sin_series(x))


def sin_cos_deg(angle_deg: float) -> tuple[float, float]:
    """(RN(sin(angle)), RN(cos(angle))) for an angle in degrees (any finite double)."""
    if not math.isfinite(angle_deg):
        raise ValueError("angle must be finite")
    with localcontext() as ctx:
        ctx.prec = _PREC
        pi = _pi()
    t = Fraction(angle_deg) % 360  # exact, in [0, 360)

    def sin_exact(th: Fraction) -> float:
        th = th % 360
        if th <= 90:
            return _sin_first_quadrant(th, pi)
        if th <= 180:
            return _sin_first_quadrant(180 - th, pi)
        if th <= 270:
            return -_sin_first_quadrant(th - 180, pi)
        return -_sin_first_quadrant(360 - th, pi)

    s = sin_exact(t)
    c = sin_exact(90 - t)  # cos(t) = sin(90 - t), exact in rationals
    return s, c


def trig_table(angles_deg) -> tuple[list[float], list[float]]:
    """Sine and cosine tables for a list of angles in degrees."""
    cache: dict[float, tuple[float, float]] = {}
    sins, coss = [], []
    for a in angles_deg:
        a = float(a)
        if a not in cache:
            cache[a] = sin_cos_deg(a)
        s, c = cache[a]
        sins.append(s)
        coss.append(c)
    return sins, coss
