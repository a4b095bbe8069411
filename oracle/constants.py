"""Exact colour-science constants for the FP64 oracle.

Test infrastructure only: nothing outside ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` leg of ``bench.py`` may import this package.

The paper (§2 Methods, Fig. 1b, Fig. 2) converts RGB to CIE L*a*b* and back
but prints no constant.  The reading taken here is sRGB (IEC 61966-2-1) with a
D65 white, written out with exact rational arithmetic so that every table is
the correctly rounded double of its real value and is the same on every host:

* ``M``      - the IEC linear-RGB -> XYZ matrix, each entry the double nearest
               to its 4-digit decimal.
* ``W``      - the white point, ``M @ (1,1,1)`` summed left to right in IEEE
               double, so that RGB (255,255,255) maps to L*=100, a*=b*=0.
* ``MI``     - the exact inverse of the double-valued ``M``, each entry rounded
               to nearest.
* ``LUT``    - 8-bit sRGB decode: ``LUT[c]`` = RN(dec(c/255)).
* ``THR``    - quantisation thresholds: ``THR[k+1]`` = RU(dec*((k+0.5)/255)) for
               k = -1..255, the smallest double whose encoded value reaches the
               rounding boundary between codes k and k+1.  Hence, for any double
               ``lin``, ``q = #{t in THR : t <= lin} - 1`` equals
               ``floor(255*enc(lin) + 1/2)`` evaluated in exact real arithmetic
               (clamped to [-1, 256]).
* CIE f() constants: ``DELTA = 6/29``; branch points are compared exactly
  against the real breakpoints; linear-branch factors are rounded to nearest.

Every value is produced by integer / Fraction arithmetic (including the 2.4
power, evaluated as an exact integer 5th root of a 12th power), never by libm.
"""
from __future__ import annotations

import math
from fractions import Fraction
from functools import lru_cache

# IEC 61966-2-1 linear-RGB -> XYZ (D65), 4-digit decimals.
_M_DEC = (
    ("0.4124", "0.3576", "0.1805"),
    ("0.2126", "0.7152", "0.0722"),
    ("0.0193", "0.1192", "0.9505"),
)


# ---------------------------------------------------------------- rounding
def _rn(x: Fraction) -> float:
    """Round an exact rational to the nearest double (ties to even)."""
    return x.numerator / x.denominator  # CPython int/int division is correctly rounded


def _next_up(x: float) -> float:
    return math.nextafter(x, math.inf)


def _next_down(x: float) -> float:
    return math.nextafter(x, -math.inf)


def _ru(x: Fraction) -> float:
    """Smallest double >= x."""
    d = _rn(x)
    return d if Fraction(d) >= x else _next_up(d)


def _rd(x: Fraction) -> float:
    """Largest double <= x."""
    d = _rn(x)
    return d if Fraction(d) <= x else _next_down(d)


def iroot(n: int, k: int) -> int:
    """floor(n ** (1/k)) for an integer n >= 0, by integer Newton iteration."""
    if n < 0:
        raise ValueError("negative radicand")
    if n < 2:
        return n
    x = 1 << ((n.bit_length() + k - 1) // k)
    while True:
        y = ((k - 1) * x + n // x ** (k - 1)) // k
        if y >= x:
            break
        x = y
    while x ** k > n:
        x -= 1
    while (x + 1) ** k <= n:
        x += 1
    return x


def pow_12_5(p: int, q: int, mode: str) -> float:
    """(p/q)**(12/5) rounded to a double: mode 'rn' (nearest-even) or 'ru' (up).

    With s chosen so that 2**52 <= y*2**s < 2**53, floor(y*2**(s+1)) is the
    integer 5th root of floor(p**12 * 2**(5(s+1)) / q**12); exactness is known
    by raising the root back to the 5th power.
    """
    assert p > 0 and q > 0
    approx = (p / q) ** 2.4
    e = math.frexp(approx)[1] - 1  # approx in [2**e, 2**(e+1))
    num12, den12 = p ** 12, q ** 12
    for _ in range(4):
        s = 52 - e
        sh = 5 * (s + 1)
        if sh >= 0:
            a, b = num12 << sh, den12
        else:
            a, b = num12, den12 << (-sh)
        n2 = iroot(a // b, 5)  # floor(y * 2**(s+1))
        if n2 >= (1 << 54):
            e += 1
            continue
        if n2 < (1 << 53):
            e -= 1
            continue
        exact2 = n2 ** 5 * b == a
        break
    else:  # pragma: no cover
        raise RuntimeError("exponent search failed")
    n, half = n2 >> 1, n2 & 1
    if mode == "ru":
        inexact = half == 1 or not exact2
        m = n + 1 if inexact else n
    elif mode == "rn":
        if half == 0:
            m = n
        elif not exact2:
            m = n + 1
        else:  # exact tie
            m = n + (n & 1)
    else:
        raise ValueError(mode)
    return math.ldexp(m, -s)


# ---------------------------------------------------------------- tables
@lru_cache(maxsize=1)
def matrices():
    """(M, W, MI) as tuples of floats; M, MI row-major 3x3, W length 3."""
    M = tuple(tuple(float(v) for v in row) for row in _M_DEC)
    W = tuple((row[0] + row[1]) + row[2] for row in M)  # IEEE double, left to right
    F = [[Fraction(v) for v in row] for row in M]
    det = (F[0][0] * (F[1][1] * F[2][2] - F[1][2] * F[2][1])
           - F[0][1] * (F[1][0] * F[2][2] - F[1][2] * F[2][0])
           + F[0][2] * (F[1][0] * F[2][1] - F[1][1] * F[2][0]))
    cof = [[None] * 3 for _ in range(3)]
    for i in range(3):
        for j in range(3):
            r = [x for x in range(3) if x != i]
            c = [x for x in range(3) if x != j]
            minor = F[r[0]][c[0]] * F[r[1]][c[1]] - F[r[0]][c[1]] * F[r[1]][c[0]]
            cof[i][j] = minor if (i + j) % 2 == 0 else -minor
    inv = [[cof[j][i] / det for j in range(3)] for i in range(3)]  # adjugate / det
    MI = tuple(tuple(_rn(inv[i][j]) for j in range(3)) for i in range(3))
    return M, W, MI


def _dec_exact_linear(num: int, den: int) -> Fraction:
    """Linear branch of the sRGB decode at y = num/den: y / 12.92."""
    return Fraction(num, den) / Fraction(1292, 100)


@lru_cache(maxsize=1)
def srgb_decode_lut():
    """LUT[c] = RN(dec(c/255)), c = 0..255 (IEC 61966-2-1 decode).

    dec(y) = y/12.92 for y <= 0.04045, else ((y+0.055)/1.055)**2.4.
    c/255 <= 0.04045 exactly for c <= 10.  For c >= 11,
    (c/255 + 0.055)/1.055 = (40c + 561)/10761.
    """
    out = []
    for c in range(256):
        if Fraction(c, 255) <= Fraction(4045, 100000):
            out.append(_rn(_dec_exact_linear(c, 255)))
        else:
            out.append(pow_12_5(40 * c + 561, 10761, "rn"))
    return tuple(out)


@lru_cache(maxsize=1)
def quant_thresholds():
    """THR[k+1] = RU(dec*((k+1/2)/255)) for k = -1..255 (257 values, increasing).

    At y = (2k+1)/510: y <= 0.04045 for k <= 9 (linear branch, including the
    negative k = -1); for k >= 10, (y+0.055)/1.055 = (40k+581)/10761.  No
    boundary falls inside the small jump of the sRGB encode at 0.0031308.
    """
    out = []
    for k in range(-1, 256):
        y = Fraction(2 * k + 1, 510)
        if y <= Fraction(4045, 100000):
            out.append(_ru(_dec_exact_linear(2 * k + 1, 510)))
        else:
            out.append(pow_12_5(40 * k + 581, 10761, "ru"))
    return tuple(out)


@lru_cache(maxsize=1)
def cie_constants():
    """Scalars of the CIE f() / f^-1() pair with DELTA = 6/29.

    f(t)    = cbrt(t)                  if t > DELTA**3
            = t * F_LIN_MUL + F_LIN_ADD  otherwise   (t/(3 DELTA^2) + 4/29)
    finv(u) = (u*u)*u                  if u > DELTA
            = (u - F_LIN_ADD) * FINV_LIN_MUL   otherwise (3 DELTA^2 (u - 4/29))
    The branch tests compare a double against the exact real breakpoint, which
    for a double t is the same as comparing against RD(breakpoint).
    """
    delta = Fraction(6, 29)
    return {
        "F_BREAK": _rd(delta ** 3),          # t > F_BREAK  <=>  t > (6/29)^3
        "FINV_BREAK": _rd(delta),            # u > FINV_BREAK <=> u > 6/29
        "F_LIN_MUL": _rn(1 / (3 * delta ** 2)),   # 841/108
        "F_LIN_ADD": _rn(Fraction(4, 29)),
        "FINV_LIN_MUL": _rn(3 * delta ** 2),      # 108/841
    }


def quantize_ref(lin: float) -> int:
    """floor(255*enc(lin) + 1/2) from the threshold table, clamped to [-1, 256]."""
    thr = quant_thresholds()
    lo, hi = 0, len(thr)
    while lo < hi:  # number of thresholds <= lin
        mid = (lo + hi) // 2
        if thr[mid] <= lin:
            lo = mid + 1
        else:
            hi = mid
    return lo - 1
