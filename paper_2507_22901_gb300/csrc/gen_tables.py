"""Generate cvs_tables.h: the FP64 constant tables of libcvsearch.

Run from the repository root after changing a definition:
    python paper_2507_22901_gb300/csrc/gen_tables.py

The paper converts RGB to L*a*b* and back (§2 Methods, Fig. 2) without giving
constants; the library takes sRGB (IEC 61966-2-1) with a D65 white.  Each table
entry is the correctly rounded double of a real number defined below, computed
here with exact rationals and integer roots, so the header is host independent:

  CVS_M[9], CVS_W[3]   sRGB linear->XYZ matrix (nearest doubles to the 4-digit
                        entries) and white = M*(1,1,1) summed left to right
  CVS_MI[9]            XYZ->linear matrix: nearest doubles to the exact inverse
                        of the double-valued M
  CVS_DECODE[256]      8-bit decode: nearest double to dec(c/255)
  CVS_QTHR[257]        CVS_QTHR[q] = least double x with 255*enc(x) >= q - 1/2,
                        q = 0..256, so code(x) = #{q : CVS_QTHR[q] <= x} - 1
  CIE f/finv scalars    breakpoints rounded down (so `x > bp` is exact),
                        linear-branch factors rounded to nearest
  CVS_PI180_HI/LO       pi/180 as a double-double
  CVS_SIN_C/CVS_COS_C   double-double Taylor coefficients (-1)^n/(2n+1)!, (-1)^n/(2n)!
"""
from __future__ import annotations

import math
import os
from decimal import Decimal, getcontext
from fractions import Fraction

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cvs_tables.h")

M_TEXT = [["0.4124", "0.3576", "0.1805"],
          ["0.2126", "0.7152", "0.0722"],
          ["0.0193", "0.1192", "0.9505"]]


def nearest(q: Fraction) -> float:
    return q.numerator / q.denominator  # exact int/int division rounds once, to nearest


def round_up(q: Fraction) -> float:
    d = nearest(q)
    return math.nextafter(d, math.inf) if Fraction(d) < q else d


def round_down(q: Fraction) -> float:
    d = nearest(q)
    return math.nextafter(d, -math.inf) if Fraction(d) > q else d


def kth_root_floor(n: int, k: int) -> int:
    """Largest integer x with x**k <= n (bisection on integers)."""
    lo, hi = 0, 1 << (n.bit_length() // k + 2)
    while lo < hi:
        mid = (lo + hi + 1) // 2
        if mid ** k <= n:
            lo = mid
        else:
            hi = mid - 1
    return lo


def rational_pow_2_4(num: int, den: int, up: bool) -> float:
    """(num/den)**2.4 = ((num/den)**12)**(1/5), rounded to nearest or up."""
    target = Fraction(num, den) ** 12  # y**5 == target
    guess = nearest(Fraction(num, den)) ** 2.4
    exp = math.frexp(guess)[1]          # y in [2**(exp-1), 2**exp) (maybe off by one)
    for e in (exp, exp - 1, exp + 1):
        scale = 53 - e + 1              # y * 2**scale has 54 significant bits
        # floor(y * 2**scale) = floor((target * 2**(5*scale)) ** (1/5))
        n = target * (Fraction(2) ** (5 * scale))
        r = kth_root_floor(n.numerator // n.denominator, 5)
        if (1 << 53) <= r < (1 << 54):
            break
    else:  # pragma: no cover
        raise RuntimeError("scale search failed")
    exact = Fraction(r) ** 5 == n
    mant, guard = r >> 1, r & 1
    if up:
        if guard or not exact:
            mant += 1
    else:
        if guard and (not exact or (mant & 1)):
            mant += 1                   # above half, or exactly half and odd
    return math.ldexp(mant, -(scale - 1))


def srgb_tables():
    decode, qthr = [], []
    brk = Fraction(4045, 100000)
    for c in range(256):
        y = Fraction(c, 255)
        if y <= brk:
            decode.append(nearest(y * Fraction(100, 1292)))
        else:  # (y + 0.055)/1.055 = (40c + 561)/10761
            decode.append(rational_pow_2_4(40 * c + 561, 10761, up=False))
    for q in range(257):
        y = Fraction(2 * q - 1, 510)    # code boundary (q - 1/2)/255
        if y <= brk:
            qthr.append(round_up(y * Fraction(100, 1292)))
        else:  # (y + 0.055)/1.055 = (40q + 541)/10761
            qthr.append(rational_pow_2_4(40 * q + 541, 10761, up=True))
    return decode, qthr


def matrices():
    M = [[float(x) for x in row] for row in M_TEXT]
    W = [(row[0] + row[1]) + row[2] for row in M]
    A = [[Fraction(x) for x in row] for row in M]
    # Gauss-Jordan elimination on exact rationals
    aug = [A[i][:] + [Fraction(int(i == j)) for j in range(3)] for i in range(3)]
    for col in range(3):
        piv = next(r for r in range(col, 3) if aug[r][col] != 0)
        aug[col], aug[piv] = aug[piv], aug[col]
        p = aug[col][col]
        aug[col] = [x / p for x in aug[col]]
        for r in range(3):
            if r != col and aug[r][col] != 0:
                f = aug[r][col]
                aug[r] = [x - f * y for x, y in zip(aug[r], aug[col])]
    MI = [[nearest(aug[i][3 + j]) for j in range(3)] for i in range(3)]
    return M, W, MI


def dd(value: Decimal):
    hi = nearest(Fraction(value))
    lo = nearest(Fraction(value) - Fraction(hi))
    return hi, lo


def trig_constants():
    getcontext().prec = 90
    # pi by the Gauss-Legendre iteration
    a, b, t, p = Decimal(1), Decimal(1) / Decimal(2).sqrt(), Decimal(1) / 4, Decimal(1)
    for _ in range(8):
        an = (a + b) / 2
        b = (a * b).sqrt()
        t -= p * (a - an) ** 2
        a, p = an, 2 * p
    pi = (a + b) ** 2 / (4 * t)
    pi180 = dd(pi / 180)
    sin_c, cos_c = [], []
    fact = Decimal(1)
    for n in range(1, 40):
        fact *= n
        if n % 2 == 1:
            sin_c.append(dd(Decimal((-1) ** ((n - 1) // 2)) / fact))
        else:
            cos_c.append(dd(Decimal((-1) ** (n // 2)) / fact))
        if fact > Decimal(10) ** 36:
            break
    return pi180, sin_c, cos_c


def hx(x: float) -> str:
    return float.hex(x)


def main():
    M, W, MI = matrices()
    decode, qthr = srgb_tables()
    delta = Fraction(6, 29)
    pi180, sin_c, cos_c = trig_constants()
    lines = [
        "/* Generated by gen_tables.py - do not edit.  FP64 constants of libcvsearch:",
        " * sRGB (IEC 61966-2-1) with D65 white, CIE 1976 L*a*b*, each value the",
        " * correctly rounded double of its exact definition (see gen_tables.py). */",
        "#pragma once",
        "",
        "#define CVS_M_INIT {" + ", ".join(hx(x) for row in M for x in row) + "}",
        "#define CVS_W_INIT {" + ", ".join(hx(x) for x in W) + "}",
        "#define CVS_MI_INIT {" + ", ".join(hx(x) for row in MI for x in row) + "}",
        f"#define CVS_F_BREAK {hx(round_down(delta ** 3))}      /* (6/29)^3, rounded down */",
        f"#define CVS_FINV_BREAK {hx(round_down(delta))}   /* 6/29, rounded down */",
        f"#define CVS_F_LIN_MUL {hx(nearest(1 / (3 * delta ** 2)))}    /* 841/108 */",
        f"#define CVS_F_LIN_ADD {hx(nearest(Fraction(4, 29)))}    /* 4/29 */",
        f"#define CVS_FINV_LIN_MUL {hx(nearest(3 * delta ** 2))} /* 108/841 */",
        f"#define CVS_PI180_HI {hx(pi180[0])}",
        f"#define CVS_PI180_LO {hx(pi180[1])}",
        f"#define CVS_N_SIN_C {len(sin_c)}",
        f"#define CVS_N_COS_C {len(cos_c)}",
        "#define CVS_SIN_C_INIT {" + ", ".join(f"{hx(h)}, {hx(l)}" for h, l in sin_c) + "}",
        "#define CVS_COS_C_INIT {" + ", ".join(f"{hx(h)}, {hx(l)}" for h, l in cos_c) + "}",
        "",
        "/* CVS_DECODE_INIT: 256 doubles; CVS_QTHR_INIT: 257 doubles */",
        "#define CVS_DECODE_INIT { \\",
    ]
    for i in range(0, 256, 4):
        sep = ", \\" if i + 4 < 256 else " }"
        lines.append("  " + ", ".join(hx(x) for x in decode[i:i + 4]) + sep)
    lines.append("#define CVS_QTHR_INIT { \\")
    for i in range(0, 257, 4):
        chunk = qthr[i:i + 4]
        sep = ", \\" if i + 4 < 257 else " }"
        lines.append("  " + ", ".join(hx(x) for x in chunk) + sep)
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")
    print("wrote", OUT)


if __name__ == "__main__":
    main()
