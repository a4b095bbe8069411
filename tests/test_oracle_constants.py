"""Pins of the oracle's colour constants against the sRGB standard and an
independent high-precision evaluation (no GPU)."""
import math
from decimal import Decimal, localcontext
from fractions import Fraction

import pytest

from oracle import constants as K

# IEC 61966-2-1 (sRGB) defining chromaticities: primaries and D65 white (x, y).
SRGB_PRIMARIES_XY = {"R": (0.64, 0.33), "G": (0.30, 0.60), "B": (0.15, 0.06)}
D65_XY = (0.3127, 0.3290)


def _xy(X, Y, Z):
    s = X + Y + Z
    return X / s, Y / s


def test_matrix_columns_match_srgb_primaries():
    M, W, _ = K.matrices()
    for col, name in enumerate("RGB"):
        x, y = _xy(M[0][col], M[1][col], M[2][col])
        ex, ey = SRGB_PRIMARIES_XY[name]
        assert abs(x - ex) < 1e-3 and abs(y - ey) < 1e-3, name


def test_white_point_is_d65_and_row_sums():
    M, W, _ = K.matrices()
    x, y = _xy(*W)
    assert abs(x - D65_XY[0]) < 2e-4 and abs(y - D65_XY[1]) < 2e-4
    assert W[1] == 1.0  # Y row of the sRGB matrix sums to exactly 1
    for i in range(3):
        assert W[i] == (M[i][0] + M[i][1]) + M[i][2]


def test_inverse_matrix():
    M, _, MI = K.matrices()
    for i in range(3):
        for j in range(3):
            s = sum(M[i][k] * MI[k][j] for k in range(3))
            assert abs(s - (1.0 if i == j else 0.0)) < 4e-16
    # the familiar 4-digit published inverse
    pub = ((3.2406, -1.5372, -0.4986), (-0.9689, 1.8758, 0.0415), (0.0557, -0.2040, 1.0570))
    for i in range(3):
        for j in range(3):
            assert abs(MI[i][j] - pub[i][j]) < 1e-4


def _dec_decimal(y: Decimal) -> Decimal:
    """IEC sRGB decode at high precision (exp/ln route, independent of the
    integer-root route used by the constants module)."""
    if y <= Decimal("0.04045"):
        return y / Decimal("12.92")
    base = (y + Decimal("0.055")) / Decimal("1.055")
    return (base.ln() * Decimal("2.4")).exp()


def _enc_decimal(x: Decimal) -> Decimal:
    if x <= Decimal("0.0031308"):
        return x * Decimal("12.92")
    return Decimal("1.055") * (x.ln() * Decimal(5) / Decimal(12)).exp() - Decimal("0.055")


def test_decode_lut_is_correctly_rounded():
    lut = K.srgb_decode_lut()
    assert lut[0] == 0.0 and lut[255] == 1.0
    with localcontext() as ctx:
        ctx.prec = 60
        for c in range(256):
            exact = Fraction(_dec_decimal(Decimal(c) / Decimal(255)))
            d = lut[c]
            err = abs(Fraction(d) - exact)
            for nb in (math.nextafter(d, 2.0), math.nextafter(d, -1.0)):
                assert err <= abs(Fraction(nb) - exact), c
            # and agrees with the libm formula (several roundings, x2.4 amplified)
            y = c / 255.0
            libm = y / 12.92 if y <= 0.04045 else ((y + 0.055) / 1.055) ** 2.4
            assert abs(libm - d) <= 8 * math.ulp(d)
    assert all(lut[i] < lut[i + 1] for i in range(255))


def test_quant_thresholds_are_exact_boundaries():
    """thr[i] is the smallest double whose encoded value reaches code i - 1/2."""
    thr = K.quant_thresholds()
    assert len(thr) == 257
    assert all(thr[i] < thr[i + 1] for i in range(256))
    with localcontext() as ctx:
        ctx.prec = 60
        for i, t in enumerate(thr):
            boundary = Decimal(2 * i - 1) / Decimal(2)  # i - 1/2
            below = math.nextafter(t, -math.inf)
            assert 255 * _enc_decimal(Decimal(t)) >= boundary, i
            assert 255 * _enc_decimal(Decimal(below)) < boundary, i


def test_quantize_inverts_decode():
    lut = K.srgb_decode_lut()
    for c in range(256):
        assert K.quantize_ref(lut[c]) == c
    assert K.quantize_ref(-1.0) == -1
    assert K.quantize_ref(2.0) == 256


def test_pow_12_5_modes():
    # exact powers: (32/1)^(12/5) = 2^12
    assert K.pow_12_5(32, 1, "rn") == 4096.0
    assert K.pow_12_5(32, 1, "ru") == 4096.0
    for p, q in [(581, 10761), (10761, 10761), (5000, 10761), (7, 3)]:
        rn, ru = K.pow_12_5(p, q, "rn"), K.pow_12_5(p, q, "ru")
        assert abs(rn - (p / q) ** 2.4) <= 4 * math.ulp(rn)
        x12 = Fraction(p, q) ** 12  # y = x^(12/5)  <=>  y^5 = x^12
        lo = (Fraction(math.nextafter(rn, 0.0)) + Fraction(rn)) / 2
        hi = (Fraction(rn) + Fraction(math.nextafter(rn, math.inf))) / 2
        assert lo ** 5 <= x12 <= hi ** 5  # nearest
        assert Fraction(ru) ** 5 >= x12  # RU is an upper bound ...
        assert Fraction(math.nextafter(ru, 0.0)) ** 5 < x12  # ... and the least one


@pytest.mark.parametrize("n,k", [(0, 5), (1, 5), (31, 5), (32, 5), (10 ** 40, 5), (2 ** 200 + 1, 3)])
def test_iroot(n, k):
    r = K.iroot(n, k)
    assert r ** k <= n < (r + 1) ** k


def test_cie_constants():
    cc = K.cie_constants()
    d = Fraction(6, 29)
    assert Fraction(cc["F_BREAK"]) <= d ** 3 < Fraction(math.nextafter(cc["F_BREAK"], 1.0))
    assert Fraction(cc["FINV_BREAK"]) <= d < Fraction(math.nextafter(cc["FINV_BREAK"], 1.0))
    assert abs(cc["F_LIN_MUL"] - 841 / 108) < 1e-15
    assert abs(cc["FINV_LIN_MUL"] * cc["F_LIN_MUL"] - 1.0) < 1e-15
    # f() is continuous at the breakpoint: t/(3 delta^2) + 4/29 = delta at t = delta^3
    t = float(d ** 3)
    assert abs(t * cc["F_LIN_MUL"] + cc["F_LIN_ADD"] - 6 / 29) < 1e-15
