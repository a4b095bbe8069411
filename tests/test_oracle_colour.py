"""Pins of the oracle's colour chain: cube root, trig table, L*a*b* and the
inverse chain (no GPU)."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import constants as K


# ------------------------------------------------------------------ cbrt
def _is_correctly_rounded_cbrt(y: float, t: float) -> bool:
    lo = (Fraction(math.nextafter(y, 0.0)) + Fraction(y)) / 2
    hi = (Fraction(y) + Fraction(math.nextafter(y, math.inf))) / 2
    T = Fraction(t)
    return lo ** 3 < T < hi ** 3


def test_cbrt_exact_cubes():
    for x in [1.0, 2.0, 3.0, 0.5, 0.75, 1.25, 0.3125]:
        assert oracle.cbrt_cr(x * x * x) == x
    assert oracle.cbrt_cr(1.0) == 1.0


def test_cbrt_correctly_rounded_random():
    rng = np.random.default_rng(123)
    ts = np.concatenate([rng.uniform(0.008, 1.1, 3000), rng.uniform(1e-3, 1e-2, 500)])
    for t in ts:
        y = oracle.cbrt_cr(float(t))
        assert _is_correctly_rounded_cbrt(y, float(t)), t
        assert abs(y - math.cbrt(t)) <= 3 * math.ulp(y)  # glibc cbrt is not correctly rounded


def test_cbrt_near_binade_edges():
    # inputs whose cube roots sit next to powers of two
    for e in (-3, -2, -1, 0):
        y0 = 2.0 ** e
        for y in (math.nextafter(y0, 0), y0, math.nextafter(y0, 1)):
            t = float(Fraction(y) ** 3)  # nearest double to y^3
            r = oracle.cbrt_cr(t)
            assert _is_correctly_rounded_cbrt(r, t)


# ------------------------------------------------------------------ trig
def test_trig_exact_angles():
    s, c = oracle.trig_table([0, 30, 90, 150, 180, 210, 270, 330, 60, 120, 240, 300])
    assert list(s[:8]) == [0.0, 0.5, 1.0, 0.5, 0.0, -0.5, -1.0, -0.5]
    assert list(c[8:]) == [0.5, -0.5, -0.5, 0.5]
    assert c[0] == 1.0 and c[2] == 0.0 and c[4] == -1.0 and c[6] == 0.0


@pytest.mark.parametrize("step,n", [(1.0, 360), (2.0, 180), (0.5, 720)])
def test_trig_grid_vs_libm_and_symmetry(step, n):
    ang = np.arange(n) * step
    s, c = oracle.trig_table(ang)
    for m in range(n):
        r = math.radians(ang[m])
        # math.radians itself rounds (error up to about ulp(r)), so allow that
        # plus a few ulps of the value
        tol_r = 2 * math.ulp(r) + 1e-300
        assert abs(s[m] - math.sin(r)) <= 4 * math.ulp(abs(s[m]) or 1e-300) + tol_r
        assert abs(c[m] - math.cos(r)) <= 4 * math.ulp(abs(c[m]) or 1e-300) + tol_r
        assert abs(s[m] ** 2 + c[m] ** 2 - 1.0) < 4e-16
    h = n // 2  # the grid is closed under +180 degrees: exact point symmetry
    assert np.array_equal(s[h:], -s[:h] + 0.0) and np.array_equal(c[h:], -c[:h] + 0.0)
    # sin(180 - x) == sin(x) exactly
    for m in range(1, h):
        assert s[h - m] == s[m]


def test_trig_negative_and_large_angles():
    s1, c1 = oracle.trig_table([-30.0, 390.0, 720.5])
    s2, c2 = oracle.trig_table([330.0, 30.0, 0.5])
    assert np.array_equal(s1, s2) and np.array_equal(c1, c2)


# ------------------------------------------------------------------ L*a*b*
def test_lab_white_black_grey_closed_forms():
    assert list(oracle.target_lab([255, 255, 255])) == [100.0, 0.0, 0.0]
    assert list(oracle.target_lab([0, 0, 0])) == [0.0, 0.0, 0.0]
    lut = K.srgb_decode_lut()
    for g in range(256):
        L, a, b = oracle.target_lab([g, g, g])
        Y = lut[g]
        Lref = 116 * math.cbrt(Y) - 16 if Y > (6 / 29) ** 3 else Y * 24389 / 27
        assert abs(L - Lref) < 1e-12
        assert abs(a) < 1e-12 and abs(b) < 1e-12


# Published CIE L*a*b* (D65) of the sRGB primaries, as tabulated in colour
# science references; tolerance covers the 4-digit matrix / white used here.
PRIMARIES_LAB = {
    (255, 0, 0): (53.24, 80.09, 67.20),
    (0, 255, 0): (87.73, -86.18, 83.18),
    (0, 0, 255): (32.30, 79.19, -107.86),
}


@pytest.mark.parametrize("rgb", list(PRIMARIES_LAB))
def test_lab_of_primaries(rgb):
    lab = oracle.target_lab(rgb)
    ref = PRIMARIES_LAB[rgb]
    assert np.allclose(lab, ref, atol=0.1), (lab, ref)


def test_roundtrip_all_colours():
    bad, err = oracle.roundtrip_all()
    assert bad == 0
    assert err < 1e-9


def test_inverse_chain_is_inverse_of_forward():
    rng = np.random.default_rng(7)
    for _ in range(2000):
        lin = rng.uniform(-0.05, 1.05, 3)
        lab = oracle.lin_to_lab(lin)
        back = oracle.lab_to_lin(*lab)
        assert np.max(np.abs(back - lin)) < 1e-12


def test_pair_lab_orientation_and_midpoint():
    """'+' colour = (L, a + r sin j, b + r cos j), '-' = (L, a - r sin j, b - r cos j):
    the unquantised pair, taken back to L*a*b*, sits where the paper puts it."""
    rng = np.random.default_rng(11)
    for _ in range(300):
        rgb = rng.integers(30, 226, 3)
        L, a, b = oracle.target_lab(rgb)
        r = float(rng.uniform(0, 20))
        ang = float(rng.choice([0.0, 90.0, 37.0, 200.0]))
        (s,), (c,) = oracle.trig_table([ang])
        lin_p = oracle.lab_to_lin(L, a + r * s, b + r * c)
        lin_m = oracle.lab_to_lin(L, a - r * s, b - r * c)
        lp, lm = oracle.lin_to_lab(lin_p), oracle.lin_to_lab(lin_m)
        assert np.allclose(lp, [L, a + r * s, b + r * c], atol=1e-9)
        assert np.allclose(lm, [L, a - r * s, b - r * c], atol=1e-9)
        assert np.allclose((lp + lm) / 2, [L, a, b], atol=1e-9)  # point symmetry
        assert abs(lp[0] - L) < 1e-9 and abs(lm[0] - L) < 1e-9  # fixed L*
    # angle 90 moves along +a* only, angle 0 along +b* only
    L, a, b = oracle.target_lab([128, 128, 128])
    lab90 = oracle.lin_to_lab(oracle.lab_to_lin(L, a + 5.0, b))
    (s,), (c,) = oracle.trig_table([90.0])
    assert s == 1.0 and c == 0.0
    assert np.allclose(lab90, [L, a + 5, b], atol=1e-9)


def test_quantize_matches_pow_formula():
    rng = np.random.default_rng(5)
    thr = K.quant_thresholds()
    xs = list(rng.uniform(-0.01, 1.01, 20000))
    for t in thr:  # both sides of every boundary, a few ulps away
        xs += [t, math.nextafter(t, -1), t + 4 * math.ulp(t), t - 4 * math.ulp(t)]
    thr_arr = np.asarray(thr)
    for x in xs:
        q = oracle.quantize(x)
        assert q == K.quantize_ref(x)
        # away from a boundary the libm formula must agree; within an ulp or two
        # of one, its own rounding may land on either side (a tie-critical value)
        if np.min(np.abs(thr_arr - x)) > 1e-12:
            assert q == oracle.quantize_pow(x), x
