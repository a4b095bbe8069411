"""The facts the angle ranges of slow-path radii rest on (CPU only).

Below delta = 6/29 the inverse CIE function f^-1 (§2 Methods, the inverse of
step 1) is the line 3 delta^2 (f - 4/29), not the cube.  The range pass bounds
how far that puts a colour's linear RGB from the cubic form:
  f^-1(f) = f^3 + e(f),  e(f) = -(delta - f)^2 (f + 2 delta) for f <= delta,
with e non-positive and its size growing as f falls on [-delta, delta], and it
relies on every f-value of a real colour at radius up to 32 lying above
-delta.  These tests check each fact exactly (rational arithmetic) and the
last one on real colours through the oracle's L*a*b*.
"""
from fractions import Fraction as Fr

import numpy as np

import oracle

DELTA = Fr(6, 29)


def finv(u: Fr) -> Fr:
    """The CIE inverse, as its definition states it."""
    return u ** 3 if u > DELTA else 3 * DELTA ** 2 * (u - Fr(4, 29))


def departure(u: Fr) -> Fr:
    return -(DELTA - u) ** 2 * (u + 2 * DELTA) if u <= DELTA else Fr(0)


def test_departure_identity_is_exact():
    for k in range(-300, 400):
        u = Fr(k, 997)  # -0.30 .. 0.40, both sides of delta
        assert finv(u) - u ** 3 == departure(u), u


def test_departure_is_non_positive_and_grows_as_f_falls():
    grid = [-DELTA + (2 * DELTA) * Fr(i, 500) for i in range(501)]  # [-delta, delta]
    vals = [departure(u) for u in grid]
    assert all(v <= 0 for v in vals)
    # |e| is non-increasing in f: its derivative -3 (delta - f)(f + delta) <= 0 there
    assert all(abs(a) >= abs(b) for a, b in zip(vals, vals[1:]))
    assert departure(DELTA) == 0 and departure(-DELTA) == -(2 * DELTA) ** 2 * DELTA


def test_departure_matches_the_oracles_piecewise_inverse():
    """The same identity against the oracle's FP64 constants (4/29 and 3 delta^2
    rounded to double): the difference is a rounding error."""
    c = oracle.consts()
    for u in np.linspace(-0.2, float(DELTA), 257):
        lin_branch = (u - c.f_lin_add) * c.finv_lin_mul
        assert abs((lin_branch - u ** 3) - float(departure(Fr(u)))) < 1e-15


def test_real_colours_keep_f_above_minus_delta_up_to_radius_32():
    """X, Z >= 0 for every 8-bit colour, so f_x, f_z >= 4/29; at radius 32 an
    f-value moves by at most 32/200, which leaves it above -delta."""
    assert Fr(4, 29) - Fr(32, 200) > -DELTA
    rng = np.random.default_rng(3)
    corners = np.array([[r, g, b] for r in (0, 255) for g in (0, 255) for b in (0, 255)],
                       np.uint8)
    rgb = np.concatenate([corners, rng.integers(0, 256, (4000, 3)).astype(np.uint8)])
    lab = oracle.target_lab_many(rgb, threads=oracle.max_threads())
    fy = (lab[:, 0] + 16.0) / 116.0
    fx, fz = fy + lab[:, 1] / 500.0, fy - lab[:, 2] / 200.0
    assert fx.min() > 4 / 29 - 1e-12 and fz.min() > 4 / 29 - 1e-12
    assert min(fx.min() - 32 / 500, fz.min() - 32 / 200) > -float(DELTA)
