"""Pins of the oracle's luminance-difference limit on the emitted pair.

The limit keeps a passing pair only if its two emitted 8-bit colours differ in
L* by at most max_dl, each L* being step 1 (pinned in test_oracle_colour)
applied to the emitted codes.  The filter is checked against an enumeration
that applies the same rule with Python-side L* values, and against fixed
points: identical colours, black against white, and no limit.
"""
import math

import numpy as np
import pytest

import oracle


def test_passes_dl_fixed_points():
    l_mid = oracle.target_lab((10, 200, 30))[0]
    assert oracle.passes_dl(l_mid, (10, 200, 30), (10, 200, 30), 0.0)
    # black and white have L* = 0 and 100 exactly
    assert not oracle.passes_dl(50.0, (0, 0, 0), (255, 255, 255), 49.999)
    assert oracle.passes_dl(50.0, (0, 0, 0), (255, 255, 255), 50.0)
    assert not oracle.passes_dl(0.0, (0, 0, 0), (255, 255, 255), 99.999)
    assert oracle.passes_dl(0.0, (0, 0, 0), (255, 255, 255), 100.0)
    assert oracle.passes_dl(0.0, (0, 0, 0), (255, 255, 255), -1.0)  # negative: no limit
    assert oracle.passes_dl(0.0, (0, 0, 0), (255, 255, 255), float("nan"))


def _pairs(rgb, radii, angles, gamut):
    lab = oracle.target_lab(rgb)
    s, c = oracle.trig_table(angles)
    out = []
    for k, r in enumerate(radii):
        for m in range(len(angles)):
            qp, qm = oracle.pair_codes(lab, r, s[m], c[m])
            pat, op, om = oracle.decide_pair(qp, qm, 50, 0.5, 0x7F, gamut)
            if pat:
                dl = max(abs(oracle.target_lab(op)[0] - lab[0]),
                         abs(oracle.target_lab(om)[0] - lab[0]))
                out.append((k, m, pat, dl))
    return out


CASES = [
    ((170, 170, 170), [12.0, 24.0, 30.0], list(np.arange(0.0, 360.0, 30.0))),
    ((240, 100, 100), [15.5, 22.0, 30.0, 31.0], list(np.arange(5.0, 360.0, 30.0))),
    ((100, 240, 240), [9.0, 26.0, 31.5], list(np.arange(3.0, 360.0, 25.0))),
    ((12, 200, 33), [18.0, 28.0, 32.0], list(np.arange(0.0, 360.0, 20.0))),
]


@pytest.mark.parametrize("rgb,radii,angles", CASES)
@pytest.mark.parametrize("gamut", [0, 1])
def test_limit_filters_the_enumeration(rgb, radii, angles, gamut):
    all_pairs = _pairs(rgb, radii, angles, gamut)
    dls = sorted({p[3] for p in all_pairs})
    limits = [0.0, 0.05, 0.2, 0.5] + (dls[len(dls) // 2:len(dls) // 2 + 1] if dls else [])
    for lim in limits:
        exp = [(k, m, pat) for k, m, pat, dl in all_pairs if dl <= lim]
        got, n = oracle.search_color(rgb, radii, angles, 50, 0.5, gamut_mode=gamut, max_dl=lim)
        assert n == len(exp)
        assert [(int(g["k"]), int(g["m"]), int(g["pattern"])) for g in got] == exp
        max_r, count, pmask = oracle.search_colors([rgb], radii, angles, 50, 0.5,
                                                   gamut_mode=gamut, max_dl=lim)
        assert count[0] == len(exp)
        assert pmask[0] == sum({1 << (p - 1) for _, _, p in exp})


def test_cases_have_pairs_on_both_sides_of_a_limit():
    dls = [p[3] for rgb, radii, angles in CASES for p in _pairs(rgb, radii, angles, 1)]
    assert min(dls) <= 0.2 < max(dls)


def test_no_limit_and_monotone_counts():
    rgb, radii, angles = CASES[1]
    base = oracle.search_colors([rgb], radii, angles, 50, 0.5, gamut_mode=1)[1][0]
    assert oracle.search_colors([rgb], radii, angles, 50, 0.5, gamut_mode=1,
                                max_dl=math.inf)[1][0] == base
    counts = [oracle.search_colors([rgb], radii, angles, 50, 0.5, gamut_mode=1, max_dl=x)[1][0]
              for x in (0.0, 0.1, 0.3, 1.0, 3.0)]
    assert counts == sorted(counts) and counts[-1] <= base
