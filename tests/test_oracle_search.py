"""Pins of the oracle's decision rule and search loops (no GPU)."""
import json
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------- decision rule
# Hand-worked cases of the embedding-signal condition (§3 Experiments): a bit
# is high if the channel difference exceeds V_th, low if it is below
# V_th * R_novib; R is the leading digit of the Table 1 pattern.
@pytest.mark.parametrize(
    "qp,qm,vth,rn,expect",
    [
        ((200, 100, 100), (100, 100, 100), 50, 0.5, 0b100),   # dR=100 high, G/B 0 low
        ((100, 200, 100), (100, 100, 100), 50, 0.5, 0b010),
        ((100, 100, 200), (100, 100, 100), 50, 0.5, 0b001),
        ((200, 200, 200), (100, 100, 100), 50, 0.5, 0b111),
        ((151, 100, 100), (100, 100, 100), 50, 0.5, 0b100),   # 51 > 50
        ((150, 100, 100), (100, 100, 100), 50, 0.5, 0),       # 50 is not > 50, not < 25
        ((130, 100, 100), (100, 100, 100), 50, 0.5, 0),       # 30: neither high nor low
        ((200, 124, 100), (100, 100, 100), 50, 0.5, 0b100),   # 24 < 25: low
        ((200, 125, 100), (100, 100, 100), 50, 0.5, 0),       # 25 is not < 25
        ((100, 100, 100), (100, 100, 100), 50, 0.5, 0),       # pattern 000 never passes
        ((100, 100, 100), (200, 100, 100), 50, 0.5, 0b100),   # |difference|
        ((255, 100, 100), (0, 100, 100), 200, 0.125, 0b100),  # 255 > 200, 0 < 25
        ((255, 125, 100), (0, 100, 100), 200, 0.125, 0),      # 25 not < 25
        ((255, 118, 100), (0, 100, 100), 150, 0.125, 0b100),  # 18 < 18.75
        ((255, 119, 100), (0, 100, 100), 150, 0.125, 0),      # 19 not < 18.75
    ],
)
def test_decide_pair_hand_cases(qp, qm, vth, rn, expect):
    pat, op, om = oracle.decide_pair(qp, qm, vth, rn)
    assert pat == expect
    if expect:
        assert list(op) == list(qp) and list(om) == list(qm)


def test_decide_pair_mask_and_gamut():
    qp, qm = (200, 100, 100), (100, 100, 100)
    assert oracle.decide_pair(qp, qm, 50, 0.5, pattern_mask=0b1110111)[0] == 0  # 100 (bit 3) masked
    assert oracle.decide_pair(qp, qm, 50, 0.5, pattern_mask=0b0001000)[0] == 4
    # out of gamut: rejected in mode 0, clamped in mode 1
    assert oracle.decide_pair((256, 100, 100), (100, 100, 100), 50, 0.5, gamut_mode=0)[0] == 0
    pat, op, om = oracle.decide_pair((256, 100, 100), (100, 100, 100), 50, 0.5, gamut_mode=1)
    assert pat == 4 and list(op) == [255, 100, 100]
    pat, op, om = oracle.decide_pair((150, 100, 100), (-1, 100, 100), 50, 0.5, gamut_mode=1)
    assert pat == 4 and list(om) == [0, 100, 100]
    assert oracle.decide_pair((150, 100, 100), (-1, 100, 100), 50, 0.5, gamut_mode=0)[0] == 0


# --------------------------------------------------------------- brute force
def _brute(rgb, radii, angles, vth, rn, mask=0x7F, gamut=0):
    """The search written out with the oracle's own primitives, one call per
    candidate, to pin the C loops' bookkeeping (order, counts, max radius)."""
    lab = oracle.target_lab(rgb)
    s, c = oracle.trig_table(angles)
    pairs = []
    for k, r in enumerate(radii):
        for m in range(len(angles)):
            qp, qm = oracle.pair_codes(lab, r, s[m], c[m])
            pat, op, om = oracle.decide_pair(qp, qm, vth, rn, mask, gamut)
            if pat:
                pairs.append((k, m, tuple(op), tuple(om), pat))
    return pairs


CASES = [
    ((170, 170, 170), [0.0, 12.0, 24.0], [0.0, 90.0, 180.0, 270.0]),
    ((240, 100, 100), [15.5, 30.0], [10.0, 100.0, 190.0, 280.0]),
    ((100, 100, 240), [20.0, 25.0, 31.0], [45.0, 135.0, 225.0, 315.0]),
    ((12, 200, 33), [5.0, 28.0], [0.0, 60.0, 120.0, 180.0, 240.0, 300.0]),
    # unsorted radii: the largest passing radius (22) comes before a smaller
    # passing one (15.5), so max_r is not simply the last passing radius
    ((240, 100, 100), [22.0, 30.0, 15.5], [10.0, 100.0, 190.0, 280.0]),
]


@pytest.mark.parametrize("rgb,radii,angles", CASES)
@pytest.mark.parametrize("gamut", [0, 1])
def test_search_color_matches_brute_force(rgb, radii, angles, gamut):
    exp = _brute(rgb, radii, angles, 50, 0.5, gamut=gamut)
    got, n = oracle.search_color(rgb, radii, angles, 50, 0.5, gamut_mode=gamut, target=7)
    assert n == len(exp) == len(got)
    for rec, e in zip(got, exp):
        assert (int(rec["k"]), int(rec["m"]), tuple(rec["plus"]), tuple(rec["minus"]),
                int(rec["pattern"])) == e
        assert rec["target"] == 7 and rec["flags"] == 0


@pytest.mark.parametrize("rgb,radii,angles", CASES)
def test_search_colors_matches_brute_force(rgb, radii, angles):
    exp = _brute(rgb, radii, angles, 50, 0.5)
    max_r, count, pmask = oracle.search_colors([rgb, rgb], radii, angles, 50, 0.5)
    assert count[0] == count[1] == len(exp)
    best = max((radii[e[0]] for e in exp), default=-1.0)
    assert max_r[0] == np.float32(best)
    assert pmask[0] == sum({1 << (e[4] - 1) for e in exp})


def test_some_brute_case_passes():
    # the tiny grids above must exercise passing candidates, not only rejections
    assert sum(len(_brute(*c, 50, 0.5)) for c in CASES) > 0
    # and the unsorted case must pass at its largest radius before a smaller one
    rgb, radii, angles = CASES[-1]
    ks = [e[0] for e in _brute(rgb, radii, angles, 50, 0.5)]
    best = max(ks, key=lambda k: radii[k])
    assert any(k > best and radii[k] < radii[best] for k in ks)


def test_radius_zero_gives_target_and_never_passes():
    rng = np.random.default_rng(3)
    for rgb in rng.integers(0, 256, (200, 3)):
        lab = oracle.target_lab(rgb)
        for ang in (0.0, 33.0, 271.0):
            (s,), (c,) = oracle.trig_table([ang])
            qp, qm = oracle.pair_codes(lab, 0.0, s, c)
            assert list(qp) == list(rgb) and list(qm) == list(rgb)
    _, n = oracle.search_color((170, 170, 170), [0.0], np.arange(360.0), 50, 0.5)
    assert n == 0


def test_truncation_reports_required_count():
    radii, ang = np.arange(61) * 0.5, np.arange(360.0)
    full, n = oracle.search_color((170, 170, 170), radii, ang, 50, 0.5)
    assert n > 100
    part, n2 = oracle.search_color((170, 170, 170), radii, ang, 50, 0.5, cap=100)
    assert n2 == n and len(part) == 100
    assert part.tobytes() == full[:100].tobytes()


def test_point_symmetry_of_search_output():
    """On a grid closed under +180 degrees, candidate (k, m + n/2) is candidate
    (k, m) with its two colours swapped (§2 Methods: point-symmetric pairs)."""
    radii, ang = np.arange(61) * 0.5, np.arange(360.0)
    for rgb in [(170, 170, 170), (240, 100, 100), (100, 240, 240)]:
        pairs, n = oracle.search_color(rgb, radii, ang, 50, 0.5)
        d = {(int(p["k"]), int(p["m"])): p for p in pairs}
        for (k, m), p in d.items():
            q = d[(k, (m + 180) % 360)]
            assert list(q["plus"]) == list(p["minus"]) and list(q["minus"]) == list(p["plus"])
            assert q["pattern"] == p["pattern"]


def test_golden_config1_regression():
    """Counts and digests of the (170,170,170) search over the 61 x 360 grid for
    all twelve Table 1 threshold combinations, written by
    tests/golden/gen_golden.py from the oracle."""
    import hashlib
    with open(os.path.join(GOLDEN, "search_color_gray170.json")) as f:
        gold = json.load(f)
    radii = np.asarray(gold["radii"], np.float64)
    ang = np.asarray(gold["angles_deg"], np.float64)
    tt = oracle.trig_table(ang)
    for entry in gold["combos"]:
        pairs, n = oracle.search_color(gold["rgb"], radii, ang, entry["v_th"], entry["r_novib"],
                                       gamut_mode=entry["gamut_mode"], trig_tab=tt)
        assert n == entry["count"]
        assert hashlib.sha256(pairs.tobytes()).hexdigest() == entry["sha256"]


def test_table2_soft_diagnostic(capsys):
    """Table 2 of the paper as a soft diagnostic: agreement is printed, not
    asserted, because the paper leaves the grid, constants and gamut handling
    unstated.  The check only requires the comparison to run."""
    with open(os.path.join(GOLDEN, "table1_search_params.json")) as f:
        t1 = json.load(f)
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "table2_presence.txt"))
            if ln.strip() and not ln.startswith("#")]
    colors = list(t1["colors_rgb"])
    radii, ang = np.arange(1, 61) * 0.5, np.arange(0.0, 360.0, 2.0)
    agree = {0: 0, 1: 0}
    for gamut in (0, 1):
        present = {}
        for name in colors:
            mask = 0
            for vth in t1["v_th"]:
                for rn in t1["r_novib"]:
                    _, _, pm = oracle.search_colors([t1["colors_rgb"][name]], radii, ang, vth, rn,
                                                    gamut_mode=gamut)
                    mask |= int(pm[0])
            present[name] = mask
        for row in rows:
            pat = int(row[0], 2)
            for ci, name in enumerate(colors):
                agree[gamut] += int(bool(present[name] >> (pat - 1) & 1) == (row[1 + ci] == "1"))
    print(f"Table 2 agreement (of 63): reject {agree[0]}, clip {agree[1]}")
    assert 0 <= agree[0] <= 63 and 0 <= agree[1] <= 63
