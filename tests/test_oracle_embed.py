"""Pins of the oracle's embedding step (Fig. 1a): per pixel, the passing pair of
the requested pattern that comes first in (radius value, k, m) order.

The choice is checked against an exhaustive enumeration written with the
oracle's per-candidate primitives (themselves pinned in test_oracle_colour and
test_oracle_search), plus invariants that follow from the geometry: on angle
lists closed under +180 degrees the chosen angle index is in the first half,
and the emitted pair re-decides to the requested pattern.
"""
import numpy as np
import pytest

import oracle

NONE = 0xFFFFFFFF


def _enumerate(rgb, radii, angles, vth, rn, mask=0x7F, gamut=0, max_dl=-1.0):
    lab = oracle.target_lab(rgb)
    s, c = oracle.trig_table(angles)
    out = []
    for k, r in enumerate(radii):
        for m in range(len(angles)):
            qp, qm = oracle.pair_codes(lab, r, s[m], c[m])
            pat, op, om = oracle.decide_pair(qp, qm, vth, rn, mask, gamut)
            if pat and oracle.passes_dl(lab[0], op, om, max_dl):
                out.append((float(r), k, m, tuple(op), tuple(om), pat))
    return out


def _expected(rgb, p, cands):
    best = min((c for c in cands if c[5] == p), default=None)  # (r, k, m) order
    if not (1 <= p <= 7) or best is None:
        return tuple(rgb), tuple(rgb), NONE
    return best[3], best[4], best[1] | (best[2] << 16)


CASES = [  # unsorted radii with repeats; angle lists not closed under +180
    ((170, 170, 170), [24.0, 12.0, 30.0, 12.0, 31.5], list(np.arange(0.0, 360.0, 30.0)) + [45.0]),
    ((240, 100, 100), [30.0, 15.5, 22.0, 31.0], list(np.arange(5.0, 360.0, 30.0))),
    ((100, 100, 240), [20.0, 25.0, 31.0, 31.0], list(np.arange(0.0, 360.0, 24.0))),
    ((12, 200, 33), [28.0, 5.0, 18.0, 32.0], list(np.arange(0.0, 360.0, 20.0))),
    ((100, 240, 240), [31.5, 26.0, 26.0, 9.0], list(np.arange(3.0, 360.0, 25.0))),
    ((240, 240, 100), [32.0, 29.0, 29.0], list(np.arange(0.0, 360.0, 15.0))),
]

@pytest.mark.parametrize("rgb,radii,angles", CASES)
@pytest.mark.parametrize("gamut", [0, 1])
def test_embed_matches_enumeration(rgb, radii, angles, gamut):
    cands = _enumerate(rgb, radii, angles, 50, 0.5, gamut=gamut)
    pats = np.array([0, 1, 2, 3, 4, 5, 6, 7, 8, 255], np.uint8)
    rgbs = np.tile(np.array(rgb, np.uint8), (len(pats), 1))
    fa, fb, ch = oracle.embed(rgbs, pats, radii, angles, 50, 0.5, gamut_mode=gamut)
    for i, p in enumerate(pats):
        ea, eb, ec = _expected(rgb, int(p), cands)
        assert (tuple(fa[i]), tuple(fb[i]), int(ch[i])) == (ea, eb, ec), (rgb, int(p))


@pytest.mark.parametrize("rgb,radii,angles", CASES)
@pytest.mark.parametrize("gamut", [0, 1])
def test_embed_with_luminance_limit_matches_enumeration(rgb, radii, angles, gamut):
    """With a luminance limit the chosen pair is the first passing pair of the
    pattern whose two colours both keep L* within the limit (the limit's pin,
    passes_dl, is in test_oracle_dl)."""
    pats = np.arange(0, 9, dtype=np.uint8)
    rgbs = np.tile(np.array(rgb, np.uint8), (len(pats), 1))
    for lim in (0.02, 0.1, 2.0):
        cands = _enumerate(rgb, radii, angles, 50, 0.5, gamut=gamut, max_dl=lim)
        fa, fb, ch = oracle.embed(rgbs, pats, radii, angles, 50, 0.5, gamut_mode=gamut, max_dl=lim)
        for i, p in enumerate(pats):
            ea, eb, ec = _expected(rgb, int(p), cands)
            assert (tuple(fa[i]), tuple(fb[i]), int(ch[i])) == (ea, eb, ec), (rgb, int(p), lim)


def test_luminance_limit_changes_some_embedding_choices():
    """The limit is not vacuous on these cases: it removes some choices, keeps
    others, and a huge limit changes nothing."""
    changed = kept = 0
    for rgb, radii, angles in CASES:
        pats = np.arange(1, 8, dtype=np.uint8)
        rgbs = np.tile(np.array(rgb, np.uint8), (7, 1))
        base = oracle.embed(rgbs, pats, radii, angles, 50, 0.5)[2]
        lim = oracle.embed(rgbs, pats, radii, angles, 50, 0.5, max_dl=0.1)[2]
        huge = oracle.embed(rgbs, pats, radii, angles, 50, 0.5, max_dl=1e9)[2]
        assert np.array_equal(huge, base)
        changed += int((lim != base).sum())
        kept += int(((lim == base) & (base != NONE)).sum())
    assert changed > 0 and kept > 0


def test_enumeration_cases_embed_something():
    got = 0
    for rgb, radii, angles in CASES:
        pats = np.arange(1, 8, dtype=np.uint8)
        _, _, ch = oracle.embed(np.tile(np.array(rgb, np.uint8), (7, 1)), pats, radii, angles,
                                50, 0.5)
        got += int((ch != NONE).sum())
    assert got >= 4


def test_masked_pattern_is_never_embedded():
    rgb, radii, angles = CASES[0]
    pats = np.arange(1, 8, dtype=np.uint8)
    rgbs = np.tile(np.array(rgb, np.uint8), (7, 1))
    _, _, ch_all = oracle.embed(rgbs, pats, radii, angles, 50, 0.5)
    assert (ch_all != NONE).any()
    _, _, ch = oracle.embed(rgbs, pats, radii, angles, 50, 0.5, pattern_mask=0)
    assert (ch == NONE).all()


def test_folded_grid_invariants_on_table1_colours():
    """60 radii x 180 angles (closed under +180): the chosen m is below 90, the
    pair at m + 90 is the same pair with the frames swapped, and the emitted
    pair re-decides to the requested pattern."""
    radii, angles = np.arange(1, 61) * 0.5, np.arange(0.0, 360.0, 2.0)
    cols = np.array([[100, 100, 100], [170, 170, 170], [240, 240, 240], [240, 100, 100],
                     [100, 240, 100], [100, 100, 240], [240, 240, 100], [100, 240, 240],
                     [240, 100, 240]], np.uint8)
    rgbs = np.repeat(cols, 7, axis=0)
    pats = np.tile(np.arange(1, 8, dtype=np.uint8), len(cols))
    fa, fb, ch = oracle.embed(rgbs, pats, radii, angles, 50, 0.5, threads=oracle.max_threads())
    s, c = oracle.trig_table(angles)
    hits = 0
    for i in range(len(rgbs)):
        if ch[i] == NONE:
            assert tuple(fa[i]) == tuple(fb[i]) == tuple(rgbs[i])
            continue
        hits += 1
        k, m = int(ch[i]) & 0xFFFF, int(ch[i]) >> 16
        assert m < 90
        pat, op, om = oracle.decide_pair(fa[i].astype(int), fb[i].astype(int), 50, 0.5)
        assert pat == pats[i]
        lab = oracle.target_lab(rgbs[i])
        qp, qm = oracle.pair_codes(lab, radii[k], s[m + 90], c[m + 90])
        assert tuple(qp) == tuple(fb[i]) and tuple(qm) == tuple(fa[i])
    assert hits >= 10
