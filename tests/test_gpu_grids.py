"""Adversarial grids for every kernel (needs a GPU).

The search loops skip work in three ways that depend on the grid: iterations
below the first radius where a pair can pass, warps whose pairs all leave the
gamut, and (for fewer than 32 angle slots) iterations that span several radii.
Tiny and irregular grids exercise all of them: one radius, one angle, angle
lists folded to 1..3 slots, unsorted and repeated radii, radii on both sides
of the prune boundary, and forced small work items.  Every result must equal
the oracle exactly, and the multi-set and embedding paths must agree with it
too.  The counters must add up: pruned + skipped <= candidates.
"""
import os

import numpy as np
import pytest

import oracle
import paper_2507_22901_gb300 as cvs
from paper_2507_22901_gb300 import binding, workloads as W

pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 1

GRIDS = {
    "one radius, one angle": (np.array([20.0]), np.array([33.0])),
    "folded to one slot": (np.array([3.0, 28.0, 12.0]), np.array([45.0, 225.0])),
    "folded to three slots": (np.arange(1, 41) * 0.75, np.array([0.0, 120.0, 240.0, 180.0, 300.0, 60.0])),
    "unfolded, five angles": (np.array([31.0, 0.0, 31.0, 2.5, 19.25, 26.0]),
                              np.array([0.0, 72.0, 144.0, 216.0, 288.0])),
    "unsorted radii, 24 slots": (np.array([30.0, 1.0, 25.0, 7.0, 30.0, 14.0, 0.5, 22.0]),
                                 np.arange(48) * 7.5),
}


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def ctx(torch_cuda):
    c = cvs.Context(0)
    yield c
    c.close()


def colours():
    cube = W.color_cube(16)
    rng = np.random.default_rng(21)
    extra = np.array([[170, 170, 170], [240, 100, 100], [0, 0, 0], [255, 255, 255],
                      [5, 250, 5]], np.uint8)
    return np.concatenate([cube[rng.choice(len(cube), 120, replace=False)], extra])


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def same(got, exp, what):
    gm, gc, gp = got
    em, ec, ep = exp
    bad = np.nonzero((gc != ec) | (gp != ep) | (gm.view(np.uint32) != em.view(np.uint32)))[0]
    assert bad.size == 0, f"{what}: {bad.size} mismatches, first {bad[:5]}"


@pytest.mark.parametrize("name", list(GRIDS))
@pytest.mark.parametrize("gamut", [0, 1])
def test_search_matches_oracle(ctx, torch_cuda, name, gamut):
    radii, ang = GRIDS[name]
    rgb = colours()
    exp = oracle.search_colors(rgb, radii, ang, 50.0, 0.5, 0x7F, gamut, threads=THREADS)
    for kchunk in (0, 1, 3):
        ctx.set_option("kchunk", kchunk)
        try:
            out = ctx.search_colors(dev(torch_cuda, rgb), radii, ang, 50.0, 0.5, 0x7F, gamut)
            torch_cuda.cuda.synchronize()
        finally:
            ctx.set_option("kchunk", 0)
        same(tuple(x.cpu().numpy() for x in out), exp, f"{name}, kchunk {kchunk}")
        ctx.synchronize()
        st = ctx.stats()
        assert 0 <= st["pruned"] and 0 <= st["skipped"]
        assert st["pruned"] + st["skipped"] <= st["candidates"]


@pytest.mark.parametrize("name", list(GRIDS))
def test_pair_lists_match_oracle(ctx, torch_cuda, name):
    radii, ang = GRIDS[name]
    for rgb in ((170, 170, 170), (240, 100, 100), (5, 250, 5)):
        got, n = ctx.search_color(rgb, radii, ang, 50.0, 0.5)
        exp, ne = oracle.search_color(rgb, radii, ang, 50.0, 0.5)
        assert n == ne
        for f in ("k", "m", "plus", "minus", "pattern"):
            assert np.array_equal(got[f], exp[f]), (name, rgb, f)


@pytest.mark.parametrize("name", list(GRIDS))
def test_multi_matches_oracle(ctx, torch_cuda, name):
    radii, ang = GRIDS[name]
    rgb = colours()
    sets = [(50.0, 0.5), (100.0, 0.25, 0b1010101), (30.0, 0.9), (150.0, 0.125)]
    got = ctx.search_colors_multi(dev(torch_cuda, rgb), radii, ang, sets)
    torch_cuda.cuda.synchronize()
    got = tuple(x.cpu().numpy() for x in got)
    for s, st in enumerate(sets):
        exp = oracle.search_colors(rgb, radii, ang, st[0], st[1], st[2] if len(st) > 2 else 0x7F,
                                   threads=THREADS)
        same(tuple(x[:, s] for x in got), exp, f"{name}, set {s}")


@pytest.mark.parametrize("name", list(GRIDS))
def test_embedding_matches_oracle(ctx, torch_cuda, name):
    torch = torch_cuda
    radii, ang = GRIDS[name]
    rgb = colours()
    n = len(rgb)
    img = np.repeat(rgb, 7, axis=0).reshape(1, n * 7, 3)
    pat = np.tile(np.arange(1, 8, dtype=np.uint8), n).reshape(1, n * 7)
    fa, fb, ch = ctx.embed_image(dev(torch, img), dev(torch, pat), radii, ang, 50.0, 0.5)
    torch.cuda.synchronize()
    ea, eb, ec = oracle.embed(img.reshape(-1, 3), pat.reshape(-1), radii, ang, 50.0, 0.5,
                              threads=THREADS)
    assert np.array_equal(fa.cpu().numpy().reshape(-1, 3), ea)
    assert np.array_equal(fb.cpu().numpy().reshape(-1, 3), eb)
    assert np.array_equal(ch.cpu().numpy().reshape(-1).view(np.uint32), ec)


@pytest.mark.parametrize("angle_ranges", [0, 1])
def test_prunes_run_on_the_cube_grid(ctx, torch_cuda, angle_ranges):
    """On the colour-cube grid the prunes must fire (else the tests above would
    not exercise them) and the results still equal the oracle: without angle
    ranges the radius bound and the out-of-gamut warp skip, with them the
    per-radius angle ranges."""
    cube = W.color_cube(16)
    radii, ang = W.grid(2)
    ctx.set_option("angle_ranges", angle_ranges)
    try:
        out = ctx.search_colors(dev(torch_cuda, cube), radii, ang, 50.0, 0.5)
        ctx.synchronize()
        st = ctx.stats()
    finally:
        ctx.set_option("angle_ranges", 2)
    cand = len(cube) * len(radii) * len(ang)
    assert st["candidates"] == cand
    if angle_ranges:
        assert st["pruned"] > 0.5 * cand
    else:
        assert st["pruned"] > 0.05 * cand and st["skipped"] > 0.2 * cand
    exp = oracle.search_colors(cube, radii, ang, 50.0, 0.5, threads=THREADS)
    same(tuple(x.cpu().numpy() for x in out), exp, "cube step 16")
