"""The angle-range walk of the FP32 search (needs a GPU).

On folded, evenly spaced angle grids in gamut-reject mode the search first
turns, per target and radius, the gamut and "some channel can be high"
bounds into slot ranges, and evaluates only those slots.  Every slot it
leaves out must certainly fail: results must equal the oracle exactly and the
plain walk (option angle_ranges = 0) bit for bit (the tests force the ranges
with angle_ranges = 1), on grids with offset first
angles, fine and coarse steps, 4096 slots, unsorted radii, restricted pattern
masks and other thresholds, in pair lists, under the luminance limit, over
images, and across several chunks of the range scratch.
"""
import os

import numpy as np
import pytest

import oracle
import paper_2507_22901_gb300 as cvs
from paper_2507_22901_gb300 import workloads as W

pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 1


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


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def sample_colours(n, seed):
    """Cube colours plus near-grey, near-edge and dark ones."""
    rng = np.random.default_rng(seed)
    cube = W.color_cube(8)
    pick = cube[rng.choice(len(cube), n, replace=False)]
    extra = np.array([[170, 170, 170], [240, 100, 100], [0, 0, 0], [255, 255, 255],
                      [5, 250, 5], [3, 3, 40], [250, 250, 2], [12, 0, 0]], np.uint8)
    return np.concatenate([pick, extra])


def both_walks(ctx, torch, rgb, radii, ang, v_th=50.0, r_novib=0.5, pattern_mask=0x7F):
    """Results and counters with the angle ranges (1) and the plain walk (0)."""
    out = {}
    for ar in (1, 0):
        ctx.set_option("angle_ranges", ar)
        try:
            o = ctx.search_colors(dev(torch, rgb), radii, ang, v_th, r_novib,
                                  pattern_mask=pattern_mask)
            ctx.synchronize()
            out[ar] = (tuple(x.cpu().numpy() for x in o), ctx.stats())
        finally:
            ctx.set_option("angle_ranges", 2)
    return out


def same(got, exp, what):
    gm, gc, gp = got
    em, ec, ep = exp
    bad = np.nonzero((gc != ec) | (gp != ep) | (gm.view(np.uint32) != em.view(np.uint32)))[0]
    assert bad.size == 0, f"{what}: {bad.size} mismatches, first {bad[:5]}"


GRIDS = {
    "1 degree from 0.5": (np.arange(1, 65) * 0.5, 0.5 + np.arange(360) * 1.0),
    "2 degrees from 1": (np.arange(1, 65) * 0.5, 1.0 + np.arange(180) * 2.0),
    "0.25 degree": (np.arange(1, 33) * 1.0, np.arange(1440) * 0.25),
    "12 degrees, radius 0 included": (np.arange(0, 41) * 0.8, np.arange(30) * 12.0),
    "unsorted radii": (np.array([30.0, 1.0, 25.0, 7.0, 31.5, 14.0, 0.5, 22.0, 12.25, 3.0]),
                       np.arange(360) * 1.0),
    # first angles far from [0, 360): the offset is reduced exactly before the
    # ranges round it to FP32 radians
    "0.5 degree from 1e6 + 0.5": (np.arange(1, 65) * 0.5, 1e6 + 0.5 + np.arange(720) * 0.5),
    "1 degree from -1e6 - 0.25": (np.arange(1, 65) * 0.5, -1e6 - 0.25 + np.arange(360) * 1.0),
}


@pytest.mark.parametrize("name", list(GRIDS))
def test_grids_match_oracle_and_plain_walk(ctx, torch_cuda, name):
    radii, ang = GRIDS[name]
    rgb = sample_colours(120, 3)
    res = both_walks(ctx, torch_cuda, rgb, radii, ang)
    exp = oracle.search_colors(rgb, radii, ang, 50.0, 0.5, threads=THREADS)
    same(res[1][0], exp, name + " (ranges)")
    same(res[0][0], exp, name + " (plain)")
    cand = len(rgb) * len(radii) * len(ang)
    assert res[1][1]["pruned"] + res[1][1]["skipped"] <= cand
    assert res[1][1]["pruned"] >= res[0][1]["pruned"]


@pytest.mark.parametrize("grid", [2, 3])
def test_dark_colours_on_slow_radii(ctx, torch_cuda, grid):
    """Dark colours, whose larger radii leave the cubic branch of f^-1: on
    those radii the ranges come from bounds widened by the departure of the
    piecewise f^-1 from its cube, and the slots they list are evaluated with
    the slow chain.  Every cube colour with channels up to 88 (step 8), and
    the darkest of each hue, against the oracle and the plain walk; the
    ranges must also prune slow-path radii (more slots than the radius bound
    alone removes)."""
    radii, ang = W.grid(grid)
    q = np.arange(0, 89, 8)
    dark = np.stack(np.meshgrid(q, q, q, indexing="ij"), -1).reshape(-1, 3).astype(np.uint8)
    hues = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 0], [0, 1, 1], [1, 0, 1],
                     [2, 1, 0], [0, 2, 1]], np.uint8)
    rgb = np.concatenate([dark, hues, hues * 3])
    res = both_walks(ctx, torch_cuda, rgb, radii, ang)
    exp = oracle.search_colors(rgb, radii, ang, 50.0, 0.5, threads=THREADS)
    same(res[1][0], exp, f"dark colours, grid {grid} (ranges)")
    same(res[0][0], exp, f"dark colours, grid {grid} (plain)")
    assert exp[1].sum() > 0
    assert res[1][1]["pruned"] > res[0][1]["pruned"]


def test_4096_slots(ctx, torch_cuda):
    radii = np.array([2.0, 9.5, 17.0, 24.5, 32.0])
    ang = np.arange(8192) * (360.0 / 8192)
    rgb = sample_colours(24, 5)
    res = both_walks(ctx, torch_cuda, rgb, radii, ang)
    same(res[1][0], res[0][0], "8192 angles")
    exp = oracle.search_colors(rgb, radii, ang, 50.0, 0.5, threads=THREADS)
    same(res[1][0], exp, "8192 angles vs oracle")


@pytest.mark.parametrize("thr", [(50.0, 0.5, 0x01), (50.0, 0.5, 0x40), (100.0, 0.25, 0x7F),
                                 (150.0, 0.125, 0x2A), (20.0, 1.0, 0x7F), (0.0, 0.5, 0x7F),
                                 (254.5, 0.125, 0x7F)])
def test_masks_and_thresholds(ctx, torch_cuda, thr):
    v_th, r_novib, mask = thr
    radii, ang = W.grid(2)
    radii = radii[::4]
    rgb = sample_colours(100, 7)
    res = both_walks(ctx, torch_cuda, rgb, radii, ang, v_th, r_novib, mask)
    out = {ar: res[ar][0] for ar in res}
    exp = oracle.search_colors(rgb, radii, ang, v_th, r_novib, pattern_mask=mask, threads=THREADS)
    same(out[1], exp, f"{thr} (ranges)")
    same(out[0], exp, f"{thr} (plain)")


def test_pair_lists(ctx, torch_cuda):
    radii, ang = W.grid(1)
    rgb = sample_colours(40, 9)
    recs, offs = ctx.search_colors_pairs(dev(torch_cuda, rgb), radii, ang, 50.0, 0.5)
    recs = recs.cpu().numpy().view(cvs.PAIR_DTYPE).reshape(-1)
    for i in range(len(rgb)):
        exp, n = oracle.search_color(rgb[i], radii, ang, 50.0, 0.5)
        got = recs[offs[i]:offs[i + 1]]
        assert len(got) == n, i
        for f in ("k", "m", "plus", "minus", "pattern"):
            assert np.array_equal(got[f], exp[f]), (i, f)


def test_luminance_limit(ctx, torch_cuda):
    radii, ang = W.grid(3)
    rgb = sample_colours(150, 11)
    out = {}
    try:
        for ar in (1, 0):
            ctx.set_option("angle_ranges", ar)
            o = ctx.search_colors(dev(torch_cuda, rgb), radii, ang, 50.0, 0.5, max_dl=0.5)
            ctx.synchronize()
            out[ar] = tuple(x.cpu().numpy() for x in o)
    finally:
        ctx.set_option("angle_ranges", 2)
    exp = oracle.search_colors(rgb, radii, ang, 50.0, 0.5, threads=THREADS, max_dl=0.5)
    same(out[1], exp, "max_dl 0.5 (ranges)")
    same(out[0], exp, "max_dl 0.5 (plain)")


def test_images(ctx, torch_cuda):
    torch = torch_cuda
    radii, ang = W.grid(3)
    params = W.image_params(3, seed=2, sizes=[(300, 200), (64, 48), (17, 5)])
    imgs = [W.render_image_torch(w, h, t, s, device="cuda") for w, h, t, s in params]
    maps = {}
    for ar in (1, 0):
        ctx.set_option("angle_ranges", ar)
        try:
            m = ctx.search_images(imgs, radii, ang, 50.0, 0.5)
            ctx.synchronize()
            maps[ar] = [tuple(x.cpu().numpy() for x in mm) for mm in m]
        finally:
            ctx.set_option("angle_ranges", 2)
    for a, b in zip(maps[1], maps[0]):
        same(tuple(x.reshape(-1) for x in a), tuple(x.reshape(-1) for x in b), "image")
    small = imgs[2].cpu().numpy().reshape(-1, 3)
    exp = oracle.search_colors(small, radii, ang, 50.0, 0.5, threads=THREADS)
    same(tuple(x.reshape(-1) for x in maps[1][2]), exp, "17 x 5 image vs oracle")


def test_several_scratch_chunks(ctx, torch_cuda):
    """4096 radii: the range scratch holds 8192 targets, so 8200 colours take
    two chunks; results equal the plain walk, and the oracle on a sample."""
    radii = np.arange(1, 4097) * (32.0 / 4096)
    ang = np.arange(36) * 10.0
    rng = np.random.default_rng(13)
    rgb = rng.integers(0, 256, (8200, 3)).astype(np.uint8)
    res = both_walks(ctx, torch_cuda, rgb, radii, ang)
    same(res[1][0], res[0][0], "two chunks")
    pick = np.concatenate([np.arange(8), np.arange(8188, 8200)])
    exp = oracle.search_colors(rgb[pick], radii, ang, 50.0, 0.5, threads=THREADS)
    same(tuple(x[pick] for x in res[1][0]), exp, "two chunks vs oracle")


def test_automatic_choice(ctx, torch_cuda):
    """angle_ranges = 2 (the default) takes the ranges where they list well
    under the slots the plain walk searches (under 0.6 of them, measured by a
    probe of the call's targets): on the colour cube, and on the colours of a
    smooth image only when the forced runs show the same clear margin."""
    torch = torch_cuda
    assert ctx.get_option("angle_ranges") == 2
    radii, ang = W.grid(3)
    cube = dev(torch, W.color_cube(8))
    ctx.search_colors(cube, radii, ang, 50.0, 0.5)
    ctx.synchronize()
    st = ctx.stats()
    assert st["pruned"] > 0.5 * st["candidates"] and st["ranges_ms"] > 0.0
    w, h, t, s = W.image_params(1, seed=0)[0]
    pix = W.render_image_torch(w, h, t, s, device="cuda").reshape(-1, 3)[:65536].contiguous()
    forced = {}
    for ar in (1, 0):
        ctx.set_option("angle_ranges", ar)
        try:
            ctx.search_colors(pix, radii, ang, 50.0, 0.25)
            ctx.synchronize()
            forced[ar] = ctx.stats()
        finally:
            ctx.set_option("angle_ranges", 2)
    listed = forced[1]["candidates"] - forced[1]["pruned"]
    walked = forced[0]["candidates"] - forced[0]["pruned"]
    ratio = listed / walked
    ctx.search_colors(pix, radii, ang, 50.0, 0.25)  # other thresholds: a new probe
    ctx.synchronize()
    auto = ctx.stats()
    print(f"image colours: ranges list {ratio:.3f} of the walked slots")
    if ratio < 0.5:
        assert auto["ranges_ms"] > 0.0 and auto["pruned"] == forced[1]["pruned"]
    elif ratio > 0.7:
        assert auto["ranges_ms"] == 0.0 and auto["pruned"] == forced[0]["pruned"]
    # a call too small to fill the GPU (the Table 1 colours, 61 radii) keeps
    # the plain walk, single-set and multi-set alike
    t1 = dev(torch, np.array(list(W.TABLE1_COLORS.values()), np.uint8))
    r1, a1 = W.grid(1)
    ctx.search_colors(t1, r1, a1, 50.0, 0.5)
    ctx.synchronize()
    assert ctx.stats()["ranges_ms"] == 0.0
    ctx.search_colors_multi(t1, r1, a1, W.table1_threshold_sets())
    ctx.synchronize()
    assert ctx.stats()["ranges_ms"] == 0.0


def test_reserve_covers_the_ranges(torch_cuda):
    """After cvs_reserve, a search within its limits (the first call of its
    kind, so with the probe) allocates no device memory."""
    torch = torch_cuda
    c = cvs.Context(0)
    try:
        radii, ang = W.grid(2)
        rgb = dev(torch, W.color_cube(8))
        n = rgb.shape[0]
        out = (torch.empty(n, dtype=torch.float32, device="cuda"),
               torch.empty(n, dtype=torch.int32, device="cuda"),
               torch.empty(n, dtype=torch.uint8, device="cuda"))
        c.reserve(radii, ang, max_targets=n)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        c.search_colors(rgb, radii, ang, 50.0, 0.5, out=out)
        c.synchronize()
        assert c.stats()["ranges_ms"] > 0.0
        assert abs(torch.cuda.mem_get_info()[0] - free0) < (1 << 20)
    finally:
        c.close()


@pytest.mark.parametrize("seed", range(12))
def test_random_grids_match_plain_walk(ctx, torch_cuda, seed):
    """Seeded random folded, evenly spaced grids (angle count, first angle),
    radii (unsorted, radius 0 included), colours, thresholds and masks: the
    range walk equals the plain walk bit for bit."""
    rng = np.random.default_rng(1000 + seed)
    n_ang = 2 * int(rng.integers(1, 361))
    ang = float(rng.uniform(0.0, 360.0 / n_ang)) + np.arange(n_ang) * (360.0 / n_ang)
    radii = rng.uniform(0.0, 32.0, int(rng.integers(1, 97)))
    radii[0] = 0.0 if seed % 3 == 0 else radii[0]
    rgb = rng.integers(0, 256, (int(rng.integers(1, 300)), 3)).astype(np.uint8)
    v_th = float(rng.choice([0.0, 20.0, 50.0, 100.0, 150.0, 254.5]))
    r_novib = float(rng.choice([0.125, 0.25, 0.5, 1.0]))
    mask = int(rng.integers(1, 128))
    res = both_walks(ctx, torch_cuda, rgb, radii, ang, v_th, r_novib, mask)
    same(res[1][0], res[0][0], f"seed {seed}: {n_ang} angles, {len(radii)} radii")
    assert res[1][1]["pruned"] >= res[0][1]["pruned"] or res[1][1]["ranges_ms"] == 0.0
