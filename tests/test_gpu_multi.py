"""The multi-threshold search, cvs_search_colors_multi (needs a GPU).

One pass decides every candidate against up to 16 threshold sets (the
experiment of §3 Experiments: the Table 1 colours under all 12 (V_th, R_novib)
combinations).  Each set's results must equal, exactly, the oracle's and the
single-set entry point's for the same colour and set.
"""
import json
import os

import numpy as np
import pytest

import oracle
import paper_2507_22901_gb300 as cvs
from paper_2507_22901_gb300 import binding, workloads as W

pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 1
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


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


def multi(ctx, torch, rgb, radii, ang, sets, gamut, prec):
    out = ctx.search_colors_multi(dev(torch, rgb), radii, ang, sets, gamut, precision=prec)
    torch.cuda.synchronize()
    return tuple(x.cpu().numpy() for x in out)


def column_equal(got, s, exp, what):
    gm, gc, gp = (x[:, s] for x in got)
    em, ec, ep = exp
    bad = np.nonzero((gc != ec) | (gp != ep) | (gm.view(np.uint32) != em.view(np.uint32)))[0]
    assert bad.size == 0, f"{what} set {s}: {bad.size} mismatches, first {bad[:5]}: " \
        f"gpu {gc[bad[:5]]} {gp[bad[:5]]} expected {ec[bad[:5]]} {ep[bad[:5]]}"


@pytest.mark.parametrize("gamut", [0, 1])
@pytest.mark.parametrize("prec", [binding.PREC_FP32_RECHECK, binding.PREC_FP64])
def test_table1_experiment_matches_oracle(ctx, torch_cuda, prec, gamut):
    """9 colours x 12 combinations on the 61-radius, 360-angle grid."""
    rgb = np.array(list(W.TABLE1_COLORS.values()), np.uint8)
    radii, ang = W.grid(1)
    sets = W.table1_threshold_sets()
    got = multi(ctx, torch_cuda, rgb, radii, ang, sets, gamut, prec)
    for s, (vth, rn) in enumerate(sets):
        exp = oracle.search_colors(rgb, radii, ang, vth, rn, 0x7F, gamut, threads=THREADS)
        column_equal(got, s, exp, "Table 1 colours")
    assert got[1].sum() > 0 and (got[1] == 0).any()


def test_table2_matrix_from_one_pass(ctx, torch_cuda):
    """The presence matrix built from one multi-set pass equals the one built
    from the oracle's per-set searches."""
    with open(os.path.join(GOLDEN, "table1_search_params.json")) as f:
        t1 = json.load(f)
    rgb = np.array([t1["colors_rgb"][k] for k in t1["colors_rgb"]], np.uint8)
    radii, ang = np.arange(1, 61) * 0.5, np.arange(0.0, 360.0, 2.0)
    sets = [(float(v), float(r)) for v in t1["v_th"] for r in t1["r_novib"]]
    got = multi(ctx, torch_cuda, rgb, radii, ang, sets, 0, binding.PREC_FP32_RECHECK)
    exp_pm = np.stack([oracle.search_colors(rgb, radii, ang, v, r, threads=THREADS)[2]
                       for v, r in sets], axis=1)
    assert np.array_equal(W.presence_matrix(got[2]), W.presence_matrix(exp_pm))


def test_cube_sample_sets_match_single_set_search(ctx, torch_cuda):
    """200 cube colours + corners on the 128 x 360 grid: every set equals the
    single-set entry point; three sets are also checked against the oracle."""
    cube = W.color_cube()
    rng = np.random.default_rng(11)
    rgb = np.concatenate([cube[rng.choice(len(cube), 200, replace=False)],
                          np.array([[0, 0, 0], [252, 252, 252], [252, 0, 0], [4, 4, 4]],
                                   np.uint8)])
    radii, ang = W.grid(2)
    sets = W.table1_threshold_sets()
    got = multi(ctx, torch_cuda, rgb, radii, ang, sets, 0, binding.PREC_FP32_RECHECK)
    for s, (vth, rn) in enumerate(sets):
        one = ctx.search_colors(dev(torch_cuda, rgb), radii, ang, vth, rn)
        torch_cuda.cuda.synchronize()
        column_equal(got, s, tuple(x.cpu().numpy() for x in one), "cube sample")
    for s in (0, 5, 11):
        exp = oracle.search_colors(rgb, radii, ang, *sets[s], threads=THREADS)
        column_equal(got, s, exp, "cube sample vs oracle")


def test_masks_per_set_and_one_set(ctx, torch_cuda):
    """Per-set pattern masks; a single set equals cvs_search_colors; 16 sets."""
    rgb = W.color_cube(step=32)
    radii, ang = W.grid(3)
    sets = [(50.0, 0.5, 0x7F), (50.0, 0.5, 0b0010101), (100.0, 0.25, 0b1000000),
            (30.0, 0.9, 0x7F), (0.0, 0.5, 0x7F), (254.5, 0.125, 0x7F)]
    sets = sets + [(20.0 + 10 * i, 0.3, 0x7F) for i in range(10)]
    assert len(sets) == 16
    for gamut in (0, 1):
        got = multi(ctx, torch_cuda, rgb, radii, ang, sets, gamut, binding.PREC_FP32_RECHECK)
        for s, (vth, rn, mask) in enumerate(sets):
            one = ctx.search_colors(dev(torch_cuda, rgb), radii, ang, vth, rn, mask, gamut)
            torch_cuda.cuda.synchronize()
            column_equal(got, s, tuple(x.cpu().numpy() for x in one), f"gamut {gamut}")
    got1 = multi(ctx, torch_cuda, rgb, radii, ang, sets[1:2], 0, binding.PREC_FP32_RECHECK)
    exp = oracle.search_colors(rgb, radii, ang, 50.0, 0.5, 0b0010101, 0, threads=THREADS)
    column_equal(got1, 0, exp, "one set")


def test_large_radii_and_ragged_grid(ctx, torch_cuda):
    """Radii above the FP32 limit (run in FP64 through option fp64_fallback); an
    odd, unfolded angle list."""
    rgb = W.color_cube(step=64)
    radii = np.array([0.0, 3.0, 40.0, 7.5, 120.0])
    ang = np.arange(0.0, 359.0, 7.0)
    sets = W.table1_threshold_sets()[:5]
    ctx.set_option("fp64_fallback", 1)
    try:
        got = multi(ctx, torch_cuda, rgb, radii, ang, sets, 0, binding.PREC_FP32_RECHECK)
    finally:
        ctx.set_option("fp64_fallback", 0)
    for s, (vth, rn) in enumerate(sets):
        exp = oracle.search_colors(rgb, radii, ang, vth, rn, threads=THREADS)
        column_equal(got, s, exp, "large radii")


def test_invalid_sets_rejected(ctx, torch_cuda):
    rgb = dev(torch_cuda, np.zeros((4, 3), np.uint8))
    radii, ang = W.grid(3)
    for sets in ([], [(50.0, 0.5)] * 17):
        with pytest.raises(cvs.CvsError) as ei:
            ctx.search_colors_multi(rgb, radii, ang, sets)
        assert ei.value.status == binding.CVS_ERR_INVALID_ARG
    with pytest.raises(cvs.CvsError) as ei:
        ctx.search_colors_multi(rgb, radii, ang, [(50.0, -1.0)])
    assert ei.value.status == binding.CVS_ERR_INVALID_ARG
    # empty input is fine
    out = ctx.search_colors_multi(dev(torch_cuda, np.zeros((0, 3), np.uint8)), radii, ang,
                                  [(50.0, 0.5)])
    assert out[0].shape == (0, 1)


@pytest.mark.parametrize("walk", [1, 0])
def test_angle_range_walk_matches_oracle(ctx, torch_cuda, walk):
    """The multi-set pass on the angle-range walk (option angle_ranges = 1:
    ranges of the union of the sets) and on the plain walk (0): every set
    equals the single-set entry point, and four sets the oracle.  The grids
    cover one and several blocks of 128 radii, unsorted radii, radius chunks
    per work item, per-set masks and luminance limits; the colours include dark
    ones whose larger radii take the slow path (walked by the plain kernel)."""
    torch = torch_cuda
    cube = W.color_cube()
    rng = np.random.default_rng(23)
    # dark colours leave the cubic branch of f^-1 part of the way up the radii
    dark = np.array([[0, 0, 0], [28, 28, 28], [40, 40, 40], [60, 20, 20], [10, 40, 60],
                     [48, 36, 80]], np.uint8)
    rgb = np.concatenate([cube[rng.choice(len(cube), 96, replace=False)], dark,
                          np.array([[252, 252, 252], [4, 200, 4]], np.uint8)])
    r2, a2 = W.grid(2)
    grids = [(r2, a2),
             (np.linspace(0.2, 30.0, 200), np.arange(0.0, 360.0, 3.0)),
             (rng.permutation(np.linspace(0.5, 24.0, 70)), np.arange(0.0, 360.0, 4.0))]
    sets = [(50.0, 0.5, 0x7F, None), (100.0, 0.25, 0x7F, None), (150.0, 0.125, 0b0101010, 0.2),
            (60.0, 0.5, 0b1000001, None), (200.0, 0.5, 0x7F, 0.05)]
    ctx.set_option("angle_ranges", walk)
    try:
        for gi, (radii, ang) in enumerate(grids):
            for kchunk in (0, 37):
                ctx.set_option("kchunk", kchunk)
                out = ctx.search_colors_multi(dev(torch, rgb), radii, ang, sets, 0)
                ctx.synchronize()
                got = tuple(x.cpu().numpy() for x in out)
                st = ctx.stats()
                assert (st["ranges_ms"] > 0.0) == (walk == 1), st
                for s, (vth, rn, mask, lim) in enumerate(sets):
                    one = ctx.search_colors(dev(torch, rgb), radii, ang, vth, rn, mask, 0,
                                            max_dl=lim)
                    torch.cuda.synchronize()
                    column_equal(got, s, tuple(x.cpu().numpy() for x in one),
                                 f"grid {gi} kchunk {kchunk}")
            for s in (0, 2, 3, 4):
                vth, rn, mask, lim = sets[s]
                exp = oracle.search_colors(rgb, radii, ang, vth, rn, mask, 0, threads=THREADS,
                                           max_dl=-1.0 if lim is None else lim)
                column_equal(got, s, exp, f"grid {gi} vs oracle")
            assert got[1].sum() > 0
    finally:
        ctx.set_option("kchunk", 0)
        ctx.set_option("angle_ranges", 2)
