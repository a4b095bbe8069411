"""The luminance-difference limit on emitted pairs (thresholds field max_dl,
given per call; needs a GPU).

With the limit on, every entry point must still equal the oracle exactly:
counts, radii and pattern masks of colours and images, pair lists, the
capacity table, the multi-set search with a limit per set, the embedding
(frames and choices) and the embedding table.  The FP32 path must equal the
all-FP64 path, calls with and without a limit on one context must not affect
each other, and invalid limits are refused.
"""
import os

import numpy as np
import pytest

import oracle
import paper_2507_22901_gb300 as cvs
from paper_2507_22901_gb300 import binding, workloads as W

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


def gpu_colors(ctx, torch, rgb, radii, ang, max_dl, prec=binding.PREC_FP32_RECHECK, gamut=0):
    out = ctx.search_colors(dev(torch, rgb), radii, ang, 50.0, 0.5, 0x7F, gamut, max_dl=max_dl,
                            precision=prec)
    torch.cuda.synchronize()
    return tuple(x.cpu().numpy() for x in out)


def same(got, exp, what):
    gm, gc, gp = got
    em, ec, ep = exp
    bad = np.nonzero((gc != ec) | (gp != ep) | (gm.view(np.uint32) != em.view(np.uint32)))[0]
    assert bad.size == 0, f"{what}: {bad.size} mismatches, first {bad[:5]}"


def cube_sample(n, seed=5):
    cube = W.color_cube()
    return cube[np.random.default_rng(seed).choice(len(cube), n, replace=False)]


@pytest.mark.parametrize("max_dl", [0.05, 0.2])
@pytest.mark.parametrize("prec", [binding.PREC_FP32_RECHECK, binding.PREC_FP64])
@pytest.mark.parametrize("gamut", [0, 1])
def test_colours_match_oracle(ctx, torch_cuda, max_dl, prec, gamut):
    rgb = cube_sample(160)
    radii, ang = W.grid(2)
    got = gpu_colors(ctx, torch_cuda, rgb, radii, ang, max_dl, prec, gamut)
    exp = oracle.search_colors(rgb, radii, ang, 50.0, 0.5, 0x7F, gamut, threads=THREADS,
                               max_dl=max_dl)
    same(got, exp, f"max_dl {max_dl}")
    base = oracle.search_colors(rgb, radii, ang, 50.0, 0.5, 0x7F, gamut, threads=THREADS)
    assert 0 < exp[1].sum() < base[1].sum()  # the limit removes some pairs, not all


def test_pair_lists_match_oracle(ctx, torch_cuda):
    radii, ang = W.grid(1)
    for rgb in W.TABLE1_COLORS.values():
        for gamut in (0, 1):
            got, n = ctx.search_color(rgb, radii, ang, 50.0, 0.5, gamut_mode=gamut, max_dl=0.1)
            exp, ne = oracle.search_color(rgb, radii, ang, 50.0, 0.5, gamut_mode=gamut,
                                          max_dl=0.1)
            assert n == ne
            for f in ("k", "m", "plus", "minus", "pattern"):
                assert np.array_equal(got[f], exp[f]), (rgb, gamut, f)


def test_images_match_oracle(ctx, torch_cuda):
    torch = torch_cuda
    radii, ang = W.grid(3)
    w, h = 41, 23
    terms = W.image_params(1, seed=3, sizes=[(w, h)])[0][2]
    img = W.render_image_numpy(w, h, terms, 3)
    maps = ctx.search_images([dev(torch, img)], radii, ang, 50.0, 0.5, max_dl=0.15)
    torch.cuda.synchronize()
    got = tuple(x.cpu().numpy().reshape(-1) for x in maps[0])
    exp = oracle.search_colors(img.reshape(-1, 3), radii, ang, 50.0, 0.5, threads=THREADS,
                               max_dl=0.15)
    same(got, exp, "image")


def test_full_cube_fp32_equals_fp64(ctx, torch_cuda):
    rgb = W.color_cube(8)
    radii, ang = W.grid(2)
    a = gpu_colors(ctx, torch_cuda, rgb, radii, ang, 0.1)
    b = gpu_colors(ctx, torch_cuda, rgb, radii, ang, 0.1, binding.PREC_FP64)
    same(a, b, "cube fp32 vs fp64 with max_dl")
    c = gpu_colors(ctx, torch_cuda, rgb, radii, ang, None)
    assert (a[1] <= c[1]).all() and a[1].sum() < c[1].sum()


def test_capacity_table_honours_the_limit(ctx, torch_cuda):
    radii, ang = W.grid(3)
    lut = ctx.build_lut(radii, ang, 50.0, 0.5, max_dl=0.2)
    rgb = cube_sample(500, seed=8)
    got = tuple(x.cpu().numpy() for x in lut.lookup_colors(dev(torch_cuda, rgb)))
    lut.close()
    direct = gpu_colors(ctx, torch_cuda, rgb, radii, ang, 0.2)
    same(got, direct, "table vs direct")


def test_limit_is_per_call(ctx, torch_cuda):
    """Calls with and without a limit, interleaved on one context and one
    stream, each get their own answer (no state carries over)."""
    rgb = cube_sample(64, seed=12)
    radii, ang = W.grid(3)
    none_ = gpu_colors(ctx, torch_cuda, rgb, radii, ang, None)
    lim = gpu_colors(ctx, torch_cuda, rgb, radii, ang, 0.2)
    again = gpu_colors(ctx, torch_cuda, rgb, radii, ang, 0.0)  # 0 = no limit
    inf = gpu_colors(ctx, torch_cuda, rgb, radii, ang, float("inf"))
    same(again, none_, "no limit after a limited call")
    same(inf, none_, "+inf = no limit")
    exp = oracle.search_colors(rgb, radii, ang, 50.0, 0.5, threads=THREADS, max_dl=0.2)
    same(lim, exp, "limited call between unlimited ones")
    assert lim[1].sum() < none_[1].sum()


def test_invalid_limits_are_refused(ctx, torch_cuda):
    rgb = dev(torch_cuda, np.zeros((2, 3), np.uint8))
    radii, ang = W.grid(3)
    for bad in (float("nan"), -0.5, -1.0):
        with pytest.raises(cvs.CvsError) as ei:
            ctx.search_colors(rgb, radii, ang, 50.0, 0.5, max_dl=bad)
        assert ei.value.status == binding.CVS_ERR_INVALID_ARG and "max_dl" in str(ei.value)


def small_image(w, h, seed):
    terms = W.image_params(1, seed=seed, sizes=[(w, h)])[0][2]
    return W.render_image_numpy(w, h, terms, seed)


@pytest.mark.parametrize("prec", [binding.PREC_FP32_RECHECK, binding.PREC_FP64])
@pytest.mark.parametrize("gamut", [0, 1])
def test_embedding_matches_oracle(ctx, torch_cuda, prec, gamut):
    """Fig. 1a under the limit: per pixel the first pair of the requested
    pattern that also keeps both colours within max_dl of the target's L*."""
    torch = torch_cuda
    radii, ang = W.grid(3)
    img = small_image(37, 23, 5)
    pat = np.random.default_rng(6).integers(0, 9, (23, 37)).astype(np.uint8)
    choices = {}
    for lim in (0.05, 0.3):
        fa, fb, ch = ctx.embed_image(dev(torch, img), dev(torch, pat), radii, ang, 50.0, 0.5,
                                     gamut_mode=gamut, max_dl=lim, precision=prec)
        torch.cuda.synchronize()
        ea, eb, ec = oracle.embed(img.reshape(-1, 3), pat.reshape(-1), radii, ang, 50.0, 0.5,
                                  gamut_mode=gamut, threads=THREADS, max_dl=lim)
        assert np.array_equal(fa.cpu().numpy().reshape(-1, 3), ea), lim
        assert np.array_equal(fb.cpu().numpy().reshape(-1, 3), eb), lim
        assert np.array_equal(ch.cpu().numpy().reshape(-1).view(np.uint32), ec), lim
        choices[lim] = ec
    base = oracle.embed(img.reshape(-1, 3), pat.reshape(-1), radii, ang, 50.0, 0.5,
                        gamut_mode=gamut, threads=THREADS)[2]
    # the tight limit changes some choices and still embeds some pixels
    assert (choices[0.05] != base).any() and (choices[0.05] != 0xFFFFFFFF).any()


@pytest.mark.parametrize("gamut", [0, 1])
def test_embedding_table_matches_direct_embedding(ctx, torch_cuda, gamut):
    torch = torch_cuda
    radii, ang = W.grid(3)
    img = dev(torch, small_image(256, 96, 7))
    pat = dev(torch, W.code_pattern(96, 256, module=8, seed=3))
    etab = ctx.build_embed_table(radii, ang, 50.0, 0.5, gamut_mode=gamut, max_dl=0.05)
    try:
        got = etab.embed_image(img, pat)
        exp = ctx.embed_image(img, pat, radii, ang, 50.0, 0.5, gamut_mode=gamut, max_dl=0.05)
        torch.cuda.synchronize()
    finally:
        etab.close()
    for a, b in zip(got, exp):
        assert torch.equal(a, b)
    unlimited = ctx.embed_image(img, pat, radii, ang, 50.0, 0.5, gamut_mode=gamut)
    torch.cuda.synchronize()
    assert not torch.equal(unlimited[2], exp[2])


@pytest.mark.parametrize("prec", [binding.PREC_FP32_RECHECK, binding.PREC_FP64])
@pytest.mark.parametrize("gamut", [0, 1])
def test_threshold_sets_with_their_own_limits(ctx, torch_cuda, prec, gamut):
    rgb = cube_sample(96, seed=14)
    radii, ang = W.grid(2)
    sets = [(50.0, 0.5, 0x7F, None), (50.0, 0.5, 0x7F, 0.1), (100.0, 0.25, 0x7F, 0.3),
            (50.0, 0.5, 0x2A, 0.05), (150.0, 0.125, 0x7F, None)]
    out = ctx.search_colors_multi(dev(torch_cuda, rgb), radii, ang, sets, gamut_mode=gamut,
                                  precision=prec)
    torch_cuda.cuda.synchronize()
    got = tuple(x.cpu().numpy() for x in out)
    for s, (vth, rn, mask, lim) in enumerate(sets):
        exp = oracle.search_colors(rgb, radii, ang, vth, rn, mask, gamut, threads=THREADS,
                                   max_dl=-1.0 if lim is None else lim)
        same(tuple(x[:, s] for x in got), exp, f"set {s}")
    assert got[1][:, 1].sum() < got[1][:, 0].sum()
