"""The luminance-difference limit on emitted pairs (option "max_dl"; needs a GPU).

With the limit on, every search entry point that supports it must still equal
the oracle exactly (counts, radii, pattern masks, pair lists), the FP32 path
must equal the all-FP64 path, and the entry points that do not support it
must refuse while it is on.
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
    ctx.set_option("max_dl", max_dl)
    out = ctx.search_colors(dev(torch, rgb), radii, ang, 50.0, 0.5, 0x7F, gamut, precision=prec)
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
    ctx.set_option("max_dl", 0.1)
    for rgb in W.TABLE1_COLORS.values():
        for gamut in (0, 1):
            got, n = ctx.search_color(rgb, radii, ang, 50.0, 0.5, gamut_mode=gamut)
            exp, ne = oracle.search_color(rgb, radii, ang, 50.0, 0.5, gamut_mode=gamut,
                                          max_dl=0.1)
            assert n == ne
            for f in ("k", "m", "plus", "minus", "pattern"):
                assert np.array_equal(got[f], exp[f]), (rgb, gamut, f)
    ctx.set_option("max_dl", -1)


def test_images_match_oracle(ctx, torch_cuda):
    torch = torch_cuda
    radii, ang = W.grid(3)
    w, h = 41, 23
    terms = W.image_params(1, seed=3, sizes=[(w, h)])[0][2]
    img = W.render_image_numpy(w, h, terms, 3)
    ctx.set_option("max_dl", 0.15)
    maps = ctx.search_images([dev(torch, img)], radii, ang, 50.0, 0.5)
    torch.cuda.synchronize()
    got = tuple(x.cpu().numpy().reshape(-1) for x in maps[0])
    exp = oracle.search_colors(img.reshape(-1, 3), radii, ang, 50.0, 0.5, threads=THREADS,
                               max_dl=0.15)
    same(got, exp, "image")
    ctx.set_option("max_dl", -1)


def test_full_cube_fp32_equals_fp64(ctx, torch_cuda):
    rgb = W.color_cube(8)
    radii, ang = W.grid(2)
    a = gpu_colors(ctx, torch_cuda, rgb, radii, ang, 0.1)
    b = gpu_colors(ctx, torch_cuda, rgb, radii, ang, 0.1, binding.PREC_FP64)
    same(a, b, "cube fp32 vs fp64 with max_dl")
    c = gpu_colors(ctx, torch_cuda, rgb, radii, ang, -1.0)
    assert (a[1] <= c[1]).all() and a[1].sum() < c[1].sum()


def test_capacity_table_honours_the_limit(ctx, torch_cuda):
    radii, ang = W.grid(3)
    ctx.set_option("max_dl", 0.2)
    lut = ctx.build_lut(radii, ang, 50.0, 0.5)
    rgb = cube_sample(500, seed=8)
    got = tuple(x.cpu().numpy() for x in lut.lookup_colors(dev(torch_cuda, rgb)))
    lut.close()
    direct = gpu_colors(ctx, torch_cuda, rgb, radii, ang, 0.2)
    same(got, direct, "table vs direct")
    ctx.set_option("max_dl", -1)


def test_unsupported_entry_points_refuse(ctx, torch_cuda):
    torch = torch_cuda
    radii, ang = W.grid(3)
    ctx.set_option("max_dl", 0.3)
    assert ctx.get_option("max_dl") == 0.3
    rgb = dev(torch, np.zeros((2, 3), np.uint8))
    with pytest.raises(cvs.CvsError) as ei:
        ctx.search_colors_multi(rgb, radii, ang, [(50.0, 0.5)])
    assert ei.value.status == binding.CVS_ERR_INVALID_ARG and "max_dl" in str(ei.value)
    img = torch.zeros((4, 5, 3), dtype=torch.uint8, device="cuda")
    pat = torch.ones((4, 5), dtype=torch.uint8, device="cuda")
    with pytest.raises(cvs.CvsError):
        ctx.embed_image(img, pat, radii, ang, 50.0, 0.5)
    with pytest.raises(cvs.CvsError):
        ctx.build_embed_table(radii, ang, 50.0, 0.5)
    with pytest.raises(cvs.CvsError):
        ctx.set_option("max_dl", float("nan"))
    ctx.set_option("max_dl", -5)
    assert ctx.get_option("max_dl") == -1.0
    ctx.search_colors_multi(rgb, radii, ang, [(50.0, 0.5)])  # works again once off
