"""The embedding step, cvs_embed_image (needs a GPU).

Per pixel the frames and the choice must equal the oracle's exactly: the first
passing pair of the requested pattern in (radius value, k, m) order.  Small
ragged images with row pitch are compared pixel by pixel; a full-HD frame is
compared on sampled pixels and checked everywhere for the properties every
correct result has (untouched pixels keep their colour, the emitted pair
re-decides to the requested pattern, the chosen angle lies in the first half
of a folded angle list).
"""
import os

import numpy as np
import pytest

import oracle
import paper_2507_22901_gb300 as cvs
from paper_2507_22901_gb300 import binding, workloads as W

pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 1
NONE = np.int32(-1)


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


def small_image(w, h, seed):
    terms = W.image_params(1, seed=seed, sizes=[(w, h)])[0][2]
    return W.render_image_numpy(w, h, terms, seed)


def gpu_embed(ctx, torch, img, pat, radii, ang, pitch_pad=0, **kw):
    h, w, _ = img.shape
    buf = np.zeros((h, w * 3 + pitch_pad), np.uint8)
    buf[:, :w * 3] = img.reshape(h, w * 3)
    d = torch.from_numpy(buf).cuda()
    dimg = d[:, :w * 3].view(h, w, 3) if pitch_pad == 0 else None
    if dimg is None:  # a strided view with row pitch 3w + pad
        dimg = torch.as_strided(d, (h, w, 3), (w * 3 + pitch_pad, 3, 1))
    fa, fb, ch = ctx.embed_image(dimg, torch.from_numpy(pat).cuda(), radii, ang, 50.0, 0.5, **kw)
    torch.cuda.synchronize()
    return fa.cpu().numpy(), fb.cpu().numpy(), ch.cpu().numpy()


def oracle_embed(img, pat, radii, ang, **kw):
    h, w, _ = img.shape
    fa, fb, ch = oracle.embed(img.reshape(-1, 3), pat.reshape(-1), radii, ang, 50.0, 0.5,
                              threads=THREADS, **kw)
    return fa.reshape(h, w, 3), fb.reshape(h, w, 3), ch.view(np.int32).reshape(h, w)


def assert_same(got, exp, what):
    for g, e, name in zip(got, exp, ("frame A", "frame B", "choice")):
        bad = np.argwhere(g != e)
        assert bad.size == 0, f"{what}: {name} differs at {bad[:4].tolist()}"


@pytest.mark.parametrize("gamut", [0, 1])
@pytest.mark.parametrize("prec", [binding.PREC_FP32_RECHECK, binding.PREC_FP64])
def test_small_images_match_oracle(ctx, torch_cuda, prec, gamut):
    radii, ang = W.grid(3)
    for (w, h), seed, pad in (((37, 23), 1, 0), ((16, 9), 2, 5)):
        img = small_image(w, h, seed)
        pat = W.code_pattern(h, w, module=3, seed=seed, fill=0.9)
        pat[0, 0], pat[-1, -1] = 8, 255  # outside 1..7: nothing embedded
        got = gpu_embed(ctx, torch_cuda, img, pat, radii, ang, pitch_pad=pad, precision=prec,
                        gamut_mode=gamut)
        exp = oracle_embed(img, pat, radii, ang, gamut_mode=gamut)
        assert_same(got, exp, f"{w}x{h} prec {prec} gamut {gamut}")
        assert (got[2] != NONE).sum() > 10


def test_unsorted_radii_and_unfolded_angles(ctx, torch_cuda):
    img = small_image(24, 14, 4)
    pat = W.code_pattern(14, 24, module=2, seed=4, fill=1.0)
    radii = np.array([20.0, 6.0, 31.0, 12.5, 6.0, 25.0, 0.0, 17.25])
    ang = np.arange(0.0, 359.0, 7.0)  # 52 angles, not closed under +180
    got = gpu_embed(ctx, torch_cuda, img, pat, radii, ang)
    exp = oracle_embed(img, pat, radii, ang)
    assert_same(got, exp, "unsorted radii")
    assert (got[2] != NONE).sum() > 10


def test_masks_and_large_radii(ctx, torch_cuda):
    img = small_image(20, 12, 6)
    pat = W.code_pattern(12, 20, module=2, seed=6, fill=1.0)
    radii, ang = np.array([10.0, 24.0, 40.0, 64.0]), np.arange(0.0, 360.0, 10.0)
    ctx.set_option("fp64_fallback", 1)  # radii above 32 run in FP64
    try:
        for mask in (0x7F, 0b1010101, 0):
            got = gpu_embed(ctx, torch_cuda, img, pat, radii, ang, pattern_mask=mask)
            exp = oracle_embed(img, pat, radii, ang, pattern_mask=mask)
            assert_same(got, exp, f"mask {mask:#x}")
    finally:
        ctx.set_option("fp64_fallback", 0)
    assert (got[2] == NONE).all()


def test_full_hd_frame_sampled_and_properties(ctx, torch_cuda):
    w, h = 1920, 1080
    terms = W.image_params(1, seed=9, sizes=[(w, h)])[0][2]
    img = W.render_image_numpy(w, h, terms, 9)
    pat = W.code_pattern(h, w, module=16, seed=9, fill=0.5)
    radii, ang = W.grid(3)
    fa, fb, ch = gpu_embed(ctx, torch_cuda, img, pat, radii, ang)
    none = ch == NONE
    assert np.array_equal(fa[none], img[none]) and np.array_equal(fb[none], img[none])
    assert (pat[~none] > 0).all()
    m = (ch[~none].astype(np.int64) >> 16)
    assert (m < len(ang) // 2).all()  # the folded partner (m + 90) has a larger index
    hi_min, lo_max = cvs.signal_bounds(50.0, 0.5)
    d = np.abs(fa[~none].astype(np.int32) - fb[~none].astype(np.int32))
    cls = np.where(d >= hi_min, 1, np.where(d <= lo_max, 0, -1))
    assert (cls >= 0).all()
    assert np.array_equal(cls[:, 0] * 4 + cls[:, 1] * 2 + cls[:, 2], pat[~none])
    # sampled pixels against the oracle (embedded and not)
    rng = np.random.default_rng(9)
    ys, xs = rng.integers(0, h, 400), rng.integers(0, w, 400)
    e = oracle.embed(img[ys, xs], pat[ys, xs], radii, ang, 50.0, 0.5, threads=THREADS)
    assert np.array_equal(fa[ys, xs], e[0]) and np.array_equal(fb[ys, xs], e[1])
    assert np.array_equal(ch[ys, xs], e[2].view(np.int32))
    assert (~none).sum() > 100000


def test_invalid_arguments(ctx, torch_cuda):
    torch = torch_cuda
    img = torch.zeros((4, 5, 3), dtype=torch.uint8, device="cuda")
    pat = torch.ones((4, 5), dtype=torch.uint8, device="cuda")
    radii, ang = W.grid(3)
    with pytest.raises(ValueError):
        ctx.embed_image(img, pat[:, :4], radii, ang, 50.0, 0.5)
    f = torch.zeros((4, 5, 3), dtype=torch.uint8, device="cuda")
    with pytest.raises(cvs.CvsError) as ei:
        ctx.embed_image(img, pat, radii, ang, 50.0, 0.5, frames=(f, f))
    assert ei.value.status == binding.CVS_ERR_INVALID_ARG


# ------------------------------------------------------------ embedding table
@pytest.fixture(scope="module")
def etab3(ctx):
    radii, ang = W.grid(3)
    t = ctx.build_embed_table(radii, ang, 50.0, 0.5)
    yield t
    t.close()


def table_embed(torch, table, img, pat):
    fa, fb, ch = table.embed_image(torch.from_numpy(img).cuda(), torch.from_numpy(pat).cuda())
    torch.cuda.synchronize()
    return fa.cpu().numpy(), fb.cpu().numpy(), ch.cpu().numpy()


def test_table_matches_oracle_on_sampled_colours(etab3, torch_cuda):
    rng = np.random.default_rng(13)
    cols = rng.integers(0, 256, (300, 3)).astype(np.uint8)
    img = np.repeat(cols, 7, axis=0).reshape(1, -1, 3)
    pat = np.tile(np.arange(1, 8, dtype=np.uint8), 300).reshape(1, -1)
    got = table_embed(torch_cuda, etab3, img, pat)
    radii, ang = W.grid(3)
    exp = oracle_embed(img, pat, radii, ang)
    assert_same(got, exp, "table vs oracle")
    assert (got[2] != NONE).sum() > 100


def test_table_equals_direct_embedding(ctx, etab3, torch_cuda):
    radii, ang = W.grid(3)
    w, h = 1920, 1080
    terms = W.image_params(1, seed=9, sizes=[(w, h)])[0][2]
    img = W.render_image_numpy(w, h, terms, 9)
    pat = W.code_pattern(h, w, module=16, seed=9, fill=0.5)
    direct = gpu_embed(ctx, torch_cuda, img, pat, radii, ang)
    assert_same(table_embed(torch_cuda, etab3, img, pat), direct, "table vs direct")


def test_clip_mode_table_equals_direct(ctx, torch_cuda):
    radii, ang = W.grid(3)
    img = small_image(64, 40, 17)
    pat = W.code_pattern(40, 64, module=2, seed=17, fill=1.0)
    t = ctx.build_embed_table(radii, ang, 50.0, 0.5, gamut_mode=1)
    try:
        got = table_embed(torch_cuda, t, img, pat)
    finally:
        t.close()
    assert_same(got, gpu_embed(ctx, torch_cuda, img, pat, radii, ang, gamut_mode=1), "clip table")
