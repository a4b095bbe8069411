"""Workloads 2, 3 and 4 compared with the FP64 CPU oracle in full (needs a GPU).

The GPU runs each workload in the launch configuration the library picks for
it (one call; FP32 with FP64 re-decision), and every target is compared with
the oracle's answer for it: counts, largest-radius bits and pattern masks, no
tolerance.
  - workload 4, the precision set: 4096 colours x 256 radii x 720 angles;
  - workload 2, the colour cube (the bench workload): 262,144 colours x 128
    radii x 360 angles, 1.2e10 candidates (about 90 s of the oracle on 16
    host cores);
  - workload 3: the smallest image of the 48-image batch (991 x 312 pixels),
    per pixel directly and with per-batch de-duplication, against the oracle
    over the image's distinct colours mapped back to the pixels.
Then the FP32 chain itself over every 8-bit colour: on the image grid (all
2^24 colours x 64 radii x 180 angles, the grid of the capacity and embedding
tables) and on the cube's 128 radii (every tenth angle), no FP32 code that
the search would take without re-deciding it may differ from FP64, and the
largest FP32 error near a rounding boundary must stay below half the window.
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


def same(got, exp, what):
    gm, gc, gp = got
    em, ec, ep = exp
    bad = np.nonzero((gc != ec) | (gp != ep) | (gm.view(np.uint32) != em.view(np.uint32)))[0]
    assert bad.size == 0, f"{what}: {bad.size} mismatches, first {bad[:5]}"


def gpu_colors(ctx, torch, rgb, radii, ang):
    out = ctx.search_colors(dev(torch, rgb), radii, ang, 50.0, 0.5)
    torch.cuda.synchronize()
    return tuple(x.cpu().numpy() for x in out)


def test_precision_set_in_full(ctx, torch_cuda):
    rgb = W.precision_colors()
    radii, ang = W.grid(4)
    got = gpu_colors(ctx, torch_cuda, rgb, radii, ang)
    exp = oracle.search_colors(rgb, radii, ang, 50.0, 0.5, threads=THREADS)
    same(got, exp, "workload 4 in full")
    assert exp[1].sum() > 0


@pytest.mark.slow
def test_colour_cube_in_full(ctx, torch_cuda):
    rgb = W.color_cube()
    radii, ang = W.grid(2)
    got = gpu_colors(ctx, torch_cuda, rgb, radii, ang)
    exp = oracle.search_colors(rgb, radii, ang, 50.0, 0.5, threads=THREADS)
    same(got, exp, "workload 2 in full")
    assert (exp[1] > 0).sum() > 1000


def smallest_batch_image():
    params = W.image_params()
    i = min(range(len(params)), key=lambda j: params[j][0] * params[j][1])
    w, h, terms, ns = params[i]
    return W.render_image_numpy(w, h, terms, ns)


@pytest.mark.slow
@pytest.mark.parametrize("dedup", [0, 1])
def test_batch_image_in_full(ctx, torch_cuda, dedup):
    torch = torch_cuda
    img = smallest_batch_image()
    h, w, _ = img.shape
    radii, ang = W.grid(3)
    ctx.set_option("dedup", dedup)
    try:
        maps = ctx.search_images([dev(torch, img)], radii, ang, 50.0, 0.5)
        torch.cuda.synchronize()
    finally:
        ctx.set_option("dedup", 2)
    got = tuple(x.cpu().numpy().reshape(-1) for x in maps[0])
    key = (img[..., 0].astype(np.uint32) << 16) | (img[..., 1].astype(np.uint32) << 8) | img[..., 2]
    uniq, inv = np.unique(key.reshape(-1), return_inverse=True)
    urgb = np.stack([(uniq >> 16) & 255, (uniq >> 8) & 255, uniq & 255], 1).astype(np.uint8)
    em, ec, ep = oracle.search_colors(urgb, radii, ang, 50.0, 0.5, threads=THREADS)
    same(got, (em[inv], ec[inv], ep[inv]), f"workload 3 image {w}x{h}, dedup {dedup}")


def all_colours():
    v = np.arange(1 << 24, dtype=np.uint32)
    return np.stack([(v >> 16) & 255, (v >> 8) & 255, v & 255], axis=1).astype(np.uint8)


@pytest.mark.slow
@pytest.mark.parametrize("grid", ["image grid", "cube radii"])
def test_fp32_window_holds_for_every_colour(ctx, torch_cuda, grid):
    if grid == "image grid":
        radii, ang = W.grid(3)
    else:
        radii, ang = W.grid(2)
        ang = ang[::10]  # 36 angles, still closed under +180 degrees
    pr = ctx.precision_probe(dev(torch_cuda, all_colours()), radii, ang)
    print(grid, pr)
    assert pr["n_values"] >= (1 << 24) * len(radii) * len(ang) * 3
    assert pr["n_unflagged_wrong"] == 0  # every unflagged FP32 code equals FP64
    assert pr["max_code_err"] < pr["window"] / 2
    assert pr["n_wrong_codes"] > 0  # the flag window is what keeps the rest exact
