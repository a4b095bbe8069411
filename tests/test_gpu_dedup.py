"""Per-batch colour de-duplication of the image search (option "dedup";
needs a GPU).  The maps must be identical to the per-pixel search's, the
number of searched targets must equal the number of distinct colours, and
small ragged images with row pitch must equal the oracle."""
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


def maps_of(ctx, torch, imgs, radii, ang, dedup):
    ctx.set_option("dedup", dedup)
    maps = ctx.search_images(imgs, radii, ang, 50.0, 0.5)
    torch.cuda.synchronize()
    ctx.synchronize()
    return [tuple(x.cpu().numpy() for x in m) for m in maps], ctx.stats()


def test_workload3_images_identical_with_and_without_dedup(torch_cuda):
    torch = torch_cuda
    ctx = cvs.Context(0)
    radii, ang = W.grid(3)
    params = W.image_params(8, seed=0)
    imgs = [W.render_image_torch(w, h, t, s, device="cuda") for w, h, t, s in params]
    direct, _ = maps_of(ctx, torch, imgs, radii, ang, 0)
    dedup, st = maps_of(ctx, torch, imgs, radii, ang, 1)
    for a, b in zip(direct, dedup):
        assert np.array_equal(a[0].view(np.uint32), b[0].view(np.uint32))
        assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
    keys = np.concatenate([((im[..., 0].long() << 16) | (im[..., 1].long() << 8) | im[..., 2].long())
                           .reshape(-1).cpu().numpy() for im in imgs])
    assert st["targets"] == len(np.unique(keys))
    ctx.close()


def test_small_ragged_images_match_oracle(torch_cuda):
    torch = torch_cuda
    ctx = cvs.Context(0)
    radii, ang = W.grid(3)
    sizes = [(37, 23), (5, 1), (1, 9), (64, 40)]
    params = W.image_params(len(sizes), seed=4, sizes=sizes)
    hosts = [W.render_image_numpy(w, h, t, s) for w, h, t, s in params]
    hosts[1][:] = hosts[1][0, 0]  # one colour only
    imgs = []
    for im in hosts:  # row pitch 3 w + 8
        h, w, _ = im.shape
        buf = torch.zeros((h, 3 * w + 8), dtype=torch.uint8, device="cuda")
        buf[:, :3 * w] = torch.from_numpy(im.reshape(h, 3 * w)).cuda()
        imgs.append(torch.as_strided(buf, (h, w, 3), (3 * w + 8, 3, 1)))
    got, _ = maps_of(ctx, torch, imgs, radii, ang, 1)
    for im, g in zip(hosts, got):
        em, ec, ep = oracle.search_colors(im.reshape(-1, 3), radii, ang, 50.0, 0.5,
                                          threads=THREADS)
        assert np.array_equal(g[1].reshape(-1), ec) and np.array_equal(g[2].reshape(-1), ep)
        assert np.array_equal(g[0].reshape(-1).view(np.uint32), em.view(np.uint32))
    ctx.close()


def same_maps(a, b):
    for x, y in zip(a, b):
        assert np.array_equal(x[0].view(np.uint32), y[0].view(np.uint32))
        assert np.array_equal(x[1], y[1]) and np.array_equal(x[2], y[2])


def test_automatic_dedup(torch_cuda):
    """The default (dedup 2) searches each distinct colour once for batches of
    at least 2^20 pixels, unless CUDA graphs are on; the maps never change."""
    torch = torch_cuda
    ctx = cvs.Context(0)
    assert ctx.get_option("dedup") == 2
    radii, ang = W.grid(3)
    (w, h, t, s), = W.image_params(1, seed=9, sizes=[(1024, 1024)])
    img = W.render_image_torch(w, h, t, s, device="cuda")
    n_distinct = len(torch.unique((img[..., 0].long() << 16) | (img[..., 1].long() << 8)
                                  | img[..., 2].long()))
    direct, st = maps_of(ctx, torch, [img], radii, ang, 0)
    assert st["targets"] == 1 << 20
    auto, st = maps_of(ctx, torch, [img], radii, ang, 2)
    assert st["targets"] == n_distinct < 1 << 20
    same_maps(direct, auto)
    below, st = maps_of(ctx, torch, [img[:1023]], radii, ang, 2)  # one row short
    assert st["targets"] == 1023 * 1024
    same_maps([tuple(x[:1023] for x in direct[0])], below)
    ctx.set_option("graphs", 1)
    try:
        graphed, st = maps_of(ctx, torch, [img], radii, ang, 2)
        assert st["targets"] == 1 << 20
        same_maps(direct, graphed)
    finally:
        ctx.set_option("graphs", 0)
    ctx.close()


def test_automatic_dedup_within_budget(torch_cuda):
    """A budget that holds the per-pixel search of a 2^20-pixel batch never
    makes the automatic mode fail: tables that do not fit leave the search
    per pixel, with the same maps, and the context stays within its budget."""
    torch = torch_cuda
    radii, ang = W.grid(3)
    (w, h, t, s), = W.image_params(1, seed=9, sizes=[(1024, 1024)])
    img = W.render_image_torch(w, h, t, s, device="cuda")
    probe = cvs.Context(0)
    direct, _ = maps_of(probe, torch, [img], radii, ang, 0)
    need = probe.get_option("mem_in_use")
    probe.close()
    for budget in (need, need + (64 << 20), need + (256 << 20)):
        ctx = cvs.Context(0, mem_budget=budget)
        got, st = maps_of(ctx, torch, [img], radii, ang, 2)
        same_maps(direct, got)
        assert ctx.get_option("mem_in_use") <= budget
        assert st["targets"] <= 1 << 20
        ctx.close()
