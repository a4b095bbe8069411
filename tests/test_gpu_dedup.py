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
