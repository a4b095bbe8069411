"""Pair lists of many colours, cvs_search_colors_pairs (needs a GPU).

The search leaves each work item's passing-slot bitmap; a scan and the emit
kernel write every record straight to its place.  Each colour's group of
records must equal the oracle's pair list for that colour exactly (radius and
angle indices, both emitted colours, pattern), in (k, m) order, with the
colour's index as the target; the group sizes must equal the per-colour
counts.  Covered: the
bench's pair-list workload in full, several radii per work item and one,
grids whose items are capped by the bitmap size, unfolded and unsorted grids,
many batches of colours, FP64, and the truncation contract.
"""
import ctypes
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


def check_groups(recs, offs, rgb, radii, ang, sample, **thr):
    recs = recs.cpu().numpy().view(cvs.PAIR_DTYPE).reshape(-1)
    _, count, _ = oracle.search_colors(rgb, radii, ang, 50.0, 0.5, threads=THREADS, **thr)
    assert np.array_equal(np.diff(offs), count.astype(np.int64))
    assert np.array_equal(recs["target"], np.repeat(np.arange(len(rgb)), count))
    for i in sample:
        exp, n = oracle.search_color(rgb[i], radii, ang, 50.0, 0.5, **thr)
        got = recs[offs[i]:offs[i + 1]]
        assert len(got) == n
        for f in ("k", "m", "plus", "minus", "pattern"):
            assert np.array_equal(got[f], exp[f]), (i, f)


@pytest.mark.parametrize("gamut", [0, 1])
def test_table1_colours_match_oracle(ctx, torch_cuda, gamut):
    rgb = np.array(list(W.TABLE1_COLORS.values()), np.uint8)
    radii, ang = W.grid(1)
    recs, offs = ctx.search_colors_pairs(torch_cuda.from_numpy(rgb).cuda(), radii, ang, 50.0, 0.5,
                                         gamut_mode=gamut)
    check_groups(recs, offs, rgb, radii, ang, range(len(rgb)), gamut_mode=gamut)
    assert offs[-1] > 0


def test_precision_grid(ctx, torch_cuda):
    """256 radii x 720 angles (16 radii per work item at most)."""
    rgb = W.precision_colors()[::10][:400]
    radii, ang = W.grid(4)
    recs, offs = ctx.search_colors_pairs(torch_cuda.from_numpy(rgb).cuda(), radii, ang, 50.0, 0.5)
    rng = np.random.default_rng(4)
    check_groups(recs, offs, rgb, radii, ang, rng.choice(len(rgb), 12, replace=False))


def test_bench_workload_in_full(ctx, torch_cuda):
    """The bench's pair-list workload: 4096 colours x 64 radii x 180 angles,
    every group against the oracle."""
    rgb = W.precision_colors()
    radii, ang = W.grid(3)
    recs, offs = ctx.search_colors_pairs(torch_cuda.from_numpy(rgb).cuda(), radii, ang, 50.0, 0.5)
    check_groups(recs, offs, rgb, radii, ang, range(len(rgb)))
    assert offs[-1] > 1_000_000


GRIDS = {
    "unsorted radii": (np.array([30.0, 1.0, 25.0, 7.0, 31.5, 14.0, 0.5, 22.0, 12.25, 3.0]),
                       np.arange(360) * 1.0),
    "unfolded, 5 angles": (np.arange(1, 33) * 1.0, np.arange(5) * 72.0),
    "4096 slots per radius": (np.array([4.0, 11.5, 19.0, 26.5, 32.0]),
                              np.arange(8192) * (360.0 / 8192)),
    "8192 unfolded angles": (np.array([6.0, 17.0, 29.0]), np.arange(8192) * (359.0 / 8191)),
}


@pytest.mark.parametrize("name", list(GRIDS))
@pytest.mark.parametrize("kchunk", [0, 1, 3])
def test_grids_and_work_item_sizes(ctx, torch_cuda, name, kchunk):
    rgb = W.precision_colors()[::64]
    radii, ang = GRIDS[name]
    ctx.set_option("kchunk", kchunk)
    try:
        recs, offs = ctx.search_colors_pairs(torch_cuda.from_numpy(rgb).cuda(), radii, ang,
                                             50.0, 0.5)
    finally:
        ctx.set_option("kchunk", 0)
    check_groups(recs, offs, rgb, radii, ang, range(0, len(rgb), 5))


@pytest.mark.parametrize("items", [1, 7, 1000])
def test_many_batches(ctx, torch_cuda, items):
    """Batches of a few work items: each batch's first record follows the
    records of the batches before it."""
    rgb = W.precision_colors()[:300:3]
    radii, ang = W.grid(1)
    ctx.set_option("list_batch_items", items)
    try:
        recs, offs = ctx.search_colors_pairs(torch_cuda.from_numpy(rgb).cuda(), radii, ang,
                                             50.0, 0.5)
    finally:
        ctx.set_option("list_batch_items", 1 << 22)
    check_groups(recs, offs, rgb, radii, ang, range(len(rgb)))


@pytest.mark.parametrize("gamut", [0, 1])
def test_fp64_lists_and_flags(ctx, torch_cuda, gamut):
    rgb = np.array(list(W.TABLE1_COLORS.values()), np.uint8)
    radii, ang = W.grid(1)
    d = torch_cuda.from_numpy(rgb).cuda()
    r64, o64 = ctx.search_colors_pairs(d, radii, ang, 50.0, 0.5, gamut_mode=gamut,
                                       precision=binding.PREC_FP64)
    r32, o32 = ctx.search_colors_pairs(d, radii, ang, 50.0, 0.5, gamut_mode=gamut)
    a = r64.cpu().numpy().view(cvs.PAIR_DTYPE).reshape(-1)
    b = r32.cpu().numpy().view(cvs.PAIR_DTYPE).reshape(-1)
    assert np.array_equal(o64, o32) and (a["flags"] == 1).all()
    assert b["flags"].max() <= 1
    a["flags"] = 0
    b["flags"] = 0
    assert a.tobytes() == b.tobytes()
    check_groups(r64, o64, rgb, radii, ang, range(len(rgb)), gamut_mode=gamut)


def test_truncation_and_empty(ctx, torch_cuda):
    torch = torch_cuda
    rgb = torch.tensor([[170, 170, 170], [240, 100, 100]], dtype=torch.uint8, device="cuda")
    radii, ang = W.grid(1)
    g, keep = binding.make_grid(radii, ang)
    t = binding.make_thresholds(50.0, 0.5)
    out = torch.empty((4, 16), dtype=torch.uint8, device="cuda")
    offs = np.zeros(3, np.int64)
    total = ctypes.c_int64()
    st = cvs.lib().cvs_search_colors_pairs(ctx._h, rgb.data_ptr(), 2, ctypes.byref(g),
                                           ctypes.byref(t), binding.PREC_FP32_RECHECK,
                                           out.data_ptr(), 4, offs.ctypes.data,
                                           ctypes.byref(total), None)
    assert st == binding.CVS_ERR_TRUNCATED and total.value == offs[2] > 4
    _, count, _ = oracle.search_colors(rgb.cpu().numpy(), radii, ang, 50.0, 0.5)
    assert list(np.diff(offs)) == list(count)
    # the records that fit are the first ones of the full list
    full, _ = ctx.search_colors_pairs(rgb, radii, ang, 50.0, 0.5)
    assert out.cpu().numpy().tobytes() == full[:4].cpu().numpy().tobytes()
    recs, offs0 = ctx.search_colors_pairs(rgb[:0], radii, ang, 50.0, 0.5)
    assert recs.shape[0] == 0 and list(offs0) == [0]
