"""Pair lists of many colours, cvs_search_colors_pairs (needs a GPU).

Each colour's group of records must equal the oracle's pair list for that
colour exactly (radius and angle indices, both emitted colours, pattern), in
(k, m) order, with the colour's index as the target; the group sizes must
equal the per-colour counts.  A grid large enough to need several batches of
dense records is covered, and the truncation contract is checked.
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


def test_several_batches(ctx, torch_cuda):
    """256 radii x 720 angles: 2.9 MB of dense records per colour, so 400
    colours need three batches."""
    rgb = W.precision_colors()[::10][:400]
    radii, ang = W.grid(4)
    recs, offs = ctx.search_colors_pairs(torch_cuda.from_numpy(rgb).cuda(), radii, ang, 50.0, 0.5)
    rng = np.random.default_rng(4)
    check_groups(recs, offs, rgb, radii, ang, rng.choice(len(rgb), 12, replace=False))


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
    recs, offs0 = ctx.search_colors_pairs(rgb[:0], radii, ang, 50.0, 0.5)
    assert recs.shape[0] == 0 and list(offs0) == [0]
