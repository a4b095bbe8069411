"""Full-size parity (needs a GPU).

The bench workload runs in exactly the launch configuration the bench times
(all 262,144 cube colours, 128 radii x 360 angles, one call), and sampled
colours are compared with the oracle one by one.  The largest grids the
library accepts (8192 radii; 8192 angles) are compared with the oracle in
full for a few colours, and one past either limit is refused.
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


def same(got, exp, what):
    gm, gc, gp = got
    em, ec, ep = exp
    bad = np.nonzero((gc != ec) | (gp != ep) | (gm.view(np.uint32) != em.view(np.uint32)))[0]
    assert bad.size == 0, f"{what}: {bad.size} mismatches, first {bad[:5]}"


def test_bench_workload_sampled_against_oracle(ctx, torch_cuda):
    cube = W.color_cube()
    radii, ang = W.grid(2)
    out = ctx.search_colors(torch_cuda.from_numpy(cube).cuda(), radii, ang, 50.0, 0.5)
    torch_cuda.cuda.synchronize()
    got = tuple(x.cpu().numpy() for x in out)
    idx = np.random.default_rng(2024).choice(len(cube), 256, replace=False)
    exp = oracle.search_colors(cube[idx], radii, ang, 50.0, 0.5, threads=THREADS)
    same(tuple(x[idx] for x in got), exp, "bench workload, sampled")
    assert exp[1].sum() > 0


@pytest.mark.parametrize("shape", ["radii", "angles"])
def test_largest_grids(ctx, torch_cuda, shape):
    rgb = np.array([[170, 170, 170], [240, 100, 100], [30, 200, 60], [100, 240, 240]], np.uint8)
    if shape == "radii":
        radii, ang = np.arange(1, 8193) * (32.0 / 8192), np.arange(0.0, 360.0, 15.0)
    else:
        radii, ang = np.array([6.0, 14.0, 22.0, 31.5]), np.arange(8192) * (360.0 / 8192)
    out = ctx.search_colors(torch_cuda.from_numpy(rgb).cuda(), radii, ang, 50.0, 0.5)
    torch_cuda.cuda.synchronize()
    exp = oracle.search_colors(rgb, radii, ang, 50.0, 0.5, threads=THREADS)
    same(tuple(x.cpu().numpy() for x in out), exp, f"largest grid ({shape})")
    assert exp[1].sum() > 0


def test_one_past_the_limits_is_refused(ctx, torch_cuda):
    rgb = torch_cuda.zeros((2, 3), dtype=torch_cuda.uint8, device="cuda")
    for radii, ang in ((np.arange(1, 8194) * 0.001, [0.0]), ([1.0], np.arange(8193) * 0.01)):
        with pytest.raises(cvs.CvsError) as ei:
            ctx.search_colors(rgb, radii, ang, 50.0, 0.5)
        assert ei.value.status == binding.CVS_ERR_INVALID_ARG and "8192" in str(ei.value)
