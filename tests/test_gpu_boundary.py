"""The context's memory budget (cvs_create's mem_budget_bytes; needs a GPU).

A context allocates its scratch lazily.  With a budget, a call whose scratch
would exceed it fails with CVS_ERR_NO_MEMORY before any device work, and the
context stays usable for calls that fit; results within the budget equal the
oracle's.
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


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def maps(out):
    return tuple(x.cpu().numpy() for x in out)


def same(got, exp, what):
    gm, gc, gp = got
    em, ec, ep = exp
    bad = np.nonzero((gc != ec) | (gp != ep) | (gm.view(np.uint32) != em.view(np.uint32)))[0]
    assert bad.size == 0, f"{what}: {bad.size} mismatches, first {bad[:5]}"


def test_budget_refuses_what_does_not_fit_and_stays_usable(torch_cuda):
    torch = torch_cuda
    budget = 4 << 20
    radii, ang = W.grid(3)
    small = W.color_cube(32)[:200]
    with cvs.Context(0, mem_budget=budget) as ctx:
        assert ctx.get_option("mem_budget") == budget
        a = maps(ctx.search_colors(dev(torch, small), radii, ang, 50.0, 0.5))
        used = ctx.get_option("mem_in_use")
        assert 0 < used <= budget
        # 262,144 targets need about 25 MB of per-target scratch
        with pytest.raises(cvs.CvsError) as ei:
            ctx.search_colors(dev(torch, W.color_cube()), radii, ang, 50.0, 0.5)
        assert ei.value.status == binding.CVS_ERR_NO_MEMORY and "budget" in str(ei.value)
        assert ctx.get_option("mem_in_use") <= budget
        b = maps(ctx.search_colors(dev(torch, small), radii, ang, 50.0, 0.5))
        same(b, a, "after a refused call")
    exp = oracle.search_colors(small, radii, ang, 50.0, 0.5, threads=THREADS)
    same(a, exp, "within the budget")


def test_luminance_table_counts_against_the_budget(torch_cuda):
    torch = torch_cuda
    radii, ang = W.grid(3)
    rgb = dev(torch, W.color_cube(32)[:16])
    with cvs.Context(0, mem_budget=64 << 20) as ctx:
        ctx.search_colors(rgb, radii, ang, 50.0, 0.5)
        with pytest.raises(cvs.CvsError) as ei:  # the L* table alone is 128 MiB
            ctx.search_colors(rgb, radii, ang, 50.0, 0.5, max_dl=0.2)
        assert ei.value.status == binding.CVS_ERR_NO_MEMORY
        ctx.search_colors(rgb, radii, ang, 50.0, 0.5)


def test_budget_too_small_for_the_context_itself(torch_cuda):
    with pytest.raises(cvs.CvsError) as ei:
        cvs.Context(0, mem_budget=64)
    assert ei.value.status == binding.CVS_ERR_NO_MEMORY


def test_unbudgeted_context_reports_its_memory(torch_cuda):
    torch = torch_cuda
    radii, ang = W.grid(3)
    with cvs.Context(0) as ctx:
        assert ctx.get_option("mem_budget") == 0
        before = ctx.get_option("mem_in_use")
        ctx.search_colors(dev(torch, W.color_cube(16)), radii, ang, 50.0, 0.5)
        ctx.synchronize()
        assert ctx.get_option("mem_in_use") > before > 0
