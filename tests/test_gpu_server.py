"""The continuous-batching request loop (needs a GPU).

Each frame's maps must be the same whether the frame is served alone or in a
mix with others on the device, and the same as a direct cvs_search_images
call; admission must wait for memory; host waits are bounded."""
import numpy as np
import pytest

import paper_2507_22901_gb300 as cvs
from paper_2507_22901_gb300 import binding, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def frames(n, seed=0):
    sizes = [(320, 240), (640, 360), (97, 53), (512, 512), (33, 600), (800, 450), (1, 1), (255, 3)]
    params = W.image_params(n, seed=seed, sizes=[sizes[i % len(sizes)] for i in range(n)])
    return [W.render_image_numpy(w, h, t, ns) for w, h, t, ns in params]


def direct(torch, fr):
    radii, ang = W.grid(3)
    ctx = cvs.Context(0)
    maps = ctx.search_images([torch.from_numpy(f).cuda() for f in fr], radii, ang, 50, 0.5)
    torch.cuda.synchronize()
    out = [tuple(x.cpu().numpy() for x in m) for m in maps]
    ctx.close()
    return out


def same(a, b):
    return (np.array_equal(a[0].view(np.uint32), b[0].view(np.uint32)) and
            np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2]))


@pytest.mark.parametrize("mode", ["search", "table", "search per distinct colour"])
def test_alone_equals_mix_equals_direct(torch_cuda, mode):
    fr = frames(8)
    ref = direct(torch_cuda, fr)
    radii, ang = W.grid(3)
    srv = cvs.Server(radii, ang, 50, 0.5, max_inflight=3, max_pixels=1 << 20,
                     mem_budget_bytes=64 << 20, use_table=(mode == "table"),
                     dedup=(mode == "search per distinct colour"))
    alone = []
    for f in fr:  # one at a time
        t = srv.submit(f)
        srv.wait(t)
        alone.append(srv.result_host(t))
        srv.release(t)
    tickets = [srv.submit(f) for f in fr]  # all at once: they overlap on the device
    mix = []
    for t in tickets:
        srv.wait(t)
        mix.append(srv.result_host(t))
        srv.release(t)
    st = srv.stats()
    srv.close()
    for r, a, m in zip(ref, alone, mix):
        assert same(r, a) and same(r, m)
    assert st["completed"] == 16 and st["failed"] == 0 and st["p99_ms"] >= st["p50_ms"] > 0


def test_admission_waits_for_memory(torch_cuda):
    fr = frames(6, seed=1)
    fr = [np.ascontiguousarray(np.broadcast_to(f[:1, :1], (400, 500, 3))) if i % 2 else f
          for i, f in enumerate(fr)]
    ref = direct(torch_cuda, fr)
    radii, ang = W.grid(3)
    px = max(f.shape[0] * f.shape[1] for f in fr)
    budget = 2 * (px * 12 + 1024)  # room for about two frames at a time
    srv = cvs.Server(radii, ang, 50, 0.5, max_inflight=4, max_pixels=px, mem_budget_bytes=budget)
    tickets = [srv.submit(f) for f in fr]
    got = {}
    pending = list(tickets)
    while pending:  # results must be released for the rest to be admitted
        t = pending.pop(0)
        srv.wait(t, 120000)
        got[t] = srv.result_host(t)
        srv.release(t)
    st = srv.stats()
    srv.close()
    assert st["peak_bytes_in_use"] <= budget
    for t, r in zip(tickets, ref):
        assert same(got[t], r)


def test_bounded_wait_and_release_rules(torch_cuda):
    radii, ang = W.grid(3)
    big = W.render_image_numpy(1600, 1200, W.image_params(1, seed=5)[0][2], 3)
    srv = cvs.Server(radii, ang, 50, 0.5, max_inflight=1, max_pixels=1600 * 1200,
                     mem_budget_bytes=2 * (1600 * 1200 * 12 + 1024))
    t1 = srv.submit(big)
    t2 = srv.submit(big)
    t3 = srv.submit(big)  # cannot be admitted while t1 and t2 hold the memory
    with pytest.raises(cvs.CvsError) as ei:
        srv.wait(t1, 0)
    assert ei.value.status == binding.CVS_ERR_TIMEOUT
    assert srv.state(t3) == binding.REQ_QUEUED
    srv.release(t3)  # cancel a queued request
    assert srv.state(t3) == binding.REQ_UNKNOWN
    srv.wait(t1, 120000)
    srv.wait(t2, 120000)
    with pytest.raises(cvs.CvsError):
        srv.submit(np.zeros((1300, 1600, 3), np.uint8))  # larger than max_pixels
    srv.release(t1)
    srv.release(t2)
    assert srv.stats()["completed"] == 2
    srv.close()
