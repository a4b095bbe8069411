"""The allocation-free entry point, cvs_search_colors_noalloc.

Some callers cannot allocate device memory - for example code hosted inside an
application whose memory manager owns the device heap, or a latency-critical
loop that cannot afford cudaMalloc's device-wide synchronisation.  For them the
library offers cvs_search_colors_noalloc, which keeps all of its scratch in one
fixed array inside the library.  This test calls it through the C ABI twice in
a row, on different inputs, and checks each result against the regular entry
point cvs_search_colors (exact equality, the tolerance of every parity test
here), then checks that sizes beyond the fixed array's limits are refused.

The file sorts last so that a run stopping at the first failure has already
run every other test.
"""
import ctypes

import numpy as np
import pytest

import paper_2507_22901_gb300 as cvs
from paper_2507_22901_gb300 import binding, workloads as W

pytestmark = pytest.mark.gpu


def _noalloc(torch, rgb, radii, ang, thr):
    """Call the C entry point directly with caller-owned device buffers."""
    n = rgb.shape[0]
    d_rgb = torch.from_numpy(np.ascontiguousarray(rgb)).cuda()
    out = (torch.full((n,), 7.0, dtype=torch.float32, device="cuda"),
           torch.full((n,), 7, dtype=torch.int32, device="cuda"),
           torch.full((n,), 7, dtype=torch.uint8, device="cuda"))
    g, keep = binding.make_grid(radii, ang)
    t = binding.make_thresholds(**thr)
    m = binding.cvs_capacity_map(out[0].data_ptr(), out[1].data_ptr(), out[2].data_ptr())
    st = cvs.lib().cvs_search_colors_noalloc(0, d_rgb.data_ptr(), n, ctypes.byref(g),
                                             ctypes.byref(t), binding.PREC_FP32_RECHECK,
                                             ctypes.byref(m), None)
    binding.check(st, "cvs_search_colors_noalloc")
    torch.cuda.synchronize()
    return tuple(x.cpu().numpy() for x in out)


def _regular(ctx, torch, rgb, radii, ang, thr):
    out = ctx.search_colors(torch.from_numpy(np.ascontiguousarray(rgb)).cuda(), radii, ang,
                            thr["v_th"], thr["r_novib"], thr["pattern_mask"], thr["gamut_mode"])
    torch.cuda.synchronize()
    return tuple(x.cpu().numpy() for x in out)


def _same(a, b):
    assert np.array_equal(a[0].view(np.uint32), b[0].view(np.uint32))
    assert np.array_equal(a[1], b[1])
    assert np.array_equal(a[2], b[2])


def test_noalloc_matches_regular_entry_point_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = cvs.Context(0)
    # first call: the 4096-colour precision set (the size limit) on the image grid
    rgb1 = W.precision_colors()
    r1, a1 = W.grid(3)
    thr1 = dict(W.DEFAULT_THRESHOLDS)
    got1 = _noalloc(torch, rgb1, r1, a1, thr1)
    _same(got1, _regular(ctx, torch, rgb1, r1, a1, thr1))
    assert got1[1].sum() > 0
    # second call in a row: other colours, grid and thresholds over the same array
    rgb2 = W.color_cube(step=32)[:300]
    r2, a2 = np.arange(1, 97) * 0.25, np.arange(360) * 1.0
    thr2 = dict(v_th=100.0, r_novib=0.25, pattern_mask=0x7F, gamut_mode=1)
    got2 = _noalloc(torch, rgb2, r2, a2, thr2)
    _same(got2, _regular(ctx, torch, rgb2, r2, a2, thr2))
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_array():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    with pytest.raises(cvs.CvsError) as ei:
        _noalloc(torch, np.zeros((4097, 3), np.uint8), [1.0], [0.0], dict(W.DEFAULT_THRESHOLDS))
    assert ei.value.status == binding.CVS_ERR_INVALID_ARG and "4096" in str(ei.value)
    with pytest.raises(cvs.CvsError) as ei:
        _noalloc(torch, np.zeros((4, 3), np.uint8), np.arange(1025) * 0.1, [0.0],
                 dict(W.DEFAULT_THRESHOLDS))
    assert ei.value.status == binding.CVS_ERR_INVALID_ARG and "1024" in str(ei.value)
