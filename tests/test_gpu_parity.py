"""Parity of the CUDA library with the FP64 CPU oracle (needs a GPU).

Every comparison is exact: 8-bit codes, pass/fail decisions, patterns, counts,
bit patterns of the largest radius, and the FP64 tables (trig, target L*a*b*).
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


def assert_maps_equal(got, exp, what=""):
    gm, gc, gp = (np.asarray(x) for x in got)
    em, ec, ep = exp
    bad = np.nonzero((gc != ec) | (gp != ep) | (gm.view(np.uint32) != em.view(np.uint32)))[0]
    assert bad.size == 0, f"{what}: {bad.size} mismatches, first {bad[:5]}: " \
        f"gpu {gc[bad[:5]]} {gm[bad[:5]]} {gp[bad[:5]]} oracle {ec[bad[:5]]} {em[bad[:5]]} {ep[bad[:5]]}"


def gpu_colors(ctx, torch, rgb, radii, ang, prec, **thr):
    t = dict(W.DEFAULT_THRESHOLDS)
    t.update(thr)
    out = ctx.search_colors(dev(torch, rgb), radii, ang, t["v_th"], t["r_novib"],
                            t["pattern_mask"], t["gamut_mode"], precision=prec)
    torch.cuda.synchronize()
    return tuple(x.cpu().numpy() for x in out)


def oracle_colors(rgb, radii, ang, **thr):
    t = dict(W.DEFAULT_THRESHOLDS)
    t.update(thr)
    return oracle.search_colors(rgb, radii, ang, t["v_th"], t["r_novib"], t["pattern_mask"],
                                t["gamut_mode"], threads=THREADS)


# ------------------------------------------------------------------ tables
def test_trig_table_bitwise(ctx):
    rng = np.random.default_rng(9)
    ang = np.concatenate([W.grid(1)[1], W.grid(3)[1], W.grid(4)[1],
                          [-30.0, -180.0, 390.0, 720.5, 1e6 + 0.25, 45.0, 89.99, 0.1, 1e-12],
                          rng.uniform(-1000, 1000, 500)])
    s, c = ctx.trig_table(ang)
    so, co = oracle.trig_table(ang)
    assert np.array_equal(s.view(np.uint64), so.view(np.uint64))
    assert np.array_equal(c.view(np.uint64), co.view(np.uint64))


def test_target_lab_all_colours_bitwise(ctx, torch_cuda):
    torch = torch_cuda
    v = np.arange(1 << 24, dtype=np.uint32)
    rgb = np.stack([(v >> 16) & 255, (v >> 8) & 255, v & 255], axis=1).astype(np.uint8)
    lab = ctx.target_lab(dev(torch, rgb))
    torch.cuda.synchronize()
    got = lab.cpu().numpy()
    exp = oracle.target_lab_many(rgb, THREADS)
    diff = np.nonzero(np.any(got.view(np.uint64) != exp.view(np.uint64), axis=1))[0]
    assert diff.size == 0, (diff[:5], rgb[diff[:5]], got[diff[:5]], exp[diff[:5]])


# ------------------------------------------------------------------ config 1
@pytest.mark.parametrize("prec", [binding.PREC_FP32_RECHECK, binding.PREC_FP64])
@pytest.mark.parametrize("gamut", [0, 1])
def test_search_color_config1_all_table1_thresholds(ctx, prec, gamut):
    radii, ang = W.grid(1)
    tt = oracle.trig_table(ang)
    for vth in W.TABLE1_VTH:
        for rn in W.TABLE1_RNOVIB:
            exp, n_exp = oracle.search_color((170, 170, 170), radii, ang, vth, rn,
                                             gamut_mode=gamut, target=11, trig_tab=tt)
            got, n = ctx.search_color((170, 170, 170), radii, ang, vth, rn, gamut_mode=gamut,
                                      precision=prec, target=11)
            assert n == n_exp, (vth, rn)
            g = got.copy()
            g["flags"] = 0
            assert g.tobytes() == exp.tobytes(), (vth, rn)


@pytest.mark.parametrize("name", list(W.TABLE1_COLORS))
def test_search_color_table1_colours(ctx, name):
    radii, ang = W.grid(1)
    rgb = W.TABLE1_COLORS[name]
    for vth, rn in [(50, 0.5), (100, 0.25)]:
        exp, n_exp = oracle.search_color(rgb, radii, ang, vth, rn)
        got, n = ctx.search_color(rgb, radii, ang, vth, rn)
        got["flags"] = 0
        assert n == n_exp and got.tobytes() == exp.tobytes()


def test_search_color_truncation(ctx):
    radii, ang = W.grid(1)
    full, n = ctx.search_color((170, 170, 170), radii, ang, 50, 0.5)
    assert n > 100
    part, n2 = ctx.search_color((170, 170, 170), radii, ang, 50, 0.5, cap=100)
    assert n2 == n and len(part) == 100 and part.tobytes() == full[:100].tobytes()


# ------------------------------------------------------------------ config 2
def cube_sample(n, seed=5):
    cube = W.color_cube()
    rng = np.random.default_rng(seed)
    idx = rng.choice(len(cube), n, replace=False)
    extra = np.array([[0, 0, 0], [252, 252, 252], [252, 0, 0], [0, 252, 0], [0, 0, 252],
                      [4, 4, 4], [8, 0, 252], [128, 128, 128]], np.uint8)
    return np.concatenate([cube[idx], extra])


@pytest.mark.parametrize("prec", [binding.PREC_FP32_RECHECK, binding.PREC_FP64])
def test_cube_sample_full_grid(ctx, torch_cuda, prec):
    rgb = cube_sample(200)
    radii, ang = W.grid(2)
    exp = oracle_colors(rgb, radii, ang)
    got = gpu_colors(ctx, torch_cuda, rgb, radii, ang, prec)
    assert_maps_equal(got, exp, "cube sample")
    assert exp[1].sum() > 0


def test_cube_full_fp32_equals_fp64(ctx, torch_cuda):
    """All 262,144 colours x 128 radii x 360 angles (1.2e10 candidates): the FP32
    path with FP64 re-decision equals the all-FP64 path everywhere."""
    rgb = W.color_cube()
    radii, ang = W.grid(2)
    a = gpu_colors(ctx, torch_cuda, rgb, radii, ang, binding.PREC_FP32_RECHECK)
    ctx.synchronize()
    st = ctx.stats()
    b = gpu_colors(ctx, torch_cuda, rgb, radii, ang, binding.PREC_FP64)
    assert_maps_equal(a, b, "cube fp32 vs fp64")
    assert st["candidates"] == len(rgb) * 128 * 360 and st["symmetric"] == 1
    print(f"flagged {st['flagged'] / st['candidates']:.3e} rechecked "
          f"{st['rechecked'] / st['candidates']:.3e}")


# ------------------------------------------------------------------ config 4
@pytest.mark.parametrize("prec", [binding.PREC_FP32_RECHECK, binding.PREC_FP64])
def test_precision_set_sample(ctx, torch_cuda, prec):
    pc = W.precision_colors()
    rgb = np.concatenate([pc[:48], pc[3072:3072 + 40], pc[3584:3584 + 40]])
    radii, ang = W.grid(4)
    exp = oracle_colors(rgb, radii, ang)
    got = gpu_colors(ctx, torch_cuda, rgb, radii, ang, prec)
    assert_maps_equal(got, exp, "precision sample")


def test_precision_set_full_fp32_equals_fp64_and_probe(ctx, torch_cuda):
    rgb = W.precision_colors()
    radii, ang = W.grid(4)
    a = gpu_colors(ctx, torch_cuda, rgb, radii, ang, binding.PREC_FP32_RECHECK)
    b = gpu_colors(ctx, torch_cuda, rgb, radii, ang, binding.PREC_FP64)
    assert_maps_equal(a, b, "precision set fp32 vs fp64")
    pr = ctx.precision_probe(dev(torch_cuda, rgb), radii, ang)
    w = ctx.get_option("fp32_window")
    print("probe", pr, "window", w)
    assert pr["max_code_err"] < w / 2  # the window keeps a margin over the measured error
    assert pr["n_unflagged_wrong"] == 0 and pr["window"] == w
    assert pr["max_lab_err"] < 1e-4 and pr["n_values"] >= len(rgb) * 256 * 720 * 3


# ------------------------------------------------------------------ images
def small_images():
    params = W.image_params(6, seed=3, sizes=[(37, 23), (64, 1), (1, 5), (130, 70), (33, 33),
                                                (16, 9)])
    return [W.render_image_numpy(w, h, terms, ns) for w, h, terms, ns in params]


@pytest.mark.parametrize("prec", [binding.PREC_FP32_RECHECK, binding.PREC_FP64])
def test_images_small_ragged_with_pitch(ctx, torch_cuda, prec):
    torch = torch_cuda
    imgs = small_images()
    dimgs = []
    for im in imgs:  # pad each row by 7 bytes to exercise the pitch
        h, w, _ = im.shape
        buf = torch.zeros((h, w * 3 + 7), dtype=torch.uint8, device="cuda")
        buf[:, :w * 3] = dev(torch, im.reshape(h, w * 3))
        dimgs.append(buf[:, :w * 3].view(h, w, 3))
    radii, ang = W.grid(3)
    maps = ctx.search_images(dimgs, radii, ang, 50, 0.5, precision=prec)
    torch.cuda.synchronize()
    allpx = np.concatenate([im.reshape(-1, 3) for im in imgs])
    uniq, inv = np.unique(allpx, axis=0, return_inverse=True)
    exp = oracle_colors(uniq, radii, ang)
    off = 0
    for im, (mr, cn, pm) in zip(imgs, maps):
        n = im.shape[0] * im.shape[1]
        sel = inv.reshape(-1)[off:off + n]
        off += n
        assert_maps_equal((mr.cpu().numpy().ravel(), cn.cpu().numpy().ravel(),
                           pm.cpu().numpy().ravel()),
                          (exp[0][sel], exp[1][sel], exp[2][sel]), "image")


def test_images_full_size_sampled(ctx, torch_cuda):
    """The 48-image workload at full size (1.19e8 pixels) in the benchmark's
    launch configuration; 600 sampled pixels against the oracle."""
    torch = torch_cuda
    params = W.image_params()
    imgs = [W.render_image_torch(w, h, terms, ns) for w, h, terms, ns in params]
    radii, ang = W.grid(3)
    maps = ctx.search_images(imgs, radii, ang, 50, 0.5)
    torch.cuda.synchronize()
    rng = np.random.default_rng(17)
    picks = []
    for _ in range(600):
        i = int(rng.integers(0, len(imgs)))
        h, w = imgs[i].shape[:2]
        picks.append((i, int(rng.integers(0, h)), int(rng.integers(0, w))))
    rgb = np.array([imgs[i][y, x].cpu().numpy() for i, y, x in picks], np.uint8)
    exp = oracle_colors(rgb, radii, ang)
    got = (np.array([maps[i][0][y, x].item() for i, y, x in picks], np.float32),
           np.array([maps[i][1][y, x].item() for i, y, x in picks], np.int32),
           np.array([maps[i][2][y, x].item() for i, y, x in picks], np.uint8))
    assert_maps_equal(got, exp, "full-size images")


def test_result_is_function_of_colour(ctx, torch_cuda):
    torch = torch_cuda
    rng = np.random.default_rng(8)
    pal = rng.integers(0, 256, (5, 3)).astype(np.uint8)
    im = pal[rng.integers(0, 5, (40, 50))]
    radii, ang = W.grid(3)
    mr, cn, pm = ctx.search_images([dev(torch, im)], radii, ang, 50, 0.5)[0]
    torch.cuda.synchronize()
    for k in range(5):
        sel = np.all(im == pal[k], axis=2)
        assert len(np.unique(cn.cpu().numpy()[sel])) == 1
        assert len(np.unique(mr.cpu().numpy()[sel])) == 1


# ------------------------------------------------------------------ edge cases
@pytest.mark.parametrize("ang", [np.arange(7) * 51.0, np.arange(180) * 1.0,
                                 np.array([10.0, 190.0, 20.0, 200.5])])
def test_unfolded_angle_lists(ctx, torch_cuda, ang):
    rgb = cube_sample(40, seed=2)
    radii = np.arange(1, 33) * 1.0
    exp = oracle_colors(rgb, radii, ang)
    got = gpu_colors(ctx, torch_cuda, rgb, radii, ang, binding.PREC_FP32_RECHECK)
    assert_maps_equal(got, exp, "unfolded")
    ctx.synchronize()
    assert ctx.stats()["symmetric"] == 0


def test_clip_mode_and_masks(ctx, torch_cuda):
    rgb = cube_sample(60, seed=4)
    radii, ang = W.grid(3)
    for thr in [dict(gamut_mode=1), dict(pattern_mask=0b0000101), dict(v_th=100, r_novib=0.25),
                dict(v_th=37.5, r_novib=0.3, gamut_mode=1)]:
        exp = oracle_colors(rgb, radii, ang, **thr)
        got = gpu_colors(ctx, torch_cuda, rgb, radii, ang, binding.PREC_FP32_RECHECK, **thr)
        assert_maps_equal(got, exp, str(thr))


def test_radius_zero_and_unsorted_radii(ctx, torch_cuda):
    rgb = cube_sample(30, seed=6)
    ang = np.arange(360) * 1.0
    got = gpu_colors(ctx, torch_cuda, rgb, np.array([0.0]), ang, binding.PREC_FP32_RECHECK)
    assert (got[1] == 0).all() and (got[0] == -1.0).all() and (got[2] == 0).all()
    radii = np.array([20.0, 3.5, 31.0, 0.0, 12.25, 31.0])
    exp = oracle_colors(rgb, radii, ang)
    assert_maps_equal(gpu_colors(ctx, torch_cuda, rgb, radii, ang, 0), exp, "unsorted")


@pytest.mark.parametrize("kchunk", [1, 7, 300])
def test_ragged_work_items(ctx, torch_cuda, kchunk):
    rgb = cube_sample(24, seed=7)
    radii, ang = W.grid(2)
    exp = oracle_colors(rgb, radii, ang)
    ctx.set_option("kchunk", kchunk)
    try:
        got = gpu_colors(ctx, torch_cuda, rgb, radii, ang, binding.PREC_FP32_RECHECK)
    finally:
        ctx.set_option("kchunk", 0)
    assert_maps_equal(got, exp, f"kchunk {kchunk}")


def test_window_sizes_do_not_change_results(ctx, torch_cuda):
    rgb = cube_sample(64, seed=12)
    radii, ang = W.grid(2)
    base = gpu_colors(ctx, torch_cuda, rgb, radii, ang, binding.PREC_FP64)
    w0 = ctx.get_option("fp32_window")
    try:
        for w in (0.01, 0.2):
            ctx.set_option("fp32_window", w)
            assert_maps_equal(gpu_colors(ctx, torch_cuda, rgb, radii, ang, 0), base, f"W {w}")
    finally:
        ctx.set_option("fp32_window", w0)


def test_empty_and_invalid_inputs(ctx, torch_cuda):
    torch = torch_cuda
    radii, ang = W.grid(2)
    out = ctx.search_colors(torch.empty((0, 3), dtype=torch.uint8, device="cuda"), radii, ang,
                            50, 0.5)
    assert out[0].numel() == 0
    rgb = dev(torch, cube_sample(4))
    for r, a in [([float("nan")], ang), ([-1.0], ang), (radii, []), ([1.0], [float("inf")]),
                 ([1000.5], ang)]:
        with pytest.raises(cvs.CvsError) as ei:
            ctx.search_colors(rgb, r, a, 50, 0.5)
        assert ei.value.status == binding.CVS_ERR_INVALID_ARG
    with pytest.raises(cvs.CvsError):
        ctx.search_colors(rgb, radii, ang, 50, 0.0)
    with pytest.raises(cvs.CvsError):
        ctx.set_option("no_such_option", 1)


def test_host_entry_point_and_stream(ctx, torch_cuda):
    torch = torch_cuda
    rgb = cube_sample(50, seed=13)
    radii, ang = W.grid(2)
    exp = oracle_colors(rgb, radii, ang)
    assert_maps_equal(ctx.search_colors_host(rgb, radii, ang, 50, 0.5), exp, "host")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        d = dev(torch, rgb)
        out = ctx.search_colors(d, radii, ang, 50, 0.5, stream=s)
    ctx.synchronize(s)
    assert_maps_equal(tuple(x.cpu().numpy() for x in out), exp, "side stream")


def test_large_radii_need_fp64(ctx, torch_cuda):
    """Radii beyond the FP32 path's validated range (32): an FP32 request is
    refused with a message naming the remedies; FP64, asked for directly or
    through option fp64_fallback, matches the oracle."""
    rgb = cube_sample(16, seed=21)
    radii = np.array([5.0, 31.5, 40.0, 64.0, 120.0])
    ang = np.arange(72) * 5.0
    exp = oracle_colors(rgb, radii, ang)
    with pytest.raises(cvs.CvsError) as ei:
        gpu_colors(ctx, torch_cuda, rgb, radii, ang, binding.PREC_FP32_RECHECK)
    assert ei.value.status == binding.CVS_ERR_INVALID_ARG
    assert "CVS_PREC_FP64" in str(ei.value) and "fp64_fallback" in str(ei.value)
    got = gpu_colors(ctx, torch_cuda, rgb, radii, ang, binding.PREC_FP64)
    assert_maps_equal(got, exp, "large radii, FP64")
    ctx.set_option("fp64_fallback", 1)
    try:
        got = gpu_colors(ctx, torch_cuda, rgb, radii, ang, binding.PREC_FP32_RECHECK)
        ctx.synchronize()
        assert ctx.stats()["precision"] == binding.PREC_FP64
    finally:
        ctx.set_option("fp64_fallback", 0)
    assert_maps_equal(got, exp, "large radii, fallback")


# ------------------------------------------------------------------ batching machinery
def test_autotune_keeps_results(ctx, torch_cuda):
    torch = torch_cuda
    rgb = cube_sample(300, seed=31)
    radii, ang = W.grid(2)
    exp = oracle_colors(rgb, radii, ang)
    best = ctx.autotune(dev(torch, rgb), radii, ang, 50, 0.5)
    assert best["block"] in (64, 128) and 1 <= best["kchunk"] <= len(radii) and best["ms"] > 0
    assert_maps_equal(gpu_colors(ctx, torch, rgb, radii, ang, 0), exp, "after autotune")


def test_lazy_autotune_option(torch_cuda):
    torch = torch_cuda
    c = cvs.Context(0)
    c.set_option("autotune", 1)
    rgb = cube_sample(64, seed=32)
    radii, ang = W.grid(3)
    exp = oracle_colors(rgb, radii, ang)
    for _ in range(2):
        assert_maps_equal(gpu_colors(c, torch, rgb, radii, ang, 0), exp, "lazy autotune")
    c.close()


def test_graph_replay_colours_and_images(torch_cuda):
    torch = torch_cuda
    c = cvs.Context(0)
    c.set_option("graphs", 1)
    radii, ang = W.grid(3)
    a, b = cube_sample(120, seed=33), cube_sample(120, seed=34)
    d = dev(torch, a)
    out = (torch.empty(len(a), dtype=torch.float32, device="cuda"),
           torch.empty(len(a), dtype=torch.int32, device="cuda"),
           torch.empty(len(a), dtype=torch.uint8, device="cuda"))
    c.search_colors(d, radii, ang, 50, 0.5, out=out)
    c.synchronize()
    assert_maps_equal(tuple(x.cpu().numpy() for x in out), oracle_colors(a, radii, ang), "graph 1")
    d.copy_(torch.from_numpy(b))  # same buffers, new contents: the replay reads them
    c.search_colors(d, radii, ang, 50, 0.5, out=out)
    c.synchronize()
    assert_maps_equal(tuple(x.cpu().numpy() for x in out), oracle_colors(b, radii, ang), "graph 2")
    assert c.get_option("graph_launches") == 2 and c.get_option("graphs_cached") == 1
    st = c.stats()
    assert st["targets"] == len(b) and st["search_ms"] > 0
    # images through a graph, twice
    imgs = [dev(torch, im) for im in small_images()]
    m1 = [tuple(x.cpu().numpy().copy() for x in m) for m in c.search_images(imgs, radii, ang, 50, 0.5)]
    c.synchronize()
    m2 = [tuple(x.cpu().numpy() for x in m) for m in c.search_images(imgs, radii, ang, 50, 0.5)]
    c.synchronize()
    ref = cvs.Context(0)
    m3 = [tuple(x.cpu().numpy() for x in m) for m in ref.search_images(imgs, radii, ang, 50, 0.5)]
    torch.cuda.synchronize()
    for x, y, z in zip(m1, m2, m3):
        for p, q, r in zip(x, y, z):
            assert np.array_equal(p, r) and np.array_equal(q, r)
    ref.close()
    c.close()


# ------------------------------------------------------------------ capacity table
@pytest.fixture(scope="module")
def lut3(ctx):
    radii, ang = W.grid(3)
    t = ctx.build_lut(radii, ang, 50, 0.5)
    yield t
    t.close()


def test_lut_colours_match_oracle(lut3, torch_cuda):
    torch = torch_cuda
    rng = np.random.default_rng(41)
    rgb = np.concatenate([rng.integers(0, 256, (1500, 3)), W.precision_colors()[3072:3172],
                          [[0, 0, 0], [255, 255, 255], [255, 0, 0], [1, 254, 3]]]).astype(np.uint8)
    radii, ang = W.grid(3)
    out = lut3.lookup_colors(dev(torch, rgb))
    torch.cuda.synchronize()
    assert_maps_equal(tuple(x.cpu().numpy() for x in out), oracle_colors(rgb, radii, ang), "lut")


def test_lut_images_match_direct_search(ctx, lut3, torch_cuda):
    torch = torch_cuda
    radii, ang = W.grid(3)
    small = [dev(torch, im) for im in small_images()]
    params = W.image_params(3, seed=0)
    big = [W.render_image_torch(w, h, terms, ns) for w, h, terms, ns in params]
    imgs = small + big
    direct = ctx.search_images(imgs, radii, ang, 50, 0.5)
    via = lut3.lookup_images(imgs)
    torch.cuda.synchronize()
    for d, v in zip(direct, via):
        for a, b in zip(d, v):
            assert torch.equal(a, b)
