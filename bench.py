#!/usr/bin/env python3
"""Benchmark of the colour-pair search (Hattori and Hiraki, §2 Methods) on GB300.

One step = one pass of the whole search over the dense colour cube: every colour
with channels 0, 4, .., 252 (262,144 targets) x 128 radii (0.25..32) x 360
angles = 1.208e10 candidate pairs: target decode to L*a*b* (FP64), the pair
chain in FP32 with FP64 re-decision near rounding boundaries, the
embedding-signal decision (V_th = 50, R_novib = 0.5, all patterns, out-of-gamut
rejected) and the per-colour reduction (count, largest radius, pattern mask).

Prints one JSON line (rank 0).  `value` is G candidate pairs/s over all ranks
with inputs resident on the device; `e2e` is the same metric through the C ABI
entry point that takes host buffers (copies inside the timed region).
`--impl reference` times the FP64 CPU oracle on a bounded sample instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

METRIC = "G candidate pairs/s & 4K images/s, FP32+recheck vs plain FP64 GPU, 1 GB300"
UNIT = "Gcand/s"
# Candidates of one 3840x2160 frame with the 64-radius x 180-angle image grid.
CAND_PER_4K_FRAME = 3840 * 2160 * 64 * 180
# Algorithmic instruction issues per candidate of the FP32 path (one colour
# conversion and half a pair decision per candidate): displacement 1, cube
# expansion 6, linear RGB 6, encode 15 FP32 + 6 MUFU, rounding and window test
# 12, half of the 27-issue pair decision 13.5.
ALG_ISSUES_PER_CAND = 59.5
# a candidate rejected before the encode (gamut reject, the warp's 32 slots all
# certainly out of range): displacement 1 + cube expansion 6 + linear RGB 6 +
# range test 6 issues
ALG_ISSUES_PER_SKIPPED = 19.0
# A coarser count per fully evaluated candidate, for comparison: 38 FMA-pipe
# + 6 MUFU + 12 integer operations.
ALG_ISSUES_COARSE = 56.0
LANES_PER_SM_CLK = 128
# DRAM bytes of one FP32 search launch on this workload, from one ncu capture
# of the search kernel on 32,768 cube colours (dram__bytes_read.sum +
# dram__bytes_write.sum), scaled by 8 to the cube's 262,144 colours since the
# traffic is proportional to the colours.  Valid only for the kernel source it
# was taken from (its hash below); otherwise the roofline reports null.
TRAFFIC_CAPTURE = {"source_sha256_16": "2772b1494c0894b5", "bytes_per_launch": 8 * 37.11232e6}


def kernel_source_hash() -> str:
    import hashlib
    from pathlib import Path
    csrc = Path(__file__).resolve().parent / "paper_2507_22901_gb300" / "csrc"
    data = b"".join((csrc / f).read_bytes()
                    for f in ("cvs_kernels.cu", "cvs_slot32.cuh", "cvs_device.cuh"))
    return hashlib.sha256(data).hexdigest()[:16]
REASON_BITS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown",
               0x2: "applications_clocks_setting", 0x1: "gpu_idle"}


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=30)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-fp64", action="store_true", help="skip the all-FP64 comparison arm")
    p.add_argument("--cpu-sample", type=int, default=32768,
                   help="colours of the cube timed on the CPU oracle")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the precision study and the one-pass image measurement")
    p.add_argument("--gather-profile", action="store_true",
                   help="only the table gathers (one 3840x2160 frame through the embedding "
                        "table, four images through the capacity table), for profiling")
    p.add_argument("--frames-profile", action="store_true",
                   help="only the per-pixel paths on one 1920x1080 frame (the image search, "
                        "the same with one search per distinct colour, and the direct "
                        "embedding), for profiling")
    p.add_argument("--sets-profile", action="store_true",
                   help="only the multi-set pass (the cube under the 12 Table 1 threshold "
                        "sets) and one embedding-table build, for profiling")
    p.add_argument("--no-frames", action="store_true",
                   help="skip the 4K-frame measurement (images_4k_per_s is then null), for "
                        "profiling runs")
    p.add_argument("--pairs-profile", action="store_true",
                   help="only the pair lists (the 4096-colour precision set on the 64 x 180 "
                        "grid, and a slice of the cube on the 128 x 360 grid), for profiling")
    p.add_argument("--cube-step", type=int, default=4, choices=[4, 8, 16],
                   help="channel step of the colour cube (4 = the 262,144-colour workload; "
                        "larger steps give the small cases used for profiling)")
    return p.parse_args()


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of the SM clock and throttle reasons while running."""

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self.proc = None
        self.thread = None

    def __enter__(self):
        cmd = ["nvidia-smi", "-i", str(self.index),
               "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active",
               "--format=csv,noheader,nounits", "-lms", "100"]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except OSError:
            self.proc = None
            return self

        def reader():
            for line in self.proc.stdout:
                parts = [x.strip() for x in line.split(",")]
                try:
                    self.samples.append((float(parts[0]), float(parts[1]), float(parts[2]),
                                         int(parts[3], 16)))
                except (ValueError, IndexError):
                    pass
        self.thread = threading.Thread(target=reader, daemon=True)
        self.thread.start()
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=5)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        busy = [s for s in self.samples if not (s[3] & 0x1)] or self.samples
        reasons = set()
        for s in busy:
            for bit, name in REASON_BITS.items():
                if s[3] & bit and name != "gpu_idle":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(s[0] for s in busy),
                "sm_max_mhz": max(s[1] for s in self.samples),
                "power_w_max": max(s[2] for s in busy),
                "reasons": sorted(reasons), "samples": len(busy)}


# ------------------------------------------------------------------ distributed
def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if os.environ.get("CVS_BENCH_BACKEND", "nccl") == "nccl" else "gloo"
        dist.init_process_group(backend)
    return world, rank, local


def max_over_ranks(value: float, world: int, device=None) -> float:
    """Largest value over all ranks (the job's wall time is its slowest rank)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64,
                     device=device if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ------------------------------------------------------------------ oracle arms
def cpu_sample(n: int):
    from paper_2507_22901_gb300 import workloads as W
    cube = W.color_cube()
    idx = np.linspace(0, len(cube) - 1, n).astype(np.int64)
    return cube[idx]


def time_oracle(n_colors: int, threads: int = 0):
    """FP64 CPU oracle over a bounded, evenly spaced sample of the cube (all
    host cores unless `threads` is given)."""
    import oracle
    from paper_2507_22901_gb300 import workloads as W
    radii, ang = W.grid(2)
    tt = oracle.trig_table(ang)
    rgb = cpu_sample(n_colors)
    threads = threads or oracle.max_threads()
    t0 = time.perf_counter()
    oracle.search_colors(rgb, radii, ang, 50.0, 0.5, threads=threads, trig_tab=tt)
    dt = time.perf_counter() - t0
    cand = n_colors * len(radii) * len(ang)
    return cand / dt / 1e9, threads, cand, dt


def run_reference(args, world, rank):
    if rank != 0:
        return
    from paper_2507_22901_gb300 import workloads as W  # noqa: F401
    n = max(16, args.cpu_sample // 16)  # about 0.7 s of oracle work per step on 16 cores
    for _ in range(args.warmup):
        time_oracle(max(8, n // 8))
    vals, cand_total, dt_total, threads = [], 0, 0.0, 1
    for _ in range(args.steps):
        v, threads, cand, dt = time_oracle(n)
        vals.append(v)
        cand_total += cand
        dt_total += dt
    value = cand_total / dt_total / 1e9
    sample = f"{n} evenly spaced colours of the 262,144-colour cube x 128 radii x 360 angles per step"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt_total / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "colour cube 262144 x 128 radii x 360 angles (sampled)",
                   "sample_colors_per_step": n},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ extras
def table2_marks():
    """The paper's Table 2 (7 patterns x 9 colours, 1 = check mark), as stored
    with its citation in tests/golden/table2_presence.txt."""
    from pathlib import Path
    path = Path(__file__).resolve().parent / "tests" / "golden" / "table2_presence.txt"
    rows = [ln.split() for ln in path.read_text().splitlines()
            if ln.strip() and not ln.startswith("#")]
    order = {int(r[0], 2): [int(x) for x in r[1:]] for r in rows}
    return np.array([order[p] for p in range(1, 8)], int)


def measure_4k_frames(ctx, torch, device, W, n_frames=4):
    """Four 3840x2160 frames rendered by the 48-image recipe (seed 31), per
    pixel 64 radii x 180 angles: timed as one batch through cvs_search_images
    with its defaults, with every pixel searched (option dedup 0), with one
    search per distinct colour (dedup 1), and through the capacity table (built
    once, its build timed apart).  The maps of the four are compared."""
    r3, a3 = W.grid(3)
    params = W.image_params(n_frames, seed=31, sizes=[(3840, 2160)] * n_frames)
    frames = [W.render_image_torch(w, h, t, ns, device=device) for w, h, t, ns in params]
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)

    def timed(fn, reps=1):
        fn()
        ctx.synchronize()
        torch.cuda.synchronize(device)
        ev0.record()
        for _ in range(reps):
            r = fn()
        ev1.record()
        ctx.synchronize()
        torch.cuda.synchronize(device)
        return ev0.elapsed_time(ev1) / 1e3 / reps, r

    ctx.set_option("dedup", 0)  # every pixel searched
    try:
        maps = ctx.search_images(frames, r3, a3, 50.0, 0.5)
        sec_direct, _ = timed(lambda: ctx.search_images(frames, r3, a3, 50.0, 0.5, maps=maps))
        ctx.set_option("dedup", 1)
        maps_d = ctx.search_images(frames, r3, a3, 50.0, 0.5)
        sec_dedup, _ = timed(lambda: ctx.search_images(frames, r3, a3, 50.0, 0.5, maps=maps_d))
        distinct = ctx.stats()["targets"]
    finally:
        ctx.set_option("dedup", 2)  # the default: automatic
    maps_a = ctx.search_images(frames, r3, a3, 50.0, 0.5)
    sec_default, _ = timed(lambda: ctx.search_images(frames, r3, a3, 50.0, 0.5, maps=maps_a))
    ev0.record()
    lut = ctx.build_lut(r3, a3, 50.0, 0.5)
    ev1.record()
    torch.cuda.synchronize(device)
    build_s = ev0.elapsed_time(ev1) / 1e3
    maps_t = lut.lookup_images(frames)
    sec_table, _ = timed(lambda: lut.lookup_images(frames, maps=maps_t), reps=20)
    lut.close()
    same = all(torch.equal(a, b) and torch.equal(a, c) and torch.equal(a, d)
               for m, md, mt, ma in zip(maps, maps_d, maps_t, maps_a)
               for a, b, c, d in zip(m, md, mt, ma))
    cand = n_frames * CAND_PER_4K_FRAME
    return {"frames": n_frames, "size": "3840x2160", "grid": "64 radii x 180 angles",
            "default_s": sec_default, "default_frames_per_s": n_frames / sec_default,
            "default_path": "cvs_search_images with its default options (per-batch "
                            "colour de-duplication for batches of 2^20 pixels or more)",
            "direct_s": sec_direct, "direct_frames_per_s": n_frames / sec_direct,
            "direct_gcand_s": cand / sec_direct / 1e9,
            "dedup_s": sec_dedup, "dedup_frames_per_s": n_frames / sec_dedup,
            "distinct_colours": int(distinct),
            "table_s": sec_table, "table_frames_per_s": n_frames / sec_table,
            "table_build_s": build_s, "maps_identical": bool(same)}


def run_extras(ctx, torch, device, W, cvs):
    """Precision study on workloads 1-4 (FP32 vs FP64 errors, re-decision
    fractions, decision mismatches) and one timed pass of the 48-image workload
    (64 radii x 180 angles per pixel), directly and through the capacity table."""
    out = {}
    params = W.image_params()
    imgs = [W.render_image_torch(w, h, terms, ns, device=device) for w, h, terms, ns in params]
    gen = torch.Generator(device="cpu").manual_seed(3)
    pix = []
    for im in imgs:  # 1366 random pixels per image
        ys = torch.randint(0, im.shape[0], (1366,), generator=gen)
        xs = torch.randint(0, im.shape[1], (1366,), generator=gen)
        pix.append(im.cpu()[ys, xs])
    cases = {
        "1_grey170": (np.array([[170, 170, 170]], np.uint8), W.grid(1)),
        "2_cube_step8": (W.color_cube(8), W.grid(2)),
        "3_image_pixels": (torch.cat(pix).numpy(), W.grid(3)),
        "4_precision_set": (W.precision_colors(), W.grid(4)),
    }
    study = {}
    for name, (rgb_h, (radii, ang)) in cases.items():
        rgb = torch.from_numpy(np.ascontiguousarray(rgb_h)).to(device)
        cand = len(rgb_h) * len(radii) * len(ang)
        res = {}
        for prec in (cvs.PREC_FP32_RECHECK, cvs.PREC_FP64):
            ctx.search_colors(rgb, radii, ang, 50.0, 0.5, precision=prec)
            o = ctx.search_colors(rgb, radii, ang, 50.0, 0.5, precision=prec)
            ctx.synchronize()
            res[prec] = (o, ctx.stats())
        (o32, st32), (o64, st64) = res[cvs.PREC_FP32_RECHECK], res[cvs.PREC_FP64]
        mism = int(((o32[0].view(torch.int32) != o64[0].view(torch.int32)) |
                    (o32[1] != o64[1]) | (o32[2] != o64[2])).sum().item())
        rep = ctx.precision_probe(rgb, radii, ang)
        study[name] = {
            "colours": len(rgb_h), "candidates": cand,
            "flagged_fraction": st32["flagged"] / cand,
            "rechecked_fraction": st32["rechecked"] / cand,
            "max_code_err_fp32": rep["max_code_err"], "max_lab_err_fp32": rep["max_lab_err"],
            "max_lin_err_fp32": rep["max_lin_err"], "raw_fp32_wrong_codes": rep["n_wrong_codes"],
            "unflagged_wrong_codes": rep["n_unflagged_wrong"],
            "decision_mismatches_vs_fp64": mism,
            "fp32_gcand_s": cand / (st32["search_ms"] / 1e3) / 1e9,
            "fp64_gcand_s": cand / (st64["search_ms"] / 1e3) / 1e9,
        }
    out["precision_study"] = study
    # one pass over the 48 full-size synthetic images
    r3, a3 = W.grid(3)
    px = sum(im.shape[0] * im.shape[1] for im in imgs)
    ctx.set_option("dedup", 0)  # every pixel searched
    maps = ctx.search_images(imgs, r3, a3, 50.0, 0.5)
    ctx.synchronize()
    torch.cuda.synchronize(device)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    ctx.search_images(imgs, r3, a3, 50.0, 0.5, maps=maps)
    t1.record()
    ctx.synchronize()
    torch.cuda.synchronize(device)
    sec = t0.elapsed_time(t1) / 1e3
    cand3 = px * len(r3) * len(a3)
    # the same batch with one search per distinct colour (option "dedup")
    ctx.set_option("dedup", 1)
    maps_d = ctx.search_images(imgs, r3, a3, 50.0, 0.5)
    ctx.synchronize()
    torch.cuda.synchronize(device)
    t0.record()
    ctx.search_images(imgs, r3, a3, 50.0, 0.5, maps=maps_d)
    t1.record()
    ctx.synchronize()
    torch.cuda.synchronize(device)
    sec_d = t0.elapsed_time(t1) / 1e3
    n_distinct = ctx.stats()["targets"]
    ctx.set_option("dedup", 2)
    same_d = all(torch.equal(a, b) for m, m2 in zip(maps, maps_d) for a, b in zip(m, m2))
    del maps_d
    out["images_dedup"] = {"seconds": sec_d, "distinct_colours": n_distinct,
                           "images_per_s": len(imgs) / sec_d,
                           "effective_gcand_s": px * len(r3) * len(a3) / sec_d / 1e9,
                           "maps_identical_to_search": same_d}
    out["images"] = {"workload": "48 images 256..3840 x 256..2160 (seed 0), 64 radii x 180 angles",
                     "pixels": px, "seconds": sec, "gcand_s": cand3 / sec / 1e9,
                     "images_per_s": len(imgs) / sec,
                     "images_4k_equiv_per_s": cand3 / CAND_PER_4K_FRAME / sec}
    # colour-keyed memoisation: one search over all 2^24 colours, then gathers
    t0.record()
    lut = ctx.build_lut(r3, a3, 50.0, 0.5)
    t1.record()
    torch.cuda.synchronize(device)
    build_s = t0.elapsed_time(t1) / 1e3
    maps2 = lut.lookup_images(imgs)
    torch.cuda.synchronize(device)
    same = all(torch.equal(a, b) for m, m2 in zip(maps, maps2) for a, b in zip(m, m2))
    reps = 20
    t0.record()
    for _ in range(reps):
        lut.lookup_images(imgs, maps=maps2)
    t1.record()
    torch.cuda.synchronize(device)
    look_s = t0.elapsed_time(t1) / 1e3 / reps
    lut.close()
    frames_4k = px / (3840 * 2160)
    out["images_via_table"] = {
        "table_build_s": build_s, "table_candidates": (1 << 24) * len(r3) * len(a3),
        "table_build_gcand_s": (1 << 24) * len(r3) * len(a3) / build_s / 1e9,
        "lookup_s_per_batch": look_s, "images_per_s": len(imgs) / look_s,
        "images_4k_equiv_per_s": frames_4k / look_s,
        "lookup_gb_s": px * 21 / look_s / 1e9,
        "maps_identical_to_search": same}
    del imgs, maps, maps2
    # the embedding step: a 2D-code-like pattern map (16-pixel modules, 60% of
    # them carrying a pattern 1..7) over a 1920x1080 and a 3840x2160 frame
    emb = {}
    for (w, h) in ((1920, 1080), (3840, 2160)):
        terms = W.image_params(1, seed=21, sizes=[(w, h)])[0][2]
        img = W.render_image_torch(w, h, terms, 21, device=device)
        pat = torch.from_numpy(W.code_pattern(h, w, module=16, seed=21)).to(device)
        fa, fb, ch = ctx.embed_image(img, pat, r3, a3, 50.0, 0.5)
        ctx.synchronize()
        reps = 3
        t0.record()
        for _ in range(reps):
            ctx.embed_image(img, pat, r3, a3, 50.0, 0.5, frames=(fa, fb))
        t1.record()
        ctx.synchronize()
        torch.cuda.synchronize(device)
        sec = t0.elapsed_time(t1) / 1e3 / reps
        req = int((pat > 0).sum().item())
        got = int((ch >= 0).sum().item())
        emb[f"{w}x{h}"] = {"seconds": sec, "frames_per_s": 1.0 / sec,
                           "mpixels_per_s": w * h / sec / 1e6,
                           "pixels_requested": req, "pixels_embedded": got,
                           "embedded_fraction_of_requested": got / max(req, 1)}
        del img, pat, fa, fb, ch
    out["embedding"] = {"workload": "synthetic frame, 16-px modules, 60% carry a pattern; "
                                    "64 radii x 180 angles, V_th 50, R_novib 0.5", **emb}
    # the same frames through the embedding table (all 2^24 colours x 7 patterns)
    t0.record()
    etab = ctx.build_embed_table(r3, a3, 50.0, 0.5)
    t1.record()
    torch.cuda.synchronize(device)
    etab_build_s = t0.elapsed_time(t1) / 1e3
    via = {"table_build_s": etab_build_s}
    for (w, h) in ((1920, 1080), (3840, 2160)):
        terms = W.image_params(1, seed=21, sizes=[(w, h)])[0][2]
        img = W.render_image_torch(w, h, terms, 21, device=device)
        pat = torch.from_numpy(W.code_pattern(h, w, module=16, seed=21)).to(device)
        d = ctx.embed_image(img, pat, r3, a3, 50.0, 0.5)
        g = etab.embed_image(img, pat)
        torch.cuda.synchronize(device)
        same = all(torch.equal(x, y) for x, y in zip(d, g))
        reps = 50
        t0.record()
        for _ in range(reps):
            etab.embed_image(img, pat, frames=(g[0], g[1]))
        t1.record()
        torch.cuda.synchronize(device)
        sec = t0.elapsed_time(t1) / 1e3 / reps
        # per pixel: colour 3 + pattern 1 + frames 6 + choice 4 bytes, plus the
        # table entry's 10 bytes (codes 6, choice 4) where a pattern is requested
        alg_bytes = w * h * 14 + int((pat > 0).sum().item()) * 10
        via[f"{w}x{h}"] = {"seconds": sec, "frames_per_s": 1.0 / sec,
                           "identical_to_direct": same,
                           "algorithmic_bytes": alg_bytes, "gb_s": alg_bytes / sec / 1e9}
        del img, pat, d, g
    etab.close()
    out["embedding_via_table"] = via
    # the luminance limit on emitted pairs (max_dl 0.1) over the bench workload
    cube = torch.from_numpy(W.color_cube()).to(device)
    r2, a2 = W.grid(2)
    base = ctx.search_colors(cube, r2, a2, 50.0, 0.5)
    ctx.synchronize()
    lim = ctx.search_colors(cube, r2, a2, 50.0, 0.5, max_dl=0.1)
    lim = ctx.search_colors(cube, r2, a2, 50.0, 0.5, max_dl=0.1, out=lim)
    ctx.synchronize()
    st_l = ctx.stats()
    cand = cube.shape[0] * len(r2) * len(a2)
    out["luminance_limit"] = {
        "workload": "262,144 cube colours x 128 radii x 360 angles, max_dl 0.1",
        "gcand_s": cand / (st_l["search_ms"] / 1e3) / 1e9,
        "pairs_without_limit": int(base[1].sum().item()),
        "pairs_with_limit": int(lim[1].sum().item())}
    del cube, base, lim
    # pair lists of many colours: every passing pair of the 4096-colour precision
    # set on the 64-radius x 180-angle grid, grouped by colour in (k, m) order
    pc = torch.from_numpy(W.precision_colors()).to(device)
    recs, offs = ctx.search_colors_pairs(pc, r3, a3, 50.0, 0.5)
    t0.record()
    recs, offs = ctx.search_colors_pairs(pc, r3, a3, 50.0, 0.5, cap=int(offs[-1]))
    t1.record()
    torch.cuda.synchronize(device)
    sec_p = t0.elapsed_time(t1) / 1e3
    out["pair_lists"] = {"workload": "4096 precision-set colours x 64 radii x 180 angles",
                         "pairs": int(offs[-1]), "seconds": sec_p,
                         "gcand_s": 4096 * len(r3) * len(a3) / sec_p / 1e9,
                         "mpairs_s": int(offs[-1]) / sec_p / 1e6}
    del pc, recs
    # the paper's own timed experiment (§3, Table 1): its 9 colours under all 12
    # (V_th, R_novib) combinations and all 7 patterns, as one multi-set pass on
    # the 61-radius x 360-angle grid (the paper does not state its grid)
    t1rgb = torch.tensor(list(W.TABLE1_COLORS.values()), dtype=torch.uint8, device=device)
    r1, a1 = W.grid(1)
    sets1 = W.table1_threshold_sets()
    res1 = ctx.search_colors_multi(t1rgb, r1, a1, sets1)
    ctx.synchronize()
    reps = 50
    t0.record()
    for _ in range(reps):
        ctx.search_colors_multi(t1rgb, r1, a1, sets1, out=res1)
    t1.record()
    torch.cuda.synchronize(device)
    sec1 = t0.elapsed_time(t1) / 1e3 / reps
    h2 = time.perf_counter()
    for _ in range(reps):
        ctx.search_colors_multi(t1rgb, r1, a1, sets1, out=res1)
        ctx.synchronize()
    host_s = (time.perf_counter() - h2) / reps
    # Table 2's presence matrix in both gamut modes, and its agreement with the
    # paper's (a soft diagnostic: the paper leaves the grid and gamut unstated)
    table2 = table2_marks()
    presence = {}
    for gamut in (0, 1):
        rg = ctx.search_colors_multi(t1rgb, r1, a1, sets1, gamut_mode=gamut)
        torch.cuda.synchronize(device)
        pm = W.presence_matrix(rg[2].cpu().numpy()).astype(int)
        presence["reject" if gamut == 0 else "clip"] = {
            "presence": pm.tolist(), "table2_agreement_of_63": int((pm == table2).sum())}
    out["table1_experiment"] = {
        "workload": "9 Table 1 colours x 12 (V_th, R_novib) x 7 patterns; 61 radii x 360 angles",
        "device_s": sec1, "call_to_result_s": host_s,
        "paper_array_method_s": 62.62, "paper_hardware": "MacBook Pro 13-inch 2019 (CPU), grid unstated",
        "gamut_modes": presence}
    del t1rgb, res1
    # the experiment of §3: every cube colour under all 12 (V_th, R_novib) sets,
    # one multi-set pass against 12 single-set passes
    cube = torch.from_numpy(W.color_cube()).to(device)
    r2, a2 = W.grid(2)
    sets = W.table1_threshold_sets()
    res = ctx.search_colors_multi(cube, r2, a2, sets)
    ctx.synchronize()
    t0.record()
    res = ctx.search_colors_multi(cube, r2, a2, sets, out=res)
    t1.record()
    ctx.synchronize()
    torch.cuda.synchronize(device)
    multi_s = t0.elapsed_time(t1) / 1e3
    st_m = ctx.stats()
    singles = [ctx.search_colors(cube, r2, a2, v, rn) for v, rn in sets]  # warm
    torch.cuda.synchronize(device)
    t0.record()
    for (v, rn), o in zip(sets, singles):
        ctx.search_colors(cube, r2, a2, v, rn, out=o)
    t1.record()
    torch.cuda.synchronize(device)
    single_s = t0.elapsed_time(t1) / 1e3
    same = all(torch.equal(res[i][:, s], singles[s][i]) for s in range(len(sets))
               for i in range(3))
    cand = cube.shape[0] * len(r2) * len(a2)
    out["threshold_sets"] = {
        "workload": "262,144 cube colours x 128 radii x 360 angles x 12 Table 1 sets",
        "multi_pass_s": multi_s, "single_passes_s": single_s, "speedup": single_s / multi_s,
        "gdecisions_s": cand * len(sets) / multi_s / 1e9,
        "flagged_fraction": st_m["flagged"] / cand,
        "rechecked_fraction": st_m["rechecked"] / cand,
        "identical_to_single_set": same,
        "table2_presence_any_colour": W.presence_matrix(res[2].cpu().numpy()).any(axis=1).tolist()}
    del cube, res, singles
    return out


# ------------------------------------------------------------------ serving
def run_serving(torch, device, W, cvs, n_table=600, n_search=24):
    """Workload 5: Poisson arrivals (seed 2, 120 frames/s) of 1920x1080 (60%),
    3840x2160 (30%) and 7680x4320 (10%) frames rendered as in workload 3, sent
    to the continuous-batching server; latency = submit -> maps resident.  With
    the capacity table (all 600 requests) and with per-frame search, per pixel
    and per distinct colour (the first n_search requests: the search alone
    cannot keep up with 120 frames/s)."""
    import threading
    reqs = W.serving_requests(n_table, seed=2, rate=120.0)
    sizes = sorted({(w, h) for _, w, h, _ in reqs})
    params = W.image_params(4 * len(sizes), seed=2, sizes=[sz for sz in sizes for _ in range(4)])
    frames = {}
    for (w, h, terms, ns) in params:
        img = W.render_image_torch(w, h, terms, ns, device=device).cpu().numpy()
        frames.setdefault((w, h), []).append(img)
    r3, a3 = W.grid(3)
    out = {}
    for mode, n in (("table", n_table), ("search", n_search), ("search_dedup", n_search)):
        srv = cvs.Server(r3, a3, 50.0, 0.5, max_inflight=4, max_pixels=7680 * 4320,
                         mem_budget_bytes=6 << 30, use_table=(mode == "table"),
                         dedup=(mode == "search_dedup"))
        tickets = []
        lock = threading.Lock()
        done_flag = [False]

        def drain():
            i = 0
            while True:
                with lock:
                    if i < len(tickets):
                        t = tickets[i]
                    elif done_flag[0]:
                        return
                    else:
                        t = None
                if t is None:
                    time.sleep(0.0005)
                    continue
                srv.wait(t, 600000)
                srv.release(t)
                i += 1
        th = threading.Thread(target=drain)
        th.start()
        t0 = time.perf_counter()
        for arrival, w, h, idx in reqs[:n]:
            delay = t0 + arrival - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            t = srv.submit(frames[(w, h)][idx % 4])
            with lock:
                tickets.append(t)
        with lock:
            done_flag[0] = True
        th.join()
        st = srv.stats()
        srv.close()
        px = sum(w * h for _, w, h, _ in reqs[:n])
        out[mode] = {"requests": n, "completed": st["completed"], "failed": st["failed"],
                     "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "max_ms": st["max_ms"],
                     "frames_per_s": st["frames_per_s"],
                     "offered_frames_per_s": n / reqs[n - 1][0],
                     "pixels": px, "peak_arena_bytes": st["peak_bytes_in_use"]}
    return {"serving": {"workload": "Poisson 120 frames/s (seed 2): 60% 1080p, 30% 4K, 10% 8K; "
                                    "64 radii x 180 angles; 4 slots", **out}}


# ------------------------------------------------------------------ our arm
def run_ours(args, world, rank, local):
    import torch
    import paper_2507_22901_gb300 as cvs
    from paper_2507_22901_gb300 import workloads as W

    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    ctx = cvs.Context(local)
    radii, ang = W.grid(2)
    rgb_h = W.color_cube(args.cube_step)
    n = len(rgb_h)
    cand = n * len(radii) * len(ang)
    rgb = torch.from_numpy(rgb_h).to(device)
    out = (torch.empty(n, dtype=torch.float32, device=device),
           torch.empty(n, dtype=torch.int32, device=device),
           torch.empty(n, dtype=torch.uint8, device=device))
    stream = torch.cuda.current_stream(device)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=device)  # > 129 MB L2

    def step(prec):
        ctx.search_colors(rgb, radii, ang, 50.0, 0.5, precision=prec, out=out, stream=stream)

    for _ in range(args.warmup):
        step(cvs.PREC_FP32_RECHECK)
    ctx.synchronize(stream)

    # ---- timed region: device-resident inputs, L2 flushed between steps
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    step_ms, kern_ms, ranges_ms, flagged, rechecked, skipped, pruned = [], [], [], 0, 0, 0, 0
    barrier(world)
    torch.cuda.synchronize(device)
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()
            start.record(stream)
            step(cvs.PREC_FP32_RECHECK)
            end.record(stream)
            ctx.synchronize(stream)
            step_ms.append(start.elapsed_time(end))
            st = ctx.stats()
            kern_ms.append(st["search_ms"] - st["ranges_ms"])
            ranges_ms.append(st["ranges_ms"])
            flagged += st["flagged"]
            rechecked += st["rechecked"]
            skipped += st["skipped"]
            pruned += st["pruned"]
    torch.cuda.synchronize(device)
    barrier(world)
    total_s = max_over_ranks(sum(step_ms) / 1e3, world, device)
    value = world * cand * args.steps / total_s / 1e9
    res32 = tuple(x.clone() for x in out)

    # ---- comparison arm: every candidate in FP64 (one timed step)
    fp64 = None
    mismatch = None
    if not args.no_fp64:
        step(cvs.PREC_FP64)
        ctx.synchronize(stream)
        flush.zero_()
        start.record(stream)
        step(cvs.PREC_FP64)
        end.record(stream)
        ctx.synchronize(stream)
        t64 = max_over_ranks(start.elapsed_time(end) / 1e3, world, device)
        fp64 = world * cand / t64 / 1e9
        mismatch = int(((res32[0].view(torch.int32) != out[0].view(torch.int32)) |
                        (res32[1] != out[1]) | (res32[2] != out[2])).sum().item())

    # ---- end to end through the host-buffer C entry point
    h_out = (np.empty(n, np.float32), np.empty(n, np.int32), np.empty(n, np.uint8))
    ctx.search_colors_host(rgb_h, radii, ang, 50.0, 0.5, out=h_out)
    barrier(world)
    e2e_s = 0.0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize(device)
        t0 = time.perf_counter()
        ctx.search_colors_host(rgb_h, radii, ang, 50.0, 0.5, out=h_out)
        e2e_s += time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, world, device)
    e2e = world * cand * args.steps / e2e_s / 1e9
    e2e_match = bool(np.array_equal(h_out[1], res32[1].cpu().numpy()))

    # ---- 4K frames: a batch of 3840x2160 frames per GPU, measured
    frames4k = {"images_4k_per_s_all_gpus": None}
    if not args.no_frames:
        frames4k = measure_4k_frames(ctx, torch, device, W)
        sec4k = max_over_ranks(frames4k["default_s"], world, device)
        frames4k["images_4k_per_s_all_gpus"] = world * frames4k["frames"] / sec4k

    # ---- extras: precision study (4096-colour set) and one pass over the images
    extras = {}
    if not args.no_extras and world == 1:
        extras = run_extras(ctx, torch, device, W, cvs)
        extras.update(run_serving(torch, device, W, cvs))

    # ---- roofline of the search kernel (issue bound)
    c = clk.summary()
    f_mhz = c["sm_mhz"] or 2070.0
    kern_avg_s = sum(kern_ms) / len(kern_ms) / 1e3
    ranges_avg_ms = sum(ranges_ms) / len(ranges_ms)
    chunks = -(-n * 128 // (1 << 25)) if ranges_avg_ms > 0 else 0  # angle-range passes per step
    skip_c = skipped / args.steps  # per launch
    prune_c = pruned / args.steps  # rejected by the per-radius bound: no per-candidate work
    alg_ops = ALG_ISSUES_PER_CAND * (cand - skip_c - prune_c) + ALG_ISSUES_PER_SKIPPED * skip_c
    achieved = alg_ops / kern_avg_s / 1e12
    alg_ops56 = ALG_ISSUES_COARSE * (cand - skip_c - prune_c) + ALG_ISSUES_PER_SKIPPED * skip_c
    with_pass_s = kern_avg_s + ranges_avg_ms / 1e3
    num_sms = torch.cuda.get_device_properties(device).multi_processor_count
    peak = num_sms * LANES_PER_SM_CLK * f_mhz * 1e6 / 1e12

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": sum(step_ms) / len(step_ms),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic",
        "config": {"workload": f"colour cube {n} colours x 128 radii (0.25..32) x 360 angles "
                               f"({cand:.4g} candidates per GPU per step)",
                   "v_th": 50, "r_novib": 0.5, "patterns": "all 7", "gamut": "reject",
                   "precision": "fp32 + fp64 re-decision", "l2": "flushed between steps "
                   "(256 MB write)", "parallelism": f"replicas x{world}"},
        "images_4k_per_s": frames4k["images_4k_per_s_all_gpus"],
        "frames_4k": frames4k,
        "fp64_gpu": {"value": fp64, "unit": UNIT,
                     "speedup": (value / fp64) if fp64 else None,
                     "decision_mismatches": mismatch},
        "recheck": {"flagged_fraction": flagged / (cand * args.steps),
                    "rechecked_fraction": rechecked / (cand * args.steps),
                    "window_code_units": ctx.get_option("fp32_window")},
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": int(rgb_h.nbytes),
                "d2h_bytes_per_step": int(n * 9), "matches_device_result": e2e_match},
        "gpu_launches": (3 + chunks) * args.steps,
        "roofline": {"bound": "alu", "kernel": "k_search<fp32>" + (" (angle ranges)" if chunks else ""),
                     "achieved": achieved,
                     "peak": peak, "unit": "Tops/s", "frac": achieved / peak,
                     "traffic": (TRAFFIC_CAPTURE["bytes_per_launch"]
                                 if kernel_source_hash() == TRAFFIC_CAPTURE["source_sha256_16"]
                                 and args.cube_step == 4 else None),
                     "peak_basis": f"{num_sms} SMs x {LANES_PER_SM_CLK} lanes x "
                                   f"{f_mhz:.0f} MHz median SM clock under load",
                     "frac_incl_ranges_pass": alg_ops / with_pass_s / 1e12 / peak,
                     "frac_56_issue_model": alg_ops56 / kern_avg_s / 1e12 / peak,
                     "frac_56_issue_model_incl_ranges_pass": alg_ops56 / with_pass_s / 1e12 / peak,
                     "ops_per_candidate": ALG_ISSUES_PER_CAND,
                     "ops_per_skipped_candidate": ALG_ISSUES_PER_SKIPPED,
                     "skipped_fraction": skip_c / cand,
                     "pruned_fraction": prune_c / cand,
                     "kernel_ms": kern_avg_s * 1e3,
                     "ranges_pass_ms": ranges_avg_ms,
                     "ranges_pass_share": ranges_avg_ms / (ranges_avg_ms + kern_avg_s * 1e3)},
        "clocks": {"sm_mhz": c["sm_mhz"], "sm_max_mhz": c["sm_max_mhz"],
                   "reasons": c["reasons"], "samples": c["samples"]},
    }
    line.update(extras)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, threads, ccand, dt = time_oracle(args.cpu_sample)
        n1 = max(8, args.cpu_sample // 32)  # one core: about 1/32 of the sample
        v1, _, ccand1, dt1 = time_oracle(n1, threads=1)
        line["cpu_baseline"] = {
            "value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{args.cpu_sample} evenly spaced colours of the cube x 128 x 360 "
                      f"({ccand:.3g} candidates, {dt:.1f} s)",
            "single_core": {"value": v1, "unit": UNIT, "cores": 1,
                            "sample": f"{n1} evenly spaced colours of the cube x 128 x 360 "
                                      f"({ccand1:.3g} candidates, {dt1:.1f} s)"}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()


def run_gather_profile(args):
    """The HBM-bound table gathers on their own: build the embedding table and
    the capacity table (64 radii x 180 angles), then gather one 3840x2160 frame
    and four 1920x1080 images `args.steps` times each.  Prints one JSON line
    with the achieved bandwidth per gather (algorithmic bytes / time)."""
    import torch
    import paper_2507_22901_gb300 as cvs
    from paper_2507_22901_gb300 import workloads as W
    dev = torch.device("cuda", 0)
    ctx = cvs.Context(0)
    r3, a3 = W.grid(3)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    terms = W.image_params(1, seed=21, sizes=[(3840, 2160)])[0][2]
    img = W.render_image_torch(3840, 2160, terms, 21, device=dev)
    pat = torch.from_numpy(W.code_pattern(2160, 3840, module=16, seed=21)).to(dev)
    etab = ctx.build_embed_table(r3, a3, 50.0, 0.5)
    fa, fb, ch = etab.embed_image(img, pat)
    torch.cuda.synchronize(dev)
    ev0.record()
    for _ in range(args.steps):
        etab.embed_image(img, pat, frames=(fa, fb))
    ev1.record()
    torch.cuda.synchronize(dev)
    t_emb = ev0.elapsed_time(ev1) / 1e3 / args.steps
    etab.close()
    lut = ctx.build_lut(r3, a3, 50.0, 0.5)
    imgs = [W.render_image_torch(1920, 1080, W.image_params(1, seed=30 + i, sizes=[(1920, 1080)])[0][2],
                                 30 + i, device=dev) for i in range(4)]
    maps = lut.lookup_images(imgs)
    torch.cuda.synchronize(dev)
    ev0.record()
    for _ in range(args.steps):
        lut.lookup_images(imgs, maps=maps)
    ev1.record()
    torch.cuda.synchronize(dev)
    t_lut = ev0.elapsed_time(ev1) / 1e3 / args.steps
    lut.close()
    px4k, pxl = 3840 * 2160, 4 * 1920 * 1080
    emb_bytes = px4k * 14 + int((pat > 0).sum().item()) * 10  # see embedding_via_table
    print(json.dumps({
        "k_etab_gather": {"pixels": px4k, "seconds": t_emb, "algorithmic_bytes": emb_bytes,
                          "gb_s": emb_bytes / t_emb / 1e9},
        "k_lut_gather_images": {"pixels": pxl, "seconds": t_lut, "bytes_per_pixel": 21,
                                "gb_s": pxl * 21 / t_lut / 1e9}}))


def run_frames_profile(args):
    """The per-pixel kernels on one synthetic 1920x1080 frame (64 radii x 180
    angles, V_th 50, R_novib 0.5): the persistent image search, the same with
    one search per distinct colour (option dedup), and the direct embedding of
    a 2D-code pattern map.  Each runs once untimed, then `args.steps` times
    under CUDA events; prints one JSON line."""
    import torch
    import paper_2507_22901_gb300 as cvs
    from paper_2507_22901_gb300 import workloads as W
    dev = torch.device("cuda", 0)
    ctx = cvs.Context(0)
    r3, a3 = W.grid(3)
    w, h = 1920, 1080
    terms = W.image_params(1, seed=21, sizes=[(w, h)])[0][2]
    img = W.render_image_torch(w, h, terms, 21, device=dev)
    pat = torch.from_numpy(W.code_pattern(h, w, module=16, seed=21)).to(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    cand = w * h * len(r3) * len(a3)

    def timed(fn):
        fn()
        ctx.synchronize()
        torch.cuda.synchronize(dev)
        ev0.record()
        for _ in range(args.steps):
            fn()
        ev1.record()
        ctx.synchronize()
        torch.cuda.synchronize(dev)
        return ev0.elapsed_time(ev1) / 1e3 / args.steps

    out = {"workload": "one synthetic 1920x1080 frame (seed 21), 64 radii x 180 angles"}
    ctx.set_option("dedup", 0)  # every pixel searched
    maps = ctx.search_images([img], r3, a3, 50.0, 0.5)
    t = timed(lambda: ctx.search_images([img], r3, a3, 50.0, 0.5, maps=maps))
    st = ctx.stats()
    out["search_images"] = {"seconds": t, "gcand_s": cand / t / 1e9,
                            "angle_ranges": st["ranges_ms"] > 0,
                            "pruned_fraction": st["pruned"] / cand,
                            "skipped_fraction": st["skipped"] / cand}
    ctx.set_option("dedup", 1)
    maps_d = ctx.search_images([img], r3, a3, 50.0, 0.5)
    t = timed(lambda: ctx.search_images([img], r3, a3, 50.0, 0.5, maps=maps_d))
    n_distinct = ctx.stats()["targets"]
    ctx.set_option("dedup", 2)
    out["search_images_dedup"] = {
        "seconds": t, "distinct_colours": n_distinct,
        "maps_identical": all(torch.equal(a, b) for a, b in zip(maps[0], maps_d[0]))}
    fa, fb, ch = ctx.embed_image(img, pat, r3, a3, 50.0, 0.5)
    t = timed(lambda: ctx.embed_image(img, pat, r3, a3, 50.0, 0.5, frames=(fa, fb)))
    out["embed_image"] = {"seconds": t, "pixels_requested": int((pat > 0).sum().item()),
                          "pixels_embedded": int((ch >= 0).sum().item())}
    ctx.close()
    print(json.dumps(out))


def run_sets_profile(args):
    """The multi-set pass on its own: the colour cube (channel step
    `args.cube_step`) x 128 radii x 360 angles under the 12 Table 1 threshold
    sets, once untimed and then `args.steps` times under CUDA events; then one
    embedding-table build (all 2^24 colours x 64 radii x 180 angles).  Prints
    one JSON line."""
    import torch
    import paper_2507_22901_gb300 as cvs
    from paper_2507_22901_gb300 import workloads as W
    dev = torch.device("cuda", 0)
    ctx = cvs.Context(0)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    cube = torch.from_numpy(W.color_cube(args.cube_step)).to(dev)
    r2, a2 = W.grid(2)
    sets = W.table1_threshold_sets()
    res = ctx.search_colors_multi(cube, r2, a2, sets)
    ctx.synchronize()
    ev0.record()
    for _ in range(args.steps):
        ctx.search_colors_multi(cube, r2, a2, sets, out=res)
    ev1.record()
    ctx.synchronize()
    torch.cuda.synchronize(dev)
    t_multi = ev0.elapsed_time(ev1) / 1e3 / args.steps
    ranges_ms = ctx.stats()["ranges_ms"]
    ctx.set_option("angle_ranges", 0)  # the plain walk, for comparison
    plain = ctx.search_colors_multi(cube, r2, a2, sets)
    ctx.synchronize()
    ev0.record()
    for _ in range(args.steps):
        ctx.search_colors_multi(cube, r2, a2, sets, out=plain)
    ev1.record()
    ctx.synchronize()
    torch.cuda.synchronize(dev)
    t_plain = ev0.elapsed_time(ev1) / 1e3 / args.steps
    ctx.set_option("angle_ranges", 2)
    same = all(torch.equal(a, b) for a, b in zip(res, plain))
    cand = cube.shape[0] * len(r2) * len(a2)
    r3, a3 = W.grid(3)
    ev0.record()
    etab = ctx.build_embed_table(r3, a3, 50.0, 0.5)
    ev1.record()
    torch.cuda.synchronize(dev)
    t_etab = ev0.elapsed_time(ev1) / 1e3
    etab.close()
    ctx.close()
    print(json.dumps({
        "multi_set_pass": {"colours": int(cube.shape[0]), "sets": len(sets), "seconds": t_multi,
                           "gdecisions_s": cand * len(sets) / t_multi / 1e9,
                           "ranges_pass_ms": ranges_ms,
                           "plain_walk_seconds": t_plain, "same_as_plain_walk": same},
        "embedding_table_build": {"colours": 1 << 24, "seconds": t_etab,
                                  "gcand_s": (1 << 24) * len(r3) * len(a3) / t_etab / 1e9}}))


def run_pairs_profile(args):
    """The pair lists on their own: every passing pair of the 4096-colour
    precision set on the 64-radius x 180-angle grid (the bench's pair-list
    workload), and of every 16th cube colour on the 128 x 360 grid; each once
    to size the output, then `args.steps` times under CUDA events.  Prints one
    JSON line (call-to-result times: the calls are synchronous)."""
    import torch
    import paper_2507_22901_gb300 as cvs
    from paper_2507_22901_gb300 import workloads as W
    dev = torch.device("cuda", 0)
    ctx = cvs.Context(0)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {}
    cases = {"precision_set_64x180": (W.precision_colors(), W.grid(3)),
             "cube_every_16th_128x360": (W.color_cube()[::16].copy(), W.grid(2))}
    for name, (rgb_h, (radii, ang)) in cases.items():
        rgb = torch.from_numpy(rgb_h).to(dev)
        recs, offs = ctx.search_colors_pairs(rgb, radii, ang, 50.0, 0.5)
        cap = int(offs[-1])
        ev0.record()
        for _ in range(args.steps):
            recs, offs = ctx.search_colors_pairs(rgb, radii, ang, 50.0, 0.5, cap=cap)
        ev1.record()
        torch.cuda.synchronize(dev)
        sec = ev0.elapsed_time(ev1) / 1e3 / args.steps
        cand = len(rgb_h) * len(radii) * len(ang)
        out[name] = {"colours": len(rgb_h), "candidates": cand, "pairs": cap, "seconds": sec,
                     "gcand_s": cand / sec / 1e9, "record_gb_s": cap * 16 / sec / 1e9}
        del recs, rgb
    ctx.close()
    print(json.dumps({"pair_lists": out}))


def main():
    args = parse_args()
    if args.gather_profile:
        return run_gather_profile(args)
    if args.frames_profile:
        return run_frames_profile(args)
    if args.pairs_profile:
        return run_pairs_profile(args)
    if args.sets_profile:
        return run_sets_profile(args)
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
