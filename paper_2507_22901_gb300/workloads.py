"""Seeded synthetic workloads for the colour-pair search.

Inputs only: this module holds none of the search's arithmetic and is shared by
the benchmark and the tests (which hand the same inputs to the CUDA library and
to the CPU oracle).  The paper's experiment (§3, Table 1) uses nine flat
colours, seven patterns, V_th in {50, 100, 150, 200} and R_novib in
{0.5, 0.25, 0.125}; its radius/angle grid is not stated.  The five workloads:

  1 single colour  (170,170,170); radii 0..30 step 0.5 (61); angles 0..359 step 1
  2 colour cube    all 262,144 colours with channels 0,4,..,252; radii 0.25..32
                   step 0.25 (128); angles 0..359 step 1 (360): 1.208e10 candidates
  3 images         48 images (seed 0), W ~ U{256..3840}, H ~ U{256..2160}; per
                   channel a sum of 4 low-frequency 2-D cosines scaled to [0,255]
                   plus integer noise U{-8..8}, clipped; radii 0.5..32 step 0.5
                   (64); angles 0..358 step 2 (180)
  4 precision set  4096 colours (seed 1): 3072 uniform, 512 near-grey (g + U{-2..2}),
                   512 near the gamut edge (one channel in {0..3, 252..255});
                   radii 0.125..32 step 0.125 (256); angles 0..359.5 step 0.5 (720)
  5 serving        Poisson arrivals (seed 2, mean 120/s) of frames 60% 1920x1080,
                   30% 3840x2160, 10% 7680x4320, content and grid as workload 3

Default thresholds for 2-5: V_th = 50, R_novib = 0.5, all seven patterns,
out-of-gamut pairs rejected (the loosest row of Table 1).
"""
from __future__ import annotations

import math

import numpy as np

TABLE1_COLORS = {
    "Black": (100, 100, 100), "Gray": (170, 170, 170), "White": (240, 240, 240),
    "Red": (240, 100, 100), "Green": (100, 240, 100), "Blue": (100, 100, 240),
    "Yellow": (240, 240, 100), "Cyan": (100, 240, 240), "Magenta": (240, 100, 240),
}
TABLE1_VTH = (50, 100, 150, 200)
TABLE1_RNOVIB = (0.5, 0.25, 0.125)
DEFAULT_THRESHOLDS = dict(v_th=50.0, r_novib=0.5, pattern_mask=0x7F, gamut_mode=0)


def table1_threshold_sets():
    """The 12 (V_th, R_novib) combinations of Table 1, V_th-major."""
    return [(float(v), float(r)) for v in TABLE1_VTH for r in TABLE1_RNOVIB]


def presence_matrix(pmask) -> np.ndarray:
    """Table 2's question from per-(colour, set) pattern masks: (7, n_colours)
    bool, row p - 1 true where some set gives colour a pair for pattern p.
    pmask: (n_colours, n_sets) uint8, bit p - 1 = pattern p has a pair."""
    any_set = np.bitwise_or.reduce(np.asarray(pmask, np.uint8), axis=1)
    return np.array([(any_set >> (p - 1)) & 1 for p in range(1, 8)], bool)


def grid(config: int):
    """(radii, angles_deg) float64 arrays of a workload."""
    if config == 1:
        return np.arange(61) * 0.5, np.arange(360) * 1.0
    if config == 2:
        return np.arange(1, 129) * 0.25, np.arange(360) * 1.0
    if config in (3, 5):
        return np.arange(1, 65) * 0.5, np.arange(180) * 2.0
    if config == 4:
        return np.arange(1, 257) * 0.125, np.arange(720) * 0.5
    raise ValueError(config)


def color_cube(step: int = 4) -> np.ndarray:
    """(n, 3) uint8: every colour whose channels are multiples of `step`."""
    v = np.arange(0, 256, step, dtype=np.uint8)
    r, g, b = np.meshgrid(v, v, v, indexing="ij")
    return np.stack([r.ravel(), g.ravel(), b.ravel()], axis=1)


def precision_colors(seed: int = 1) -> np.ndarray:
    rng = np.random.default_rng(seed)
    uni = rng.integers(0, 256, (3072, 3))
    g = rng.integers(0, 256, (512, 1))
    grey = np.clip(g + rng.integers(-2, 3, (512, 3)), 0, 255)
    edge = rng.integers(0, 256, (512, 3))
    ch = rng.integers(0, 3, 512)
    edge_vals = np.concatenate([np.arange(0, 4), np.arange(252, 256)])
    edge[np.arange(512), ch] = rng.choice(edge_vals, 512)
    return np.concatenate([uni, grey, edge]).astype(np.uint8)


def image_params(n: int = 48, seed: int = 0, sizes=None):
    """Per image: (width, height, params) with params[c] = list of 4 cosine terms
    (amplitude, fx, fy, phase) and a noise seed."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        if sizes is None:
            w = int(rng.integers(256, 3841))
            h = int(rng.integers(256, 2161))
        else:
            w, h = sizes[i]
        terms = []
        for _c in range(3):
            terms.append([(float(rng.uniform(0.2, 1.0)), float(rng.uniform(0, 2)),
                           float(rng.uniform(0, 2)), float(rng.uniform(0, 2 * math.pi)))
                          for _ in range(4)])
        out.append((w, h, terms, int(rng.integers(0, 2 ** 31))))
    return out


def render_image_numpy(w: int, h: int, terms, noise_seed: int) -> np.ndarray:
    """(h, w, 3) uint8 image from image_params (CPU; for small sizes)."""
    y = np.arange(h, dtype=np.float64)[:, None] / h
    x = np.arange(w, dtype=np.float64)[None, :] / w
    img = np.empty((h, w, 3), np.float64)
    for c in range(3):
        s = np.zeros((h, w))
        amp = 0.0
        for A, fx, fy, ph in terms[c]:
            s += A * np.cos(2 * math.pi * (fx * x + fy * y) + ph)
            amp += A
        img[:, :, c] = (s + amp) / (2 * amp) * 255.0
    noise = np.random.default_rng(noise_seed).integers(-8, 9, (h, w, 3))
    return np.clip(np.rint(img) + noise, 0, 255).astype(np.uint8)


def render_image_torch(w: int, h: int, terms, noise_seed: int, device="cuda"):
    """The same recipe on a torch device (fast for full-size images); the noise
    comes from torch's generator, so pixels differ from render_image_numpy."""
    import torch
    y = (torch.arange(h, device=device, dtype=torch.float32) / h)[:, None]
    x = (torch.arange(w, device=device, dtype=torch.float32) / w)[None, :]
    chans = []
    for c in range(3):
        s = torch.zeros((h, w), device=device, dtype=torch.float32)
        amp = 0.0
        for A, fx, fy, ph in terms[c]:
            s += A * torch.cos(2 * math.pi * (fx * x + fy * y) + ph)
            amp += A
        chans.append((s + amp) / (2 * amp) * 255.0)
    img = torch.stack(chans, dim=2)
    gen = torch.Generator(device=device)
    gen.manual_seed(noise_seed)
    noise = torch.randint(-8, 9, (h, w, 3), generator=gen, device=device, dtype=torch.int16)
    return torch.clamp(torch.round(img).to(torch.int16) + noise, 0, 255).to(torch.uint8)


def code_pattern(h: int, w: int, module: int = 8, seed: int = 0, fill: float = 0.6) -> np.ndarray:
    """(h, w) uint8 requested-pattern map of a 2D-code-like embedding: square
    modules of `module` pixels, each carrying one 3-bit pattern 1..7 with
    probability `fill`, else 0 (nothing embedded)."""
    rng = np.random.default_rng(seed)
    mh, mw = -(-h // module), -(-w // module)
    cells = rng.integers(1, 8, (mh, mw)).astype(np.uint8)
    cells[rng.random((mh, mw)) >= fill] = 0
    return np.ascontiguousarray(np.repeat(np.repeat(cells, module, 0), module, 1)[:h, :w])


def serving_requests(n: int = 600, seed: int = 2, rate: float = 120.0):
    """Poisson arrivals: list of (arrival_time_s, width, height, image_param_index)."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, n))
    kind = rng.choice(3, n, p=[0.6, 0.3, 0.1])
    sizes = [(1920, 1080), (3840, 2160), (7680, 4320)]
    return [(float(t[i]), sizes[kind[i]][0], sizes[kind[i]][1], i) for i in range(n)]
