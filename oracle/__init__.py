"""FP64 CPU oracle of the colour-pair search (test infrastructure).

TEST INFRASTRUCTURE ONLY.  The only code allowed to import, call, link or run
anything in this package is ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``.  The CUDA library
(``paper_2507_22901_gb300``) never imports it and shares no code with it.

Layout:
  constants.py   exact colour constants and tables (integer / Fraction maths)
  trig.py        correctly rounded sin / cos of degree angles (decimal maths)
  cvs_oracle.c   the plain serial-loop FP64 search (gcc, -ffp-contract=off)
  this file      builds cvs_oracle.c and exposes it through ctypes

Every function here follows the paper's §2 Methods: target -> L*a*b*, add and
subtract D_a = i sin j, D_b = i cos j at fixed L*, convert both colours back to
8-bit RGB, keep the pairs whose per-channel RGB difference encodes a Table 1
pattern under the V_th / R_novib rule of §3 Experiments.

Pins (tests/test_oracle_*.py, run with ``-m "not gpu"``): the constants
against the sRGB standard's primaries and white chromaticities and an
independent high-precision evaluation; the cube root against exact rational
arithmetic; the trig table against exact angles and libm; L*a*b* against the
CIE closed form for greys and the published L*a*b* of the sRGB primaries; the
inverse chain by round trip over all 2^24 colours and the forward / inverse
identity; the decision rule by hand-worked cases; the search loops by brute
force over tiny grids.  tests/test_oracle_mutants.py plants plausible mistakes
in a copy of this package and checks that each one fails a pin.  Agreement with
the paper itself can only be soft: its one printed result (Table 2) is reported
as a diagnostic, not a pin.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from pathlib import Path

import numpy as np

from . import constants, trig

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "cvs_oracle.c"
_BUILD = _HERE / "_build"
_LIB_PATH = _BUILD / "liborcvs.so"
_lock = threading.Lock()
_lib = None
_consts = None

PAIR_DTYPE = np.dtype(
    [("k", "<u2"), ("m", "<u2"), ("plus", "u1", 3), ("minus", "u1", 3),
     ("pattern", "u1"), ("flags", "u1"), ("target", "<u4")]
)
assert PAIR_DTYPE.itemsize == 16


class _Consts(ctypes.Structure):
    _fields_ = [
        ("M", ctypes.c_double * 9),
        ("W", ctypes.c_double * 3),
        ("MI", ctypes.c_double * 9),
        ("lut", ctypes.c_double * 256),
        ("thr", ctypes.c_double * 257),
        ("f_break", ctypes.c_double),
        ("finv_break", ctypes.c_double),
        ("f_lin_mul", ctypes.c_double),
        ("f_lin_add", ctypes.c_double),
        ("finv_lin_mul", ctypes.c_double),
    ]


def build(force: bool = False) -> Path:
    """Compile cvs_oracle.c into oracle/_build/liborcvs.so (idempotent)."""
    _BUILD.mkdir(exist_ok=True)
    if (not force and _LIB_PATH.exists()
            and _LIB_PATH.stat().st_mtime >= _SRC.stat().st_mtime):
        return _LIB_PATH
    tmp = _BUILD / f"liborcvs.{os.getpid()}.tmp.so"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
           "-shared", "-o", str(tmp), str(_SRC), "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(str(path))
            P = ctypes.POINTER
            d, i32, i64, u32 = ctypes.c_double, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
            vp = ctypes.c_void_p
            L.orc_cbrt_cr.argtypes = [d]
            L.orc_cbrt_cr.restype = d
            L.orc_target_lab.argtypes = [P(_Consts), vp, vp]
            L.orc_target_lab.restype = None
            L.orc_target_lab_many.argtypes = [P(_Consts), vp, i64, vp, ctypes.c_int]
            L.orc_target_lab_many.restype = None
            L.orc_lin_to_lab.argtypes = [P(_Consts), vp, vp]
            L.orc_lin_to_lab.restype = None
            L.orc_lab_to_lin.argtypes = [P(_Consts), d, d, d, vp]
            L.orc_lab_to_lin.restype = None
            L.orc_quantize.argtypes = [P(_Consts), d]
            L.orc_quantize.restype = ctypes.c_int
            L.orc_quantize_pow.argtypes = [d]
            L.orc_quantize_pow.restype = ctypes.c_int
            L.orc_pair_codes.argtypes = [P(_Consts), vp, d, d, d, vp, vp]
            L.orc_pair_codes.restype = None
            L.orc_search_color.argtypes = [P(_Consts), vp, u32, vp, i32, vp, vp, i32, d, d,
                                           u32, ctypes.c_int, d, vp, i64]
            L.orc_search_color.restype = i64
            L.orc_search_colors.argtypes = [P(_Consts), vp, i64, vp, i32, vp, vp, i32, d, d,
                                            u32, ctypes.c_int, d, vp, vp, vp, ctypes.c_int]
            L.orc_search_colors.restype = None
            L.orc_decide_pair.argtypes = [vp, vp, d, d, u32, ctypes.c_int, vp, vp]
            L.orc_decide_pair.restype = ctypes.c_int
            L.orc_passes_dl.argtypes = [P(_Consts), d, vp, vp, d]
            L.orc_passes_dl.restype = ctypes.c_int
            L.orc_embed.argtypes = [P(_Consts), vp, vp, i64, vp, i32, vp, vp, i32, d, d, u32,
                                    ctypes.c_int, d, vp, vp, vp, ctypes.c_int]
            L.orc_embed.restype = None
            L.orc_roundtrip_all.argtypes = [P(_Consts), P(d), ctypes.c_int]
            L.orc_roundtrip_all.restype = i64
            L.orc_openmp_max_threads.argtypes = []
            L.orc_openmp_max_threads.restype = ctypes.c_int
            _lib = L
        return _lib


def consts() -> _Consts:
    """The constants struct handed to every C entry point."""
    global _consts
    if _consts is None:
        M, W, MI = constants.matrices()
        c = _Consts()
        for i in range(3):
            c.W[i] = W[i]
            for j in range(3):
                c.M[3 * i + j] = M[i][j]
                c.MI[3 * i + j] = MI[i][j]
        for i, v in enumerate(constants.srgb_decode_lut()):
            c.lut[i] = v
        for i, v in enumerate(constants.quant_thresholds()):
            c.thr[i] = v
        cc = constants.cie_constants()
        c.f_break = cc["F_BREAK"]
        c.finv_break = cc["FINV_BREAK"]
        c.f_lin_mul = cc["F_LIN_MUL"]
        c.f_lin_add = cc["F_LIN_ADD"]
        c.finv_lin_mul = cc["FINV_LIN_MUL"]
        _consts = c
    return _consts


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


# ---------------------------------------------------------------- primitives
def cbrt_cr(t: float) -> float:
    """Correctly rounded cube root (positive normal input)."""
    return lib().orc_cbrt_cr(float(t))


def target_lab(rgb) -> np.ndarray:
    """8-bit sRGB -> (L*, a*, b*) in FP64 (step 1 of §2 Methods)."""
    src = np.ascontiguousarray(np.asarray(rgb, dtype=np.uint8).reshape(3))
    out = np.zeros(3, np.float64)
    lib().orc_target_lab(ctypes.byref(consts()), _ptr(src), _ptr(out))
    return out


def target_lab_many(rgbs, threads: int = 0) -> np.ndarray:
    """(n, 3) L*a*b* of an (n, 3) uint8 array."""
    src = np.ascontiguousarray(np.asarray(rgbs, np.uint8).reshape(-1, 3))
    out = np.zeros(src.shape, np.float64)
    lib().orc_target_lab_many(ctypes.byref(consts()), _ptr(src), src.shape[0], _ptr(out),
                              int(threads or max_threads()))
    return out


def lin_to_lab(lin) -> np.ndarray:
    """Linear RGB -> (L*, a*, b*) in FP64."""
    src = np.ascontiguousarray(np.asarray(lin, np.float64).reshape(3))
    out = np.zeros(3, np.float64)
    lib().orc_lin_to_lab(ctypes.byref(consts()), _ptr(src), _ptr(out))
    return out


def lab_to_lin(L: float, a: float, b: float) -> np.ndarray:
    """(L*, a*, b*) -> linear RGB in FP64 (step 3 of §2 Methods, before quantisation)."""
    out = np.zeros(3, np.float64)
    lib().orc_lab_to_lin(ctypes.byref(consts()), float(L), float(a), float(b), _ptr(out))
    return out


def quantize(lin: float) -> int:
    return lib().orc_quantize(ctypes.byref(consts()), float(lin))


def quantize_pow(lin: float) -> int:
    return lib().orc_quantize_pow(float(lin))


def pair_codes(lab, r: float, s: float, c: float):
    """Raw 8-bit codes (in [-1, 256]) of the '+' and '-' colours of one candidate."""
    lab = np.ascontiguousarray(np.asarray(lab, np.float64).reshape(3))
    qp = np.zeros(3, np.int32)
    qm = np.zeros(3, np.int32)
    lib().orc_pair_codes(ctypes.byref(consts()), _ptr(lab), float(r), float(s), float(c),
                         _ptr(qp), _ptr(qm))
    return qp, qm


def decide_pair(q_plus, q_minus, v_th, r_novib, pattern_mask=0x7F, gamut_mode=0):
    """(pattern or 0, emitted plus codes, emitted minus codes) for raw codes."""
    qp = np.ascontiguousarray(q_plus, np.int32).reshape(3)
    qm = np.ascontiguousarray(q_minus, np.int32).reshape(3)
    op = np.zeros(3, np.uint8)
    om = np.zeros(3, np.uint8)
    pat = lib().orc_decide_pair(_ptr(qp), _ptr(qm), float(v_th), float(r_novib),
                                int(pattern_mask), int(gamut_mode), _ptr(op), _ptr(om))
    return pat, op, om


def passes_dl(target_l, plus, minus, max_dl) -> bool:
    """True if both 8-bit colours' L* lie within max_dl of target_l (< 0: no limit)."""
    a = np.ascontiguousarray(np.asarray(plus, np.uint8).reshape(3))
    b = np.ascontiguousarray(np.asarray(minus, np.uint8).reshape(3))
    return bool(lib().orc_passes_dl(ctypes.byref(consts()), float(target_l), _ptr(a), _ptr(b),
                                    float(max_dl)))


def roundtrip_all(threads: int = 0):
    """(number of 8-bit colours whose RGB->Lab->RGB codes differ, max |lin - LUT|)."""
    err = ctypes.c_double(0.0)
    n = lib().orc_roundtrip_all(ctypes.byref(consts()), ctypes.byref(err),
                                int(threads or max_threads()))
    return int(n), err.value


def trig_table(angles_deg):
    s, c = trig.trig_table(angles_deg)
    return np.asarray(s, np.float64), np.asarray(c, np.float64)


# ---------------------------------------------------------------- searches
def search_color(rgb, radii, angles_deg, v_th, r_novib, pattern_mask=0x7F, gamut_mode=0,
                 target=0, cap=None, trig_tab=None, max_dl=-1.0):
    """All passing pairs of one target, sorted by (k, m), as a PAIR_DTYPE array."""
    radii = np.ascontiguousarray(radii, np.float64)
    s, c = trig_tab if trig_tab is not None else trig_table(angles_deg)
    s = np.ascontiguousarray(s, np.float64)
    c = np.ascontiguousarray(c, np.float64)
    src = np.ascontiguousarray(np.asarray(rgb, np.uint8).reshape(3))
    if cap is None:
        cap = len(radii) * len(s)
    out = np.zeros(max(cap, 1), PAIR_DTYPE)
    n = lib().orc_search_color(ctypes.byref(consts()), _ptr(src), int(target), _ptr(radii),
                               len(radii), _ptr(s), _ptr(c), len(s), float(v_th),
                               float(r_novib), int(pattern_mask), int(gamut_mode), float(max_dl),
                               _ptr(out), int(cap))
    return out[:min(n, cap)], int(n)


def search_colors(rgbs, radii, angles_deg, v_th, r_novib, pattern_mask=0x7F, gamut_mode=0,
                  threads=1, trig_tab=None, max_dl=-1.0):
    """Per-target (max_r float32, count int32, pmask uint8) for an (n,3) uint8 array."""
    rgbs = np.ascontiguousarray(np.asarray(rgbs, np.uint8).reshape(-1, 3))
    radii = np.ascontiguousarray(radii, np.float64)
    s, c = trig_tab if trig_tab is not None else trig_table(angles_deg)
    s = np.ascontiguousarray(s, np.float64)
    c = np.ascontiguousarray(c, np.float64)
    n = rgbs.shape[0]
    max_r = np.zeros(n, np.float32)
    count = np.zeros(n, np.int32)
    pmask = np.zeros(n, np.uint8)
    lib().orc_search_colors(ctypes.byref(consts()), _ptr(rgbs), n, _ptr(radii), len(radii),
                            _ptr(s), _ptr(c), len(s), float(v_th), float(r_novib),
                            int(pattern_mask), int(gamut_mode), float(max_dl), _ptr(max_r),
                            _ptr(count), _ptr(pmask), int(threads))
    return max_r, count, pmask


def max_threads() -> int:
    return lib().orc_openmp_max_threads()


def embed(rgbs, patterns, radii, angles_deg, v_th, r_novib, pattern_mask=0x7F, gamut_mode=0,
          threads=1, trig_tab=None, max_dl=-1.0):
    """Embedding of requested patterns (Fig. 1a): per pixel (frame_a (n,3) uint8,
    frame_b (n,3) uint8, choice uint32 = k | m << 16 or 0xFFFFFFFF).  max_dl >= 0:
    only pairs within the luminance limit count (< 0: no limit)."""
    rgbs = np.ascontiguousarray(np.asarray(rgbs, np.uint8).reshape(-1, 3))
    pats = np.ascontiguousarray(np.asarray(patterns, np.uint8).reshape(-1))
    n = rgbs.shape[0]
    if pats.shape[0] != n:
        raise ValueError("one pattern per pixel")
    radii = np.ascontiguousarray(radii, np.float64)
    s, c = trig_tab if trig_tab is not None else trig_table(angles_deg)
    s = np.ascontiguousarray(s, np.float64)
    c = np.ascontiguousarray(c, np.float64)
    fa = np.zeros((n, 3), np.uint8)
    fb = np.zeros((n, 3), np.uint8)
    choice = np.zeros(n, np.uint32)
    lib().orc_embed(ctypes.byref(consts()), _ptr(rgbs), _ptr(pats), n, _ptr(radii), len(radii),
                    _ptr(s), _ptr(c), len(s), float(v_th), float(r_novib), int(pattern_mask),
                    int(gamut_mode), float(max_dl), _ptr(fa), _ptr(fb), _ptr(choice),
                    int(threads))
    return fa, fb, choice
