"""ctypes binding of libcvsearch (include/cvsearch.h).

Argument marshalling only: every step of the search runs in the CUDA library.
The raw C functions are available under their C names on ``lib()``; the
``Context`` class wraps them for PyTorch tensors (device memory and streams)
and NumPy arrays (host buffers).
"""
from __future__ import annotations

import ctypes
import re
from pathlib import Path

import numpy as np

from . import _build

CVS_OK, CVS_ERR_INVALID_ARG, CVS_ERR_NO_MEMORY, CVS_ERR_CUDA = 0, 1, 2, 3
CVS_ERR_TRUNCATED, CVS_ERR_TIMEOUT, CVS_ERR_NUMERIC = 4, 5, 6
PREC_FP32_RECHECK, PREC_FP64 = 0, 1

STATUS_NAMES = {0: "CVS_OK", 1: "CVS_ERR_INVALID_ARG", 2: "CVS_ERR_NO_MEMORY", 3: "CVS_ERR_CUDA",
                4: "CVS_ERR_TRUNCATED", 5: "CVS_ERR_TIMEOUT", 6: "CVS_ERR_NUMERIC"}

PAIR_DTYPE = np.dtype(
    [("k", "<u2"), ("m", "<u2"), ("plus", "u1", 3), ("minus", "u1", 3),
     ("pattern", "u1"), ("flags", "u1"), ("target", "<u4")]
)


class CvsError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class cvs_grid(ctypes.Structure):
    _fields_ = [("radii", ctypes.POINTER(ctypes.c_double)), ("n_radii", ctypes.c_int32),
                ("angles_deg", ctypes.POINTER(ctypes.c_double)), ("n_angles", ctypes.c_int32)]


class cvs_thresholds(ctypes.Structure):
    _fields_ = [("v_th", ctypes.c_double), ("r_novib", ctypes.c_double),
                ("pattern_mask", ctypes.c_uint32), ("gamut_mode", ctypes.c_int32),
                ("max_dl", ctypes.c_double)]


class cvs_pair(ctypes.Structure):
    _fields_ = [("k", ctypes.c_uint16), ("m", ctypes.c_uint16), ("plus", ctypes.c_uint8 * 3),
                ("minus", ctypes.c_uint8 * 3), ("pattern", ctypes.c_uint8),
                ("flags", ctypes.c_uint8), ("target", ctypes.c_uint32)]


class cvs_capacity_map(ctypes.Structure):
    _fields_ = [("max_r", ctypes.c_void_p), ("count", ctypes.c_void_p), ("pmask", ctypes.c_void_p)]


class cvs_image(ctypes.Structure):
    _fields_ = [("rgb", ctypes.c_void_p), ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("pitch_bytes", ctypes.c_int64)]


class cvs_stats(ctypes.Structure):
    _fields_ = [("candidates", ctypes.c_int64), ("colors_fp32", ctypes.c_int64),
                ("flagged", ctypes.c_int64), ("rechecked", ctypes.c_int64),
                ("targets", ctypes.c_int64), ("symmetric", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("search_ms", ctypes.c_double),
                ("skipped", ctypes.c_int64), ("pruned", ctypes.c_int64),
                ("ranges_ms", ctypes.c_double)]


class cvs_precision_report(ctypes.Structure):
    _fields_ = [("max_code_err", ctypes.c_double), ("max_lin_err", ctypes.c_double),
                ("max_lab_err", ctypes.c_double), ("n_wrong_codes", ctypes.c_int64),
                ("n_values", ctypes.c_int64), ("n_unflagged_wrong", ctypes.c_int64),
                ("window", ctypes.c_double)]


class cvs_launch_shape(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("kchunk", ctypes.c_int32), ("reserved", ctypes.c_int32), ("ms", ctypes.c_double)]


class cvs_server_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("max_inflight", ctypes.c_int32),
                ("max_pixels", ctypes.c_int64), ("mem_budget_bytes", ctypes.c_int64),
                ("use_table", ctypes.c_int32), ("dedup", ctypes.c_int32)]


class cvs_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("failed", ctypes.c_int64), ("queued", ctypes.c_int64),
                ("inflight", ctypes.c_int64), ("bytes_in_use", ctypes.c_int64),
                ("peak_bytes_in_use", ctypes.c_int64), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("frames_per_s", ctypes.c_double)]


REQ_QUEUED, REQ_RUNNING, REQ_DONE, REQ_FAILED, REQ_UNKNOWN = 0, 1, 2, 3, 4

assert ctypes.sizeof(cvs_pair) == 16 and PAIR_DTYPE.itemsize == 16

_lib = None


def header_functions() -> list[str]:
    """Names of the functions declared in include/cvsearch.h."""
    text = (Path(_build.INCLUDE) / "cvsearch.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cvs_[a-z_0-9]+)\s*\(", text)))


def lib() -> ctypes.CDLL:
    """Load libcvsearch.so (building it first if the sources are newer)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not _build.up_to_date():
        try:
            path = _build.build()
        except Exception as exc:  # no compiler: fail loudly, never fall back
            raise RuntimeError(f"libcvsearch is not built and cannot be built: {exc}") from exc
    L = ctypes.CDLL(str(path))
    P, vp = ctypes.POINTER, ctypes.c_void_p
    i32, i64, u32, d, st = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_double, ctypes.c_int
    sig = {
        "cvs_create": ([P(vp), ctypes.c_int, ctypes.c_size_t], st),
        "cvs_destroy": ([vp], None),
        "cvs_last_error": ([], ctypes.c_char_p),
        "cvs_version": ([], ctypes.c_char_p),
        "cvs_signal_bounds": ([P(cvs_thresholds), P(i32), P(i32)], st),
        "cvs_trig_table": ([vp, P(d), i32, P(d), P(d)], st),
        "cvs_target_lab": ([vp, vp, i64, vp, vp], st),
        "cvs_search_color": ([vp, P(ctypes.c_uint8), u32, P(cvs_grid), P(cvs_thresholds), st,
                              vp, ctypes.c_size_t, P(ctypes.c_size_t)], st),
        "cvs_search_colors": ([vp, vp, i64, P(cvs_grid), P(cvs_thresholds), st,
                               P(cvs_capacity_map), vp], st),
        "cvs_search_colors_pairs": ([vp, vp, i64, P(cvs_grid), P(cvs_thresholds), st, vp, i64,
                                     vp, P(i64), vp], st),
        "cvs_search_colors_host": ([vp, vp, i64, P(cvs_grid), P(cvs_thresholds), st, vp, vp, vp],
                                   st),
        "cvs_search_colors_multi": ([vp, vp, i64, P(cvs_grid), P(cvs_thresholds), i32, st,
                                     P(cvs_capacity_map), vp], st),
        "cvs_embed_image": ([vp, P(cvs_image), vp, i64, P(cvs_grid), P(cvs_thresholds), st, vp,
                             vp, i64, vp, vp], st),
        "cvs_search_images": ([vp, P(cvs_image), i32, P(cvs_grid), P(cvs_thresholds), st,
                               P(cvs_capacity_map), vp], st),
        "cvs_synchronize": ([vp, vp], st),
        "cvs_get_stats": ([vp, P(cvs_stats)], st),
        "cvs_precision_probe": ([vp, vp, i64, P(cvs_grid), P(cvs_precision_report)], st),
        "cvs_set_option": ([vp, ctypes.c_char_p, d], st),
        "cvs_get_option": ([vp, ctypes.c_char_p, P(d)], st),
        "cvs_lut_build": ([vp, P(cvs_grid), P(cvs_thresholds), st, P(vp), vp], st),
        "cvs_lut_lookup_images": ([vp, P(cvs_image), i32, P(cvs_capacity_map), vp], st),
        "cvs_lut_lookup_colors": ([vp, vp, i64, P(cvs_capacity_map), vp], st),
        "cvs_lut_destroy": ([vp], None),
        "cvs_etab_build": ([vp, P(cvs_grid), P(cvs_thresholds), st, P(vp), vp], st),
        "cvs_etab_embed_image": ([vp, P(cvs_image), vp, i64, vp, vp, i64, vp, vp], st),
        "cvs_etab_destroy": ([vp], None),
        "cvs_reserve": ([vp, P(cvs_grid), i64, i32], st),
        "cvs_server_create": ([P(vp), P(cvs_server_config), P(cvs_grid), P(cvs_thresholds), st], st),
        "cvs_server_destroy": ([vp], None),
        "cvs_server_submit": ([vp, vp, i32, i32, i64, P(ctypes.c_uint64)], st),
        "cvs_server_state": ([vp, ctypes.c_uint64, P(i32)], st),
        "cvs_server_wait": ([vp, ctypes.c_uint64, i32], st),
        "cvs_server_result": ([vp, ctypes.c_uint64, P(cvs_capacity_map), P(i32), P(i32)], st),
        "cvs_server_copy_result": ([vp, ctypes.c_uint64, vp, vp, vp], st),
        "cvs_server_release": ([vp, ctypes.c_uint64], st),
        "cvs_server_get_stats": ([vp, P(cvs_server_stats)], st),
        "cvs_autotune": ([vp, vp, i64, P(cvs_grid), P(cvs_thresholds), st, P(cvs_launch_shape)], st),
        "cvs_search_colors_noalloc": ([ctypes.c_int, vp, i64, P(cvs_grid), P(cvs_thresholds), st,
                                       P(cvs_capacity_map), vp], st),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def last_error() -> str:
    return lib().cvs_last_error().decode()


def check(status: int, where: str):
    if status != CVS_OK:
        raise CvsError(status, where, last_error())


def make_grid(radii, angles_deg):
    """(cvs_grid, keep-alive arrays) from sequences of radii and angles."""
    r = np.ascontiguousarray(radii, np.float64)
    a = np.ascontiguousarray(angles_deg, np.float64)
    g = cvs_grid(r.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(r),
                 a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(a))
    return g, (r, a)


def make_thresholds(v_th, r_novib, pattern_mask=0x7F, gamut_mode=0, max_dl=None):
    """A cvs_thresholds struct; max_dl None (or 0, or inf) = no luminance limit."""
    return cvs_thresholds(float(v_th), float(r_novib), int(pattern_mask), int(gamut_mode),
                          0.0 if max_dl is None else float(max_dl))


def signal_bounds(v_th, r_novib, pattern_mask=0x7F, gamut_mode=0, max_dl=None):
    """(hi_min, lo_max) integer bounds of the embedding-signal condition."""
    t = make_thresholds(v_th, r_novib, pattern_mask, gamut_mode, max_dl)
    hi, lo = ctypes.c_int32(), ctypes.c_int32()
    check(lib().cvs_signal_bounds(ctypes.byref(t), ctypes.byref(hi), ctypes.byref(lo)),
          "cvs_signal_bounds")
    return hi.value, lo.value


def _stream_ptr(stream) -> int | None:
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


class Context:
    """A libcvsearch context on one CUDA device."""

    def __init__(self, device: int = 0, mem_budget: int = 0):
        """mem_budget: cap in bytes on the device memory the context allocates
        (0 = none)."""
        self._h = ctypes.c_void_p()
        check(lib().cvs_create(ctypes.byref(self._h), int(device), int(mem_budget)), "cvs_create")
        self.device = device

    def close(self):
        if self._h:
            lib().cvs_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    # -------------------------------------------------------------- options
    def reserve(self, radii=None, angles_deg=None, max_targets=0, max_images=0):
        """Allocate ahead of time what searches up to max_targets colours or
        pixels (and batches of max_images images) on this grid need."""
        g = None
        if radii is not None:
            g, keep = make_grid(radii, angles_deg)
        check(lib().cvs_reserve(self._h, ctypes.byref(g) if g is not None else None,
                                int(max_targets), int(max_images)), "cvs_reserve")

    def set_option(self, name: str, value: float):
        check(lib().cvs_set_option(self._h, name.encode(), float(value)), "cvs_set_option")

    def get_option(self, name: str) -> float:
        v = ctypes.c_double()
        check(lib().cvs_get_option(self._h, name.encode(), ctypes.byref(v)), "cvs_get_option")
        return v.value

    # -------------------------------------------------------------- helpers
    def trig_table(self, angles_deg):
        a = np.ascontiguousarray(angles_deg, np.float64)
        s = np.zeros_like(a)
        c = np.zeros_like(a)
        dp = ctypes.POINTER(ctypes.c_double)
        check(lib().cvs_trig_table(self._h, a.ctypes.data_as(dp), len(a), s.ctypes.data_as(dp),
                                   c.ctypes.data_as(dp)), "cvs_trig_table")
        return s, c

    def target_lab(self, rgb_dev, out=None, stream=None):
        import torch
        n = rgb_dev.numel() // 3
        if out is None:
            out = torch.empty((n, 3), dtype=torch.float64, device=rgb_dev.device)
        check(lib().cvs_target_lab(self._h, rgb_dev.data_ptr(), n, out.data_ptr(),
                                   _stream_ptr(stream)), "cvs_target_lab")
        return out

    # -------------------------------------------------------------- searches
    def search_color(self, rgb, radii, angles_deg, v_th, r_novib, pattern_mask=0x7F,
                     gamut_mode=0, max_dl=None, precision=PREC_FP32_RECHECK, target=0, cap=None):
        """All passing pairs of one colour, sorted by (k, m): (PAIR_DTYPE array, total)."""
        g, keep = make_grid(radii, angles_deg)
        t = make_thresholds(v_th, r_novib, pattern_mask, gamut_mode, max_dl)
        src = (ctypes.c_uint8 * 3)(*[int(x) for x in rgb])
        if cap is None:
            cap = len(keep[0]) * len(keep[1])
        out = np.zeros(max(cap, 1), PAIR_DTYPE)
        n = ctypes.c_size_t()
        st = lib().cvs_search_color(self._h, src, int(target), ctypes.byref(g), ctypes.byref(t),
                                    int(precision), out.ctypes.data, cap, ctypes.byref(n))
        if st not in (CVS_OK, CVS_ERR_TRUNCATED):
            check(st, "cvs_search_color")
        return out[:min(n.value, cap)], n.value

    def search_colors(self, rgb_dev, radii, angles_deg, v_th, r_novib, pattern_mask=0x7F,
                      gamut_mode=0, max_dl=None,
                      precision=PREC_FP32_RECHECK, out=None, stream=None):
        """Per-colour (max_r, count, pmask) device tensors for an (n, 3) uint8 CUDA tensor."""
        import torch
        n = rgb_dev.numel() // 3
        dev = rgb_dev.device
        if out is None:
            out = (torch.empty(n, dtype=torch.float32, device=dev),
                   torch.empty(n, dtype=torch.int32, device=dev),
                   torch.empty(n, dtype=torch.uint8, device=dev))
        g, keep = make_grid(radii, angles_deg)
        t = make_thresholds(v_th, r_novib, pattern_mask, gamut_mode, max_dl)
        m = cvs_capacity_map(out[0].data_ptr(), out[1].data_ptr(), out[2].data_ptr())
        check(lib().cvs_search_colors(self._h, rgb_dev.data_ptr(), n, ctypes.byref(g),
                                      ctypes.byref(t), int(precision), ctypes.byref(m),
                                      _stream_ptr(stream)), "cvs_search_colors")
        return out

    def search_colors_pairs(self, rgb_dev, radii, angles_deg, v_th, r_novib, pattern_mask=0x7F,
                            gamut_mode=0, max_dl=None,
                            precision=PREC_FP32_RECHECK, cap=None, stream=None):
        """Every passing pair of n colours: (records (total, 16) uint8 CUDA tensor
        viewable as PAIR_DTYPE, offsets int64 NumPy array of n + 1)."""
        import torch
        n = rgb_dev.numel() // 3
        g, keep = make_grid(radii, angles_deg)
        t = make_thresholds(v_th, r_novib, pattern_mask, gamut_mode, max_dl)
        offs = np.zeros(n + 1, np.int64)
        total = ctypes.c_int64()
        if cap is None:  # ask for the size first
            st = lib().cvs_search_colors_pairs(self._h, rgb_dev.data_ptr(), n, ctypes.byref(g),
                                               ctypes.byref(t), int(precision), None, 0,
                                               offs.ctypes.data, ctypes.byref(total),
                                               _stream_ptr(stream))
            if st not in (CVS_OK, CVS_ERR_TRUNCATED):
                check(st, "cvs_search_colors_pairs")
            cap = total.value
        out = torch.empty((max(cap, 1), 16), dtype=torch.uint8, device=rgb_dev.device)
        st = lib().cvs_search_colors_pairs(self._h, rgb_dev.data_ptr(), n, ctypes.byref(g),
                                           ctypes.byref(t), int(precision), out.data_ptr(), cap,
                                           offs.ctypes.data, ctypes.byref(total),
                                           _stream_ptr(stream))
        check(st, "cvs_search_colors_pairs")
        return out[:total.value], offs

    def search_colors_multi(self, rgb_dev, radii, angles_deg, thresholds, gamut_mode=0,
                            precision=PREC_FP32_RECHECK, out=None, stream=None):
        """Per-colour results under several threshold sets in one pass.

        thresholds: sequence of (v_th, r_novib), (v_th, r_novib, pattern_mask) or
        (v_th, r_novib, pattern_mask, max_dl).
        Returns (max_r, count, pmask) device tensors of shape (n, n_sets)."""
        import torch
        n = rgb_dev.numel() // 3
        sets = [tuple(x) for x in thresholds]
        arr = (cvs_thresholds * max(len(sets), 1))()
        for i, x in enumerate(sets):
            arr[i] = make_thresholds(x[0], x[1], x[2] if len(x) > 2 else 0x7F, gamut_mode,
                                     x[3] if len(x) > 3 else None)
        dev = rgb_dev.device
        shape = (n, len(sets))
        if out is None:
            out = (torch.empty(shape, dtype=torch.float32, device=dev),
                   torch.empty(shape, dtype=torch.int32, device=dev),
                   torch.empty(shape, dtype=torch.uint8, device=dev))
        g, keep = make_grid(radii, angles_deg)
        m = cvs_capacity_map(out[0].data_ptr(), out[1].data_ptr(), out[2].data_ptr())
        check(lib().cvs_search_colors_multi(self._h, rgb_dev.data_ptr(), n, ctypes.byref(g), arr,
                                            len(sets), int(precision), ctypes.byref(m),
                                            _stream_ptr(stream)), "cvs_search_colors_multi")
        return out

    def search_colors_host(self, rgb, radii, angles_deg, v_th, r_novib, pattern_mask=0x7F,
                           gamut_mode=0, max_dl=None, precision=PREC_FP32_RECHECK, out=None):
        """As search_colors, with host NumPy buffers (copies inside the call)."""
        rgb = np.ascontiguousarray(np.asarray(rgb, np.uint8).reshape(-1, 3))
        n = rgb.shape[0]
        if out is None:
            out = (np.empty(n, np.float32), np.empty(n, np.int32), np.empty(n, np.uint8))
        g, keep = make_grid(radii, angles_deg)
        t = make_thresholds(v_th, r_novib, pattern_mask, gamut_mode, max_dl)
        check(lib().cvs_search_colors_host(self._h, rgb.ctypes.data, n, ctypes.byref(g),
                                           ctypes.byref(t), int(precision), out[0].ctypes.data,
                                           out[1].ctypes.data, out[2].ctypes.data),
              "cvs_search_colors_host")
        return out

    def embed_image(self, image, pattern, radii, angles_deg, v_th, r_novib, pattern_mask=0x7F,
                    gamut_mode=0, max_dl=None,
                    precision=PREC_FP32_RECHECK, frames=None, choice=True,
                    stream=None):
        """The two alternating frames of an (H, W, 3) uint8 CUDA image carrying a
        per-pixel pattern ((H, W) uint8 CUDA tensor, 1..7, 0 = none).
        Returns (frame_a, frame_b, choice) CUDA tensors; choice (H, W) int32 view
        of k | m << 16 (-1 where nothing was embedded) or None."""
        im, frames, ch = _embed_buffers(image, pattern, frames, choice)
        g, keep = make_grid(radii, angles_deg)
        t = make_thresholds(v_th, r_novib, pattern_mask, gamut_mode, max_dl)
        check(lib().cvs_embed_image(self._h, ctypes.byref(im), pattern.data_ptr(), pattern.stride(0),
                                    ctypes.byref(g), ctypes.byref(t), int(precision),
                                    frames[0].data_ptr(), frames[1].data_ptr(),
                                    frames[0].stride(0), ch.data_ptr() if ch is not None else None,
                                    _stream_ptr(stream)), "cvs_embed_image")
        return frames[0], frames[1], ch

    def search_images(self, images, radii, angles_deg, v_th, r_novib, pattern_mask=0x7F,
                      gamut_mode=0, max_dl=None,
                      precision=PREC_FP32_RECHECK, maps=None, stream=None):
        """Per-pixel maps for a list of (H, W, 3) uint8 CUDA tensors (row pitch from stride)."""
        import torch
        n = len(images)
        descs = (cvs_image * n)()
        if maps is None:
            maps = []
            for im in images:
                h, w = im.shape[0], im.shape[1]
                maps.append((torch.empty((h, w), dtype=torch.float32, device=im.device),
                             torch.empty((h, w), dtype=torch.int32, device=im.device),
                             torch.empty((h, w), dtype=torch.uint8, device=im.device)))
        cmaps = (cvs_capacity_map * n)()
        for i, im in enumerate(images):
            if im.dtype != torch.uint8 or im.dim() != 3 or im.shape[2] != 3 or im.stride(2) != 1 \
                    or im.stride(1) != 3:
                raise ValueError("images must be (H, W, 3) uint8 with packed pixels")
            descs[i] = cvs_image(im.data_ptr(), im.shape[1], im.shape[0], im.stride(0))
            cmaps[i] = cvs_capacity_map(maps[i][0].data_ptr(), maps[i][1].data_ptr(),
                                        maps[i][2].data_ptr())
        g, keep = make_grid(radii, angles_deg)
        t = make_thresholds(v_th, r_novib, pattern_mask, gamut_mode, max_dl)
        check(lib().cvs_search_images(self._h, descs, n, ctypes.byref(g), ctypes.byref(t),
                                      int(precision), cmaps, _stream_ptr(stream)),
              "cvs_search_images")
        return maps

    def synchronize(self, stream=None):
        check(lib().cvs_synchronize(self._h, _stream_ptr(stream)), "cvs_synchronize")

    def stats(self) -> dict:
        s = cvs_stats()
        check(lib().cvs_get_stats(self._h, ctypes.byref(s)), "cvs_get_stats")
        return {f: getattr(s, f) for f, _ in cvs_stats._fields_}

    def autotune(self, rgb_dev, radii, angles_deg, v_th, r_novib, pattern_mask=0x7F,
                 gamut_mode=0, max_dl=None, precision=PREC_FP32_RECHECK) -> dict:
        """Time launch shapes on these colours and keep the fastest (see cvs_autotune)."""
        g, keep = make_grid(radii, angles_deg)
        t = make_thresholds(v_th, r_novib, pattern_mask, gamut_mode, max_dl)
        best = cvs_launch_shape()
        n = rgb_dev.numel() // 3
        check(lib().cvs_autotune(self._h, rgb_dev.data_ptr(), n, ctypes.byref(g), ctypes.byref(t),
                                 int(precision), ctypes.byref(best)), "cvs_autotune")
        return {f: getattr(best, f) for f, _ in cvs_launch_shape._fields_}

    def build_lut(self, radii, angles_deg, v_th, r_novib, pattern_mask=0x7F, gamut_mode=0,
                  max_dl=None, precision=PREC_FP32_RECHECK, stream=None) -> "CapacityTable":
        """Capacity table of all 2^24 colours for this grid and thresholds."""
        g, keep = make_grid(radii, angles_deg)
        t = make_thresholds(v_th, r_novib, pattern_mask, gamut_mode, max_dl)
        h = ctypes.c_void_p()
        check(lib().cvs_lut_build(self._h, ctypes.byref(g), ctypes.byref(t), int(precision),
                                  ctypes.byref(h), _stream_ptr(stream)), "cvs_lut_build")
        return CapacityTable(h)

    def build_embed_table(self, radii, angles_deg, v_th, r_novib, pattern_mask=0x7F,
                          gamut_mode=0, max_dl=None, precision=PREC_FP32_RECHECK,
                          stream=None) -> "EmbedTable":
        """Embedding table of all 2^24 colours x 7 patterns for this grid and thresholds."""
        g, keep = make_grid(radii, angles_deg)
        t = make_thresholds(v_th, r_novib, pattern_mask, gamut_mode, max_dl)
        h = ctypes.c_void_p()
        check(lib().cvs_etab_build(self._h, ctypes.byref(g), ctypes.byref(t), int(precision),
                                   ctypes.byref(h), _stream_ptr(stream)), "cvs_etab_build")
        return EmbedTable(h)

    def precision_probe(self, rgb_dev, radii, angles_deg) -> dict:
        """FP32-vs-FP64 error report of every plus colour (see cvs_precision_probe)."""
        g, keep = make_grid(radii, angles_deg)
        rep = cvs_precision_report()
        n = rgb_dev.numel() // 3
        check(lib().cvs_precision_probe(self._h, rgb_dev.data_ptr(), n, ctypes.byref(g),
                                        ctypes.byref(rep)), "cvs_precision_probe")
        return {f: getattr(rep, f) for f, _ in cvs_precision_report._fields_}


class CapacityTable:
    """Per-colour results of all 2^24 colours (cvs_lut); images become gathers."""

    def __init__(self, handle):
        self._h = handle

    def close(self):
        if self._h:
            lib().cvs_lut_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def lookup_colors(self, rgb_dev, out=None, stream=None):
        import torch
        n = rgb_dev.numel() // 3
        dev = rgb_dev.device
        if out is None:
            out = (torch.empty(n, dtype=torch.float32, device=dev),
                   torch.empty(n, dtype=torch.int32, device=dev),
                   torch.empty(n, dtype=torch.uint8, device=dev))
        m = cvs_capacity_map(out[0].data_ptr(), out[1].data_ptr(), out[2].data_ptr())
        check(lib().cvs_lut_lookup_colors(self._h, rgb_dev.data_ptr(), n, ctypes.byref(m),
                                          _stream_ptr(stream)), "cvs_lut_lookup_colors")
        return out

    def lookup_images(self, images, maps=None, stream=None):
        import torch
        n = len(images)
        descs = (cvs_image * n)()
        cmaps = (cvs_capacity_map * n)()
        if maps is None:
            maps = [(torch.empty(im.shape[:2], dtype=torch.float32, device=im.device),
                     torch.empty(im.shape[:2], dtype=torch.int32, device=im.device),
                     torch.empty(im.shape[:2], dtype=torch.uint8, device=im.device))
                    for im in images]
        for i, im in enumerate(images):
            if im.dtype != torch.uint8 or im.dim() != 3 or im.shape[2] != 3 or im.stride(2) != 1 \
                    or im.stride(1) != 3:
                raise ValueError("images must be (H, W, 3) uint8 with packed pixels")
            descs[i] = cvs_image(im.data_ptr(), im.shape[1], im.shape[0], im.stride(0))
            cmaps[i] = cvs_capacity_map(maps[i][0].data_ptr(), maps[i][1].data_ptr(),
                                        maps[i][2].data_ptr())
        check(lib().cvs_lut_lookup_images(self._h, descs, n, cmaps, _stream_ptr(stream)),
              "cvs_lut_lookup_images")
        return maps


def _embed_buffers(image, pattern, frames, choice):
    import torch
    if image.dim() != 3 or image.shape[2] != 3 or image.dtype != torch.uint8:
        raise ValueError("image must be an (H, W, 3) uint8 tensor")
    h, w = image.shape[0], image.shape[1]
    if tuple(pattern.shape) != (h, w) or pattern.dtype != torch.uint8:
        raise ValueError("pattern must be an (H, W) uint8 tensor")
    if image.stride(2) != 1 or image.stride(1) != 3 or pattern.stride(1) != 1:
        raise ValueError("rows must be dense (HWC image, row-major pattern)")
    if frames is None:
        frames = (torch.empty((h, w, 3), dtype=torch.uint8, device=image.device),
                  torch.empty((h, w, 3), dtype=torch.uint8, device=image.device))
    ch = torch.empty((h, w), dtype=torch.int32, device=image.device) if choice else None
    return cvs_image(image.data_ptr(), w, h, image.stride(0)), frames, ch


class EmbedTable:
    """The embedding's pair for every colour and pattern (cvs_etab); frames
    become gathers identical to Context.embed_image."""

    def __init__(self, handle):
        self._h = handle

    def close(self):
        if self._h:
            lib().cvs_etab_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def embed_image(self, image, pattern, frames=None, choice=True, stream=None):
        im, frames, ch = _embed_buffers(image, pattern, frames, choice)
        check(lib().cvs_etab_embed_image(self._h, ctypes.byref(im), pattern.data_ptr(),
                                         pattern.stride(0), frames[0].data_ptr(),
                                         frames[1].data_ptr(), frames[0].stride(0),
                                         ch.data_ptr() if ch is not None else None,
                                         _stream_ptr(stream)), "cvs_etab_embed_image")
        return frames[0], frames[1], ch


class Server:
    """Continuous-batching request loop (cvs_server): submit host frames, wait,
    read the device-resident maps, release."""

    def __init__(self, radii, angles_deg, v_th, r_novib, pattern_mask=0x7F, gamut_mode=0,
                 max_dl=None, precision=PREC_FP32_RECHECK, device=0, max_inflight=2,
                 max_pixels=7680 * 4320, mem_budget_bytes=4 << 30, use_table=False,
                 dedup=False):
        g, self._keep = make_grid(radii, angles_deg)
        t = make_thresholds(v_th, r_novib, pattern_mask, gamut_mode, max_dl)
        cfg = cvs_server_config(int(device), int(max_inflight), int(max_pixels),
                                int(mem_budget_bytes), int(bool(use_table)), int(bool(dedup)))
        self._h = ctypes.c_void_p()
        self._frames = {}
        check(lib().cvs_server_create(ctypes.byref(self._h), ctypes.byref(cfg), ctypes.byref(g),
                                      ctypes.byref(t), int(precision)), "cvs_server_create")

    def close(self):
        if self._h:
            lib().cvs_server_destroy(self._h)
            self._h = ctypes.c_void_p()
            self._frames.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, frame) -> int:
        """Queue an (H, W, 3) uint8 host frame; it is kept alive until released."""
        frame = np.ascontiguousarray(frame, np.uint8)
        h, w = frame.shape[:2]
        tk = ctypes.c_uint64()
        check(lib().cvs_server_submit(self._h, frame.ctypes.data, w, h, w * 3, ctypes.byref(tk)),
              "cvs_server_submit")
        self._frames[tk.value] = frame
        return tk.value

    def state(self, ticket) -> int:
        s = ctypes.c_int32()
        check(lib().cvs_server_state(self._h, ticket, ctypes.byref(s)), "cvs_server_state")
        return s.value

    def wait(self, ticket, timeout_ms=60000):
        check(lib().cvs_server_wait(self._h, ticket, int(timeout_ms)), "cvs_server_wait")

    def result_host(self, ticket):
        frame = self._frames[ticket]
        h, w = frame.shape[:2]
        out = (np.empty((h, w), np.float32), np.empty((h, w), np.int32), np.empty((h, w), np.uint8))
        check(lib().cvs_server_copy_result(self._h, ticket, out[0].ctypes.data, out[1].ctypes.data,
                                           out[2].ctypes.data), "cvs_server_copy_result")
        return out

    def release(self, ticket):
        check(lib().cvs_server_release(self._h, ticket), "cvs_server_release")
        self._frames.pop(ticket, None)

    def stats(self) -> dict:
        s = cvs_server_stats()
        check(lib().cvs_server_get_stats(self._h, ctypes.byref(s)), "cvs_server_get_stats")
        return {f: getattr(s, f) for f, _ in cvs_server_stats._fields_}
