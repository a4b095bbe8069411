"""libcvsearch host-side checks that need no GPU: the library builds, loads and
exports every declared symbol; threshold resolution and constant tables agree
with the oracle; calls fail cleanly without a device."""
import ctypes
import re
import subprocess
import sys
from pathlib import Path

import numpy as np
import pytest

import oracle
from oracle import constants as K
import paper_2507_22901_gb300 as cvs
from paper_2507_22901_gb300 import binding

ROOT = Path(__file__).resolve().parent.parent


def test_library_builds_and_exports_header_symbols():
    L = cvs.lib()
    names = cvs.header_functions()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    assert L.cvs_version().decode().count(".") == 2


def test_header_declares_documented_entry_points():
    names = set(cvs.header_functions())
    for n in ["cvs_create", "cvs_destroy", "cvs_search_color", "cvs_search_colors",
              "cvs_search_images", "cvs_last_error", "cvs_synchronize"]:
        assert n in names


def _oracle_class(d, vth, rn):
    """1 high, 0 low, -1 neither, by the oracle's decision rule."""
    pat, _, _ = oracle.decide_pair((d, 0, 0), (0, 0, 0), vth, rn, pattern_mask=0x7F)
    if pat == 4:
        return 1
    pat2, _, _ = oracle.decide_pair((d, 255, 0), (0, 0, 0), vth, rn, pattern_mask=0x7F)
    # with G high (255 > vth when vth < 255) and B low, R low gives pattern 010
    return 0 if pat2 == 2 else -1


@pytest.mark.parametrize("vth,rn", [(50, 0.5), (100, 0.25), (150, 0.125), (200, 0.125),
                                    (50, 0.125), (37.5, 0.3), (49.999, 0.5000001)])
def test_signal_bounds_match_oracle_rule(vth, rn):
    hi, lo = cvs.signal_bounds(vth, rn)
    for d in range(256):
        cls = 1 if d >= hi else (0 if d <= lo else -1)
        if vth < 255:
            assert cls == _oracle_class(d, vth, rn), (d, hi, lo)


def test_signal_bounds_exact_products():
    # product exactly an integer: d < 25 is low, 25 is not
    assert cvs.signal_bounds(50, 0.5) == (51, 24)
    # 150 * 0.125 = 18.75
    assert cvs.signal_bounds(150, 0.125) == (151, 18)
    # a product that rounds to an integer but is slightly above it in exact terms
    v, r = 3.0, 1.0 / 3.0  # 3 * RN(1/3) < 1 exactly
    hi, lo = cvs.signal_bounds(v, r)
    assert lo == 0  # d = 0 < 0.999..., d = 1 is not
    rng = np.random.default_rng(4)
    cases = [(0.0, 0.5), (255.0, 1.0), (254.5, 1.0)]
    cases += [(float(rng.uniform(0, 260)), float(rng.uniform(1e-3, 1.0))) for _ in range(300)]
    for v, r in cases:
        hi, lo = cvs.signal_bounds(v, r)
        from fractions import Fraction
        p = Fraction(v) * Fraction(r)
        assert all((Fraction(d) < p) == (d <= lo) for d in range(0, 256))
        assert all((d > v) == (d >= hi) for d in range(0, 256))


@pytest.mark.parametrize("bad", [dict(v_th=float("nan")), dict(v_th=-1.0), dict(r_novib=0.0),
                                 dict(r_novib=1.5), dict(pattern_mask=0x80), dict(gamut_mode=2),
                                 dict(max_dl=float("nan")), dict(max_dl=-0.25)])
def test_signal_bounds_rejects_invalid(bad):
    args = dict(v_th=50.0, r_novib=0.5, pattern_mask=0x7F, gamut_mode=0)
    args.update(bad)
    with pytest.raises(cvs.CvsError) as ei:
        cvs.signal_bounds(**args)
    assert ei.value.status == binding.CVS_ERR_INVALID_ARG


@pytest.mark.parametrize("max_dl", [None, 0.0, 0.1, float("inf")])
def test_signal_bounds_accepts_luminance_limits(max_dl):
    assert cvs.signal_bounds(50, 0.5, max_dl=max_dl) == (51, 24)


def _grab(txt, name):
    m = re.search(r"#define " + name + r" \{(.*?)\}", txt, re.S)
    vals = m.group(1).replace("\\", " ").split(",")
    return [float.fromhex(v.strip()) for v in vals if v.strip()]


def test_library_tables_equal_oracle_tables():
    txt = (ROOT / "paper_2507_22901_gb300" / "csrc" / "cvs_tables.h").read_text()
    assert _grab(txt, "CVS_DECODE_INIT") == list(K.srgb_decode_lut())
    assert _grab(txt, "CVS_QTHR_INIT") == list(K.quant_thresholds())
    M, W, MI = K.matrices()
    assert _grab(txt, "CVS_M_INIT") == [x for r in M for x in r]
    assert _grab(txt, "CVS_W_INIT") == list(W)
    assert _grab(txt, "CVS_MI_INIT") == [x for r in MI for x in r]
    cc = K.cie_constants()
    for key, name in [("F_BREAK", "CVS_F_BREAK"), ("FINV_BREAK", "CVS_FINV_BREAK"),
                      ("F_LIN_MUL", "CVS_F_LIN_MUL"), ("F_LIN_ADD", "CVS_F_LIN_ADD"),
                      ("FINV_LIN_MUL", "CVS_FINV_LIN_MUL")]:
        m = re.search(r"#define " + name + r" (\S+)", txt)
        assert float.fromhex(m.group(1)) == cc[key], name


def test_generated_header_is_current(tmp_path):
    src = ROOT / "paper_2507_22901_gb300" / "csrc" / "gen_tables.py"
    code = src.read_text().replace(
        'OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cvs_tables.h")',
        f'OUT = {str(tmp_path / "t.h")!r}')
    gen = tmp_path / "gen.py"
    gen.write_text(code)
    subprocess.run([sys.executable, str(gen)], check=True, capture_output=True)
    committed = (ROOT / "paper_2507_22901_gb300" / "csrc" / "cvs_tables.h").read_text()
    assert (tmp_path / "t.h").read_text() == committed


def test_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(cvs.CvsError) as ei:
        cvs.Context(0)
    assert ei.value.status in (binding.CVS_ERR_CUDA, binding.CVS_ERR_INVALID_ARG)
    assert cvs.binding.last_error()


def test_null_context_rejected():
    L = cvs.lib()
    s = binding.cvs_stats()
    assert L.cvs_get_stats(None, ctypes.byref(s)) == binding.CVS_ERR_INVALID_ARG
    assert L.cvs_synchronize(None, None) == binding.CVS_ERR_INVALID_ARG
    g, keep = binding.make_grid([1.0], [0.0])
    t = binding.make_thresholds(50, 0.5)
    m = binding.cvs_capacity_map(None, None, None)
    assert L.cvs_search_colors(None, None, 1, ctypes.byref(g), ctypes.byref(t), 0,
                               ctypes.byref(m), None) == binding.CVS_ERR_INVALID_ARG


def test_workload_shapes():
    from paper_2507_22901_gb300 import workloads as W
    assert W.color_cube().shape == (262144, 3)
    r, a = W.grid(2)
    assert len(r) == 128 and len(a) == 360 and r[0] == 0.25 and r[-1] == 32.0
    r, a = W.grid(4)
    assert len(r) == 256 and len(a) == 720
    r, a = W.grid(3)
    assert len(r) == 64 and len(a) == 180 and a[-1] == 358.0
    pc = W.precision_colors()
    assert pc.shape == (4096, 3) and pc.dtype == np.uint8
    ip = W.image_params()
    assert len(ip) == 48 and all(256 <= w <= 3840 and 256 <= h <= 2160 for w, h, _, _ in ip)
    img = W.render_image_numpy(37, 23, ip[0][2], 5)
    assert img.shape == (23, 37, 3) and img.dtype == np.uint8
    req = W.serving_requests()
    assert len(req) == 600 and all(req[i][0] < req[i + 1][0] for i in range(599))


STRUCTS = ["cvs_grid", "cvs_thresholds", "cvs_pair", "cvs_capacity_map", "cvs_image", "cvs_stats",
           "cvs_precision_report", "cvs_launch_shape", "cvs_server_config", "cvs_server_stats"]


def test_binding_structs_match_the_header(tmp_path):
    """Size and field offsets of every public struct, as the C compiler lays
    them out from include/cvsearch.h, equal the binding's ctypes layouts."""
    import shutil
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "cvsearch.h"', "int main(void) {"]
    for name in STRUCTS:
        st = getattr(binding, name)
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in st._fields_:
            lines.append(f'printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    include = str(Path(__file__).resolve().parent.parent / "include")
    subprocess.run([gcc, "-std=c11", "-I", include, str(src), "-o", str(exe)], check=True)
    got = {}
    for row in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n"):
        if row:
            name, key, val = row.split()
            got[(name, key)] = int(val)
    for name in STRUCTS:
        st = getattr(binding, name)
        assert got[(name, "size")] == ctypes.sizeof(st), name
        for field, _ in st._fields_:
            assert got[(name, field)] == getattr(st, field).offset, (name, field)
