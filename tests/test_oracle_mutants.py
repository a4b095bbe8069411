"""Mutation check of the oracle's pins (no GPU).

Each case plants one plausible mistake in a private copy of the oracle and
then runs the oracle's pin tests (tests/test_oracle_*.py) against that copy.
The mistakes are of the usual kinds:
- a dropped term;
- a wrong sign, index or operand order;
- an off-by-one comparison.

The check is that at least one pin fails for every planted mistake. The copy
lives in a temporary directory, so the oracle itself is never modified. A
control run of the unmodified copy must pass, which shows that the copy itself
is sound.
"""
import os
import re
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

ROOT = Path(__file__).resolve().parents[1]
PIN_FILES = ["test_oracle_search.py", "test_oracle_embed.py", "test_oracle_dl.py",
             "test_oracle_colour.py", "test_oracle_constants.py"]
C = "oracle/cvs_oracle.c"

# (name, file, text to replace, replacement); the text occurs exactly once
MUTANTS = [
    # colour chain (§2 Methods, step 1 and step 3)
    ("finv drops the cube", C, "return (u * u) * u;", "return u * u;"),
    ("finv linear branch drops 4/29", C, "return (u - C->f_lin_add) * C->finv_lin_mul;",
     "return u * C->finv_lin_mul;"),
    ("f linear branch drops 4/29", C, "return t * C->f_lin_mul + C->f_lin_add;",
     "return t * C->f_lin_mul;"),
    ("inverse a* sign", C, "double fx = fy + a / 500.0;", "double fx = fy - a / 500.0;"),
    ("inverse b* sign", C, "double fz = fy - b / 200.0;", "double fz = fy + b / 200.0;"),
    ("forward a* operand order", C, "lab[1] = 500.0 * (fx - fy);", "lab[1] = 500.0 * (fy - fx);"),
    ("forward b* scale", C, "lab[2] = 200.0 * (fy - fz);", "lab[2] = 500.0 * (fy - fz);"),
    ("L* offset dropped", C, "lab[0] = 116.0 * fy - 16.0;", "lab[0] = 116.0 * fy;"),
    ("inverse matrix transposed", C,
     "lin[c] = (C->MI[c][0] * X + C->MI[c][1] * Y) + C->MI[c][2] * Z;",
     "lin[c] = (C->MI[0][c] * X + C->MI[1][c] * Y) + C->MI[2][c] * Z;"),
    ("forward matrix transposed", C,
     "xyz[i] = (C->M[i][0] * lin[0] + C->M[i][1] * lin[1]) + C->M[i][2] * lin[2];",
     "xyz[i] = (C->M[0][i] * lin[0] + C->M[1][i] * lin[1]) + C->M[2][i] * lin[2];"),
    ("white point index", C, "double fz = cie_f(C, xyz[2] / C->W[2]);",
     "double fz = cie_f(C, xyz[2] / C->W[0]);"),
    ("decode channel index", C, "C->lut[rgb[1]], C->lut[rgb[2]]};",
     "C->lut[rgb[1]], C->lut[rgb[1]]};"),
    ("cube root left uncorrected", C, "for (int it = 0; it < 8; ++it) {",
     "for (int it = 0; it < 0; ++it) {"),
    # quantisation (§2 Methods, step 3)
    ("threshold compared strictly", C, "if (C->thr[mid] <= lin) lo = mid + 1;",
     "if (C->thr[mid] < lin) lo = mid + 1;"),
    ("code off by one", C, "    return lo - 1;\n}", "    return lo;\n}"),
    # pair construction (§2 Methods, step 2)
    ("sin and cos swapped", C, "double da = r * s, db = r * c;", "double da = r * c, db = r * s;"),
    ("minus colour b* sign", C, "orc_lab_to_lin(C, lab[0], lab[1] - da, lab[2] - db, lin);",
     "orc_lab_to_lin(C, lab[0], lab[1] - da, lab[2] + db, lin);"),
    # embedding-signal condition (§3 Experiments, Table 1)
    ("high not strict", C, "if (d > v_th) return 1;", "if (d >= v_th) return 1;"),
    ("low not strict", C, "if (fma(v_th, r_novib, -d) > 0.0) return 0;",
     "if (fma(v_th, r_novib, -d) >= 0.0) return 0;"),
    ("low threshold drops R_novib", C, "if (fma(v_th, r_novib, -d) > 0.0) return 0;",
     "if (fma(v_th, 1.0, -d) > 0.0) return 0;"),
    ("pattern bit order", C, "pattern |= cls << (2 - c);", "pattern |= cls << c;"),
    ("pattern mask index", C, "if (!((pattern_mask >> (pattern - 1)) & 1u)) return 0;",
     "if (!((pattern_mask >> pattern) & 1u)) return 0;"),
    ("gamut upper bound", C, "|| m[c] < 0 || m[c] > 255) {", "|| m[c] < 0 || m[c] > 256) {"),
    ("signed difference", C, "int diff = p[c] > m[c] ? p[c] - m[c] : m[c] - p[c];",
     "int diff = p[c] - m[c];"),
    ("clip keeps the minus colour's low codes", C, "if (m[c] < 0) m[c] = 0;",
     "if (m[c] < -1) m[c] = 0;"),
    # search loops and outputs (Table 2 quantities)
    ("largest radius = last passing radius", C, "if (radii[k] > best) best = radii[k];",
     "best = radii[k];"),
    ("pattern set bit index", C, "mask |= (uint8_t)(1u << (pat - 1));",
     "mask |= (uint8_t)(1u << pat);"),
    ("record k and m swapped", C, "rec.k = (uint16_t)k;\n                rec.m = (uint16_t)m;",
     "rec.k = (uint16_t)m;\n                rec.m = (uint16_t)k;"),
    # luminance limit
    ("luminance limit strict", C, "return fabs(lp[0] - L_target) <= max_dl && fabs(lm[0] - L_target) <= max_dl;",
     "return fabs(lp[0] - L_target) < max_dl && fabs(lm[0] - L_target) < max_dl;"),
    ("luminance limit checks one colour", C,
     "return fabs(lp[0] - L_target) <= max_dl && fabs(lm[0] - L_target) <= max_dl;",
     "return fabs(lp[0] - L_target) <= max_dl;"),
    # embedding (Fig. 1a)
    ("embedding: equal radius replaces", C, "if (found && !(radii[k] < best_r)) continue;",
     "if (found && !(radii[k] <= best_r)) continue;"),
    ("embedding: frames swapped", C, "memcpy(best_plus, op, 3);\n                    memcpy(best_minus, om, 3);",
     "memcpy(best_plus, om, 3);\n                    memcpy(best_minus, op, 3);"),
    ("embedding: last angle of the radius", C, "break;  /* the smallest m of this radius */",
     "/* no break */"),
    ("clip emits the unclamped code", C, "out_plus[c] = (uint8_t)p[c];",
     "out_plus[c] = (uint8_t)q_plus[c];"),
    ("search ignores the luminance limit", C,
     "if (!pat || !passes_dl(C, lab[0], rec.plus, rec.minus, max_dl)) continue;",
     "if (!pat) continue;"),
    ("embedding: any pattern", C,
     "if (decide_pair(qp, qm, v_th, r_novib, pattern_mask, gamut_mode, op, om) != p ||",
     "if (decide_pair(qp, qm, v_th, r_novib, pattern_mask, gamut_mode, op, om) == 0 ||"),
    ("embedding ignores the luminance limit", C,
     "!= p ||\n                        !passes_dl(C, lab[0], op, om, max_dl))",
     "!= p)"),
    ("embedding: first radius in list order", C, "best_r = radii[k];", "best_r = 0.0;"),
    # constants and tables (Python side)
    ("thresholds rounded to nearest (linear branch)", "oracle/constants.py",
     "out.append(_ru(_dec_exact_linear(2 * k + 1, 510)))",
     "out.append(_rn(_dec_exact_linear(2 * k + 1, 510)))"),
    ("thresholds rounded to nearest (power branch)", "oracle/constants.py",
     'out.append(pow_12_5(40 * k + 581, 10761, "ru"))',
     'out.append(pow_12_5(40 * k + 581, 10761, "rn"))'),
    ("white point from column sums", "oracle/constants.py",
     "W = tuple((row[0] + row[1]) + row[2] for row in M)",
     "W = tuple((M[0][j] + M[1][j]) + M[2][j] for j in range(3))"),
    ("inverse without the transpose", "oracle/constants.py",
     "inv = [[cof[j][i] / det for j in range(3)] for i in range(3)]",
     "inv = [[cof[i][j] / det for j in range(3)] for i in range(3)]"),
    ("decode linear branch divisor", "oracle/constants.py",
     "return Fraction(num, den) / Fraction(1292, 100)",
     "return Fraction(num, den) / Fraction(1292, 1000)"),
    ("cosine sign", "oracle/trig.py", "c = sin_exact(90 - t)", "c = sin_exact(t - 90)"),
    ("second quadrant reduction", "oracle/trig.py", "return _sin_first_quadrant(180 - th, pi)",
     "return _sin_first_quadrant(th - 90, pi)"),
    ("search wrapper swaps the tables", "oracle/__init__.py",
     "_ptr(s), _ptr(c), len(s), float(v_th), float(r_novib),\n                            int(pattern_mask)",
     "_ptr(c), _ptr(s), len(s), float(v_th), float(r_novib),\n                            int(pattern_mask)"),
]


def _sandbox(base: Path, name: str, mutation) -> Path:
    dst = base / re.sub(r"[^a-z0-9]+", "_", name.lower())
    shutil.copytree(ROOT / "oracle", dst / "oracle",
                    ignore=shutil.ignore_patterns("_build", "__pycache__"))
    (dst / "tests").mkdir()
    for f in ["conftest.py", *PIN_FILES]:
        shutil.copy(ROOT / "tests" / f, dst / "tests" / f)
    shutil.copytree(ROOT / "tests" / "golden", dst / "tests" / "golden")
    if mutation is not None:
        path, old, new = mutation
        p = dst / path
        text = p.read_text()
        assert text.count(old) == 1, (name, old)
        p.write_text(text.replace(old, new))
    return dst


def _run_pins(dst: Path) -> tuple[int, str]:
    env = dict(os.environ, OMP_NUM_THREADS="2", PYTHONDONTWRITEBYTECODE="1")
    env.pop("PYTHONPATH", None)
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
           "-k", "not table2", *[f"tests/{f}" for f in PIN_FILES]]
    r = subprocess.run(cmd, cwd=dst, env=env, capture_output=True, text=True, timeout=900)
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    return r.returncode, lines[-1] if lines else r.stderr[-300:]


def _caught(rc: int, summary: str) -> bool:
    # a failed pin, not a broken copy (an import or build error)
    return rc == 1 and " failed" in summary and "error" not in summary


def test_pins_catch_planted_mistakes(tmp_path):
    jobs = [("control", None)] + [(n, (f, o, w)) for n, f, o, w in MUTANTS]
    dirs = [(n, _sandbox(tmp_path, n, m)) for n, m in jobs]
    workers = max(1, min(8, (os.cpu_count() or 2) // 2))
    with ThreadPoolExecutor(max_workers=workers) as ex:
        results = list(ex.map(lambda nd: (nd[0],) + _run_pins(nd[1]), dirs))
    control = results[0]
    assert control[1] == 0, f"the unmodified copy fails its pins: {control[2]}"
    survivors = [(n, rc, s) for n, rc, s in results[1:] if not _caught(rc, s)]
    assert not survivors, "planted mistakes no pin catches: " + "; ".join(
        f"{n} (rc {rc}: {s})" for n, rc, s in survivors)
