"""Write the oracle-derived golden files in this folder.

Calls only the oracle package.  Run from the repository root:
    python tests/golden/gen_golden.py
"""
import hashlib
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402


def search_color_gray170():
    """Target (170,170,170), radii 0..30 step 0.5 (61), angles 0..359 step 1,
    the twelve (V_th, R_novib) combinations of Table 1, all seven patterns,
    both gamut modes."""
    radii = [0.5 * i for i in range(61)]
    ang = [float(a) for a in range(360)]
    tt = oracle.trig_table(ang)
    combos = []
    for gamut in (0, 1):
        for vth in (50, 100, 150, 200):
            for rn in (0.5, 0.25, 0.125):
                pairs, n = oracle.search_color((170, 170, 170), np.asarray(radii), np.asarray(ang),
                                               vth, rn, gamut_mode=gamut, trig_tab=tt)
                combos.append({"v_th": vth, "r_novib": rn, "gamut_mode": gamut, "count": n,
                               "sha256": hashlib.sha256(pairs.tobytes()).hexdigest()})
    return {"rgb": [170, 170, 170], "radii": radii, "angles_deg": ang,
            "record": "16-byte records: u16 k, u16 m, u8 plus[3], u8 minus[3], u8 pattern, "
                      "u8 flags, u32 target (little endian)",
            "combos": combos}


if __name__ == "__main__":
    with open(os.path.join(HERE, "search_color_gray170.json"), "w") as f:
        json.dump(search_color_gray170(), f, indent=1)
    print("wrote search_color_gray170.json")
