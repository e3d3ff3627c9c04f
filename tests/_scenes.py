"""Helpers shared by the tests: scenes from the golden fixture."""
import json
import os

import numpy as np

from paper_1808_02414_gb300.synth import Scene

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def golden_entries():
    with open(os.path.join(GOLDEN, "tiny_gt.json")) as f:
        data = json.load(f)
    out = []
    for e in data:
        sc = Scene(np.array(e["cams"]), np.array(e["pts"]),
                   np.array(e["obs_cam"], dtype=np.int32), np.array(e["obs_pt"], dtype=np.int32),
                   np.array(e["obs_u"]), float(e["sigma"]),
                   None if e["obs_cov"] is None else np.array(e["obs_cov"]), {"kind": e["name"]})
        gt = np.array([[[float(v) for v in row] for row in blk] for blk in e["sigma_P_blocks"]])
        out.append((e["name"], sc, gt))
    return out
