"""Writes tests/golden/tiny_gt.json: extended-precision ground truth for two
tiny scenes, computed only by oracle.brute (the paper's ground-truth procedure,
Sec. 6: SVD of the dense M, exactly the last seven singular values set to zero,
the rest inverted, in many-digit arithmetic).  Scene inputs are stored beside
the values so that the fixture does not depend on the generator's bits.

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import mpmath as mp  # noqa: E402
import numpy as np  # noqa: E402

from oracle import brute  # noqa: E402
from paper_1808_02414_gb300 import synth  # noqa: E402

DPS = 40


def entry(sc, name):
    M = brute.information_mp(sc, dps=DPS)
    P, sv, _ = brute.pinv_svd_mp(M, dps=DPS)
    n = sc.n
    blocks = [[[mp.nstr(P[9 * i + a, 9 * i + b], 30) for b in range(9)] for a in range(9)]
              for i in range(n)]
    return {
        "name": name,
        "citation": "Sec. 6 (accuracy paragraph) and Table 2 Alg. 1: M-P inverse of M "
                    "by SVD with the last 7 singular values zeroed, extended precision",
        "digits": DPS,
        "cams": sc.cams.tolist(), "pts": sc.pts.tolist(),
        "obs_cam": sc.obs_cam.tolist(), "obs_pt": sc.obs_pt.tolist(),
        "obs_u": sc.obs_u.tolist(), "sigma": sc.sigma,
        "obs_cov": None if sc.obs_cov is None else sc.obs_cov.tolist(),
        "singular_values_tail": [mp.nstr(s, 10) for s in sv[-9:]],
        "sigma_P_blocks": blocks,
    }


def main():
    out = [entry(synth.tiny_scene(n=4, m=14, track_len=3, seed=0), "tiny_iso"),
           entry(synth.tiny_scene(n=4, m=12, track_len=3, seed=3, anisotropic=True), "tiny_aniso")]
    with open(os.path.join(os.path.dirname(__file__), "tiny_gt.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
