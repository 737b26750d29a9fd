"""Writes lattice_report.json: how far the oracle's lattice is from the exact sum.

Appendix A of the paper reports, for another implementation's constants, the
ratio brute force / lattice of the filtered ones vector and that the two are
collinear.  This script computes the same quantities for the lattice
conventions used here, with the oracle only:
    python tests/golden/lattice_report.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import crf  # noqa: E402
from oracle import permutohedral as P  # noqa: E402
from paper_1608_06192_gb300 import synthetic as S  # noqa: E402


def report(problem, name):
    fb, fs = crf.features(problem.rgb, *problem.thetas)
    out = {}
    rng = np.random.default_rng(0)
    v = rng.uniform(size=(problem.n_pixels, 1))
    for kname, f in (("bilateral", fb), ("spatial", fs)):
        lat = P.Permutohedral(crf.to_fp32_features(f))
        brute = crf.BruteGaussian([f], [1.0])
        ones = np.ones((problem.n_pixels, 1))
        kb, kl = brute.apply(ones)[:, 0], lat.filter(ones)[:, 0]
        vb, vl = brute.apply(v)[:, 0], lat.filter(v)[:, 0]
        out[kname] = {
            "vertices": int(lat.m),
            "ratio_brute_over_lattice_ones_mean": float(np.mean(kb / kl)),
            "ratio_brute_over_lattice_ones_median": float(np.median(kb / kl)),
            "cosine_ones": float(kb @ kl / np.linalg.norm(kb) / np.linalg.norm(kl)),
            "cosine_random_input": float(vb @ vl / np.linalg.norm(vb) / np.linalg.norm(vl)),
        }
    return {name: out}


if __name__ == "__main__":
    res = {}
    res.update(report(S.qp_small(), "64x48"))
    res.update(report(S.qp_cccp_medium(), "320x213"))
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lattice_report.json")
    json.dump(res, open(path, "w"), indent=1)
    print(json.dumps(res, indent=1))
