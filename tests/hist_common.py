"""Weighted-histogram comparison used by the distribution tests."""
from __future__ import annotations

import json
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_golden(name: str) -> dict:
    with open(os.path.join(GOLDEN, "oracle_hists_%s.json" % name)) as f:
        g = json.load(f)
    g["sumw"] = np.array(g["sumw"])
    g["sumw2"] = np.array(g["sumw2"])
    return g


def chi2_per_hist(a_w, a_w2, na, b_w, b_w2, nb):
    """chi^2 and ndf per histogram of two weighted samples normalised per event;
    variances from the sums of squared weights of both samples. Under- and
    overflow bins are included; bins empty in both samples are skipped."""
    out = []
    for h in range(a_w.shape[0]):
        ma, mb = a_w[h] / na, b_w[h] / nb
        va, vb = a_w2[h] / na ** 2, b_w2[h] / nb ** 2
        use = (va + vb) > 0
        chi2 = float(np.sum((ma[use] - mb[use]) ** 2 / (va[use] + vb[use])))
        out.append((chi2, int(use.sum())))
    return out


def chi2_summary(per_hist):
    chi2 = sum(c for c, _ in per_hist)
    ndf = sum(n for _, n in per_hist)
    return chi2 / max(ndf, 1), chi2, ndf
