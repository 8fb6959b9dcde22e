"""Writes the oracle's reference histograms (tests/golden/oracle_hists_<name>.json)
used by the distribution tests of the mixed-precision and learned-proposal
showers. Calls only the FP64 oracle (seed 2, independent of the GPU runs).

    python tests/golden/make_oracle_hists.py [--threads N] [--only NAME]

Histogram definitions (observable index, axis, range, regular bins) are the
ones the library reports through gaps_hist_binning; the distribution tests
check that the two tables agree.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

# (lo, hi, nbins, observable index, log10 axis)
BINNING = {
    "ee": [(0.0, 0.5, 50, 0, 0), (-5.0, 0.0, 50, 1, 1), (-5.0, 0.0, 50, 2, 1),
           (-0.5, 63.5, 64, 3, 0), (-0.5, 63.5, 64, 4, 0), (-4.0, 0.0, 40, 0, 1)],
    "pp": [(-1.0, 3.0, 40, 0, 1), (-6.0, 6.0, 48, 1, 0), (-math.pi, math.pi, 32, 2, 0),
           (-0.5, 15.5, 16, 3, 0), (0.5, 3.5, 30, 4, 1), (-0.5, 127.5, 64, 6, 0)],
}
NBINS = 66

# name: (process, sqrt_s, events, t_cut[, seed]); seed 2 unless given
WORKLOADS = {
    "ee91": (0, 91.2, 10_000_000, 1.0),
    "ee500": (0, 500.0, 10_000_000, 1.0),
    "pp_lo": (1, 13600.0, 10_000_000, 1.0),
    "pp_nlo": (2, 13600.0, 10_000_000, 1.0),
    # pp -> gamma*/Z -> e- e+, LO, dilepton mass 66-116 GeV
    "pp_ll": (3, 13600.0, 10_000_000, 1.0),
    # the e+e- rows of the mixed batch (their own cutoffs)
    "ee91_tc0.5": (0, 91.2, 10_000_000, 0.5),
    "ee500_tc4": (0, 500.0, 10_000_000, 4.0),
    # the same seed and events as the GPU runs of the precision comparison
    # (events 0 .. 1e6 - 1 of seed 1): the mixed-precision path's error per
    # observable on the same events
    "pp_nlo_seed1": (2, 13600.0, 1_000_000, 1.0, 1),
    # NLO pp -> Z with the thresholded synthetic table (c and b densities that
    # vanish at their masses): the heavy-quark measure correction of App. A.2
    "pp_nlo_hq": (2, 13600.0, 2_000_000, 1.0, 2, "thresholds"),
}
SEED = 2


def bin_index(v: np.ndarray, lo: float, hi: float, nb: int, logx: int) -> np.ndarray:
    """underflow 0, regular bins 1..nb, overflow nb+1 (same rule as the library)."""
    v = np.asarray(v, dtype=np.float64)
    out = np.zeros(v.shape, dtype=np.int64)
    with np.errstate(divide="ignore", invalid="ignore"):
        if logx:
            pos = v > 0.0
            vv = np.where(pos, np.log10(np.where(pos, v, 1.0)), -np.inf)
        else:
            vv = v
        ok = vv >= lo
        f = (vv - lo) / (hi - lo)
        b = np.floor(f * nb)
    b = np.where(ok, b, -1.0)
    out = np.where(~ok, 0, np.where(b >= nb, nb + 1, b + 1)).astype(np.int64)
    return out


def fill(hsum, hsum2, obs, w, family):
    for h, (lo, hi, nb, oi, lg) in enumerate(BINNING[family]):
        idx = bin_index(obs[:, oi], lo, hi, nb, lg)
        np.add.at(hsum[h], idx, w)
        np.add.at(hsum2[h], idx, w * w)


def make(name: str, threads: int, n_override: int | None = None) -> dict:
    from oracle import oracle as O
    from paper_2511_19633_gb300 import inputs
    process, sqrt_s, n, t_cut = WORKLOADS[name][:4]
    seed = WORKLOADS[name][4] if len(WORKLOADS[name]) > 4 else SEED
    thresholds = len(WORKLOADS[name]) > 5 and WORKLOADS[name][5] == "thresholds"
    if n_override:
        n = n_override
    pdf = inputs.synthetic_pdf_grid(thresholds=thresholds)
    family = "ee" if process == 0 else "pp"
    st = O.Settings(process=process, sqrt_s=sqrt_s, t_cut=t_cut, nmax=128, seed=seed)
    hsum = np.zeros((6, NBINS))
    hsum2 = np.zeros((6, NBINS))
    counters = np.zeros(6, dtype=np.int64)
    bad = 0
    chunk = 20_000
    t0 = time.time()
    for first in range(0, n, chunk):
        m = min(chunk, n - first)
        r = O.run(st, first, m, pdf if process else None, threads=threads)
        done = r["status"] == 1
        bad += int((~done).sum())
        fill(hsum, hsum2, r["obs"][done], r["weight"][done], family)
        counters += r["counters"].astype(np.int64).sum(0)
    return {"workload": name, "process": process, "sqrt_s": sqrt_s, "t_cut": t_cut, "events": n, "seed": seed,
            "pdf": "thresholded" if thresholds else "plain",
            "not_done": bad, "binning": BINNING[family], "sumw": hsum.tolist(), "sumw2": hsum2.tolist(),
            "oracle_counters": dict(zip(("steps", "trials", "isr_trials", "vetoes", "accepts",
                                         "violations"), counters.tolist())),
            "seconds": time.time() - t0, "threads": threads,
            "command": "python tests/golden/make_oracle_hists.py --only %s" % name}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--only", default=None)
    args = ap.parse_args()
    names = [args.only] if args.only else list(WORKLOADS)
    for name in names:
        res = make(name, args.threads)
        path = os.path.join(HERE, "oracle_hists_%s.json" % name)
        with open(path, "w") as f:
            json.dump(res, f)
        print(name, res["events"], "events in %.0f s" % res["seconds"], flush=True)


if __name__ == "__main__":
    main()
