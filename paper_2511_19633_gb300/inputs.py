"""Synthetic, seeded inputs shared by the CUDA library binding, the tests and
the benchmark.

This module holds input data only: the synthetic parton-density table that
stands in for the CT14lo grid of the paper (Section 4.1, Fig. 4 caption) and
the workload presets. It contains none of the shower's arithmetic.

PDF table: x f_i(x, Q^2) = N_i x^{a_i} (1 - x)^{b_i}, independent of Q^2,
tabulated on 100 nodes uniform in ln x over [1e-6, 1 - 1e-6] and 50 nodes
uniform in ln Q^2 over [0.5, 13600^2] GeV^2, stored as float32 with layout
[flavour][x node][Q^2 node]. Flavour order: g, d, u, s, c, b, dbar, ubar,
sbar, cbar, bbar.
  gluon   (a, b) = (-0.2, 5), N = 1.7
  valence (a, b) = (0.5, 3),  N_uv = 2 / B(0.5, 4), N_dv = 1 / B(0.5, 4)
          (so that the valence number sum rules give 2 and 1)
  sea     (a, b) = (-0.2, 7), N = 0.1 (every antiquark, s, c, b)
  u = u_v + sea, d = d_v + sea
With heavy-quark thresholds (synthetic_pdf_grid(thresholds=True), the
stand-in for a PDF whose c and b densities vanish at their masses, App. A.2):
the c, b, cbar and bbar densities are sea(x) (1 - m_q^2/Q^2) above m_q^2 and
zero at and below it, with m_c^2 and m_b^2 on Q^2 nodes 3 and 9 of the grid
(1.674 and 18.73 GeV^2, m_c = 1.29 GeV, m_b = 4.33 GeV), so that the
interpolated density vanishes exactly at the mass.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

PDF_NX = 100
PDF_NQ = 50
PDF_NFL = 11
PDF_X_MIN = 1e-6
PDF_X_MAX = 1.0 - 1e-6
PDF_Q2_MIN = 0.5
PDF_Q2_MAX = 13600.0 ** 2

FLAVOURS = ("g", "d", "u", "s", "c", "b", "dbar", "ubar", "sbar", "cbar", "bbar")


def _beta(a: float, b: float) -> float:
    return math.exp(math.lgamma(a) + math.lgamma(b) - math.lgamma(a + b))


PDF_PARAMS = {
    "g": (1.7, -0.2, 5.0),
    "uv": (2.0 / _beta(0.5, 4.0), 0.5, 3.0),
    "dv": (1.0 / _beta(0.5, 4.0), 0.5, 3.0),
    "sea": (0.1, -0.2, 7.0),
}


def x_nodes() -> np.ndarray:
    lx = np.log(PDF_X_MIN) + np.arange(PDF_NX) * (np.log(PDF_X_MAX) - np.log(PDF_X_MIN)) / (PDF_NX - 1)
    return np.exp(lx)


def q2_nodes() -> np.ndarray:
    lq = np.log(PDF_Q2_MIN) + np.arange(PDF_NQ) * (np.log(PDF_Q2_MAX) - np.log(PDF_Q2_MIN)) / (PDF_NQ - 1)
    return np.exp(lq)


def synthetic_xf(name: str, x: np.ndarray) -> np.ndarray:
    """x f(x) of one synthetic component ('g', 'uv', 'dv', 'sea'), float64."""
    n, a, b = PDF_PARAMS[name]
    return n * np.power(x, a) * np.power(1.0 - x, b)


def synthetic_flavour_xf(flavour: str, x: np.ndarray) -> np.ndarray:
    if flavour == "g":
        return synthetic_xf("g", x)
    sea = synthetic_xf("sea", x)
    if flavour == "u":
        return synthetic_xf("uv", x) + sea
    if flavour == "d":
        return synthetic_xf("dv", x) + sea
    return sea


# Q^2 node of each heavy flavour's mass (thresholded table)
HQ_THRESHOLD_NODE = {"c": 3, "b": 9, "cbar": 3, "bbar": 9}


def synthetic_pdf_grid(thresholds: bool = False) -> np.ndarray:
    """float32 array [11][100][50] of x f(x, Q^2) on the grid nodes."""
    x = x_nodes()
    q2 = q2_nodes()
    grid = np.empty((PDF_NFL, PDF_NX, PDF_NQ), dtype=np.float64)
    for i, fl in enumerate(FLAVOURS):
        grid[i] = synthetic_flavour_xf(fl, x)[:, None]
        if thresholds and fl in HQ_THRESHOLD_NODE:
            k0 = HQ_THRESHOLD_NODE[fl]
            h = np.zeros(PDF_NQ)
            h[k0 + 1:] = 1.0 - q2[k0] / q2[k0 + 1:]
            grid[i] *= h[None, :]
    return np.ascontiguousarray(grid.astype(np.float32))


# ---------------------------------------------------------------------------
# workload presets (process codes: 0 = e+e- -> q qbar, 1 = pp -> Z LO,
# 2 = pp -> Z NLO-matched)
# ---------------------------------------------------------------------------
PROC_EE = 0
PROC_PP_LO = 1
PROC_PP_NLO = 2


@dataclass
class Workload:
    name: str
    process: int
    sqrt_s: float
    n_events: int
    t_cut: float = 1.0
    alpha_s_mz: float = 0.118
    nf: int = 5
    seed: int = 1
    p_s: float = 0.5
    nmax: int = 64
    extra: dict = field(default_factory=dict)


WORKLOADS = {
    "ee91": Workload("e+e- -> q qbar at 91.2 GeV, final-state shower, 1e4 events",
                     PROC_EE, 91.2, 10_000),
    "pp_lo": Workload("pp -> Z at 13.6 TeV, LO + initial/final shower, 1e6 events",
                      PROC_PP_LO, 13600.0, 1_000_000),
    "pp_nlo": Workload("NLO-matched pp -> Z at 13.6 TeV, 1e7 events",
                       PROC_PP_NLO, 13600.0, 10_000_000),
    "ee500": Workload("e+e- -> q qbar at 500 GeV, final-state shower",
                      PROC_EE, 500.0, 10_000),
}
