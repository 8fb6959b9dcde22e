"""Pins of the oracle's pp -> gamma*/Z -> e- e+ process (the LO process GAPS 2
provides besides on-shell Z production, Sec. 4.1). No GPU needed.

- The partonic cross section against an independent form of the same matrix
  element: helicity amplitudes Q_q Q_e + 4 kappa g_i^q g_j^e s/(s - m_Z^2 + i m_Z
  Gamma_Z), weighted by (1 + cos)^2 for equal and (1 - cos)^2 for opposite
  helicities (the oracle writes it with V/A couplings and chi_1, chi_2).
- The hadronic cross section in the mass window and dsigma/dcos(theta*) in
  bins by quadrature against the weighted events, cos(theta*) taken from the
  event's lepton momenta.
- Event records: momentum conservation, masses in the window, flavours.
"""
import math

import numpy as np
import pytest
from scipy import integrate, stats

MZ, GZ, S2W, GF, AEM, NC = 91.1876, 2.4952, 0.2312, 1.16638e-5, 1.0 / 128.9, 3.0
GEV2PB = 0.3893794e9
LO, HI = 66.0, 116.0


def helicity_dsigma(s, f, c):
    up = f in (2, 4)
    Qq, T3q = (2.0 / 3.0, 0.5) if up else (-1.0 / 3.0, -0.5)
    Qe, T3e = -1.0, -0.5
    gq = {"L": T3q - Qq * S2W, "R": -Qq * S2W}
    ge = {"L": T3e - Qe * S2W, "R": -Qe * S2W}
    kappa = math.sqrt(2.0) * GF * MZ ** 2 / (4.0 * math.pi * AEM)
    prop = s / complex(s - MZ ** 2, MZ * GZ)
    tot = 0.0
    for i in "LR":
        for j in "LR":
            amp = Qq * Qe + 4.0 * kappa * gq[i] * ge[j] * prop
            tot += abs(amp) ** 2 * ((1.0 + c) ** 2 if i == j else (1.0 - c) ** 2)
    return math.pi * AEM ** 2 / (8.0 * s) * tot / NC


@pytest.mark.parametrize("m", [40.0, 70.0, MZ, 100.0, 150.0, 500.0])
@pytest.mark.parametrize("f", [1, 2, 3, 4, 5])
def test_partonic_cross_section_equals_helicity_amplitudes(oracle_mod, m, f):
    for c in (-0.95, -0.4, 0.0, 0.3, 0.99):
        assert oracle_mod.ll_dsigma(m * m, f, c) == pytest.approx(helicity_dsigma(m * m, f, c), rel=1e-12)


@pytest.mark.parametrize("m", [20.0, MZ, 200.0, 500.0])
@pytest.mark.parametrize("f", [1, 2, 3, 4, 5])
def test_ee_to_qq_cross_section_equals_helicity_amplitudes(oracle_mod, m, f):
    """e+e- -> q qbar (the e+e- hard process): the same helicity amplitudes
    with the sum N_c over the outgoing colours in place of the average 1/N_c;
    cos(theta) between the electron and the quark."""
    for c in (-0.9, -0.2, 0.0, 0.5, 0.97):
        assert oracle_mod.ee_dsigma(m * m, f, c) == pytest.approx(helicity_dsigma(m * m, f, c) * NC * NC, rel=1e-12)


def test_partonic_photon_limit(oracle_mod):
    """Far below the pole the photon term dominates: sigma = 4 pi alpha^2 Q^2 / (3 s N_c)."""
    s = 2.0 ** 2
    sig = integrate.quad(lambda c: oracle_mod.ll_dsigma(s, 2, c), -1.0, 1.0)[0]
    assert sig == pytest.approx(4.0 * math.pi * AEM ** 2 * (4.0 / 9.0) / (3.0 * s * NC), rel=2e-3)


def _pairs():
    out = []
    for k in range(10):
        q = k % 5 + 1
        out.append((q, -q) if k < 5 else (-q, q))
    return out


def _density(oracle_mod, pdf, sqrt_s, m2, y, c):
    """sum over ordered pairs of F_a F_b / m^2 dsigma/dcos, cos from beam 1's side."""
    m = math.sqrt(m2)
    ea, eb = math.exp(y) * m / sqrt_s, math.exp(-y) * m / sqrt_s
    tot = 0.0
    for fa, fb in _pairs():
        Fa = oracle_mod.pdf_xf(pdf, _pdf_index(fa), ea, m2)
        Fb = oracle_mod.pdf_xf(pdf, _pdf_index(fb), eb, m2)
        tot += Fa * Fb * oracle_mod.ll_dsigma(m2, abs(fa), c if fa > 0 else -c)
    return tot / m2


def _pdf_index(fl):
    return fl if fl > 0 else 5 - fl


def _quadrature(oracle_mod, pdf, sqrt_s, c_lo, c_hi, n_r=24, n_y=24):
    """int dm^2 dy dcos over the window (Gauss-Legendre in the Breit-Wigner
    variable and in y, exact 3-point rule in cos: the density is quadratic)."""
    mg = MZ * GZ
    r_lo, r_hi = math.atan((LO * LO - MZ * MZ) / mg), math.atan((HI * HI - MZ * MZ) / mg)
    xr, wr = np.polynomial.legendre.leggauss(n_r)
    xy, wy = np.polynomial.legendre.leggauss(n_y)
    xc, wc = np.polynomial.legendre.leggauss(3)
    total = 0.0
    for a, wa in zip(xr, wr):
        rho = 0.5 * (r_lo + r_hi) + 0.5 * (r_hi - r_lo) * a
        m2 = MZ * MZ + mg * math.tan(rho)
        jac_m = mg / math.cos(rho) ** 2 * 0.5 * (r_hi - r_lo)
        Y = math.log(sqrt_s / math.sqrt(m2))
        for b, wb in zip(xy, wy):
            y = Y * b
            for cc, wcc in zip(xc, wc):
                c = 0.5 * (c_lo + c_hi) + 0.5 * (c_hi - c_lo) * cc
                total += wa * wb * wcc * jac_m * Y * 0.5 * (c_hi - c_lo) * _density(oracle_mod, pdf, sqrt_s, m2, y, c)
    return total * GEV2PB


def test_hadronic_cross_section_and_angular_bins(oracle_mod, pdf):
    sqrt_s = 13600.0
    st = oracle_mod.Settings(process=3, sqrt_s=sqrt_s, mll_lo=LO, mll_hi=HI)
    n = 100_000
    r = oracle_mod.run(st, 0, n, pdf, hard_only=True, threads=4)
    w = r["weight"]
    sigma = _quadrature(oracle_mod, pdf, sqrt_s, -1.0, 1.0)
    assert w.mean() == pytest.approx(sigma, rel=5 * w.std() / math.sqrt(n) / sigma)
    # cos(theta*) of the electron in the dilepton frame from the momenta:
    # at LO the pair has no pT, so cos = tanh(y_e - y_pair)
    P = r["p"]
    el, po = P[:, 2, :], P[:, 3, :]
    pair = el + po
    y_pair = 0.5 * np.log((pair[:, 0] + pair[:, 3]) / (pair[:, 0] - pair[:, 3]))
    y_e = 0.5 * np.log((el[:, 0] + el[:, 3]) / (el[:, 0] - el[:, 3]))
    cth = np.tanh(y_e - y_pair)
    edges = np.linspace(-1.0, 1.0, 5)
    hw, _ = np.histogram(cth, edges, weights=w)
    hw2, _ = np.histogram(cth, edges, weights=w * w)
    expect = np.array([_quadrature(oracle_mod, pdf, sqrt_s, a, b, 16, 16) for a, b in zip(edges[:-1], edges[1:])]) * n
    chi2 = np.sum((hw - expect) ** 2 / hw2)
    assert stats.chi2.sf(chi2, len(hw)) > 1e-4, (chi2, hw / expect)


def test_dilepton_events(oracle_mod, pdf):
    st = oracle_mod.Settings(process=3, sqrt_s=13600.0, mll_lo=LO, mll_hi=HI)
    r = oracle_mod.run(st, 0, 5000, pdf, hard_only=True, threads=2)
    P = r["p"]
    assert np.all(r["npart"] == 4)
    assert np.all(r["flav"][:, 2] == 11) and np.all(r["flav"][:, 3] == -11)
    assert np.all(r["flav"][:, 0] == -r["flav"][:, 1])
    assert np.abs(P[:, 0] + P[:, 1] - P[:, 2] - P[:, 3]).max() < 1e-9
    pair = P[:, 2] + P[:, 3]
    m = np.sqrt(pair[:, 0] ** 2 - (pair[:, 1:] ** 2).sum(1))
    assert m.min() > LO and m.max() < HI
    for k in (2, 3):  # massless leptons
        mm = P[:, k, 0] ** 2 - (P[:, k, 1:] ** 2).sum(1)
        assert np.abs(mm).max() < 1e-7 * P[:, k, 0].max() ** 2
    assert np.all(r["weight"] > 0)
