"""Pins of the oracle's veto algorithm against the paper's Sudakov form factors.

For an isolated colour dipole the probability of no emission between the
starting scale and the cutoff, and the distribution of the first emission
scale, follow from the Sudakov form factors of Appendix A.1 / B.2-B.5. The
reference values come from quadrature of those formulas (sudakov_ref.py),
independent of the oracle's overestimates, trial sampling and PDF-ratio
bounds; a dropped Jacobian, a wrong z limit, kernel or PDF ratio fails them.
"""
import math

import numpy as np
import pytest
from scipy import stats

from tests import sudakov_ref as R

N_EVENTS = 30000
SQRT_S = 13600.0


def run_case(oracle_mod, pdf, dipole, flq, s, eta, mask, t_c, process=1, fixed_alpha=False,
             seed=7):
    st = oracle_mod.Settings(process=process, sqrt_s=SQRT_S, t_cut=t_c, channel_mask=mask,
                             fixed_alpha=fixed_alpha, seed=seed)
    return st, oracle_mod.first_emission(st, pdf, dipole, flq, s, eta, N_EVENTS)


def check(tfirst, ends, t_c, t_start, nbins=8):
    tmax = max(R.t_limit(e.kind, e.s, e.eta) for e in ends)
    tmax = min(tmax, t_start)
    edges = np.exp(np.linspace(math.log(t_c), math.log(tmax), nbins + 1))
    pb, p0_ref = R.first_emission_bins(ends, edges, t_start)
    p0_mc = float(np.mean(tfirst == 0.0))
    sig = math.sqrt(p0_ref * (1 - p0_ref) / len(tfirst))
    assert abs(p0_mc - p0_ref) < 4.5 * sig, (p0_mc, p0_ref, sig)
    em = tfirst[tfirst > 0]
    assert em.min() >= t_c and em.max() <= tmax * (1 + 1e-12)
    counts, _ = np.histogram(em, bins=edges)
    exp = pb * len(tfirst)
    keep = exp > 5
    chi2 = float(np.sum((counts[keep] - exp[keep]) ** 2 / exp[keep]))
    ndf = int(keep.sum())
    pval = stats.chi2.sf(chi2, ndf)
    assert pval > 1e-4, (chi2, ndf, counts, exp)
    return p0_mc, p0_ref, chi2 / max(ndf, 1)


def pdf_fn(oracle_mod, pdf):
    return lambda f, x, t: oracle_mod.pdf_xf_batch(pdf, f, x, t)


def test_ff_quark_fixed_coupling(oracle_mod, pdf):
    """FF q -> qg, fixed alpha_s: both ends of a q qbar dipole (paper's P1)."""
    s, tc = 91.2 ** 2, 5.0
    st, tf = run_case(oracle_mod, None, 0, 1, s, 0.0, 1 << 0, tc, process=0, fixed_alpha=True)
    fixed = lambda t: 0.118
    ends = [R.End("FF", "qg", s, alpha=fixed, mult=2)]
    check(tf, ends, tc, SQRT_S ** 2)


def test_ff_quark_running(oracle_mod, pdf):
    s, tc = 91.2 ** 2, 5.0
    st, tf = run_case(oracle_mod, None, 0, 2, s, 0.0, 1 << 0, tc, process=0)
    ends = [R.End("FF", "qg", s, mult=2)]
    check(tf, ends, tc, SQRT_S ** 2)


def test_ff_gluons(oracle_mod, pdf):
    """g g colour singlet: four dipole ends, each with g->gg and g->q qbar."""
    s, tc = 60.0 ** 2, 9.0
    st, tf = run_case(oracle_mod, None, 0, 21, s, 0.0, (1 << 1) | (1 << 2), tc, process=0)
    ends = [R.End("FF", "gg", s, mult=4), R.End("FF", "qq", s, mult=4)]
    check(tf, ends, tc, SQRT_S ** 2)


@pytest.mark.parametrize("flq,eta", [(2, 0.05), (-1, 0.2)])
def test_fi_quark(oracle_mod, pdf, flq, eta):
    """FI: final quark radiating against an incoming quark (spectator PDF ratio)."""
    s, tc = 3000.0, 4.0
    st, tf = run_case(oracle_mod, pdf, 1, flq, s, eta, 1 << 0, tc)
    fs = flq if flq > 0 else 5 - flq
    ends = [R.End("FI", "qg", s, eta=eta, fspec=fs, pdf=pdf_fn(oracle_mod, pdf))]
    check(tf, ends, tc, SQRT_S ** 2)


@pytest.mark.parametrize("flq,eta", [(2, 0.05), (1, 0.3), (-2, 0.02)])
def test_if_quark(oracle_mod, pdf, flq, eta):
    """IF: incoming quark radiating (q->qg and q->g qbar) against a final quark."""
    s, tc = 3000.0, 4.0
    st, tf = run_case(oracle_mod, pdf, 1, flq, s, eta, (1 << 3) | (1 << 4), tc)
    fq = flq if flq > 0 else 5 - flq
    P = pdf_fn(oracle_mod, pdf)
    ends = [R.End("IF", "qg", s, eta=eta, fq=fq, pdf=P), R.End("IF", "gq", s, eta=eta, fq=fq, pdf=P)]
    check(tf, ends, tc, SQRT_S ** 2)


def test_fi_if_gluons(oracle_mod, pdf):
    """final gluon + incoming gluon (two colour lines): FI g->gg, g->qqbar with the
    gluon spectator ratio, and IF g->gg, g->qq with the summed quark ratio."""
    s, tc, eta = 2000.0, 4.0, 0.08
    P = pdf_fn(oracle_mod, pdf)
    st, tf = run_case(oracle_mod, pdf, 1, 21, s, eta, (1 << 1) | (1 << 2), tc)
    ends = [R.End("FI", "gg", s, eta=eta, fspec=0, pdf=P, mult=2),
            R.End("FI", "qq", s, eta=eta, fspec=0, pdf=P, mult=2)]
    check(tf, ends, tc, SQRT_S ** 2)
    st, tf = run_case(oracle_mod, pdf, 1, 21, s, eta, (1 << 5) | (1 << 6), tc)
    ends = [R.End("IF", "gg", s, eta=eta, pdf=P, mult=2), R.End("IF", "qq", s, eta=eta, pdf=P, mult=2)]
    check(tf, ends, tc, SQRT_S ** 2)


@pytest.mark.parametrize("flq,eta_a", [(2, 0.02), (1, 0.0067)])
def test_ii_quarks(oracle_mod, pdf, flq, eta_a):
    """II: q (beam 1) qbar (beam 2) at s = m_Z^2; both legs, q->qg and q->g qbar."""
    s, tc = R.MZ ** 2, 4.0
    eta_b = s / (eta_a * SQRT_S ** 2)
    P = pdf_fn(oracle_mod, pdf)
    st, tf = run_case(oracle_mod, pdf, 2, flq, s, eta_a, (1 << 3) | (1 << 4), tc)
    fa = flq
    fb = 5 + flq  # antiquark of the same flavour
    ends = [R.End("II", "qg", s, eta=eta_a, fq=fa, pdf=P), R.End("II", "gq", s, eta=eta_a, fq=fa, pdf=P),
            R.End("II", "qg", s, eta=eta_b, fq=fb, pdf=P), R.End("II", "gq", s, eta=eta_b, fq=fb, pdf=P)]
    check(tf, ends, tc, SQRT_S ** 2)


def test_ii_gluons(oracle_mod, pdf):
    s, tc, eta_a = 200.0 ** 2, 4.0, 0.03
    eta_b = s / (eta_a * SQRT_S ** 2)
    P = pdf_fn(oracle_mod, pdf)
    st, tf = run_case(oracle_mod, pdf, 2, 21, s, eta_a, (1 << 5) | (1 << 6), tc)
    ends = []
    for eta in (eta_a, eta_b):
        ends += [R.End("II", "gg", s, eta=eta, pdf=P, mult=2), R.End("II", "qq", s, eta=eta, pdf=P, mult=2)]
    check(tf, ends, tc, SQRT_S ** 2)
