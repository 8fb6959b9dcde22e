"""Pins of the heavy-quark measure correction (App. A.2) in the oracle, with
the thresholded synthetic table (c and b densities that vanish at their
masses, on Q^2 nodes of the grid).

The correction draws an incoming c or b's q <- q and q <- g trials in
dt/(t - m^2) and multiplies the PDF ratio by (t - m^2)/t. The product is the
plain density dt/t x ratio, so the first emission of such an end must follow
the plain Sudakov form factor (App. A.1), down to the floor where the
corrected trials end (m^2 (1 + 1e-3), a reading: the paper is silent). The
reference integrates the plain density by quadrature in u = ln(t - m^2),
independent of the oracle's trials, bounds and measure.
"""
import math

import numpy as np
import pytest
from scipy import integrate, stats

from tests import sudakov_ref as R

SQRT_S = 13600.0
FLOOR = 1e-3


@pytest.fixture(scope="module")
def hq_pdf():
    from paper_2511_19633_gb300 import inputs
    return inputs.synthetic_pdf_grid(thresholds=True)


def _m2(node):
    from paper_2511_19633_gb300 import inputs
    return float(inputs.q2_nodes()[node])


def test_thresholded_table_vanishes_at_the_mass(oracle_mod, hq_pdf):
    """The interpolated c and b densities are zero at and below their masses
    and equal the closed form sea(x) (1 - m^2/Q^2) on the nodes above."""
    from paper_2511_19633_gb300 import inputs
    q2 = inputs.q2_nodes()
    x = inputs.x_nodes()[40]
    for f, node in ((4, 3), (5, 9), (9, 3), (10, 9)):
        m2 = q2[node]
        for q in (0.6, 0.9 * m2):
            assert oracle_mod.pdf_xf(hq_pdf, f, x, q) == 0.0
        # at the mass itself: zero up to the rounding of ln Q^2
        assert abs(oracle_mod.pdf_xf(hq_pdf, f, x, m2)) < 1e-12 * oracle_mod.pdf_xf(hq_pdf, f, x, q2[node + 1])
        for k in (node + 1, node + 5, 49):
            expect = inputs.synthetic_xf("sea", np.array([x]))[0] * (1.0 - m2 / q2[k])
            assert oracle_mod.pdf_xf(hq_pdf, f, x, q2[k]) == pytest.approx(expect, rel=2e-7)
        # just above the mass the density rises linearly in ln Q^2
        t = m2 * math.exp(0.1 * (math.log(q2[node + 1]) - math.log(m2)))
        assert 0.0 < oracle_mod.pdf_xf(hq_pdf, f, x, t) < oracle_mod.pdf_xf(hq_pdf, f, x, q2[node + 1])


@pytest.mark.parametrize("num,den", [(0, 4), (4, 4), (0, 5), (5, 5), (11, 0)])
def test_heavy_bound_holds_on_a_dense_grid(oracle_mod, hq_pdf, num, den):
    """The certified bound of the corrected ratio (t - m^2)/t x f_num(x', t) /
    f_den(eta, t) (for a heavy denominator; the plain ratio otherwise) holds
    for every x' >= eta and t above the mass, checked by brute force."""
    m2 = {4: _m2(3), 5: _m2(9)}.get(den, 0.0)
    lo = max(0.5, m2 * (1 + 1e-9))
    ts = np.exp(np.linspace(math.log(lo), math.log(1e5), 400))
    for eta in (3e-5, 1e-3, 0.04, 0.3, 0.77):
        B = oracle_mod.pdf_bound(hq_pdf, num, den, eta)
        assert B > 0.0
        xs = np.exp(np.linspace(math.log(eta), math.log(0.999999), 60))
        for t in ts:
            f0 = oracle_mod.pdf_xf(hq_pdf, den, eta, t)
            if f0 <= 0.0:
                continue
            f1 = oracle_mod.pdf_xf_batch(hq_pdf, num, xs, np.full_like(xs, t))
            corr = (t - m2) / t if m2 > 0 else 1.0
            assert np.all(corr * f1 / f0 <= B * (1 + 1e-12)), (eta, t)


class HeavyEnd(R.End):
    """A heavy-quark IF end whose density is integrated from the floor of the
    corrected trials, in u = ln(t - m^2) (the density is steep at the mass)."""

    def __init__(self, *a, m2=0.0, **k):
        super().__init__(*a, **k)
        self.m2 = m2

    def exponent(self, t_lo, t_hi):
        tk = R.t_limit(self.kind, self.s, self.eta)
        lo, hi = max(t_lo, self.m2 * (1 + FLOOR)), min(t_hi, tk)
        if hi <= lo:
            return 0.0
        m2 = self.m2

        def f(u):
            t = m2 + math.exp(u)
            return self.z_integral(t) * math.exp(u) / t  # dt/t = e^u du / t
        val, _ = integrate.quad(f, math.log(lo - m2), math.log(hi - m2), limit=200, epsabs=1e-9,
                                epsrel=1e-7)
        return self.mult * val


@pytest.mark.parametrize("flq,eta", [(4, 0.05), (-4, 0.01), (5, 0.03)])
def test_heavy_quark_first_emission_follows_the_plain_sudakov(oracle_mod, hq_pdf, flq, eta):
    """IF dipole of an incoming c, cbar or b and a final quark of the same
    flavour, channels q <- q and q <- g, cutoff 1 GeV^2 below the mass: the
    oracle's corrected trials against the plain density's quadrature."""
    s, tc = 3000.0, 1.0
    m2 = _m2(3) if abs(flq) == 4 else _m2(9)
    st = oracle_mod.Settings(process=1, sqrt_s=SQRT_S, t_cut=tc, channel_mask=(1 << 3) | (1 << 4), seed=11)
    n = 30000
    tf = oracle_mod.first_emission(st, hq_pdf, 1, flq, s, eta, n)
    fq = abs(flq) if flq > 0 else 5 + abs(flq)
    P = lambda f, x, t: oracle_mod.pdf_xf_batch(hq_pdf, f, x, t)
    ends = [HeavyEnd("IF", "qg", s, eta=eta, fq=fq, pdf=P, m2=m2), HeavyEnd("IF", "gq", s, eta=eta, fq=fq, pdf=P, m2=m2)]
    tmax = min(R.t_limit("IF", s, eta), SQRT_S ** 2)
    # bins uniform in ln(t - m^2) from the floor
    lo = m2 * (1 + FLOOR)
    edges = m2 + np.exp(np.linspace(math.log(lo - m2), math.log(tmax - m2), 11))
    pb, p0_ref = R.first_emission_bins(ends, edges, SQRT_S ** 2)
    p0_mc = float(np.mean(tf == 0.0))
    sig = math.sqrt(max(p0_ref * (1 - p0_ref), 1e-12) / n)
    assert abs(p0_mc - p0_ref) < 4.5 * sig + 1e-9, (p0_mc, p0_ref, sig)
    em = tf[tf > 0]
    assert em.size > 1000 and em.min() > lo * (1 - 1e-12)
    counts, _ = np.histogram(em, bins=edges)
    exp = pb * n
    keep = exp > 5
    chi2 = float(np.sum((counts[keep] - exp[keep]) ** 2 / exp[keep]))
    assert stats.chi2.sf(chi2, int(keep.sum())) > 1e-4, (chi2, counts, exp)


def test_heavy_quarks_convert_in_nlo_events(oracle_mod, hq_pdf):
    """NLO pp -> Z with the thresholded table: every event ends, no acceptance
    weight exceeds one, and most incoming c and b quarks of the hard process
    have turned into gluons by the end of the shower."""
    st = oracle_mod.Settings(process=2, sqrt_s=SQRT_S, nmax=128)
    n = 20000
    hard = oracle_mod.run(st, 0, n, hq_pdf, hard_only=True, threads=4)
    r = oracle_mod.run(st, 0, n, hq_pdf, threads=4)
    assert np.all(r["status"] == 1)
    assert int(r["counters"][:, 5].sum()) == 0  # violations
    heavy0 = np.isin(np.abs(hard["flav"][:, :2]), [4, 5]).sum()
    heavy1 = np.isin(np.abs(r["flav"][:, :2]), [4, 5]).sum()
    assert heavy0 > 1000 and heavy1 < 0.5 * heavy0, (heavy0, heavy1)
