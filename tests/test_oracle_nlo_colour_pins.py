"""Pins of oracle pieces that the other tests reach only through the oracle
itself: the collinear functions h^qq and h^qg of the NLO S events (App. C.3),
the flavour choices of the g -> q qbar and g <- q splittings, and the colour
flow after one emission (App. B, leading colour).

The references here are written from the paper's operators and from the
leading-colour rule, not from the oracle's own formulas:
  - K-bar, K-tilde and P of App. C.3 are restated term by term, each split
    into its plus-distribution, regular and delta(1-x) parts; h is the sum of
    the regular parts and g of the plus parts. Integrals are done by sympy.
  - The S-event weight is checked against the K + P distributions acting on
    the PDF-ratio test function, with the plus prescription applied by its
    definition (no A, B, g or h of the oracle enters).
  - The initial-state g <- q flavour is drawn in proportion to the parent
    density at eta / x; the final-state g -> q qbar flavour uniformly.
  - After one emission the colour tags form the planar chain or loop that
    leading colour prescribes, whatever the tag values.
"""
import math

import numpy as np
import pytest
from scipy import integrate, stats

CF, TR = 4.0 / 3.0, 0.5
AS = 0.118
MZ = 91.1876


# --------------------------------------------------------------------------
# App. C.3: the K and P operators for an incoming quark, term by term.
# Each returns (plus-part coefficient G(x), regular part R(x), delta coefficient D)
# without the prefactor C alpha_s / 2 pi.
# --------------------------------------------------------------------------
def Kbar_qq(x):
    l = math.log((1 - x) / x)
    return 2 / (1 - x) * l, -(1 + x) * l + (1 - x), -(5 - math.pi ** 2)


def Ktilde_qq(x):
    l = math.log(1 - x)
    return 2 / (1 - x) * l, -(1 + x) * l, -math.pi ** 2 / 3


def P_qq(x, L):
    return -L * 2 / (1 - x), L * (1 + x), -L * 1.5


def Kbar_gq(x):
    return 0.0, (x * x + (1 - x) ** 2) * math.log((1 - x) / x) + 2 * x * (1 - x), 0.0


def Ktilde_gq(x):
    return 0.0, (x * x + (1 - x) ** 2) * math.log(1 - x), 0.0


def P_gq(x, L):
    return 0.0, -L * (x * x + (1 - x) ** 2), 0.0


def parts_qq(x, L):
    terms = (Kbar_qq(x), Ktilde_qq(x), P_qq(x, L))
    return tuple(sum(t[k] for t in terms) for k in range(3))


def parts_gq(x, L):
    terms = (Kbar_gq(x), Ktilde_gq(x), P_gq(x, L))
    return tuple(sum(t[k] for t in terms) for k in range(3))


@pytest.mark.parametrize("L", [0.0, 0.7, -1.3])
def test_h_and_g_are_the_regular_and_plus_parts_of_K_plus_P(oracle_mod, L):
    pre_f, pre_t = CF * AS / (2 * math.pi), TR * AS / (2 * math.pi)
    for x in (1e-5, 0.003, 0.1, 0.37, 0.5, 0.77, 0.99, 1 - 1e-7):
        G, R, _ = parts_qq(x, L)
        assert oracle_mod.collinear(AS, L, "hqq", x) == pytest.approx(pre_f * R, rel=1e-12, abs=1e-15)
        assert oracle_mod.collinear(AS, L, "g", x) == pytest.approx(pre_f * G, rel=1e-12, abs=1e-15)
        _, Rg, _ = parts_gq(x, L)
        assert oracle_mod.collinear(AS, L, "hqg", x) == pytest.approx(pre_t * Rg, rel=1e-12, abs=1e-15)
    # A collects the delta(1-x) coefficients
    assert oracle_mod.collinear(AS, L, "A") == pytest.approx(pre_f * parts_qq(0.5, L)[2], rel=1e-13)


def test_h_moments_against_closed_forms(oracle_mod):
    """int_0^1 x^k h(x) dx, k = 0, 1, 2, from the operators' regular parts
    integrated symbolically (sympy), against quadrature of the oracle's h."""
    sp = pytest.importorskip("sympy")
    x, L = sp.symbols("x L", positive=True)
    lq = sp.log((1 - x) / x)
    l1 = sp.log(1 - x)
    reg_qq = (-(1 + x) * lq + (1 - x)) + (-(1 + x) * l1) + L * (1 + x)
    pgq = x ** 2 + (1 - x) ** 2
    reg_gq = (pgq * lq + 2 * x * (1 - x)) + pgq * l1 - L * pgq
    pre_f, pre_t = CF * AS / (2 * math.pi), TR * AS / (2 * math.pi)
    for k in range(3):
        cq = sp.integrate(sp.expand(x ** k * reg_qq), (x, 0, 1))
        cg = sp.integrate(sp.expand(x ** k * reg_gq), (x, 0, 1))
        for Lv in (0.0, 0.9):
            eq = float(cq.subs(L, Lv)) * pre_f
            eg = float(cg.subs(L, Lv)) * pre_t
            vq, _ = integrate.quad(lambda t: t ** k * oracle_mod.collinear(AS, Lv, "hqq", t), 0, 1,
                                   limit=400, epsabs=1e-14, epsrel=1e-12)
            vg, _ = integrate.quad(lambda t: t ** k * oracle_mod.collinear(AS, Lv, "hqg", t), 0, 1,
                                   limit=400, epsabs=1e-14, epsrel=1e-12)
            assert vq == pytest.approx(eq, rel=1e-9, abs=1e-13), (k, Lv)
            assert vg == pytest.approx(eg, rel=1e-9, abs=1e-13), (k, Lv)
    # the k = 0 values written out: 11/4 + 3L/2 and -7/18 - 2L/3
    assert sp.nsimplify(sp.integrate(sp.expand(reg_qq), (x, 0, 1)) - (sp.Rational(11, 4) + 3 * L / 2)) == 0
    assert sp.nsimplify(sp.integrate(sp.expand(reg_gq), (x, 0, 1)) - (-sp.Rational(7, 18) - 2 * L / 3)) == 0


def _xf(pdf, f, x):
    """x f(x) of the Q^2-independent synthetic table, bilinear in ln x (the
    table's own interpolation rule, restated here)."""
    lx0, lx1 = math.log(1e-6), math.log(1 - 1e-6)
    x = np.asarray(x, dtype=np.float64)
    u = (np.log(x) - lx0) / ((lx1 - lx0) / 99)
    ix = np.clip(np.floor(u).astype(int), 0, 98)
    fx = u - ix
    col = pdf[f, :, 0].astype(np.float64)
    v = (1 - fx) * col[ix] + fx * col[ix + 1]
    return np.where((x >= 1e-6) & (x <= 1 - 1e-6), v, 0.0)


def _leg_from_operators(pdf, fq, eta):
    """int_0^1 dx [K + P](x) phi(x), phi(x) = ratio of the parent density at
    eta/x to the Born density at eta (zero below x = eta), for a quark leg of
    table index fq: the qq operators act on the quark ratio, the gq ones on
    the gluon ratio. The plus prescription by its definition:
    int G_+ phi = int_0^1 G(x) (phi(x) - phi(1)) dx, phi(1) = 1."""
    F0 = float(_xf(pdf, fq, eta))
    pre_f, pre_t = CF * AS / (2 * math.pi), TR * AS / (2 * math.pi)

    def rq(x):
        return float(_xf(pdf, fq, eta / x)) / F0 if x > eta else 0.0

    def rg(x):
        return float(_xf(pdf, 0, eta / x)) / F0 if x > eta else 0.0

    def plus_and_regular(x):
        G, R, _ = parts_qq(x, 0.0)
        _, Rg, _ = parts_gq(x, 0.0)
        return pre_f * (G * (rq(x) - 1.0) + R * rq(x)) + pre_t * Rg * rg(x)

    below, _ = integrate.quad(lambda x: pre_f * parts_qq(x, 0.0)[0] * (-1.0), 0, eta, limit=400,
                              epsabs=1e-13, epsrel=1e-11)
    above, _ = integrate.quad(plus_and_regular, eta, 1, limit=400, epsrel=1e-10)
    delta = pre_f * parts_qq(0.5, 0.0)[2]
    return below + above + delta


def test_s_event_weight_against_the_operators(oracle_mod, pdf):
    """Mean weight of S events at fixed rapidity and flavour pair against
    B (1 + C_F as/2pi * 2) + B sum over both legs of the K + P distributions
    acting on the PDF ratio (App. C.3, reading: kappa_C without a second
    coupling prefactor)."""
    sqrt_s, y, pair = 13600.0, 0.6, 1  # pair 1 = (u from beam 1, ubar from beam 2)
    st_s = oracle_mod.Settings(process=2, sqrt_s=sqrt_s, p_s=1.0, y_fixed=y, pair_fixed=pair)
    st_b = oracle_mod.Settings(process=1, sqrt_s=sqrt_s, y_fixed=y, pair_fixed=pair)
    n = 200_000
    ws = oracle_mod.run(st_s, 0, n, pdf, hard_only=True, threads=4)["weight"]
    wb = oracle_mod.run(st_b, 0, 4, pdf, hard_only=True)["weight"][0]
    ea, eb = math.exp(y) * MZ / sqrt_s, math.exp(-y) * MZ / sqrt_s
    expect = wb * (1 + CF * AS / (2 * math.pi) * 2 + _leg_from_operators(pdf, 2, ea)
                   + _leg_from_operators(pdf, 7, eb))
    assert ws.mean() == pytest.approx(expect, rel=5 * ws.std() / math.sqrt(n) / expect)


# --------------------------------------------------------------------------
# flavour choices
# --------------------------------------------------------------------------
QUARKS = [1, 2, 3, 4, 5, -1, -2, -3, -4, -5]


def _table_index(fl):
    return fl if fl > 0 else 5 - fl


@pytest.mark.parametrize("dipole", [1, 2])
def test_initial_gluon_from_quark_flavour_follows_parent_density(oracle_mod, pdf, dipole):
    """g <- q (channel 6): an incoming gluon at eta came from a quark of
    flavour q at eta/x, drawn in proportion to x f_q(eta/x) among the ten
    quark and antiquark flavours; the emitted final parton has the same
    flavour (Appendix B.4, B.5)."""
    st = oracle_mod.Settings(process=1, sqrt_s=13600.0, channel_mask=1 << 6, nmax=8)
    r = oracle_mod.first_emission_record(st, pdf, dipole, 21, 1e4, 0.05, 40000)
    em = r["t"] > 0
    assert em.sum() > 10000
    fl0 = r["flav"][em, 0] if dipole == 1 else None
    if dipole == 2:
        # either incoming gluon may have converted
        conv = np.where(r["flav"][em, 0] != 21, 0, 1)
        fl0 = r["flav"][em][np.arange(em.sum()), conv]
        eta_new = r["eta"][em][np.arange(em.sum()), conv]
    else:
        eta_new = r["eta"][em, 0]
    assert np.all(r["flav"][em, 2] == fl0)   # the emitted parton keeps the flavour
    dens = np.stack([_xf(pdf, _table_index(q), eta_new) for q in QUARKS])  # [10][events]
    prob = dens / dens.sum(0)
    expected = prob.sum(1)
    observed = np.array([(fl0 == q).sum() for q in QUARKS])
    chi2 = np.sum((observed - expected) ** 2 / expected)
    assert stats.chi2.sf(chi2, len(QUARKS) - 1) > 1e-4, (observed, expected)
    # the same test against the density at eta itself (a plausible mistake) fails
    wrong = np.stack([_xf(pdf, _table_index(q), np.full(em.sum(), 0.05)) for q in QUARKS])
    we = (wrong / wrong.sum(0)).sum(1)
    assert stats.chi2.sf(np.sum((observed - we) ** 2 / we), len(QUARKS) - 1) < 1e-6


def test_final_gluon_splitting_flavour_is_uniform(oracle_mod):
    """g -> q qbar in the final state (channel 2): flavour uniform among the
    n_f = 5 light flavours, a quark and its antiquark."""
    st = oracle_mod.Settings(process=0, sqrt_s=91.2, channel_mask=1 << 2, nmax=8)
    r = oracle_mod.first_emission_record(st, None, 0, 21, 91.2 ** 2, 0.0, 20000)
    em = r["t"] > 0
    fl = r["flav"][em]
    q = np.abs(fl[fl != 21])
    assert q.size == 2 * em.sum()
    pairs = np.sort(fl[fl != 21].reshape(-1, 2), axis=1)
    assert np.all(pairs[:, 0] == -pairs[:, 1])
    counts = np.bincount(pairs[:, 1], minlength=6)[1:]
    assert stats.chisquare(counts).pvalue > 1e-4, counts


# --------------------------------------------------------------------------
# colour flow after one emission (leading colour, all-outgoing view: an
# incoming quark counts as an outgoing antiquark and vice versa)
# --------------------------------------------------------------------------
def _check_topology(fl, col, acol, initial, kind):
    tags = [t for t in list(col) + list(acol) if t != 0]
    # every colour line joins exactly two partons
    for t in set(tags):
        assert list(col).count(t) == 1 and list(acol).count(t) == 1, (col, acol)
    # the tags a parton holds match what it is in the all-outgoing view
    for f, c, a, ini in zip(fl, col, acol, initial):
        quark_like = (f > 0) != bool(ini) if f != 21 else None
        if f == 21:
            assert c != 0 and a != 0
        elif quark_like:
            assert c != 0 and a == 0
        else:
            assert c == 0 and a != 0
    edges = {(i, k) for i in range(3) for k in range(3) if i != k and col[i] != 0 and col[i] == acol[k]}
    if kind == "loop":
        assert len(edges) == 3 and all(f == 21 for f in fl)
        # one directed 3-cycle
        nxt = {i: k for i, k in edges}
        assert len(nxt) == 3 and nxt[nxt[nxt[0]]] == 0 and nxt[0] != 0
    else:
        assert len(edges) == 2
        g = [i for i in range(3) if fl[i] == 21]
        assert len(g) == 1
        q = [i for i in range(3) if col[i] != 0 and acol[i] == 0][0]
        a = [i for i in range(3) if acol[i] != 0 and col[i] == 0][0]
        assert edges == {(q, g[0]), (g[0], a)}


CASES = [
    # (dipole, flq, channel, topology, which slot is the gluon of a chain)
    (0, 1, 0, "chain", 2),     # FF q -> q g
    (0, 21, 1, "loop", None),  # FF g -> g g
    (0, 21, 2, "chain", None),  # FF g -> q qbar
    (1, 1, 0, "chain", 2),     # FI: final quark emits
    (1, 1, 3, "chain", 2),     # IF q <- q, final gluon
    (1, 1, 4, "chain", 0),     # IF g <- q: the incoming parton becomes a gluon
    (1, 21, 5, "loop", None),  # IF g <- g
    (1, 21, 6, "chain", 1),    # IF q <- g: the final gluon is the chain's gluon
    (1, 21, 1, "loop", None),  # FI: final gluon emits a gluon
    (2, 1, 3, "chain", 2),     # II q <- q
    (2, 1, 4, "chain", None),  # II g <- q
    (2, 21, 5, "loop", None),  # II g <- g
    (2, 21, 6, "chain", None),  # II q <- g
]


@pytest.mark.parametrize("dipole,flq,channel,kind,gslot", CASES)
def test_colour_flow_after_one_emission(oracle_mod, pdf, dipole, flq, channel, kind, gslot):
    pp = dipole != 0
    st = oracle_mod.Settings(process=1 if pp else 0, sqrt_s=13600.0 if pp else 91.2,
                             channel_mask=1 << channel, nmax=8)
    r = oracle_mod.first_emission_record(st, pdf if pp else None, dipole, flq,
                                         1e4 if pp else 91.2 ** 2, 0.05, 400)
    em = np.nonzero(r["t"] > 0)[0]
    assert em.size > 50
    for e in em:
        fl, col, acol, ini = r["flav"][e], r["col"][e], r["acol"][e], r["initial"][e]
        _check_topology(fl, col, acol, ini, kind)
        if gslot is not None:
            assert fl[gslot] == 21
        # flavour bookkeeping of the channel
        if channel in (0, 1, 3, 5):
            assert fl[2] == 21
        if channel == 4:
            conv = [s for s in (0, 1) if ini[s] and fl[s] == 21 and r["flav"][e][s] == 21]
            assert fl[2] != 21 and conv
        if channel == 6:
            assert fl[2] != 21 and (fl[0] == fl[2] or fl[1] == fl[2])
