"""The trial schemes of the mixed shower (GAPS_TRIALS_REDRAW, KEEP, SELECT and
VETOMAX) give the first accepted emission the same distribution. This is the
reason the GPU kernel may keep losing trials, draw one trial from the summed
rate, or run each channel's own veto algorithm and take the largest accepted
scale (Sec. 2, Fig. 1 and its remarks on veto-max and generate-select).

A toy veto algorithm checks it against closed forms, with no GPU and none of
the library's code. K channels have overestimate rates c_i in ln t below their
own maximum scales T_i and acceptance probabilities a_i(t) <= 1. The first
accepted emission below T0 then has the survival function
    S(t) = exp(-sum_i c_i int_{ln t}^{min(ln T0, ln T_i)} a_i(e^u) du),
and the channel is i with density c_i a_i(t) S(t). Each scheme is sampled in
plain Python. Its scales go through a Kolmogorov-Smirnov test against S, and
its channel fractions are compared with the closed form.
"""
import math

import numpy as np
import pytest
from scipy import integrate, stats

RATES = np.array([0.35, 0.8, 0.15, 0.5])
LN_CAPS = np.array([9.0, 6.5, 8.0, 4.0])  # ln T_i, different per channel
LN_T0, LN_TC = 8.5, 0.0


def accept(i, lt):
    # smooth acceptance probabilities in (0, 1]
    return (0.3 + 0.6 / (1.0 + math.exp(lt - 3.0 - i)), 0.9 * math.exp(-0.05 * lt), 0.5, 0.2 + 0.1 * math.sin(lt))[i]


def rate_integral(lt):
    """sum_i c_i int_{lt}^{min(ln T0, ln T_i)} a_i du"""
    tot = 0.0
    for i in range(len(RATES)):
        hi = min(LN_T0, LN_CAPS[i])
        if hi > lt:
            tot += RATES[i] * integrate.quad(lambda u: accept(i, u), lt, hi)[0]
    return tot


def survival(lt):
    return math.exp(-rate_integral(lt))


def channel_fractions():
    """P(first accepted emission above the cutoff belongs to channel i)."""
    out = []
    for i in range(len(RATES)):
        hi = min(LN_T0, LN_CAPS[i])
        out.append(integrate.quad(lambda u: RATES[i] * accept(i, u) * survival(u), LN_TC, hi, limit=200)[0])
    return np.array(out)


def draw(rng, lnT, i):
    """first point below lnT of channel i's overestimate process (or -inf)"""
    top = min(lnT, LN_CAPS[i])
    return top + math.log(rng.random()) / RATES[i]


def redraw(rng):
    lnT = LN_T0
    while True:
        trials = [draw(rng, lnT, i) for i in range(len(RATES))]
        i = int(np.argmax(trials))
        lnT = trials[i]
        if lnT < LN_TC:
            return None
        if rng.random() < accept(i, lnT):
            return lnT, i


def keep(rng):
    lnT = LN_T0
    trials = [draw(rng, lnT, i) for i in range(len(RATES))]
    while True:
        i = int(np.argmax(trials))
        lnT = trials[i]
        if lnT < LN_TC:
            return None
        if rng.random() < accept(i, lnT):
            return lnT, i
        trials[i] = draw(rng, lnT, i)  # only the vetoed winner draws again


def select(rng):
    lnT = LN_T0
    while lnT > LN_TC:
        active = LN_CAPS >= lnT
        R = RATES[active].sum()
        below = LN_CAPS[~active]
        t1 = below.max() if below.size else -math.inf
        if R > 0.0:
            lt = lnT + math.log(rng.random()) / R
            if lt >= t1:
                idx = np.nonzero(active)[0]
                i = int(idx[np.searchsorted(np.cumsum(RATES[idx]), rng.random() * R, side="right")])
                lnT = lt
                if lnT < LN_TC:
                    return None
                if rng.random() < accept(i, lnT):
                    return lnT, i
                continue
        lnT = t1  # nothing above the next maximum scale: restart there
    return None


def vetomax(rng):
    """each channel runs its own veto algorithm from the starting scale to its
    first accepted point; the largest accepted point wins"""
    best, bi = -math.inf, None
    for i in range(len(RATES)):
        lnT = LN_T0
        while True:
            lnT = draw(rng, lnT, i)
            if lnT < LN_TC:
                break
            if rng.random() < accept(i, lnT):
                if lnT > best:
                    best, bi = lnT, i
                break
    return None if bi is None else (best, bi)


@pytest.mark.parametrize("scheme", [redraw, keep, select, vetomax])
def test_first_emission_distribution(scheme):
    rng = np.random.default_rng(12345)
    n = 20000
    res = [scheme(rng) for _ in range(n)]
    got = [r for r in res if r is not None]
    # fraction with no emission above the cutoff
    p_none = survival(LN_TC)
    k_none = n - len(got)
    assert abs(k_none - n * p_none) < 5 * math.sqrt(n * p_none * (1 - p_none)), (k_none, n * p_none)
    # scale: KS against the conditional CDF of the emission scale
    lts = np.array([r[0] for r in got])

    def cdf(x):
        return (np.vectorize(survival)(x) - p_none) / (1.0 - p_none)
    grid = np.linspace(LN_TC, LN_T0, 400)
    table = cdf(grid)
    p = stats.kstest(lts, lambda x: np.interp(x, grid, table)).pvalue
    assert p > 1e-3, p
    # channel fractions
    frac = channel_fractions()
    counts = np.bincount([r[1] for r in got], minlength=len(RATES))
    expect = frac * n
    chi2 = ((counts - expect) ** 2 / expect).sum()
    assert stats.chi2.sf(chi2, len(RATES) - 1) > 1e-3, (counts, expect)


def test_kept_trials_and_select_draw_fewer_uniforms():
    """The point of the two schemes: fewer draws per accepted emission."""
    class Counting:
        def __init__(self, seed):
            self.rng = np.random.default_rng(seed)
            self.n = 0

        def random(self):
            self.n += 1
            return self.rng.random()
    counts = {}
    for scheme in (redraw, keep, select):
        c = Counting(7)
        for _ in range(3000):
            scheme(c)
        counts[scheme.__name__] = c.n
    assert counts["keep"] < counts["redraw"] and counts["select"] < counts["redraw"], counts


def test_vetomax_evaluates_every_channel():
    """Veto-max evaluates the acceptance of every channel's trials down to its
    first accepted point (or the cutoff), max-veto only the winners'."""
    def count_accepts(scheme, seed):
        calls = [0]
        global accept
        orig = accept

        def counted(i, lt):
            calls[0] += 1
            return orig(i, lt)
        accept = counted
        try:
            rng = np.random.default_rng(seed)
            for _ in range(2000):
                scheme(rng)
        finally:
            accept = orig
        return calls[0]
    assert count_accepts(vetomax, 3) > 1.5 * count_accepts(keep, 3)
