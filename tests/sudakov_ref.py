"""No-emission probabilities of a single colour dipole computed by quadrature of
the paper's Sudakov form factors (Appendix A.1 and B.2-B.5):

  Delta = exp( - int dt/t int_{z-}^{z+} dz alpha_s(t)/(2 pi) J P f(eta/x)/f(eta) )

with the kernels P, Jacobians J, variable maps and z limits as printed for
FF, FI, IF and II dipoles. Independent of the oracle's veto algorithm
(trial sampling, overestimates, PDF-ratio bounds); the interpolated PDF is
the oracle's own (pinned separately against the closed form).
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate

CF, CA, TR = 4.0 / 3.0, 3.0, 0.5
MZ = 91.1876

_GL_X, _GL_W = np.polynomial.legendre.leggauss(64)


def alpha_s(t, as0=0.118, nf=5):
    beta0 = (33.0 - 2.0 * nf) / (12.0 * math.pi)
    return as0 / (1.0 + as0 * beta0 * math.log(t / (MZ * MZ)))


def z_range(kind, t, s, eta):
    """Paper's z+- (naive form, fine at the moderate t/s used here)."""
    if kind == "FF":
        d = 1.0 - 4.0 * t / s
        if d <= 0:
            return None
        return 0.5 * (1 - math.sqrt(d)), 0.5 * (1 + math.sqrt(d))
    if kind == "FI":
        d = 1.0 - 4.0 * t / s * eta / (1.0 - eta)
        if d <= 0:
            return None
        return 0.5 * (1 - math.sqrt(d)), 0.5 * (1 + math.sqrt(d))
    if kind == "IF":
        d = 1.0 - 4.0 * t * eta / (s * (1.0 - eta))
    else:
        d = 1.0 - 4.0 * t * eta / (s * (1.0 - eta) ** 2)
    if d <= 0:
        return None
    return 0.5 * ((1 + eta) - (1 - eta) * math.sqrt(d)), 0.5 * ((1 + eta) + (1 - eta) * math.sqrt(d))


def t_limit(kind, s, eta):
    if kind == "FF":
        return s / 4.0
    if kind in ("FI", "IF"):
        return s / 4.0 * (1.0 - eta) / eta
    return s / 4.0 * (1.0 - eta) ** 2 / eta


class End:
    """One radiating dipole end: kind FF/FI/IF/II, channel name, invariant s,
    momentum fraction eta (spectator's for FI, emitter's for IF/II) and the PDF
    table indices used in the ratio."""

    def __init__(self, kind, channel, s, eta=0.0, fq=None, fspec=None, pdf=None, nf=5,
                 alpha=alpha_s, mult=1):
        self.kind, self.ch, self.s, self.eta = kind, channel, s, eta
        self.fq, self.fspec, self.pdf, self.nf, self.alpha = fq, fspec, pdf, nf, alpha
        self.mult = mult  # number of identical dipole ends this object stands for

    def F(self, f, x, t):
        """x f(x, t) for table index f (11 = sum of the ten quark densities)."""
        if f == 11:
            return sum(self.pdf(k, x, t) for k in range(1, 11))
        return self.pdf(f, x, t)

    def integrand(self, t, z):
        """kernel x Jacobian x PDF ratio at scale t for an array of z."""
        kind, ch, s, eta = self.kind, self.ch, self.s, self.eta
        z = np.asarray(z, dtype=np.float64)
        out = np.zeros_like(z)
        if kind == "FF":
            y = t / (z * (1 - z) * s)
            ok = (y > 0) & (y < 1)
            den = 1 - z * (1 - y)
            if ch == "qg":
                k = CF * (2 / den - (1 + z))
            elif ch == "gg":
                k = CA / 2 * (2 / den - 2 + z * (1 - z))
            else:
                k = self.nf * TR / 2 * (1 - 2 * z * (1 - z))
            return np.where(ok, np.maximum(k, 0.0) * (1 - y), 0.0)
        if kind == "FI":
            rho = t / (z * (1 - z) * s)
            x = 1 / (1 + rho)
            den = 1 - z + (1 - x)
            if ch == "qg":
                k = CF * (2 / den - (1 + z))
            elif ch == "gg":
                k = CA / 2 * (2 / den - 2 + z * (1 - z))
            else:
                k = self.nf * TR / 2 * (1 - 2 * z * (1 - z))
            f0 = self.F(self.fspec, np.full_like(z, eta), t)
            f1 = self.F(self.fspec, eta / x, t)
            pdfr = x * f1 / f0  # f(eta/x)/f(eta) with F = x f
            return np.maximum(k, 0.0) * pdfr
        r = t / s
        if kind == "IF":
            q = 1 - z + r
            x = q / (2 * r) * (1 - np.sqrt(np.maximum(0.0, 1 - 4 * r * z * (1 - z) / q ** 2)))
            u = x * r / (1 - z)
            J = 1.0 / (u + x - 2 * u * x)
            soft = 1 - x + u
        else:
            x = z * (1 - z) / (1 - z + r)
            J = 1.0 / z
            soft = 1 - x
        ok = (x > eta) & (x < 1)
        x = np.where(ok, x, 0.5)
        if ch == "qg":
            k = CF * (2 / soft - (1 + x)); num, den = self.fq, self.fq
        elif ch == "gq":
            k = TR * (1 - 2 * x * (1 - x)); num, den = 0, self.fq
        elif ch == "gg":
            k = CA * (1 / soft + (1 - x) / x - 1 + x * (1 - x)); num, den = 0, 0
        else:
            k = CF / 2 * (x + 2 * (1 - x) / x); num, den = 11, 0
        f0 = self.F(den, np.full_like(z, eta), t)
        f1 = self.F(num, eta / x, t)
        pdfr = x * f1 / f0
        return np.where(ok, np.maximum(k, 0.0) * J * pdfr, 0.0)

    def z_integral(self, t):
        zr = z_range(self.kind, t, self.s, self.eta)
        if zr is None:
            return 0.0
        zm, zp = zr
        lm, lp = math.log(zm / (1 - zm)), math.log(zp / (1 - zp))
        L = 0.5 * (lp - lm) * _GL_X + 0.5 * (lp + lm)
        z = 1.0 / (1.0 + np.exp(-L))
        vals = self.integrand(t, z) * z * (1 - z)
        return 0.5 * (lp - lm) * float(np.dot(_GL_W, vals)) * self.alpha(t) / (2 * math.pi)

    def exponent(self, t_lo, t_hi):
        """int_{t_lo}^{t_hi} dt/t int dz ..., clipped to the kinematic limit."""
        tk = t_limit(self.kind, self.s, self.eta)
        hi = min(t_hi, tk)
        if hi <= t_lo:
            return 0.0
        val, _ = integrate.quad(lambda lt: self.z_integral(math.exp(lt)), math.log(max(t_lo, 1e-300)),
                                math.log(hi), limit=100, epsabs=1e-8, epsrel=1e-6)
        return self.mult * val


def cumulative(ends, edges, t_start):
    """sum over ends of the exponent from each edge up to t_start (edges increasing)."""
    pts = list(edges) + [t_start]
    seg = np.array([sum(e.exponent(pts[i], pts[i + 1]) for e in ends) for i in range(len(edges))])
    return np.cumsum(seg[::-1])[::-1]


def no_emission(ends, t_c, t_start):
    return math.exp(-sum(e.exponent(t_c, t_start) for e in ends))


def first_emission_bins(ends, edges, t_start):
    """P(first emission scale in [edges[i], edges[i+1]]) for increasing edges,
    and the no-emission probability above edges[0]."""
    surv = np.exp(-cumulative(ends, edges, t_start))  # P(no emission above each edge)
    return surv[1:] - surv[:-1], float(surv[0])
