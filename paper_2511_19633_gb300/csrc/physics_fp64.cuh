// FP64 device physics of the dipole shower (Appendices A and B of
// arXiv:2511.19633): PDF interpolation and its certified ratio bound, the
// one-loop coupling, the z limits, overestimate shapes, the transverse basis.
// Compiled without FMA contraction so that results agree with a plain FP64
// CPU evaluation of the same formulas up to the rounding of libm calls.
#pragma once

#include "common.cuh"
#include "gmath.cuh"

namespace gaps {

// --- PDF: bilinear interpolation of x f in (ln x, ln Q^2), zero off-grid ----
__device__ __forceinline__ double pdf_node(const DevParams& P, int f, int ix, int iq) {
  if (f == 11) {
    double s = 0.0;
    for (int k = 1; k <= 10; ++k) s += (double)__ldg(&P.grid[((size_t)k * kNX + ix) * kNQ + iq]);
    return s;
  }
  return (double)__ldg(&P.grid[((size_t)f * kNX + ix) * kNQ + iq]);
}

__device__ __forceinline__ bool pdf_locate_x(const DevParams& P, double x, int& ix, double& fx) {
  if (!(x >= kXMin && x <= kXMax)) return false;
  double u = (gm_log(x) - P.lxmin) / P.dlx;
  ix = (int)floor(u);
  if (ix < 0) ix = 0;
  if (ix > kNX - 2) ix = kNX - 2;
  fx = u - (double)ix;
  return true;
}

__device__ __forceinline__ bool pdf_locate_q(const DevParams& P, double q2, int& iq, double& fq) {
  if (!(q2 >= kQ2Min && q2 <= kQ2Max)) return false;
  double u = (gm_log(q2) - P.lqmin) / P.dlq;
  iq = (int)floor(u);
  if (iq < 0) iq = 0;
  if (iq > kNQ - 2) iq = kNQ - 2;
  fq = u - (double)iq;
  return true;
}

// a point's cell and fractions on the grid, found once for several flavours
// (pdf_xf's arithmetic, so the values are the same bits)
struct PdfLoc {
  int ix, iq;
  double fx, fq;
  bool ok;
};
__device__ __forceinline__ PdfLoc pdf_locate(const DevParams& P, double x, double q2) {
  PdfLoc L;
  L.ix = L.iq = 0;
  L.fx = L.fq = 0.0;
  L.ok = pdf_locate_x(P, x, L.ix, L.fx) && pdf_locate_q(P, q2, L.iq, L.fq);
  return L;
}
__device__ __forceinline__ double pdf_at(const DevParams& P, int f, const PdfLoc& L) {
  if (f < 0 || f > 11 || !L.ok) return 0.0;
  double lo = (1.0 - L.fx) * pdf_node(P, f, L.ix, L.iq) + L.fx * pdf_node(P, f, L.ix + 1, L.iq);
  double hi = (1.0 - L.fx) * pdf_node(P, f, L.ix, L.iq + 1) + L.fx * pdf_node(P, f, L.ix + 1, L.iq + 1);
  return lo * (1.0 - L.fq) + hi * L.fq;
}

__device__ __forceinline__ double pdf_xf(const DevParams& P, int f, double x, double q2) {
  int ix, iq;
  double fx, fq;
  if (f < 0 || f > 11) return 0.0;
  if (!pdf_locate_x(P, x, ix, fx) || !pdf_locate_q(P, q2, iq, fq)) return 0.0;
  double lo = (1.0 - fx) * pdf_node(P, f, ix, iq) + fx * pdf_node(P, f, ix + 1, iq);
  double hi = (1.0 - fx) * pdf_node(P, f, ix, iq + 1) + fx * pdf_node(P, f, ix + 1, iq + 1);
  return lo * (1.0 - fq) + hi * fq;
}

// Upper bound of x' f_num(x', Q^2) / (eta f_den(eta, Q^2)) for all Q^2 and all
// x' >= eta, from per-node extrema over Q^2 (the interpolant is linear in
// ln x inside a cell at fixed Q^2). 0 when eta is off the grid.
__device__ __forceinline__ double pdf_ratio_bound(const DevParams& P, int num, int den, double eta) {
  int ix;
  double fx;
  if (num < 0 || num > 11 || den < 0 || den > 11) return 0.0;
  if (!pdf_locate_x(P, eta, ix, fx)) return 0.0;
  double uin = (1.0 - fx) * __ldg(&P.umax[num * kNX + ix]) + fx * __ldg(&P.umax[num * kNX + ix + 1]);
  double un = fmax(uin, __ldg(&P.sufmax[num * (kNX + 1) + ix + 1]));
  double ld = (1.0 - fx) * __ldg(&P.lmin[den * kNX + ix]) + fx * __ldg(&P.lmin[den * kNX + ix + 1]);
  if (!(ld > 0.0)) return 0.0;
  if (P.thr[den] >= 0) {
    // heavy denominator with a threshold: the bound of the ratio times
    // (t - m^2)/t, dlq x numerator / first in the first cell above the mass,
    // numerator / lmin above it (App. A.2)
    double fd = (1.0 - fx) * __ldg(&P.first[den * kNX + ix]) + fx * __ldg(&P.first[den * kNX + ix + 1]);
    if (!(fd > 0.0)) return 0.0;
    return un * fmax(P.dlq / fd, 1.0 / ld);
  }
  return un / ld;
}

// one-loop alpha_s(t) from alpha_s(m_Z^2)
__device__ __forceinline__ double alpha_s(const DevParams& P, double t) {
  return P.as_mz / (1.0 + P.as_mz * P.beta0 * gm_log(t / (kMZ * kMZ)));
}

// --- dipole types, channels and overestimates -----------------------------
enum DipType { kFF = 0, kFI = 1, kIF = 2, kII = 3 };
enum Shape { kSoft = 0, kFlat = 1, kBoth = 2, kInv = 3 };

// channel 0 q->qg, 1 g->gg, 2 g->qqbar (final emitters); 3 q->qg, 4 q->g qbar,
// 5 g->gg, 6 g->qq (initial emitters). Shape and coefficient of Pover.
__device__ __forceinline__ void channel_over(int ch, int type, int nf, int& shape, double& coef) {
  switch (ch) {
    case 0: shape = kSoft; coef = 2.0 * kCF; break;
    case 1: shape = kSoft; coef = kCA; break;
    case 2: shape = kFlat; coef = nf * kTR / 2.0; break;
    case 3: shape = kSoft; coef = 2.0 * kCF; break;
    case 4: if (type == kIF) { shape = kSoft; coef = kTR; } else { shape = kFlat; coef = kTR; } break;
    case 5: shape = kBoth; coef = kCA; break;
    default: if (type == kIF) { shape = kBoth; coef = kCF; } else { shape = kInv; coef = kCF; } break;
  }
}

// z- and Delta = 1 - z+ at scale t (Appendix B.2-B.5 kinematic limits,
// rationalised: 1 - sqrt(D) = (1 - D)/(1 + sqrt(D))); false above the limit
__device__ __forceinline__ bool z_limits(int type, double t, double s, double eta, double& zm,
                                         double& delta) {
  double e;
  if (type == kFF) e = 4.0 * t / s;
  else if (type == kFI) e = 4.0 * t / s * eta / (1.0 - eta);
  else if (type == kIF) e = 4.0 * t * eta / (s * (1.0 - eta));
  else e = 4.0 * t * eta / (s * (1.0 - eta) * (1.0 - eta));
  double D = 1.0 - e;
  if (!(D > 0.0)) return false;
  double sq = sqrt(D);
  if (type == kFF || type == kFI) {
    delta = 0.5 * e / (1.0 + sq);
    zm = delta;
  } else {
    delta = 0.5 * (1.0 - eta) * e / (1.0 + sq);
    zm = eta + delta;
  }
  return true;
}

__device__ __forceinline__ double t_kin_max(int type, double s, double eta) {
  if (type == kFF) return s / 4.0;
  if (type == kFI || type == kIF) return s / 4.0 * (1.0 - eta) / eta;
  return s / 4.0 * (1.0 - eta) * (1.0 - eta) / eta;
}

__device__ __forceinline__ double shape_integral(int sh, double zm, double delta) {
  double zp = 1.0 - delta;
  switch (sh) {
    case kSoft: return gm_log((1.0 - zm) / delta);
    case kFlat: return zp - zm;
    case kBoth: return gm_log(zp / zm) + gm_log((1.0 - zm) / delta);
    default: return gm_log(zp / zm);
  }
}

__device__ __forceinline__ void shape_sample(int sh, double zm, double delta, double R, double& z,
                                             double& omz) {
  double zp = 1.0 - delta;
  switch (sh) {
    case kSoft:
      omz = (1.0 - zm) * gm_exp(R * gm_log(delta / (1.0 - zm)));
      z = 1.0 - omz;
      break;
    case kFlat:
      z = zm + R * (zp - zm);
      omz = 1.0 - z;
      break;
    case kBoth: {
      double lm = gm_log(zm / (1.0 - zm)), lp = gm_log(zp / delta);
      double L = lm + R * (lp - lm);
      double em = gm_exp(-L);
      z = 1.0 / (1.0 + em);
      omz = em / (1.0 + em);
      break;
    }
    default:
      z = zm * gm_exp(R * gm_log(zp / zm));
      omz = 1.0 - z;
      break;
  }
}

__device__ __forceinline__ double shape_value(int sh, double coef, double z, double omz) {
  switch (sh) {
    case kSoft: return coef / omz;
    case kFlat: return coef;
    case kBoth: return coef / (z * omz);
    default: return coef / z;
  }
}

// initial-state PDF-ratio flavours: numerator = new incoming parton,
// denominator = current incoming parton (11 = sum of quarks)
__device__ __forceinline__ void isr_pdf_indices(int ch, int fl_emitter, int& num, int& den) {
  int fe = pdf_index(fl_emitter);
  switch (ch) {
    case 3: num = fe; den = fe; break;
    case 4: num = 0; den = fe; break;
    case 5: num = 0; den = 0; break;
    default: num = 11; den = 0; break;
  }
}

// Appendix B.4 map (t, z) -> (x, u) in the cancellation-free form
__device__ __forceinline__ bool if_map(double r, double z, double omz, double& x, double& omx,
                                       double& u, double& omu) {
  double q = omz + r;
  double disc = 1.0 - 4.0 * r * z * omz / (q * q);
  if (!(disc >= 0.0)) return false;
  x = 2.0 * z * omz / (q * (1.0 + sqrt(disc)));
  u = x * r / omz;
  omu = 1.0 - u;
  if (!(omu > 0.0)) return false;
  omx = omz / omu;
  return true;
}

// eq. ii-jacobian map (t, z) -> (x, v)
__device__ __forceinline__ bool ii_map(double r, double z, double omz, double& x, double& omx,
                                       double& v) {
  x = z * omz / (omz + r);
  omx = (omz * omz + r) / (omz + r);
  v = x * r / omz;
  return omx - v > 0.0;
}

// Transverse basis e1, e2 of a dipole (P, K lightlike): project the spatial
// axis with the largest -r_perp^2 = 1 + 2 P_i K_i / P.K, then the next one,
// Gram-Schmidt in Minkowski space.
__device__ __forceinline__ void transverse_basis(const double P[4], const double K[4], double e1[4],
                                                 double e2[4]) {
  double PK = dot4(P, K);
  double N1 = 1.0 + 2.0 * P[1] * K[1] / PK;
  double N2 = 1.0 + 2.0 * P[2] * K[2] / PK;
  double N3 = 1.0 + 2.0 * P[3] * K[3] / PK;
  int a = 1;
  double Na = N1;
  if (N2 > Na) { a = 2; Na = N2; }
  if (N3 > Na) { a = 3; Na = N3; }
  int b;
  if (a == 1) b = (N3 > N2) ? 3 : 2;
  else if (a == 2) b = (N3 > N1) ? 3 : 1;
  else b = (N2 > N1) ? 2 : 1;
  double na = sqrt(Na);
  double Ka = K[a], Pa = P[a], Kb = K[b], Pb = P[b];
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    double r = (mu == a) ? 1.0 : 0.0;
    e1[mu] = (r + (Ka / PK) * P[mu] + (Pa / PK) * K[mu]) / na;
  }
  double e1b = e1[b];
  double e2p[4];
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    double r = (mu == b) ? 1.0 : 0.0;
    double rperp = r + (Kb / PK) * P[mu] + (Pb / PK) * K[mu];
    e2p[mu] = rperp - e1b * e1[mu];
  }
  double n2 = sqrt(-dot4(e2p, e2p));
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) e2[mu] = e2p[mu] / n2;
}

}  // namespace gaps
