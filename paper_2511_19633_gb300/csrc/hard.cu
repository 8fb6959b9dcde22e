// Hard events, one thread per event: e+e- -> q qbar (textbook LO with
// Z/gamma interference), pp -> Z at LO (Appendix C.1) and the NLO S and H
// events of the MC@NLO-like matching (Appendix C.2-C.4).
#include "physics_fp64.cuh"

namespace gaps {
namespace {

struct EWq { double Q, T3; };
__device__ __forceinline__ EWq quark_ew(int f) {
  bool up = (f == 2 || f == 4);
  return up ? EWq{2.0 / 3.0, 0.5} : EWq{-1.0 / 3.0, -0.5};
}

// Born |M|^2 of q qbar -> Z (Appendix C.1): (1/N_c)(1/4) sqrt2 G_F m^4 (V^2 + A^2)
// with V = 2 T3 - 4 Q sin^2(theta_W), A = 2 T3
__device__ double born_me2(int f) {
  EWq e = quark_ew(f < 0 ? -f : f);
  double V = 2.0 * e.T3 - 4.0 * e.Q * kSin2W, A = 2.0 * e.T3;
  double m4 = kMZ * kMZ * kMZ * kMZ;
  return (1.0 / kNc) * 0.25 * sqrt(2.0) * kGF * m4 * (V * V + A * A);
}

// e+e- -> q qbar angular distribution with Z/gamma interference (LO textbook)
__device__ double ee_dsigma_dcos(double s, int f, double c) {
  EWq q = quark_ew(f);
  double Ve = -0.5 + 2.0 * kSin2W, Ae = -0.5;
  double Vf = q.T3 - 2.0 * q.Q * kSin2W, Af = q.T3;
  double kappa = sqrt(2.0) * kGF * kMZ * kMZ / (4.0 * kPi * kAlphaEM);
  double den = (s - kMZ * kMZ) * (s - kMZ * kMZ) + kGZ * kGZ * kMZ * kMZ;
  double chi1 = kappa * s * (s - kMZ * kMZ) / den;
  double chi2 = kappa * kappa * s * s / den;
  double a = q.Q * q.Q - 2.0 * q.Q * Ve * Vf * chi1 + (Ae * Ae + Ve * Ve) * (Af * Af + Vf * Vf) * chi2;
  double b = -2.0 * q.Q * Ae * Af * chi1 + 4.0 * Ae * Ve * Af * Vf * chi2;
  return kNc * kPi * kAlphaEM * kAlphaEM / (2.0 * s) * ((1.0 + c * c) * a + 2.0 * c * b);
}

// q qbar -> gamma*/Z -> e- e+: the expression above read backwards in time,
// with the average 1/N_c over the incoming colours in place of the sum N_c
// over the outgoing ones; c = cosine between incoming quark and electron
__device__ double ll_dsigma_dcos(double s, int f, double c) {
  return ee_dsigma_dcos(s, f, c) / (kNc * kNc);
}

// ordered Born pairs: (q, qbar) for q = d u s c b, then (qbar, q)
__device__ __forceinline__ void born_pair(int k, int& fa, int& fb) {
  int q = (k % 5) + 1;
  if (k < 5) { fa = q; fb = -q; } else { fa = -q; fb = q; }
}

// pi (eta_a f_a)(eta_b f_b) |M|^2 / m^4 for one ordered pair (Appendix C.1)
// (la, lb: the grid cells of eta_a, eta_b at Q^2 = m_Z^2)
__device__ double born_pair_density(const DevParams& P, int k, const PdfLoc& la, const PdfLoc& lb) {
  int fa, fb;
  born_pair(k, fa, fb);
  double mz2 = kMZ * kMZ;
  double Fa = pdf_at(P, pdf_index(fa), la);
  double Fb = pdf_at(P, pdf_index(fb), lb);
  return kPi * Fa * Fb * born_me2(fa) / (mz2 * mz2);
}

// ---- the hard process of GAPS_MIXED contexts (FAST): the same formulas in
// FP32 where the result is an event weight or a density (FP64 runs at 1/64 of
// the FP32 rate on GB300), FP64 for the momenta. The FP64 kernel keeps the
// oracle's arithmetic, operation by operation.

// Born |M|^2 per quark class, folded at compile time (born_me2's formula)
__host__ __device__ constexpr double born_me2_const(double Q, double T3) {
  return (1.0 / kNc) * 0.25 * 1.4142135623730951 * kGF * (kMZ * kMZ * kMZ * kMZ) *
         ((2.0 * T3 - 4.0 * Q * kSin2W) * (2.0 * T3 - 4.0 * Q * kSin2W) + (2.0 * T3) * (2.0 * T3));
}
__device__ __forceinline__ float born_me2_f(int f) {
  constexpr float up = (float)born_me2_const(2.0 / 3.0, 0.5);
  constexpr float down = (float)born_me2_const(-1.0 / 3.0, -0.5);
  const int a = f < 0 ? -f : f;
  return (a == 2 || a == 4) ? up : down;
}

// a point's grid cell with FP32 logarithms, and the FP32 bilinear density
struct PdfLocF {
  int ix, iq;
  float fx, fq;
  bool ok;
};
__device__ __forceinline__ PdfLocF pdf_locate_f(const DevParams& P, double x, double q2) {
  PdfLocF L;
  L.ix = L.iq = 0;
  L.fx = L.fq = 0.0f;
  L.ok = x >= kXMin && x <= kXMax && q2 >= kQ2Min && q2 <= kQ2Max;
  if (!L.ok) return L;
  const float u = (logf((float)x) - (float)P.lxmin) / (float)P.dlx;
  const float w = (logf((float)q2) - (float)P.lqmin) / (float)P.dlq;
  L.ix = min(max((int)floorf(u), 0), kNX - 2);
  L.iq = min(max((int)floorf(w), 0), kNQ - 2);
  L.fx = u - (float)L.ix;
  L.fq = w - (float)L.iq;
  return L;
}
__device__ __forceinline__ float pdf_at_f(const DevParams& P, int f, const PdfLocF& L) {
  if (f < 0 || f > 11 || !L.ok) return 0.0f;
  auto node = [&](int ix, int iq) { return (float)pdf_node(P, f, ix, iq); };
  const float lo = (1.0f - L.fx) * node(L.ix, L.iq) + L.fx * node(L.ix + 1, L.iq);
  const float hi = (1.0f - L.fx) * node(L.ix, L.iq + 1) + L.fx * node(L.ix + 1, L.iq + 1);
  return lo * (1.0f - L.fq) + hi * L.fq;
}

// Li2(x) for 0 <= x <= 1/2 from the series in u = -ln(1 - x) with Bernoulli
// coefficients, Li2 = sum_n B_n u^(n+1) / (n+1)! (B_1 = -1/2, odd B_n > 1
// vanish): u <= ln 2 < 2 pi, twelve terms reach the FP32 rounding
__device__ __forceinline__ float li2_bernoulli(float x) {
  const float u = -log1pf(-x), u2 = u * u;
  // B_2k / (2k+1)! for k = 1..6 (B_2 = 1/6, B_4 = -1/30, B_6 = 1/42,
  // B_8 = -1/30, B_10 = 5/66, B_12 = -691/2730)
  const float c1 = 1.0f / 36.0f, c2 = -1.0f / 3600.0f, c3 = 1.0f / 211680.0f, c4 = -1.0f / 10886400.0f,
              c5 = 1.0f / 526901760.0f, c6 = -4.0647616e-11f;
  const float tail = u2 * (c1 + u2 * (c2 + u2 * (c3 + u2 * (c4 + u2 * (c5 + u2 * c6)))));
  return u - 0.25f * u2 + u * tail;
}
__device__ __forceinline__ float li2_f(float x) {
  if (x == 0.0f) return 0.0f;
  const float pi2_6 = (float)(kPi * kPi / 6.0);
  if (x == 1.0f) return pi2_6;
  if (x > 0.5f) return pi2_6 - logf(x) * log1pf(-x) - li2_bernoulli(1.0f - x);
  return li2_bernoulli(x);
}

// collinear_leg in FP32 (FAST)
__device__ float collinear_leg_f(const DevParams& P, int fl, double eta_d, double R) {
  const float eta = (float)eta_d;
  const float pf = (float)(kCF * P.as_mz / (2.0 * kPi)), pt = (float)(kTR * P.as_mz / (2.0 * kPi));
  const double mz2 = kMZ * kMZ;
  const double xd = eta_d + R * (1.0 - eta_d);
  const float x = (float)xd, omx = (float)((1.0 - eta_d) * (1.0 - R));  // 1 - x without cancellation
  const PdfLocF l0 = pdf_locate_f(P, eta_d, mz2), lx = pdf_locate_f(P, eta_d / xd, mz2);
  const float Fq = pdf_at_f(P, pdf_index(fl), l0);
  const float rq = pdf_at_f(P, pdf_index(fl), lx) / Fq;
  const float rg = pdf_at_f(P, 0, lx) / Fq;
  const float logs = logf(omx / x) + logf(omx);
  const float g = pf * (2.0f / omx * logs);
  const float hqq = pf * (-(1.0f + x) * logs + omx);
  const float hqg = pt * (2.0f * x * omx + (x * x + omx * omx) * logs);
  const float A = pf * (-5.0f + (float)(2.0 * kPi * kPi / 3.0));
  const float l1 = log1pf(-eta);
  const float B = pf * (2.0f * ((float)(kPi * kPi / 6.0) - l1 * l1 - li2_f(1.0f - eta)));
  const float integrand = (rq - 1.0f) * g + rq * hqq + rg * hqg;
  return A - B + (1.0f - eta) * integrand;
}

// sum x^k/k^2 until a term falls below 1e-17 of the sum (x <= 1/2)
__device__ double li2_series(double x) {
  double sum = 0.0, xk = x;
  for (int k = 1; k < 200; ++k) {
    double term = xk / ((double)k * (double)k);
    sum += term;
    if (term < 1e-17 * sum) break;
    xk *= x;
  }
  return sum;
}

// dilogarithm on [0,1]: series up to 1/2, Euler's reflection above
__device__ double li2(double x) {
  if (x == 0.0) return 0.0;
  if (x == 1.0) return kPi * kPi / 6.0;
  if (x > 0.5) {
    double y = 1.0 - x;
    double r = (y == 0.0) ? 0.0 : li2_series(y);
    return kPi * kPi / 6.0 - gm_log(x) * gm_log(1.0 - x) - r;
  }
  return li2_series(x);
}

// Collinear K+P terms of one quark leg (Appendix C.3) with mu_F = m_Z:
// A - B(eta) + (1 - eta) [(r_q - 1) g(x) + r_q h_qq(x) + r_g h_qg(x)],
// x = eta + R (1 - eta); each term carries its own coupling prefactor.
__device__ double collinear_leg(const DevParams& P, int fl, double eta, double R) {
  const double L = 0.0;
  double pf = kCF * P.as_mz / (2.0 * kPi);
  double pt = kTR * P.as_mz / (2.0 * kPi);
  double mz2 = kMZ * kMZ;
  double x = eta + R * (1.0 - eta);
  double Fq = pdf_xf(P, pdf_index(fl), eta, mz2);
  const PdfLoc lx = pdf_locate(P, eta / x, mz2);
  double rq = pdf_at(P, pdf_index(fl), lx) / Fq;
  double rg = pdf_at(P, 0, lx) / Fq;
  double logs = gm_log((1.0 - x) / x) + gm_log(1.0 - x) - L;
  double g = pf * (2.0 / (1.0 - x) * logs);
  double hqq = pf * (-(1.0 + x) * logs + (1.0 - x));
  double hqg = pt * (2.0 * x * (1.0 - x) + (x * x + (1.0 - x) * (1.0 - x)) * logs);
  double A = pf * (-5.0 + 2.0 * kPi * kPi / 3.0 - 1.5 * L);
  double l1 = gm_log(1.0 - eta);
  double B = pf * (2.0 * (l1 * L + kPi * kPi / 6.0 - l1 * l1 - li2(1.0 - eta)));
  double integrand = (rq - 1.0) * g + rq * hqq + rg * hqg;
  return A - B + (1.0 - eta) * integrand;
}

struct Rec {
  // record being written
  const DevEvents& E;
  uint64_t e;
  __device__ void set(int slot, double E0, double px, double py, double pz, int fl, int c, int a) const {
    E.P(0, slot, e) = E0; E.P(1, slot, e) = px; E.P(2, slot, e) = py; E.P(3, slot, e) = pz;
    E.F(slot, e) = fl; E.C(slot, e) = c; E.A(slot, e) = a;
  }
};

__device__ __forceinline__ void incoming_quark_tags(int fl, int tag, int& c, int& a) {
  if (fl > 0) { c = 0; a = tag; } else { c = tag; a = 0; }
}

template <bool FAST>
__global__ void k_generate_hard(const __grid_constant__ DevParams P, DevEvents E, uint64_t first, uint64_t n) {
  uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  uint64_t id = first + e;
  // the event's row of a mixed batch: its process and energy (the other
  // fields are common; no per-thread copy of the parameters)
  int process = P.process;
  double sqrt_s = P.sqrt_s;
  if (P.n_rows > 1) {
    const RowParams& R = P.rows[mix_row(P, id)];
    process = R.process;
    sqrt_s = R.sqrt_s;
  }
  Rng rng;
  rng.init(P.seed, id, kHardDrawBase);
  double R0, R1, R2, R3, R4, R5;
  rng.next2(R0, R1);
  rng.next2(R2, R3);
  rng.next2(R4, R5);
  double s = sqrt_s * sqrt_s;
  Rec rec{E, e};
  E.status[e] = GAPS_STATUS_ACTIVE;
  E.n_emit[e] = 0;
  E.t[e] = s;
  E.draw[e] = 0;
  E.eta[e] = 0.0;
  E.eta[E.cap + e] = 0.0;
  if (process == GAPS_EE_QQ) {
    double c = 2.0 * R0 - 1.0;
    double cph, sph;
    gm_sincos2pi(R1, cph, sph);  // phi = 2 pi R1
    int f = 1 + (int)floor(R2 * P.nf);
    if (f > P.nf) f = P.nf;
    double st = sqrt((1.0 - c) * (1.0 + c));
    double En = 0.5 * sqrt_s;
    double n0 = st * cph, n1 = st * sph, n2 = c;
    rec.set(0, En, En * n0, En * n1, En * n2, f, 1, 0);
    rec.set(1, En, -En * n0, -En * n1, -En * n2, -f, 0, 1);
    E.npart[e] = 2;
    E.weight[e] = ee_dsigma_dcos(s, f, c) * 2.0 * P.nf * kGeV2pb;
    return;
  }
  if (process == GAPS_PP_LL) {
    // m^2 by the Breit-Wigner map m^2 = m_Z^2 + m_Z Gamma_Z tan(2 pi r), y
    // uniform in [-Y, Y], cos(theta*) and phi of the electron uniform in the
    // dilepton rest frame (quark along +z when it comes from beam 1); the
    // flavour pair by its share of the density
    double r = P.ll_rlo + R0 * (P.ll_rhi - P.ll_rlo);
    double cr, sr;
    gm_sincos2pi(r, cr, sr);
    double mg = kMZ * kGZ;
    double m2 = kMZ * kMZ + mg * (sr / cr);
    double m = sqrt(m2);
    double Y = gm_log(sqrt_s / m);
    double y = (2.0 * R1 - 1.0) * Y;
    double tau = m / sqrt_s;
    double ey = gm_exp(y), iey = gm_exp(-y);
    double ea = ey * tau, eb = iey * tau;
    double c = 2.0 * R3 - 1.0;
    double dens[10], tot = 0.0;
    const PdfLoc la = pdf_locate(P, ea, m2), lb = pdf_locate(P, eb, m2);
    for (int k = 0; k < 10; ++k) {
      int fa, fb;
      born_pair(k, fa, fb);
      double Fa = pdf_at(P, pdf_index(fa), la), Fb = pdf_at(P, pdf_index(fb), lb);
      dens[k] = Fa * Fb * ll_dsigma_dcos(m2, fa > 0 ? fa : fb, fa > 0 ? c : -c);
      tot += dens[k];
    }
    int pick = 9;
    double target = R2 * tot, acc = 0.0;
    for (int k = 0; k < 10; ++k) { acc += dens[k]; if (target < acc) { pick = k; break; } }
    int fa, fb;
    born_pair(pick, fa, fb);
    double Ea = ea * 0.5 * sqrt_s, Eb = eb * 0.5 * sqrt_s;
    int c0, a0, c1, a1;
    incoming_quark_tags(fa, 1, c0, a0);
    incoming_quark_tags(fb, 1, c1, a1);
    rec.set(0, Ea, 0.0, 0.0, Ea, fa, c0, a0);
    rec.set(1, Eb, 0.0, 0.0, -Eb, fb, c1, a1);
    double cph, sph;
    gm_sincos2pi(R4, cph, sph);  // phi = 2 pi R4
    double st = sqrt((1.0 - c) * (1.0 + c));
    double ch = 0.5 * (ey + iey), sh = 0.5 * (ey - iey);
    double hm = 0.5 * m;
    rec.set(2, hm * (ch + c * sh), hm * (st * cph), hm * (st * sph), hm * (sh + c * ch), 11, 0, 0);
    rec.set(3, hm * (ch - c * sh), -(hm * (st * cph)), -(hm * (st * sph)), hm * (sh - c * ch), -11, 0, 0);
    E.eta[e] = ea;
    E.eta[E.cap + e] = eb;
    E.npart[e] = 4;
    // dsigma = sum_k F_a F_b / m^2 dsigma_k/dc dm^2 dy dc, with dm^2 = 2 pi m_Z Gamma_Z / cos^2 dr
    E.weight[e] = tot / m2 * (kGmTwoPi * mg / (cr * cr)) * (P.ll_rhi - P.ll_rlo) * (2.0 * Y) * 2.0 * kGeV2pb;
    return;
  }
  double mz2 = kMZ * kMZ;
  bool hevent = false;
  double wsel = 1.0;
  if (process == GAPS_PP_Z_NLO) {
    hevent = !(R0 < P.p_s);
    wsel = hevent ? 1.0 / (1.0 - P.p_s) : 1.0 / P.p_s;
  }
  if (!hevent) {
    double Y = FAST ? log(sqrt_s / kMZ) : gm_log(sqrt_s / kMZ);
    double y = (2.0 * R1 - 1.0) * Y;
    double tau = kMZ / sqrt_s;
    double ea = (FAST ? exp(y) : gm_exp(y)) * tau, eb = (FAST ? exp(-y) : gm_exp(-y)) * tau;
    double dens[10], tot = 0.0;
    if constexpr (FAST) {
      const PdfLocF la = pdf_locate_f(P, ea, kMZ * kMZ), lb = pdf_locate_f(P, eb, kMZ * kMZ);
      constexpr float norm = (float)(kPi / (kMZ * kMZ * kMZ * kMZ));
      float tf = 0.0f;
      for (int k = 0; k < 10; ++k) {
        int fa, fb;
        born_pair(k, fa, fb);
        const float d = pdf_at_f(P, pdf_index(fa), la) * pdf_at_f(P, pdf_index(fb), lb) * born_me2_f(fa) * norm;
        dens[k] = d;
        tf += d;
      }
      tot = tf;
    } else {
      const PdfLoc la = pdf_locate(P, ea, kMZ * kMZ), lb = pdf_locate(P, eb, kMZ * kMZ);
      for (int k = 0; k < 10; ++k) { dens[k] = born_pair_density(P, k, la, lb); tot += dens[k]; }
    }
    int pick = 9;
    double target = R2 * tot, acc = 0.0;
    for (int k = 0; k < 10; ++k) { acc += dens[k]; if (target < acc) { pick = k; break; } }
    int fa, fb;
    born_pair(pick, fa, fb);
    double Ea = ea * 0.5 * sqrt_s, Eb = eb * 0.5 * sqrt_s;
    int c0, a0, c1, a1;
    incoming_quark_tags(fa, 1, c0, a0);
    incoming_quark_tags(fb, 1, c1, a1);
    rec.set(0, Ea, 0.0, 0.0, Ea, fa, c0, a0);
    rec.set(1, Eb, 0.0, 0.0, -Eb, fb, c1, a1);
    rec.set(2, Ea + Eb, 0.0 + 0.0, 0.0 + 0.0, Ea + (-Eb), 23, 0, 0);
    E.eta[e] = ea;
    E.eta[E.cap + e] = eb;
    E.npart[e] = 3;
    double w = tot * 2.0 * Y * kGeV2pb;
    if (process == GAPS_PP_Z_NLO) {
      double corr = 1.0 + kCF * P.as_mz / (2.0 * kPi) * 2.0;
      if constexpr (FAST) {
        corr += collinear_leg_f(P, fa, ea, R3);
        corr += collinear_leg_f(P, fb, eb, R4);
      } else {
        corr += collinear_leg(P, fa, ea, R3);
        corr += collinear_leg(P, fb, eb, R4);
      }
      w = w * corr * wsel;
    }
    E.weight[e] = w;
    return;
  }
  // H event: x, v, phi, rapidity of the hard system, II map with j = 2
  double xlo = mz2 / s;
  double x = xlo + R3 * (1.0 - xlo);
  double v = R4 * (1.0 - x);
  double sbar = mz2 / x;
  double Y = 0.5 * (FAST ? log(s / sbar) : gm_log(s / sbar));
  double y = (2.0 * R1 - 1.0) * Y;
  double rt = sqrt(sbar / s);
  double e1 = (FAST ? exp(y) : gm_exp(y)) * rt, e2 = (FAST ? exp(-y) : gm_exp(-y)) * rt;
  double as = P.as_mz;
  double m2 = mz2;
  // 0..9 q qbar -> Z g, 10..14 g q, 15..19 g qbar (gluon from beam 1),
  // 20..24 q g, 25..29 qbar g
  double tot = 0.0;
  double cpick = 0.0;
  {
    double cs[30];
    if constexpr (FAST) {
      // the 30 channels in FP32: the common factors once
      const PdfLocF l1 = pdf_locate_f(P, e1, mz2), l2 = pdf_locate_f(P, e2, mz2);
      const float pre = (float)(8.0 * kPi * as / m2 / (16.0 * kPi) / m2);
      const float fqq = pre * (float)kCF * -2.0f;
      const float fqg = pre * (float)kTR * (float)((2.0 * m2 + v * sbar) / sbar);
      float tf = 0.0f;
      for (int k = 0; k < 30; ++k) {
        int fa, fb;
        float rs;
        if (k < 10) {
          born_pair(k, fa, fb);
          rs = fqq * born_me2_f(fa);
        } else {
          const int q = ((k - 10) % 5) + 1;
          const int grp = (k - 10) / 5;
          const int fq = (grp == 0 || grp == 2) ? q : -q;
          if (grp < 2) { fa = 21; fb = fq; } else { fa = fq; fb = 21; }
          rs = fqg * born_me2_f(q);
        }
        const float c = pdf_at_f(P, pdf_index(fa), l1) * pdf_at_f(P, pdf_index(fb), l2) * rs;
        cs[k] = c;
        tf += fabsf(c);
      }
      tot = tf;
    } else {
    const PdfLoc l1 = pdf_locate(P, e1, mz2), l2 = pdf_locate(P, e2, mz2);
    for (int k = 0; k < 30; ++k) {
      int fa, fb;
      double rs;
      if (k < 10) {
        born_pair(k, fa, fb);
        rs = 8.0 * kPi * as * kCF / m2 * born_me2(fa) * (-2.0);
      } else {
        int q = ((k - 10) % 5) + 1;
        int grp = (k - 10) / 5;
        int fq = (grp == 0 || grp == 2) ? q : -q;
        if (grp < 2) { fa = 21; fb = fq; } else { fa = fq; fb = 21; }
        double ubar = -v * sbar;
        rs = 8.0 * kPi * as * kTR / m2 * born_me2(q) * ((2.0 * m2 - ubar) / sbar);
      }
      double Fa = pdf_at(P, pdf_index(fa), l1);
      double Fb = pdf_at(P, pdf_index(fb), l2);
      cs[k] = Fa * Fb * rs / (16.0 * kPi) / m2;
      tot += fabs(cs[k]);
    }
    }
    int pick = 29;
    double target = R2 * tot, acc = 0.0;
    for (int k = 0; k < 30; ++k) { acc += fabs(cs[k]); if (target < acc) { pick = k; break; } }
    cpick = cs[pick];
    double jac = 2.0 * Y * (1.0 - xlo) * (1.0 - x);
    E.weight[e] = (cpick < 0.0 ? -tot : tot) * jac * kGeV2pb * wsel;
    int fa, fb, fj, emitter;
    if (pick < 10) {
      born_pair(pick, fa, fb);
      fj = 21;
      emitter = 0;
    } else {
      int q = ((pick - 10) % 5) + 1;
      int grp = (pick - 10) / 5;
      int fq = (grp == 0 || grp == 2) ? q : -q;
      if (grp < 2) { fa = 21; fb = fq; emitter = 0; } else { fa = fq; fb = 21; emitter = 1; }
      fj = fq;
    }
    double E1 = e1 * 0.5 * sqrt_s, E2 = e2 * 0.5 * sqrt_s;
    double pa[4] = {E1, 0.0, 0.0, E1};
    double pb[4] = {E2, 0.0, 0.0, -E2};
    const double* pe = emitter == 0 ? pa : pb;
    const double* ps = emitter == 0 ? pb : pa;
    double Pt[4], Bt[4];
    for (int mu = 0; mu < 4; ++mu) { Pt[mu] = x * pe[mu]; Bt[mu] = ps[mu]; }
    double ea4[4], eb4[4];
    transverse_basis(Pt, Bt, ea4, eb4);
    double t = v * (1.0 - x - v) / x * m2;
    double st = sqrt(t), cph, sph;
    gm_sincos2pi(R5, cph, sph);  // phi = 2 pi R5
    double pj[4], pz[4];
    for (int mu = 0; mu < 4; ++mu) {
      double kt = st * (cph * ea4[mu] + sph * eb4[mu]);
      pj[mu] = ((1.0 - x - v) / x) * Pt[mu] + v * Bt[mu] - kt;
    }
    for (int mu = 0; mu < 4; ++mu) pz[mu] = (pa[mu] + pb[mu]) - pj[mu];
    // colours (crossed for incoming partons)
    int c0, a0, c1, a1, cj, aj;
    if (pick < 10) {
      if (fa > 0) { c0 = 0; a0 = 1; c1 = 2; a1 = 0; cj = 1; aj = 2; }
      else { c0 = 1; a0 = 0; c1 = 0; a1 = 2; cj = 2; aj = 1; }
    } else {
      int fq = emitter == 0 ? fb : fa;
      int cg, ag, cq, aq;
      if (fq > 0) { cq = 0; aq = 1; cg = 1; ag = 2; cj = 2; aj = 0; }
      else { cq = 1; aq = 0; cg = 2; ag = 1; cj = 0; aj = 2; }
      if (emitter == 0) { c0 = cg; a0 = ag; c1 = cq; a1 = aq; }
      else { c0 = cq; a0 = aq; c1 = cg; a1 = ag; }
    }
    rec.set(0, pa[0], pa[1], pa[2], pa[3], fa, c0, a0);
    rec.set(1, pb[0], pb[1], pb[2], pb[3], fb, c1, a1);
    rec.set(2, pz[0], pz[1], pz[2], pz[3], 23, 0, 0);
    rec.set(3, pj[0], pj[1], pj[2], pj[3], fj, cj, aj);
    E.eta[e] = e1;
    E.eta[E.cap + e] = e2;
    E.npart[e] = 4;
  }
}

}  // namespace

// fast: the FP32 weights of GAPS_MIXED contexts
cudaError_t launch_generate_hard(const DevParams& P, const DevEvents& E, uint64_t first, uint64_t n, int fast,
                                 cudaStream_t stream) {
  if (n == 0) return cudaSuccess;
  int bs = 128;
  unsigned grid = (unsigned)((n + bs - 1) / bs);
  if (fast) k_generate_hard<true><<<grid, bs, 0, stream>>>(P, E, first, n);
  else k_generate_hard<false><<<grid, bs, 0, stream>>>(P, E, first, n);
  return cudaGetLastError();
}

}  // namespace gaps
