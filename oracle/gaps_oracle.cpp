// GAPS oracle: a plain, single-threaded FP64 CPU implementation of the
// parton-shower veto algorithm with initial- and final-state dipoles, the
// PDF-ratio veto, Catani-Seymour recoil kinematics and the MC@NLO-like
// matching for on-shell Z production (Seymour & Sule, "An NLO-Matched Initial
// and Final State Parton Shower on a GPU", arXiv:2511.19633).
//
// THIS FILE IS TEST INFRASTRUCTURE. It exists to check the CUDA library
// against the paper. Only the test suite, the smoke check and the CPU
// baseline of the benchmark may load it. It shares no code, header, table or
// constant generator with the CUDA path; everything here is written from the
// paper's formulas (cited per function) and textbook definitions.
//
// Readings of the paper that are not fixed by its text are marked "reading:".
// The e+e- and Drell-Yan angular cross sections are pinned by the tests
// against helicity amplitudes; the observable binning is a choice (no pin).
//
// Conventions
//   four-vectors (E, px, py, pz), metric (+,-,-,-), GeV.
//   incoming partons are stored with their physical (positive-energy) momenta
//   and an "initial" flag; their colour tags are stored crossed (an incoming
//   quark carries an anticolour tag), so that two partons form a dipole when
//   col(i) == acol(k) or acol(i) == col(k), whatever their initial/final state.
//   pp events: slot 0 = parton from beam 1 (+z), slot 1 = beam 2 (-z),
//   slot 2 = the Z boson. e+e- events: slot 0 = quark, slot 1 = antiquark.

#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>
#include <algorithm>
#include <array>
#include <limits>

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kCF = 4.0 / 3.0, kCA = 3.0, kTR = 0.5, kNc = 3.0;
constexpr double kMZ = 91.1876, kGZ = 2.4952;
constexpr double kSin2W = 0.2312, kGF = 1.16638e-5, kAlphaEM = 1.0 / 128.9;
constexpr double kGeV2pb = 0.3893794e9;

// PDF grid geometry: 100 nodes uniform in ln x over [1e-6, 1-1e-6],
// 50 nodes uniform in ln Q^2 over [0.5, 13600^2] GeV^2, value = x f(x, Q^2).
constexpr int kNX = 100, kNQ = 50, kNFL = 11;
constexpr double kXMin = 1e-6, kXMax = 1.0 - 1e-6;
constexpr double kQ2Min = 0.5, kQ2Max = 13600.0 * 13600.0;

constexpr int kStatusActive = 0, kStatusDone = 1;
constexpr int kErrCapacity = -2, kErrIterCap = -3, kErrNumeric = -4;
constexpr long kMaxSteps = 200000;
constexpr double kHqFloor = 1e-3;  // heavy-quark trials end at m_q^2 (1 + kHqFloor)

// ---------------------------------------------------------------------------
// Random numbers: Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), written
// from its published definition: ten rounds of two 32x32->64 multiplications
// with the multipliers 0xD2511F53 and 0xCD9E8D57, an S-box free permutation,
// and a Weyl key schedule with increments 0x9E3779B9 and 0xBB67AE85.
// Stream contract: key = (seed_lo, seed_hi), counter = (event_lo, event_hi,
// draw_lo, draw_hi); every block advances the per-event draw counter by one.
// ---------------------------------------------------------------------------
void philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
    uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
    uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
    uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
    uint32_t n0 = hi1 ^ c[1] ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c[3] ^ k1;
    uint32_t n3 = lo0;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

// A uniform double in the open interval (0,1) from two 32-bit words: the top
// 53 bits of (hi:lo), offset by one half: (k + 0.5) * 2^-53.
double uniform_from_words(uint32_t lo, uint32_t hi) {
  uint64_t w = ((uint64_t)hi << 32) | (uint64_t)lo;
  uint64_t k = w >> 11;
  return ((double)k + 0.5) * (1.0 / 9007199254740992.0);
}

struct Stream {
  uint64_t seed, event, draw;
  // one Philox block -> two uniforms (words 0,1 and words 2,3)
  void next2(double& a, double& b) {
    uint32_t ctr[4] = {(uint32_t)event, (uint32_t)(event >> 32), (uint32_t)draw,
                       (uint32_t)(draw >> 32)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t w[4];
    philox4x32_10(ctr, key, w);
    draw += 1;
    a = uniform_from_words(w[0], w[1]);
    b = uniform_from_words(w[2], w[3]);
  }
};
constexpr uint64_t kHardDrawBase = 0x8000000000000000ull;  // hard process draws

// ---------------------------------------------------------------------------
// Elementary functions of the shower and the hard process, built only from
// IEEE-754 operations that are exactly rounded (+ - * / sqrt, floor, frexp,
// ldexp), so that every evaluation of the same steps gives the same bits:
//   ex(x): Cody-Waite reduction x = k ln2 + r with ln2 split into a 32-bit
//          head and a tail, then the Taylor series of e^r to degree 14
//          (|r| <= 0.35, truncation < 1e-19), scaled by 2^k;
//   lg(x): x = m 2^e with m in [1/sqrt2, sqrt2), ln m = 2 atanh(s),
//          s = (m-1)/(m+1), odd series to s^23 (|s| < 0.172);
//   cos/sin(2 pi R): exact reduction of R to v in [-1/8, 1/8] plus a
//          quadrant, Taylor series of cos (degree 18) and sin (degree 19) on
//          |2 pi v| <= pi/4.
// Accuracy (about 1 ulp) is pinned against the C library in the tests.
// ---------------------------------------------------------------------------
constexpr double kLn2Hi = 0x1.62e42fee00000p-1;
constexpr double kLn2Lo = 0x1.a39ef35793c76p-33;
constexpr double kInvLn2 = 0x1.71547652b82fep+0;
constexpr double kTwoPi = 0x1.921fb54442d18p+2;
constexpr double kSqrtHalf = 0x1.6a09e667f3bcdp-1;

double ex(double x) {
  if (!(x == x)) return x;
  if (x > 709.8) return std::numeric_limits<double>::infinity();
  if (x < -745.2) return 0.0;
  double k = std::floor(x * kInvLn2 + 0.5);
  double r = (x - k * kLn2Hi) - k * kLn2Lo;
  // Taylor coefficients 1/j!, j = 14 .. 1
  const double c[14] = {1.0 / 87178291200.0, 1.0 / 6227020800.0, 1.0 / 479001600.0,
                        1.0 / 39916800.0, 1.0 / 3628800.0, 1.0 / 362880.0, 1.0 / 40320.0,
                        1.0 / 5040.0, 1.0 / 720.0, 1.0 / 120.0, 1.0 / 24.0, 1.0 / 6.0, 1.0 / 2.0, 1.0};
  double p = c[0];
  for (int j = 1; j < 14; ++j) p = p * r + c[j];
  p = p * r + 1.0;
  return std::ldexp(p, (int)k);
}

double lg(double x) {
  if (!(x == x) || x < 0.0) return std::numeric_limits<double>::quiet_NaN();
  if (x == 0.0) return -std::numeric_limits<double>::infinity();
  if (x > 1.7976931348623157e308) return x;
  int e;
  double m = std::frexp(x, &e);  // x = m 2^e, m in [0.5, 1)
  if (m < kSqrtHalf) { m = m * 2.0; e -= 1; }
  double s = (m - 1.0) / (m + 1.0);
  double z = s * s;
  // 1/(2j+1), j = 11 .. 1
  const double c[11] = {1.0 / 23.0, 1.0 / 21.0, 1.0 / 19.0, 1.0 / 17.0, 1.0 / 15.0, 1.0 / 13.0,
                        1.0 / 11.0, 1.0 / 9.0, 1.0 / 7.0, 1.0 / 5.0, 1.0 / 3.0};
  double p = c[0];
  for (int j = 1; j < 11; ++j) p = p * z + c[j];
  p = p * z + 1.0;
  double lm = 2.0 * s * p;
  double de = (double)e;
  return de * kLn2Hi + (de * kLn2Lo + lm);
}

// cos(2 pi R) and sin(2 pi R)
void sincos2pi(double R, double& c, double& s) {
  double u = R - std::floor(R + 0.5);        // [-1/2, 1/2), exact
  double n = std::floor(4.0 * u + 0.5);      // quadrant in {-2, ..., 2}
  double v = u - 0.25 * n;                   // [-1/8, 1/8], exact
  double th = kTwoPi * v;
  double z = th * th;
  // sin: th (1 - z/3! + z^2/5! - ... - z^9/19!); cos: 1 - z/2! + ... + z^9/18!
  const double cs[9] = {-1.0 / 121645100408832000.0, 1.0 / 355687428096000.0, -1.0 / 1307674368000.0,
                        1.0 / 6227020800.0, -1.0 / 39916800.0, 1.0 / 362880.0, -1.0 / 5040.0,
                        1.0 / 120.0, -1.0 / 6.0};
  const double cc[9] = {1.0 / 6402373705728000.0, -1.0 / 20922789888000.0, 1.0 / 87178291200.0,
                        -1.0 / 479001600.0, 1.0 / 3628800.0, -1.0 / 40320.0, 1.0 / 720.0,
                        -1.0 / 24.0, 1.0 / 2.0};
  double ps = cs[0], pc = cc[0];
  for (int j = 1; j < 9; ++j) { ps = ps * z + cs[j]; pc = pc * z + cc[j]; }
  double sn = th + th * (z * ps);
  double cn = 1.0 - z * pc;
  int q = (int)n;
  if (q == 0) { c = cn; s = sn; }
  else if (q == 1) { c = -sn; s = cn; }
  else if (q == -1) { c = sn; s = -cn; }
  else { c = -cn; s = -sn; }
}

// ---------------------------------------------------------------------------
// Flavours: PDG-like codes 21 = gluon, 1..5 = d u s c b, negative = antiquark,
// 23 = Z. PDF table index: g -> 0, q -> 1..5, qbar -> 6..10, and 11 = the sum
// of all ten quark and antiquark densities (used by the g <- q backward step).
// ---------------------------------------------------------------------------
int pdf_index(int fl) {
  if (fl == 21) return 0;
  if (fl >= 1 && fl <= 5) return fl;
  if (fl <= -1 && fl >= -5) return 5 - fl;
  return -1;
}

// Bilinear interpolation of x f(x, Q^2) in (ln x, ln Q^2); zero outside the
// grid (the paper turns off x extrapolation and sets the PDF to zero outside
// its Q^2 limits, Appendix B.6).
struct Pdf {
  const float* grid;  // [11][100][50]
  double lxmin, dlx, lqmin, dlq;
  // certified bound tables (see pdf_ratio_bound)
  double umax[12][kNX];   // max over Q^2 nodes of the node value
  double sufmax[12][kNX + 1];  // max over x nodes j >= k of umax
  double lmin[12][kNX];   // min over Q^2 nodes of the node value (above the
                          // threshold for a heavy flavour with one)
  // Heavy-quark thresholds (App. A.2; c, b, cbar, bbar only): a flavour whose
  // nodes vanish for every x at all Q^2 nodes up to thr[f] and are positive
  // above has its mass m2[f] on node thr[f]; first[f][ix] is its node value
  // on node thr[f] + 1. thr[f] = -1: no threshold.
  int thr[12];
  double m2[12];
  double first[12][kNX];

  double node(int f, int ix, int iq) const {
    return (double)grid[((size_t)f * kNX + ix) * kNQ + iq];
  }
  double node_sum(int ix, int iq) const {  // sum over the ten (anti)quarks
    double s = 0.0;
    for (int f = 1; f <= 10; ++f) s += node(f, ix, iq);
    return s;
  }
  double node_any(int f, int ix, int iq) const {
    return f == 11 ? node_sum(ix, iq) : node(f, ix, iq);
  }

  // threshold node of a heavy flavour, or -1
  int find_threshold(int f) const {
    if (f != 4 && f != 5 && f != 9 && f != 10) return -1;
    int k0 = -1;
    for (int iq = 0; iq < kNQ; ++iq) {
      bool zero = true;
      for (int ix = 0; ix < kNX && zero; ++ix) zero = node(f, ix, iq) == 0.0;
      if (!zero) break;
      k0 = iq;
    }
    if (k0 < 0 || k0 >= kNQ - 1) return -1;
    for (int iq = k0 + 1; iq < kNQ; ++iq)
      for (int ix = 0; ix < kNX; ++ix)
        if (!(node(f, ix, iq) > 0.0)) return -1;
    return k0;
  }

  void init(const float* g) {
    grid = g;
    lxmin = lg(kXMin);
    dlx = (lg(kXMax) - lxmin) / (kNX - 1);
    lqmin = lg(kQ2Min);
    dlq = (lg(kQ2Max) - lqmin) / (kNQ - 1);
    for (int f = 0; f < 12; ++f) {
      thr[f] = f < 11 ? find_threshold(f) : -1;
      m2[f] = thr[f] >= 0 ? ex(lqmin + (double)thr[f] * dlq) : 0.0;
      for (int ix = 0; ix < kNX; ++ix) {
        first[f][ix] = thr[f] >= 0 ? node(f, ix, thr[f] + 1) : 0.0;
        double mx = -1.0, mn = 0.0;
        for (int iq = 0; iq < kNQ; ++iq) {
          double v = node_any(f, ix, iq);
          if (iq == 0 || v > mx) mx = v;
          if (iq <= thr[f]) continue;  // the minimum over the nodes above a threshold
          if (iq == thr[f] + 1 || iq == 0 || v < mn) mn = v;
        }
        umax[f][ix] = mx;
        lmin[f][ix] = mn;
      }
      sufmax[f][kNX] = 0.0;
      for (int ix = kNX - 1; ix >= 0; --ix)
        sufmax[f][ix] = std::max(umax[f][ix], sufmax[f][ix + 1]);
    }
  }

  // locate x in the grid: cell index and the fraction inside the cell
  bool locate_x(double x, int& ix, double& fx) const {
    if (!(x >= kXMin && x <= kXMax)) return false;
    double u = (lg(x) - lxmin) / dlx;
    ix = (int)std::floor(u);
    if (ix < 0) ix = 0;
    if (ix > kNX - 2) ix = kNX - 2;
    fx = u - (double)ix;
    return true;
  }
  bool locate_q(double q2, int& iq, double& fq) const {
    if (!(q2 >= kQ2Min && q2 <= kQ2Max)) return false;
    double u = (lg(q2) - lqmin) / dlq;
    iq = (int)std::floor(u);
    if (iq < 0) iq = 0;
    if (iq > kNQ - 2) iq = kNQ - 2;
    fq = u - (double)iq;
    return true;
  }

  // x f(x, Q^2) for table index f (0..11)
  double xf(int f, double x, double q2) const {
    int ix, iq;
    double fx, fq;
    if (!locate_x(x, ix, fx) || !locate_q(q2, iq, fq)) return 0.0;
    double lo = (1.0 - fx) * node_any(f, ix, iq) + fx * node_any(f, ix + 1, iq);
    double hi = (1.0 - fx) * node_any(f, ix, iq + 1) + fx * node_any(f, ix + 1, iq + 1);
    return lo * (1.0 - fq) + hi * fq;
  }

  // Upper bound, valid for every Q^2 and every x' in [eta, 1], of
  //   x' f_num(x', Q^2) / (eta f_den(eta, Q^2)).
  // The paper fits its bound to the 99 and 99.99 percentiles of sampled ratios
  // (eqs. pdfmax, pdfmax_ud), which is not a strict bound; reading: the plain
  // shower uses a certified bound built from the grid. At fixed Q^2 the
  // interpolant is linear in ln x inside a cell, so
  //   numerator   <= max(interp of per-node maxima at eta, max of nodes above the cell)
  //   denominator >= interp of per-node minima at eta.
  // Returns 0 when eta is off the grid or the denominator bound vanishes.
  //
  // Heavy denominator with a threshold (App. A.2): the bound is of the ratio
  // times (t - m^2)/t, the measure correction's factor, for t > m^2. In the
  // first cell above the mass the denominator is phi * first(eta) with
  // phi = ln(t/m^2)/dlq in (0, 1] and (t - m^2)/t = 1 - exp(-phi dlq) <= phi
  // dlq, so the corrected ratio is at most dlq * numerator / first(eta);
  // above that cell it is at most numerator / lmin(eta) (the factor is at
  // most one). The same bound holds for the uncorrected ratio of two
  // densities of this flavour at one t (the final-initial spectator), which
  // is at most numerator / first in the first cell.
  double ratio_bound(int num, int den, double eta) const {
    int ix;
    double fx;
    if (!locate_x(eta, ix, fx)) return 0.0;
    double uin = (1.0 - fx) * umax[num][ix] + fx * umax[num][ix + 1];
    double un = std::max(uin, sufmax[num][ix + 1]);
    double ld = (1.0 - fx) * lmin[den][ix] + fx * lmin[den][ix + 1];
    if (!(ld > 0.0)) return 0.0;
    if (thr[den] >= 0) {
      double fd = (1.0 - fx) * first[den][ix] + fx * first[den][ix + 1];
      if (!(fd > 0.0)) return 0.0;
      return un * std::max(dlq / fd, 1.0 / ld);
    }
    return un / ld;
  }
};

// ---------------------------------------------------------------------------
// Strong coupling. The paper uses alpha_s(t) in the veto and alpha_s(t_c) in
// the overestimate (Appendix A.2) and does not print the running; reading:
// one-loop running with n_f = 5 from alpha_s(m_Z^2).
// ---------------------------------------------------------------------------
struct Config {
  int process;           // 0 = e+e- -> q qbar, 1 = pp -> Z LO, 2 = pp -> Z NLO,
                         // 3 = pp -> gamma*/Z -> e- e+ LO
  int nf;
  int nmax;
  int fixed_alpha;       // test switch: alpha_s(t) = alpha_s(m_Z) everywhere
  uint32_t channel_mask; // test switch: bit per channel, 0 = all channels
  int pair_fixed;        // test switch: >= 0 forces the Born flavour pair
  double sqrt_s, alpha_s_mz, t_cut, p_s;
  double t_start;        // test switch: > 0 overrides the starting scale
  double y_fixed;        // test switch: finite forces the Born rapidity
  uint64_t seed;
  const float* pdf;
  double mll_lo, mll_hi; // process 3: dilepton mass window (GeV)
};

struct Physics {
  Config cfg;
  Pdf pdf;
  double s_had;
  double as_over;
  double beta0;

  double alpha_s(double t) const {
    if (cfg.fixed_alpha) return cfg.alpha_s_mz;
    return cfg.alpha_s_mz / (1.0 + cfg.alpha_s_mz * beta0 * lg(t / (kMZ * kMZ)));
  }
};

// ---------------------------------------------------------------------------
// Events
// ---------------------------------------------------------------------------
struct Parton {
  double p[4];
  int fl, col, acol;
  bool initial;
};

struct Counters {
  uint64_t steps, trials, isr_trials, vetoes, accepts, violations;
};

struct Event {
  std::vector<Parton> parts;
  double eta[2];   // momentum fractions of slots 0 and 1 (pp only)
  double t;        // current evolution scale
  double weight;
  double t_first;  // scale of the first accepted emission (0 if none)
  Stream rng;
  int status;
  int n_emit;
  bool pp;
  Counters cnt;
};

double dot4(const double a[4], const double b[4]) {
  return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
}

// ---------------------------------------------------------------------------
// Hard processes
// ---------------------------------------------------------------------------
struct EWq { double Q, T3; };
EWq quark_ew(int f) {  // f = 1..5 (d u s c b)
  bool up = (f == 2 || f == 4);
  return up ? EWq{2.0 / 3.0, 0.5} : EWq{-1.0 / 3.0, -0.5};
}

// Born |M|^2 for q qbar -> Z (Appendix C.1):
//   (1/N_c)(1/4) sqrt(2) G_F m^4 (V_q^2 + A_q^2).
// Reading: the 1/4 goes with V_q = 2 T3 - 4 Q sin^2(theta_W), A_q = 2 T3.
double born_me2(int f) {
  EWq e = quark_ew(std::abs(f));
  double V = 2.0 * e.T3 - 4.0 * e.Q * kSin2W, A = 2.0 * e.T3;
  double m4 = kMZ * kMZ * kMZ * kMZ;
  return (1.0 / kNc) * 0.25 * std::sqrt(2.0) * kGF * m4 * (V * V + A * A);
}

// e+e- -> Z/gamma* -> q qbar angular cross section (textbook LO formula with
// Z/gamma interference; the paper defers this process to GAPS 1).
double ee_dsigma_dcos(double s, int f, double c) {
  EWq q = quark_ew(f);
  double Ve = -0.5 + 2.0 * kSin2W, Ae = -0.5;
  double Vf = q.T3 - 2.0 * q.Q * kSin2W, Af = q.T3;
  double kappa = std::sqrt(2.0) * kGF * kMZ * kMZ / (4.0 * kPi * kAlphaEM);
  double den = (s - kMZ * kMZ) * (s - kMZ * kMZ) + kGZ * kGZ * kMZ * kMZ;
  double chi1 = kappa * s * (s - kMZ * kMZ) / den;
  double chi2 = kappa * kappa * s * s / den;
  double a = q.Q * q.Q - 2.0 * q.Q * Ve * Vf * chi1 + (Ae * Ae + Ve * Ve) * (Af * Af + Vf * Vf) * chi2;
  double b = -2.0 * q.Q * Ae * Af * chi1 + 4.0 * Ae * Ve * Af * Vf * chi2;
  return kNc * kPi * kAlphaEM * kAlphaEM / (2.0 * s) * ((1.0 + c * c) * a + 2.0 * c * b);
}

// q qbar -> gamma*/Z -> e- e+ (the process GAPS 2 provides besides on-shell Z
// production, Sec. 4.1): the e+e- -> q qbar expression above read backwards
// in time, with the average 1/N_c over the incoming colours in place of the
// sum N_c over the outgoing ones. c = cosine of the angle between the
// incoming quark and the electron in their centre-of-mass frame.
double ll_dsigma_dcos(double s, int f, double c) {
  return ee_dsigma_dcos(s, f, c) / (kNc * kNc);
}

// Breit-Wigner map of the dilepton mass: m^2 = m_Z^2 + m_Z Gamma_Z tan(2 pi r),
// r uniform between the window's images (computed once per configuration)
void ll_window(double mll_lo, double mll_hi, double& r_lo, double& r_hi) {
  double mg = kMZ * kGZ, mz2 = kMZ * kMZ;
  r_lo = std::atan((mll_lo * mll_lo - mz2) / mg) / kTwoPi;
  r_hi = std::atan((mll_hi * mll_hi - mz2) / mg) / kTwoPi;
}

void set_beam_parton(Event& ev, int slot, double eta, double sqrt_s) {
  Parton& P = ev.parts[slot];
  double E = eta * 0.5 * sqrt_s;
  P.p[0] = E; P.p[1] = 0.0; P.p[2] = 0.0; P.p[3] = (slot == 0) ? E : -E;
  P.initial = true;
  ev.eta[slot] = eta;
}

// crossed colour tag of an incoming (anti)quark: a physical incoming quark
// carries an anticolour tag, an incoming antiquark a colour tag
void set_incoming_quark_colour(Parton& P, int tag) {
  if (P.fl > 0) { P.col = 0; P.acol = tag; } else { P.col = tag; P.acol = 0; }
}

// The ten ordered Born flavour pairs (a from beam 1, b from beam 2):
// (q, qbar) for q = d u s c b, then (qbar, q).
void born_pair(int k, int& fa, int& fb) {
  int q = (k % 5) + 1;
  if (k < 5) { fa = q; fb = -q; } else { fa = -q; fb = q; }
}

// Hadronic Born density per unit rapidity and per pair (Appendix C.1):
//   dsigma/dy = pi * (eta_a f_a)(eta_b f_b) |M|^2 / m^4, summed over ordered
// pairs. Reading: the paper's factor 2 for the two orientations is the sum
// over the ten ordered pairs, each taken once.
double born_pair_density(const Physics& ph, int k, double eta_a, double eta_b) {
  int fa, fb;
  born_pair(k, fa, fb);
  double mz2 = kMZ * kMZ;
  double Fa = ph.pdf.xf(pdf_index(fa), eta_a, mz2);
  double Fb = ph.pdf.xf(pdf_index(fb), eta_b, mz2);
  return kPi * Fa * Fb * born_me2(fa) / (mz2 * mz2);
}

// Collinear (K+P) terms per incoming quark leg (Appendix C.3), with
// mu_F = mu_R = m_Z so ln(mu_F^2/m^2) = 0. Each term already carries its own
// prefactor (C_F or T_R times alpha_s/2pi); reading: kappa_C is the bracket
// of the final combination with those prefactors divided out, so no coupling
// is counted twice.
double li2(double x);  // dilogarithm, defined below
struct Collinear {
  double as;
  double L = 0.0;
  double pre_f() const { return kCF * as / (2.0 * kPi); }
  double pre_t() const { return kTR * as / (2.0 * kPi); }
  double A() const { return pre_f() * (-5.0 + 2.0 * kPi * kPi / 3.0 - 1.5 * L); }
  double B(double eta) const {
    double l1 = lg(1.0 - eta);
    return pre_f() * (2.0 * (l1 * L + kPi * kPi / 6.0 - l1 * l1 - li2(1.0 - eta)));
  }
  double logs(double x) const { return lg((1.0 - x) / x) + lg(1.0 - x) - L; }
  double g(double x) const { return pre_f() * (2.0 / (1.0 - x) * logs(x)); }
  double hqq(double x) const { return pre_f() * (-(1.0 + x) * logs(x) + (1.0 - x)); }
  double hqg(double x) const {
    return pre_t() * (2.0 * x * (1.0 - x) + (x * x + (1.0 - x) * (1.0 - x)) * logs(x));
  }
};

// one-sample estimate of A - B(eta) + int_eta^1 dx [(r_q - 1) g + r_q h_qq + r_g h_qg]
// for a leg of Born flavour fl at momentum fraction eta, with x = eta + R (1 - eta)
double collinear_leg(const Physics& ph, int fl, double eta, double R) {
  Collinear C{ph.cfg.alpha_s_mz};
  double mz2 = kMZ * kMZ;
  double x = eta + R * (1.0 - eta);
  double Fq = ph.pdf.xf(pdf_index(fl), eta, mz2);
  double rq = ph.pdf.xf(pdf_index(fl), eta / x, mz2) / Fq;
  double rg = ph.pdf.xf(0, eta / x, mz2) / Fq;
  double integrand = (rq - 1.0) * C.g(x) + rq * C.hqq(x) + rg * C.hqg(x);
  return C.A() - C.B(eta) + (1.0 - eta) * integrand;
}

// Dilogarithm Li2(x) for x in [0, 1]: the power series sum x^k/k^2 for
// x <= 1/2 (summed until a term falls below 1e-17 of the sum) and Euler's
// reflection Li2(x) = pi^2/6 - ln x ln(1-x) - Li2(1-x) above.
double li2(double x) {
  if (x == 0.0) return 0.0;
  if (x == 1.0) return kPi * kPi / 6.0;
  if (x > 0.5) return kPi * kPi / 6.0 - lg(x) * lg(1.0 - x) - li2(1.0 - x);
  // the remaining tail after a term t is below t x/(1-x) <= t for x <= 1/2
  double sum = 0.0, xk = x;
  for (int k = 1; k < 200; ++k) {
    double term = xk / ((double)k * (double)k);
    sum += term;
    if (term < 1e-17 * sum) break;
    xk *= x;
  }
  return sum;
}

// ---------------------------------------------------------------------------
// Orthonormal transverse basis for a dipole (reading: the paper does not fix
// it). For lightlike P, K and each spatial axis r, r_perp = r - (r.K/P.K) P -
// (r.P/P.K) K is orthogonal to both, with -r_perp^2 = 1 + 2 P_i K_i / P.K.
// e1 comes from the axis with the largest norm, e2 from the next one made
// orthogonal to e1 (Gram-Schmidt in Minkowski space).
// ---------------------------------------------------------------------------
void transverse_basis(const double P[4], const double K[4], double e1[4], double e2[4]) {
  double PK = dot4(P, K);
  double N[4] = {0.0, 0.0, 0.0, 0.0};
  for (int i = 1; i <= 3; ++i) N[i] = 1.0 + 2.0 * P[i] * K[i] / PK;
  int a = 1;
  for (int i = 2; i <= 3; ++i) if (N[i] > N[a]) a = i;
  int b = -1;
  for (int i = 1; i <= 3; ++i) {
    if (i == a) continue;
    if (b < 0 || N[i] > N[b]) b = i;
  }
  double na = std::sqrt(N[a]);
  for (int mu = 0; mu < 4; ++mu) {
    double r = (mu == a) ? 1.0 : 0.0;
    e1[mu] = (r + (K[a] / PK) * P[mu] + (P[a] / PK) * K[mu]) / na;
  }
  double e2p[4];
  for (int mu = 0; mu < 4; ++mu) {
    double r = (mu == b) ? 1.0 : 0.0;
    double rperp = r + (K[b] / PK) * P[mu] + (P[b] / PK) * K[mu];
    e2p[mu] = rperp - e1[b] * e1[mu];
  }
  double n2 = std::sqrt(-dot4(e2p, e2p));
  for (int mu = 0; mu < 4; ++mu) e2[mu] = e2p[mu] / n2;
}

// ---------------------------------------------------------------------------
// Dipole shower (Appendix B). Channels, per emitting dipole end:
//   final emitter   quark: 0 q->qg;  gluon: 1 g->gg, 2 g->q qbar (all flavours)
//   initial emitter quark: 3 q->qg (a=q, j=g), 4 q->g qbar (a=g, j=qbar)
//                   gluon: 5 g->gg, 6 g->qq (a=q, j=q, all ten flavours)
// Overestimate of the emission density in (t, z) for each channel:
//   (1/t) * alpha_s(t_c)/(2 pi) * B * Pover(z),  c = alpha_s(t_c)/(2pi) B int Pover
// with B the certified PDF-ratio bound (1 for final-final) and Pover one of
//   soft: C/(1-z)   flat: C   both: C/(z(1-z))   inv: C/z.
// Each Pover bounds kernel * Jacobian * (x for initial-state emitters) over
// the whole (x, u) or (x, v) domain (analytic bounds, checked by the Sudakov
// pins), so the acceptance weight never exceeds one when B is a true bound.
// ---------------------------------------------------------------------------
enum Shape { kSoft = 0, kFlat = 1, kBoth = 2, kInv = 3 };
enum DipType { kFF = 0, kFI = 1, kIF = 2, kII = 3 };

struct ChannelOver { Shape shape; double coef; };
ChannelOver channel_over(int ch, int type, int nf) {
  switch (ch) {
    case 0: return {kSoft, 2.0 * kCF};
    case 1: return {kSoft, kCA};
    case 2: return {kFlat, nf * kTR / 2.0};
    case 3: return {kSoft, 2.0 * kCF};
    case 4: return type == kIF ? ChannelOver{kSoft, kTR} : ChannelOver{kFlat, kTR};
    case 5: return {kBoth, kCA};
    default: return type == kIF ? ChannelOver{kBoth, kCF} : ChannelOver{kInv, kCF};
  }
}

// Overestimate z range at t: z- and Delta = 1 - z+ (kinematic limits of
// Appendix B, rationalised so that no small difference of nearly equal
// numbers is formed: 1 - sqrt(D) = (1 - D)/(1 + sqrt(D))).
//   FF: z+- = (1 +- sqrt(1 - 4t/s))/2
//   FI: z+- = (1 +- sqrt(1 - 4t/s eta/(1-eta)))/2
//   IF: z+- = ((1+eta) +- (1-eta) sqrt(1 - 4 t eta/(s (1-eta))))/2
//   II: z+- = ((1+eta) +- (1-eta) sqrt(1 - 4 t eta/(s (1-eta)^2)))/2
// Returns false when t is above the kinematic limit.
bool z_limits(int type, double t, double s, double eta, double& zm, double& delta) {
  double e = 0.0, D;
  if (type == kFF) {
    e = 4.0 * t / s;
  } else if (type == kFI) {
    e = 4.0 * t / s * eta / (1.0 - eta);
  } else if (type == kIF) {
    e = 4.0 * t * eta / (s * (1.0 - eta));
  } else {
    e = 4.0 * t * eta / (s * (1.0 - eta) * (1.0 - eta));
  }
  D = 1.0 - e;
  if (!(D > 0.0)) return false;
  double sq = std::sqrt(D);
  if (type == kFF || type == kFI) {
    delta = 0.5 * e / (1.0 + sq);
    zm = delta;
  } else {
    delta = 0.5 * (1.0 - eta) * e / (1.0 + sq);
    zm = eta + delta;
  }
  return true;
}

// kinematic upper limit of t for a dipole (Appendix B): s/4 (FF),
// s/4 (1-eta)/eta (FI, IF), s/4 (1-eta)^2/eta (II)
double t_kin_max(int type, double s, double eta) {
  if (type == kFF) return s / 4.0;
  if (type == kFI || type == kIF) return s / 4.0 * (1.0 - eta) / eta;
  return s / 4.0 * (1.0 - eta) * (1.0 - eta) / eta;
}

double shape_integral(Shape sh, double zm, double delta) {
  double zp = 1.0 - delta;
  switch (sh) {
    case kSoft: return lg((1.0 - zm) / delta);
    case kFlat: return zp - zm;
    case kBoth: return lg(zp / zm) + lg((1.0 - zm) / delta);
    default: return lg(zp / zm);
  }
}

// sample z from Pover on [zm, 1-delta] with the uniform R; returns z and 1-z,
// each formed without cancellation where the shape is singular
void shape_sample(Shape sh, double zm, double delta, double R, double& z, double& omz) {
  double zp = 1.0 - delta;
  switch (sh) {
    case kSoft:
      omz = (1.0 - zm) * ex(R * lg(delta / (1.0 - zm)));
      z = 1.0 - omz;
      break;
    case kFlat:
      z = zm + R * (zp - zm);
      omz = 1.0 - z;
      break;
    case kBoth: {
      double lm = lg(zm / (1.0 - zm)), lp = lg(zp / delta);
      double L = lm + R * (lp - lm);
      double em = ex(-L);
      z = 1.0 / (1.0 + em);
      omz = em / (1.0 + em);
      break;
    }
    default:
      z = zm * ex(R * lg(zp / zm));
      omz = 1.0 - z;
      break;
  }
}

double shape_value(Shape sh, double coef, double z, double omz) {
  switch (sh) {
    case kSoft: return coef / omz;
    case kFlat: return coef;
    case kBoth: return coef / (z * omz);
    default: return coef / z;
  }
}

// Initial-final map (Appendix B.4): (t, z) -> (x, u) with r = t/s,
//   x = (1-z+r)/(2r) [1 - sqrt(1 - 4 r z(1-z)/(1-z+r)^2)],  u = x r/(1-z),
// written as x = 2 z(1-z) / ((1-z+r)(1 + sqrt(...))) (same value, no
// cancellation for small r); 1-x = (1-z)/(1-u) from z = 1-(1-x)(1-u).
bool if_map(double r, double z, double omz, double& x, double& omx, double& u, double& omu) {
  double q = omz + r;
  double disc = 1.0 - 4.0 * r * z * omz / (q * q);
  if (!(disc >= 0.0)) return false;
  x = 2.0 * z * omz / (q * (1.0 + std::sqrt(disc)));
  u = x * r / omz;
  omu = 1.0 - u;
  if (!(omu > 0.0)) return false;
  omx = omz / omu;
  return true;
}

// Initial-initial map (eq. ii-jacobian): x = z(1-z)/(1-z+r), v = x r/(1-z),
// 1-x = ((1-z)^2 + r)/(1-z+r)
bool ii_map(double r, double z, double omz, double& x, double& omx, double& v) {
  x = z * omz / (omz + r);
  omx = (omz * omz + r) / (omz + r);
  v = x * r / omz;
  return omx - v > 0.0;
}

// PDF-ratio channel flavours: numerator (new incoming parton a) and
// denominator (current incoming parton) table indices
void isr_pdf_indices(int ch, int fl_emitter, int& num, int& den) {
  int fe = pdf_index(fl_emitter);
  switch (ch) {
    case 3: num = fe; den = fe; break;   // q <- q
    case 4: num = 0; den = fe; break;    // q <- g
    case 5: num = 0; den = 0; break;     // g <- g
    default: num = 11; den = 0; break;   // g <- sum of quarks
  }
}

struct Trial {
  int i, k, side, ch, type;
  double t, Rz, c;
  Shape shape;
  double coef, zm, delta;
  double s, eta;  // dipole invariant and the relevant momentum fraction
  double B;       // PDF bound used
  double m2;      // heavy-quark measure dt/(t - m2) of the trial, 0: dt/t
};

bool is_coloured(const Parton& P) { return P.col != 0 || P.acol != 0; }
bool is_gluon(const Parton& P) { return P.fl == 21; }

// partner on a colour side: side 0 = partner whose acol equals my col,
// side 1 = partner whose col equals my acol
int find_partner(const Event& ev, int i, int side) {
  const Parton& P = ev.parts[i];
  int tag = side == 0 ? P.col : P.acol;
  if (tag == 0) return -1;
  for (int k = 0; k < (int)ev.parts.size(); ++k) {
    if (k == i) continue;
    const Parton& Q = ev.parts[k];
    if (side == 0 && Q.acol == tag) return k;
    if (side == 1 && Q.col == tag) return k;
  }
  return -1;
}

int n_channels_of(const Parton& P, int& first) {
  if (!P.initial) { first = is_gluon(P) ? 1 : 0; return is_gluon(P) ? 2 : 1; }
  first = is_gluon(P) ? 5 : 3;
  return 2;
}

double beam_eta(const Event& ev, int slot) { return ev.eta[slot]; }

// One emission attempt of the max-veto algorithm (Section 2, Fig. 1):
// generate a trial for every dipole end and channel, pick the highest scale,
// test the cutoff, compute the acceptance weight (with the PDF ratio for
// initial-state legs) and, if accepted, build the emission.
void shower_step(const Physics& ph, Event& ev) {
  const Config& cf = ph.cfg;
  ev.cnt.steps += 1;
  Trial best{};
  best.t = -1.0;
  best.i = -1;
  int n = (int)ev.parts.size();
  for (int i = 0; i < n; ++i) {
    const Parton& Pi = ev.parts[i];
    if (!is_coloured(Pi)) continue;
    for (int side = 0; side < 2; ++side) {
      int tag = side == 0 ? Pi.col : Pi.acol;
      if (tag == 0) continue;
      int k = find_partner(ev, i, side);
      if (k < 0) continue;
      const Parton& Pk = ev.parts[k];
      int type = Pi.initial ? (Pk.initial ? kII : kIF) : (Pk.initial ? kFI : kFF);
      double s = 2.0 * dot4(Pi.p, Pk.p);
      double eta = 0.0;
      if (type == kFI) eta = beam_eta(ev, k);
      if (type == kIF || type == kII) eta = beam_eta(ev, i);
      int first;
      int nch = n_channels_of(Pi, first);
      for (int c = 0; c < nch; ++c) {
        int ch = first + c;
        double Rt, Rz;
        ev.rng.next2(Rt, Rz);
        if (cf.channel_mask != 0 && !((cf.channel_mask >> ch) & 1u)) continue;
        double tmax = std::min(ev.t, t_kin_max(type, s, eta));
        if (!(tmax > cf.t_cut)) continue;
        // Heavy-quark measure correction (App. A.2): an incoming c or b whose
        // density has a threshold draws its q <- q and q <- g trials in
        // dt/(t - m_q^2), with the PDF ratio times (t - m_q^2)/t. Reading
        // (the paper is silent): the channel's trials end at the floor
        // m_q^2 (1 + kHqFloor) (or the cutoff, if higher), where the
        // backward step to a gluon may be kinematically closed and the
        // trials would otherwise pile up at m_q^2 without end.
        double mq2 = 0.0;
        if ((type == kIF || type == kII) && (ch == 3 || ch == 4)) {
          int fe = pdf_index(Pi.fl);
          if (fe >= 0 && ph.pdf.thr[fe] >= 0) mq2 = ph.pdf.m2[fe];
        }
        if (mq2 > 0.0 && !(tmax > mq2 * (1.0 + kHqFloor))) continue;
        double zm, delta;
        if (!z_limits(type, cf.t_cut, s, eta, zm, delta)) continue;
        ChannelOver ov = channel_over(ch, type, cf.nf);
        double B = 1.0;
        if (type == kFI) {
          int f = pdf_index(Pk.fl);
          B = ph.pdf.ratio_bound(f, f, eta);
        } else if (type == kIF || type == kII) {
          int num, den;
          isr_pdf_indices(ch, Pi.fl, num, den);
          B = ph.pdf.ratio_bound(num, den, eta);
        }
        if (!(B > 0.0)) continue;
        double cc = ph.as_over / (2.0 * kPi) * B * ov.coef * shape_integral(ov.shape, zm, delta);
        if (!(cc > 0.0)) continue;
        ev.cnt.trials += 1;
        if (type != kFF && type != kFI) ev.cnt.isr_trials += 1;
        double tt = mq2 > 0.0 ? mq2 + (tmax - mq2) * ex(lg(Rt) / cc) : tmax * ex(lg(Rt) / cc);
        if (mq2 > 0.0 && !(tt > mq2 * (1.0 + kHqFloor))) continue;  // below the channel's floor
        if (tt > best.t) {
          best.i = i; best.k = k; best.side = side; best.ch = ch; best.type = type;
          best.t = tt; best.Rz = Rz; best.c = cc; best.shape = ov.shape; best.coef = ov.coef;
          best.zm = zm; best.delta = delta; best.s = s; best.eta = eta; best.B = B; best.m2 = mq2;
        }
      }
    }
  }
  if (best.i < 0 || best.t < cf.t_cut) {
    ev.status = kStatusDone;
    return;
  }
  if (!std::isfinite(best.t)) { ev.status = kErrNumeric; return; }
  double Rveto, Rphi, Rfl, Rcol;
  ev.rng.next2(Rveto, Rphi);
  ev.rng.next2(Rfl, Rcol);
  (void)Rcol;
  double t = best.t;
  ev.t = t;

  double z, omz;
  shape_sample(best.shape, best.zm, best.delta, best.Rz, z, omz);
  // true limits at the trial scale
  double zm_t, delta_t;
  if (!z_limits(best.type, t, best.s, best.eta, zm_t, delta_t) || !(omz > delta_t) ||
      !(z > zm_t)) {
    ev.cnt.vetoes += 1;
    return;
  }
  double pover = shape_value(best.shape, best.coef, z, omz);
  double as_ratio = ph.alpha_s(t) / ph.as_over;
  Parton& Pi = ev.parts[best.i];
  Parton& Pk = ev.parts[best.k];
  int type = best.type, ch = best.ch;
  double s = best.s;

  // kinematic variables and acceptance weight
  double w = 0.0;
  double y = 0.0, rho = 0.0, x = 1.0, omx = 0.0, u = 0.0, omu = 1.0, v = 0.0;
  int new_fl_i = Pi.fl, fl_j = 21;
  double sumF = 0.0;  // for channel 6
  if (type == kFF) {
    // Appendix B.2: y from t = z(1-z) y s, weight (1-y) P(z,y)
    y = t / (z * omz * s);
    double k;
    double den = omz + z * y;  // 1 - z(1-y)
    if (ch == 0) k = kCF * (2.0 / den - (1.0 + z));
    else if (ch == 1) k = kCA / 2.0 * (2.0 / den - 2.0 + z * omz);
    else k = cf.nf * kTR / 2.0 * (1.0 - 2.0 * z * omz);
    w = as_ratio * (1.0 - y) * k / pover;
  } else if (type == kFI) {
    // Appendix B.3: t = z(1-z)(1-x)/x s_ija, weight P(z,x) f_a(eta/x)/f_a(eta)
    rho = t / (z * omz * s);  // (1-x)/x
    x = 1.0 / (1.0 + rho);
    omx = rho / (1.0 + rho);
    double k;
    double den = omz + omx;
    if (ch == 0) k = kCF * (2.0 / den - (1.0 + z));
    else if (ch == 1) k = kCA / 2.0 * (2.0 / den - 2.0 + z * omz);
    else k = cf.nf * kTR / 2.0 * (1.0 - 2.0 * z * omz);
    int f = pdf_index(Pk.fl);
    double eta = best.eta;
    double F1 = ph.pdf.xf(f, eta * (1.0 + rho), t);
    double F0 = ph.pdf.xf(f, eta, t);
    double ratio = (F0 > 0.0) ? x * F1 / F0 : 0.0;  // f(eta/x)/f(eta) = x F(eta/x)/F(eta)
    w = as_ratio * k / pover * ratio / best.B;
  } else {
    double r = t / s;
    double J;
    if (type == kIF) {
      // Appendix B.4: Jacobian 1/(u + x - 2ux) = 1/(x(1-u) + u(1-x))
      if (!if_map(r, z, omz, x, omx, u, omu)) { ev.cnt.vetoes += 1; return; }
      J = 1.0 / (x * omu + u * omx);
    } else {
      // Appendix B.5: Jacobian 1/z
      if (!ii_map(r, z, omz, x, omx, v)) { ev.cnt.vetoes += 1; return; }
      J = 1.0 / z;
    }
    double eta = best.eta;
    if (!(x > eta)) { ev.cnt.vetoes += 1; return; }
    double k;
    double soft = (type == kIF) ? (omx + u) : omx;  // 1-x+u (IF) or 1-x (II)
    if (ch == 3) k = kCF * (2.0 / soft - (1.0 + x));
    else if (ch == 4) k = kTR * (1.0 - 2.0 * x * omx);
    else if (ch == 5) k = kCA * (1.0 / soft + omx / x - 1.0 + x * omx);
    else k = kCF / 2.0 * (x + 2.0 * omx / x);  // reading: half per gluon dipole end
    int num, den;
    isr_pdf_indices(ch, Pi.fl, num, den);
    double F0 = ph.pdf.xf(den, eta, t);
    double F1;
    if (ch == 6) {
      F1 = 0.0;
      for (int f = 1; f <= 10; ++f) F1 += ph.pdf.xf(f, eta / x, t);
      sumF = F1;
    } else {
      F1 = ph.pdf.xf(num, eta / x, t);
    }
    double Fratio = (F0 > 0.0) ? F1 / F0 : 0.0;
    // heavy-quark measure correction: the ratio times (t - m_q^2)/t
    if (best.m2 > 0.0) Fratio = Fratio * ((t - best.m2) / t);
    // f_a(eta/x)/f(eta) = x F_a(eta/x)/F(eta): the factor x is part of the
    // bounded kernel product
    w = as_ratio * k * J * x / pover * Fratio / best.B;
    if (ch == 4) { new_fl_i = 21; fl_j = -Pi.fl; }
    if (ch == 5) { new_fl_i = 21; fl_j = 21; }
  }
  if (!std::isfinite(w)) { ev.status = kErrNumeric; return; }
  if (w > 1.0) ev.cnt.violations += 1;
  if (!(Rveto < w)) { ev.cnt.vetoes += 1; return; }

  // ---- accepted: flavours ----
  if (ch == 2) {
    int f = 1 + (int)std::floor(Rfl * cf.nf);
    if (f > cf.nf) f = cf.nf;
    new_fl_i = f; fl_j = -f;
  } else if (ch == 6) {
    // flavour of the new incoming quark chosen in proportion to its density
    double target = Rfl * sumF, acc = 0.0;
    int pick = 10;
    for (int f = 1; f <= 10; ++f) {
      acc += ph.pdf.xf(f, best.eta / x, t);
      if (target < acc) { pick = f; break; }
    }
    int fl = pick <= 5 ? pick : -(pick - 5);
    new_fl_i = fl; fl_j = fl;
  }
  if ((int)ev.parts.size() >= cf.nmax) { ev.status = kErrCapacity; return; }

  // ---- kinematics ----
  double P[4], K[4];
  std::memcpy(P, Pi.p, sizeof P);
  std::memcpy(K, Pk.p, sizeof K);
  double e1[4], e2[4];
  transverse_basis(P, K, e1, e2);
  double st = std::sqrt(t), cph, sph;
  sincos2pi(Rphi, cph, sph);  // phi = 2 pi R_phi
  double kt[4];
  for (int mu = 0; mu < 4; ++mu) kt[mu] = st * (cph * e1[mu] + sph * e2[mu]);
  Parton J;
  J.initial = false;
  J.fl = fl_j;
  J.col = 0; J.acol = 0;
  if (type == kFF) {
    for (int mu = 0; mu < 4; ++mu) {
      Pi.p[mu] = z * P[mu] + (y * omz) * K[mu] + kt[mu];
      J.p[mu] = omz * P[mu] + (y * z) * K[mu] - kt[mu];
      Pk.p[mu] = (1.0 - y) * K[mu];
    }
  } else if (type == kFI) {
    double xinv = 1.0 + rho;
    for (int mu = 0; mu < 4; ++mu) {
      Pi.p[mu] = z * P[mu] + (omz * rho) * K[mu] + kt[mu];
      J.p[mu] = omz * P[mu] + (z * rho) * K[mu] - kt[mu];
      Pk.p[mu] = xinv * K[mu];
    }
    ev.eta[best.k] = ev.eta[best.k] * xinv;
  } else if (type == kIF) {
    for (int mu = 0; mu < 4; ++mu) {
      Pi.p[mu] = P[mu] / x;
      J.p[mu] = (omu * omx / x) * P[mu] + u * K[mu] - kt[mu];
      Pk.p[mu] = (u * omx / x) * P[mu] + omu * K[mu] + kt[mu];
    }
    ev.eta[best.i] = ev.eta[best.i] / x;
  } else {
    for (int mu = 0; mu < 4; ++mu) {
      Pi.p[mu] = P[mu] / x;
      J.p[mu] = ((omx - v) / x) * P[mu] + v * K[mu] - kt[mu];
    }
    ev.eta[best.i] = ev.eta[best.i] / x;
    // Lorentz "kick" of every other final-state particle (eq. IIkinematics3):
    //   Lambda = g - 2 (K'+K)(K'+K)/(K'+K)^2 + 2 K K'/K'^2,
    //   K' = p~_aj + p~_b, K = p_a + p_b - p_j
    double Kp[4], Kn[4], KK[4];
    for (int mu = 0; mu < 4; ++mu) {
      Kp[mu] = P[mu] + K[mu];
      Kn[mu] = (Pi.p[mu] + Pk.p[mu]) - J.p[mu];
      KK[mu] = Kp[mu] + Kn[mu];
    }
    double KK2 = dot4(KK, KK), Kp2 = dot4(Kp, Kp);
    for (int m = 0; m < (int)ev.parts.size(); ++m) {
      Parton& Q = ev.parts[m];
      if (Q.initial) continue;
      double a = 2.0 * dot4(KK, Q.p) / KK2;
      double b = 2.0 * dot4(Kp, Q.p) / Kp2;
      double q[4];
      for (int mu = 0; mu < 4; ++mu) q[mu] = Q.p[mu] - a * KK[mu] + b * Kn[mu];
      std::memcpy(Q.p, q, sizeof q);
    }
  }

  // ---- colours (leading colour; the new tag is 100 + slot of j) ----
  int T = 100 + (int)ev.parts.size();
  if (ch == 0 || ch == 1 || ch == 3 || ch == 5) {
    // a gluon is emitted between the emitter and its spectator
    if (best.side == 0) { J.col = Pi.col; J.acol = T; Pi.col = T; }
    else { J.acol = Pi.acol; J.col = T; Pi.acol = T; }
  } else if (ch == 2) {
    // final g -> q qbar: i keeps the colour tag, j the anticolour tag
    J.acol = Pi.acol; J.col = 0; Pi.acol = 0;
  } else if (ch == 4) {
    // incoming q becomes an incoming gluon, the emitted j is the antiparton
    if (Pi.acol != 0) { Pi.col = T; J.acol = T; J.col = 0; }
    else { Pi.acol = T; J.col = T; J.acol = 0; }
  } else {
    // incoming gluon (crossed tags col A, acol B) becomes an incoming quark
    // of flavour f and emits a final parton of the same flavour
    int A = Pi.col, Bt = Pi.acol;
    if (new_fl_i > 0) { Pi.col = 0; Pi.acol = Bt; J.col = A; J.acol = 0; }
    else { Pi.col = A; Pi.acol = 0; J.col = 0; J.acol = Bt; }
  }
  Pi.fl = new_fl_i;
  ev.parts.push_back(J);
  ev.n_emit += 1;
  ev.cnt.accepts += 1;
  if (ev.n_emit == 1) ev.t_first = t;
}

// ---------------------------------------------------------------------------
// Hard event generation
// ---------------------------------------------------------------------------
void generate_hard(const Physics& ph, Event& ev, uint64_t event_id) {
  const Config& cf = ph.cfg;
  ev.parts.clear();
  ev.rng = Stream{cf.seed, event_id, kHardDrawBase};
  ev.status = kStatusActive;
  ev.n_emit = 0;
  ev.t_first = 0.0;
  ev.eta[0] = ev.eta[1] = 0.0;
  ev.cnt = Counters{0, 0, 0, 0, 0, 0};
  double s = cf.sqrt_s * cf.sqrt_s;
  ev.t = cf.t_start > 0.0 ? cf.t_start : s;
  double R0, R1, R2, R3, R4, R5;
  ev.rng.next2(R0, R1);
  ev.rng.next2(R2, R3);
  ev.rng.next2(R4, R5);
  if (cf.process == 0) {
    ev.pp = false;
    double c = 2.0 * R0 - 1.0;
    double cph, sph;
    sincos2pi(R1, cph, sph);  // phi = 2 pi R1
    int f = 1 + (int)std::floor(R2 * cf.nf);
    if (f > cf.nf) f = cf.nf;
    double st = std::sqrt((1.0 - c) * (1.0 + c));
    double E = 0.5 * cf.sqrt_s;
    double n[3] = {st * cph, st * sph, c};
    Parton q{{E, E * n[0], E * n[1], E * n[2]}, f, 1, 0, false};
    Parton qb{{E, -E * n[0], -E * n[1], -E * n[2]}, -f, 0, 1, false};
    ev.parts.push_back(q);
    ev.parts.push_back(qb);
    ev.weight = ee_dsigma_dcos(s, f, c) * 2.0 * cf.nf * kGeV2pb;
    return;
  }
  ev.pp = true;
  if (cf.process == 3) {
    // m^2 by the Breit-Wigner map, y uniform in [-Y, Y], cos(theta*) and phi
    // of the electron uniform in the dilepton rest frame (quark along +z if
    // it comes from beam 1); flavour pair by its share of the density
    double r_lo, r_hi;
    ll_window(cf.mll_lo, cf.mll_hi, r_lo, r_hi);
    double r = r_lo + R0 * (r_hi - r_lo);
    double cr, sr;
    sincos2pi(r, cr, sr);
    double mg = kMZ * kGZ;
    double m2 = kMZ * kMZ + mg * (sr / cr);
    double m = std::sqrt(m2);
    double Y = lg(cf.sqrt_s / m);
    double y = (2.0 * R1 - 1.0) * Y;
    double tau = m / cf.sqrt_s;
    double ey = ex(y), iey = ex(-y);
    double ea = ey * tau, eb = iey * tau;
    double c = 2.0 * R3 - 1.0;
    double dens[10], tot = 0.0;
    for (int k = 0; k < 10; ++k) {
      int fa, fb;
      born_pair(k, fa, fb);
      double Fa = ph.pdf.xf(pdf_index(fa), ea, m2), Fb = ph.pdf.xf(pdf_index(fb), eb, m2);
      dens[k] = Fa * Fb * ll_dsigma_dcos(m2, fa > 0 ? fa : fb, fa > 0 ? c : -c);
      tot += dens[k];
    }
    int pick = 9;
    double target = R2 * tot, acc = 0.0;
    for (int k = 0; k < 10; ++k) { acc += dens[k]; if (target < acc) { pick = k; break; } }
    int fa, fb;
    born_pair(pick, fa, fb);
    ev.parts.resize(4);
    ev.parts[0].fl = fa; ev.parts[1].fl = fb;
    set_beam_parton(ev, 0, ea, cf.sqrt_s);
    set_beam_parton(ev, 1, eb, cf.sqrt_s);
    set_incoming_quark_colour(ev.parts[0], 1);
    set_incoming_quark_colour(ev.parts[1], 1);
    double cph, sph;
    sincos2pi(R4, cph, sph);  // phi = 2 pi R4
    double st = std::sqrt((1.0 - c) * (1.0 + c));
    double ch = 0.5 * (ey + iey), sh = 0.5 * (ey - iey);
    double hm = 0.5 * m;
    Parton& el = ev.parts[2];
    Parton& po = ev.parts[3];
    el.p[0] = hm * (ch + c * sh); el.p[1] = hm * (st * cph); el.p[2] = hm * (st * sph); el.p[3] = hm * (sh + c * ch);
    po.p[0] = hm * (ch - c * sh); po.p[1] = -(hm * (st * cph)); po.p[2] = -(hm * (st * sph)); po.p[3] = hm * (sh - c * ch);
    el.fl = 11; po.fl = -11;
    el.col = el.acol = po.col = po.acol = 0;
    el.initial = po.initial = false;
    // dsigma = sum_k F_a F_b / m^2 dsigma_k/dc dm^2 dy dc, with dm^2 = 2 pi m_Z Gamma_Z / cos^2 dr
    ev.weight = tot / m2 * (kTwoPi * mg / (cr * cr)) * (r_hi - r_lo) * (2.0 * Y) * 2.0 * kGeV2pb;
    return;
  }
  double mz2 = kMZ * kMZ;
  bool hevent = false;
  double wsel = 1.0;
  if (cf.process == 2) {
    hevent = !(R0 < cf.p_s);
    wsel = hevent ? 1.0 / (1.0 - cf.p_s) : 1.0 / cf.p_s;
  }
  if (!hevent) {
    // Born kinematics: y uniform in [-Y, Y], eta_{1,2} = e^{+-y} m_Z/sqrt(s)
    double Y = lg(cf.sqrt_s / kMZ);
    double y = std::isfinite(cf.y_fixed) ? cf.y_fixed : (2.0 * R1 - 1.0) * Y;
    double tau = kMZ / cf.sqrt_s;
    double ea = ex(y) * tau, eb = ex(-y) * tau;
    double dens[10], tot = 0.0;
    for (int k = 0; k < 10; ++k) { dens[k] = born_pair_density(ph, k, ea, eb); tot += dens[k]; }
    int pick = 9;
    if (cf.pair_fixed >= 0) {
      pick = cf.pair_fixed;
    } else {
      double target = R2 * tot, acc = 0.0;
      for (int k = 0; k < 10; ++k) { acc += dens[k]; if (target < acc) { pick = k; break; } }
    }
    int fa, fb;
    born_pair(pick, fa, fb);
    ev.parts.resize(3);
    ev.parts[0].fl = fa; ev.parts[1].fl = fb;
    set_beam_parton(ev, 0, ea, cf.sqrt_s);
    set_beam_parton(ev, 1, eb, cf.sqrt_s);
    set_incoming_quark_colour(ev.parts[0], 1);
    set_incoming_quark_colour(ev.parts[1], 1);
    Parton& Z = ev.parts[2];
    for (int mu = 0; mu < 4; ++mu) Z.p[mu] = ev.parts[0].p[mu] + ev.parts[1].p[mu];
    Z.fl = 23; Z.col = 0; Z.acol = 0; Z.initial = false;
    double w = tot * 2.0 * Y * kGeV2pb;
    if (cf.process == 2) {
      // S event: B (1 + C_F alpha_s/2pi * 2) + collinear terms (eq. lhc-nlo-bvic)
      double as = cf.alpha_s_mz;
      double corr = 1.0 + kCF * as / (2.0 * kPi) * 2.0;
      corr += collinear_leg(ph, fa, ea, R3);
      corr += collinear_leg(ph, fb, eb, R4);
      w = w * corr * wsel;
    }
    ev.weight = w;
    return;
  }
  // H event (Appendix C.2): x in [m^2/s, 1), v in [0, 1-x], phi, y of the
  // hard system in [-Y(x), Y(x)], eta_{1,2} = e^{+-y} sqrt(sbar/s)
  double xlo = mz2 / s;
  double x = xlo + R3 * (1.0 - xlo);
  double v = R4 * (1.0 - x);

  double sbar = mz2 / x;
  double Y = 0.5 * lg(s / sbar);
  double y = (2.0 * R1 - 1.0) * Y;
  double rt = std::sqrt(sbar / s);
  double e1 = ex(y) * rt, e2 = ex(-y) * rt;
  double as = cf.alpha_s_mz;
  double m2 = mz2;
  // thirty ordered pairs: 0..9 q qbar -> Z g (pair k as in born_pair),
  // 10..14 g q, 15..19 g qbar (gluon from beam 1), 20..24 q g, 25..29 qbar g
  double c[30], tot = 0.0;
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
      // (R - S)^{gq -> Zq} with ubar = -v sbar (the gluon is the II emitter)
      double ubar = -v * sbar;
      rs = 8.0 * kPi * as * kTR / m2 * born_me2(q) * ((2.0 * m2 - ubar) / sbar);
    }
    double Fa = ph.pdf.xf(pdf_index(fa), e1, mz2);
    double Fb = ph.pdf.xf(pdf_index(fb), e2, mz2);
    c[k] = Fa * Fb * rs / (16.0 * kPi) / m2;
    tot += std::fabs(c[k]);
  }
  int pick = 29;
  {
    double target = R2 * tot, acc = 0.0;
    for (int k = 0; k < 30; ++k) { acc += std::fabs(c[k]); if (target < acc) { pick = k; break; } }
  }
  double jac = 2.0 * Y * (1.0 - xlo) * (1.0 - x);
  ev.weight = (c[pick] < 0.0 ? -tot : tot) * jac * kGeV2pb * wsel;
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
  ev.parts.resize(4);
  ev.parts[0].fl = fa; ev.parts[1].fl = fb;
  set_beam_parton(ev, 0, e1, cf.sqrt_s);
  set_beam_parton(ev, 1, e2, cf.sqrt_s);
  // Born momenta from the II map run backwards: p~_emitter = x p_emitter
  int spec = 1 - emitter;
  double Pt[4], Bt[4];
  for (int mu = 0; mu < 4; ++mu) {
    Pt[mu] = x * ev.parts[emitter].p[mu];
    Bt[mu] = ev.parts[spec].p[mu];
  }
  double ea[4], eb[4];
  transverse_basis(Pt, Bt, ea, eb);
  double t = v * (1.0 - x - v) / x * m2;
  double st = std::sqrt(t), cph, sph;
  sincos2pi(R5, cph, sph);  // phi = 2 pi R5
  Parton& J = ev.parts[3];
  Parton& Z = ev.parts[2];
  for (int mu = 0; mu < 4; ++mu) {
    double kt = st * (cph * ea[mu] + sph * eb[mu]);
    J.p[mu] = ((1.0 - x - v) / x) * Pt[mu] + v * Bt[mu] - kt;
  }
  for (int mu = 0; mu < 4; ++mu)
    Z.p[mu] = (ev.parts[0].p[mu] + ev.parts[1].p[mu]) - J.p[mu];
  Z.fl = 23; Z.col = 0; Z.acol = 0; Z.initial = false;
  J.fl = fj; J.initial = false;
  // colours (crossed for incoming partons)
  if (pick < 10) {
    // q qbar -> Z g: incoming quark - gluon - incoming antiquark chain
    Parton& A = ev.parts[0];
    Parton& Bp = ev.parts[1];
    if (A.fl > 0) { A.col = 0; A.acol = 1; Bp.col = 2; Bp.acol = 0; J.col = 1; J.acol = 2; }
    else { A.col = 1; A.acol = 0; Bp.col = 0; Bp.acol = 2; J.col = 2; J.acol = 1; }
  } else {
    Parton& G = ev.parts[emitter];
    Parton& Q = ev.parts[spec];
    if (Q.fl > 0) { Q.col = 0; Q.acol = 1; G.col = 1; G.acol = 2; J.col = 2; J.acol = 0; }
    else { Q.col = 1; Q.acol = 0; G.col = 2; G.acol = 1; J.col = 0; J.acol = 2; }
  }
}

// ---------------------------------------------------------------------------
// Observables (Section 4.1; GAPS 1 for e+e-). Brute force, O(n^3) or worse.
// ---------------------------------------------------------------------------
double norm3(const double p[4]) { return std::sqrt(p[1] * p[1] + p[2] * p[2] + p[3] * p[3]); }

// thrust T = max over unit n of sum |p.n| / sum |p| = max over subsets S of
// 2 |sum_S p| / sum |p|. All subsets for n <= 12; above, the exact
// construction with candidate axes p_i x p_j and the four sign choices for i, j.
double thrust(const std::vector<std::array<double, 4>>& ps) {
  int n = (int)ps.size();
  double sum = 0.0;
  for (auto& p : ps) sum += norm3(p.data());
  if (n < 2 || !(sum > 0.0)) return 1.0;
  double best = 0.0;
  if (n <= 12) {
    for (uint32_t m = 0; m < (1u << (n - 1)); ++m) {
      double v[3] = {0.0, 0.0, 0.0};
      for (int i = 0; i < n; ++i)
        if ((m >> i) & 1u) { v[0] += ps[i][1]; v[1] += ps[i][2]; v[2] += ps[i][3]; }
      double l = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
      best = std::max(best, l);
    }
  } else {
    for (int i = 0; i < n; ++i) {
      for (int j = i + 1; j < n; ++j) {
        double ax[3] = {ps[i][2] * ps[j][3] - ps[i][3] * ps[j][2],
                        ps[i][3] * ps[j][1] - ps[i][1] * ps[j][3],
                        ps[i][1] * ps[j][2] - ps[i][2] * ps[j][1]};
        double base[3] = {0.0, 0.0, 0.0};
        for (int k = 0; k < n; ++k) {
          if (k == i || k == j) continue;
          double d = ps[k][1] * ax[0] + ps[k][2] * ax[1] + ps[k][3] * ax[2];
          if (d > 0.0) { base[0] += ps[k][1]; base[1] += ps[k][2]; base[2] += ps[k][3]; }
        }
        for (int si = 0; si < 2; ++si) {
          for (int sj = 0; sj < 2; ++sj) {
            double v[3] = {base[0], base[1], base[2]};
            if (si) { v[0] += ps[i][1]; v[1] += ps[i][2]; v[2] += ps[i][3]; }
            if (sj) { v[0] += ps[j][1]; v[1] += ps[j][2]; v[2] += ps[j][3]; }
            double l = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
            best = std::max(best, l);
          }
        }
      }
    }
  }
  return 2.0 * best / sum;
}

// Durham (k_T) clustering in the E-scheme:
//   y_ij = 2 min(E_i^2, E_j^2)(1 - cos theta_ij) / E_vis^2;
// ymerge[m] = the smallest y_ij when m+1 objects are merged to m.
void durham(const std::vector<std::array<double, 4>>& in, double& y23, double& y34) {
  std::vector<std::array<double, 4>> ps = in;
  double evis = 0.0;
  for (auto& p : ps) evis += p[0];
  y23 = 0.0; y34 = 0.0;
  while (ps.size() > 1) {
    int m = (int)ps.size();
    double ymin = std::numeric_limits<double>::infinity();
    int bi = -1, bj = -1;
    for (int i = 0; i < m; ++i) {
      for (int j = i + 1; j < m; ++j) {
        double ni = norm3(ps[i].data()), nj = norm3(ps[j].data());
        double cth = (ps[i][1] * ps[j][1] + ps[i][2] * ps[j][2] + ps[i][3] * ps[j][3]) / (ni * nj);
        double emin = std::min(ps[i][0], ps[j][0]);
        double y = 2.0 * emin * emin * (1.0 - cth) / (evis * evis);
        if (y < ymin) { ymin = y; bi = i; bj = j; }
      }
    }
    if (m == 3) y23 = ymin;
    if (m == 4) y34 = ymin;
    for (int mu = 0; mu < 4; ++mu) ps[bi][mu] += ps[bj][mu];
    ps.erase(ps.begin() + bj);
  }
}

// anti-kT (Cacciari, Salam, Soyez 2008), E-scheme, rapidity-azimuth distance
struct Jet { double p[4]; };
void antikt(const std::vector<std::array<double, 4>>& in, double R, std::vector<Jet>& jets) {
  std::vector<std::array<double, 4>> ps;
  for (auto& p : in)
    if (p[1] * p[1] + p[2] * p[2] > 0.0) ps.push_back(p);
  jets.clear();
  auto kin = [](const std::array<double, 4>& p, double& pt2, double& y, double& phi) {
    pt2 = p[1] * p[1] + p[2] * p[2];
    y = 0.5 * std::log((p[0] + p[3]) / (p[0] - p[3]));
    phi = std::atan2(p[2], p[1]);
  };
  while (!ps.empty()) {
    int m = (int)ps.size();
    double dmin = std::numeric_limits<double>::infinity();
    int bi = -1, bj = -1;
    for (int i = 0; i < m; ++i) {
      double pti2, yi, phii;
      kin(ps[i], pti2, yi, phii);
      double diB = 1.0 / pti2;
      if (diB < dmin) { dmin = diB; bi = i; bj = -1; }
      for (int j = i + 1; j < m; ++j) {
        double ptj2, yj, phij;
        kin(ps[j], ptj2, yj, phij);
        double dphi = std::fabs(phii - phij);
        if (dphi > kPi) dphi = 2.0 * kPi - dphi;
        double dr2 = (yi - yj) * (yi - yj) + dphi * dphi;
        double dij = std::min(1.0 / pti2, 1.0 / ptj2) * dr2 / (R * R);
        if (dij < dmin) { dmin = dij; bi = i; bj = j; }
      }
    }
    if (bj < 0) {
      Jet J;
      for (int mu = 0; mu < 4; ++mu) J.p[mu] = ps[bi][mu];
      jets.push_back(J);
      ps.erase(ps.begin() + bi);
    } else {
      for (int mu = 0; mu < 4; ++mu) ps[bi][mu] += ps[bj][mu];
      ps.erase(ps.begin() + bj);
    }
  }
}

constexpr int kNObs = 8;
// Per-event observables.
//   e+e-: [0] 1-T, [1] y23, [2] y34, [3] final partons, [4] emissions
//   pp  : [0] Z pT, [1] Z y, [2] Z phi (0 when pT = 0), [3] jets with
//         pT > 5 GeV and |eta| < 5, [4] leading such jet pT (0 if none),
//         [5] its pseudorapidity (0 if none), [6] final partons, [7] emissions
void observables(const Event& ev, double obs[kNObs]) {
  for (int i = 0; i < kNObs; ++i) obs[i] = 0.0;
  std::vector<std::array<double, 4>> fin;
  double Z[4] = {0.0, 0.0, 0.0, 0.0};  // the colourless final state: Z, or the lepton pair
  for (auto& P : ev.parts) {
    if (P.initial) continue;
    if (P.fl == 23 || P.fl == 11 || P.fl == -11) {
      for (int mu = 0; mu < 4; ++mu) Z[mu] += P.p[mu];
      continue;
    }
    fin.push_back({P.p[0], P.p[1], P.p[2], P.p[3]});
  }
  if (!ev.pp) {
    obs[0] = 1.0 - thrust(fin);
    durham(fin, obs[1], obs[2]);
    obs[3] = (double)fin.size();
    obs[4] = (double)ev.n_emit;
    return;
  }
  double pt = std::sqrt(Z[1] * Z[1] + Z[2] * Z[2]);
  obs[0] = pt;
  obs[1] = 0.5 * std::log((Z[0] + Z[3]) / (Z[0] - Z[3]));
  obs[2] = pt > 0.0 ? std::atan2(Z[2], Z[1]) : 0.0;
  std::vector<Jet> jets;
  antikt(fin, 0.4, jets);
  int nj = 0;
  double lead = 0.0, lead_eta = 0.0;
  for (auto& J : jets) {
    double jpt = std::sqrt(J.p[1] * J.p[1] + J.p[2] * J.p[2]);
    double jeta = std::asinh(J.p[3] / jpt);
    if (jpt > 5.0 && std::fabs(jeta) < 5.0) {
      nj += 1;
      if (jpt > lead) { lead = jpt; lead_eta = jeta; }
    }
  }
  obs[3] = (double)nj;
  obs[4] = lead;
  obs[5] = lead_eta;
  obs[6] = (double)fin.size();
  obs[7] = (double)ev.n_emit;
}

Physics make_physics(const Config& c) {
  Physics ph;
  ph.cfg = c;
  if (c.pdf) ph.pdf.init(c.pdf);
  ph.s_had = c.sqrt_s * c.sqrt_s;
  ph.beta0 = (33.0 - 2.0 * 5.0) / (12.0 * kPi);
  ph.as_over = c.fixed_alpha ? c.alpha_s_mz : 0.0;
  if (!c.fixed_alpha) {
    ph.as_over = c.alpha_s_mz / (1.0 + c.alpha_s_mz * ph.beta0 * lg(c.t_cut / (kMZ * kMZ)));
  }
  return ph;
}

// Mixed batch (one launch over several processes, Sec. 3 on heterogeneous
// batches). The paper does not say how events are assigned to processes.
// Reading: event `id` belongs to row r of a table of (process, sqrt_s, t_c,
// fraction) rows, r = the first row whose cumulative fraction exceeds the
// uniform of Philox block (seed, id, draw 2^62), words 0 and 1; the last row
// takes the remainder. The event is then exactly event `id` of a run with
// that row's settings and the same seed.
constexpr uint64_t kMixDraw = 0x4000000000000000ull;

int mix_row(uint64_t seed, uint64_t id, const double* fractions, int n_rows) {
  Stream r{seed, id, kMixDraw};
  double u, unused;
  r.next2(u, unused);
  double cum = 0.0;
  for (int k = 0; k + 1 < n_rows; ++k) {
    cum += fractions[k];
    if (u < cum) return k;
  }
  return n_rows - 1;
}

void run_event(const Physics& ph, uint64_t id, Event& ev) {
  generate_hard(ph, ev, id);
  ev.rng.draw = 0;
  long steps = 0;
  while (ev.status == kStatusActive) {
    shower_step(ph, ev);
    if (++steps >= kMaxSteps && ev.status == kStatusActive) ev.status = kErrIterCap;
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// C interface used by the Python test wrapper (oracle/oracle.py)
// ---------------------------------------------------------------------------
extern "C" {

struct OracleConfig {
  int process, nf, nmax, fixed_alpha;
  uint32_t channel_mask;
  int pair_fixed;
  double sqrt_s, alpha_s_mz, t_cut, p_s, t_start, y_fixed;
  uint64_t seed;
  const float* pdf;
  double mll_lo, mll_hi;
};

// Per-event output, array-of-structures, caller allocated.
struct OracleOut {
  double* p;        // [n][nmax][4]
  int32_t* flav;    // [n][nmax]
  int32_t* col;     // [n][nmax]
  int32_t* acol;    // [n][nmax]
  int32_t* initial; // [n][nmax]
  int32_t* npart;   // [n]
  int32_t* status;  // [n]
  int32_t* n_emit;  // [n]
  double* weight;   // [n]
  double* eta;      // [n][2]
  double* t_first;  // [n]
  double* obs;      // [n][8]
  uint64_t* counters; // [n][6]: steps, trials, isr trials, vetoes, accepts, violations
};

static Config to_config(const OracleConfig* c) {
  Config k;
  k.process = c->process; k.nf = c->nf; k.nmax = c->nmax; k.fixed_alpha = c->fixed_alpha;
  k.channel_mask = c->channel_mask; k.pair_fixed = c->pair_fixed;
  k.sqrt_s = c->sqrt_s; k.alpha_s_mz = c->alpha_s_mz; k.t_cut = c->t_cut; k.p_s = c->p_s;
  k.t_start = c->t_start; k.y_fixed = c->y_fixed; k.seed = c->seed; k.pdf = c->pdf;
  k.mll_lo = c->mll_lo; k.mll_hi = c->mll_hi;
  return k;
}

static void store_event(const Event& ev, int nmax, uint64_t i, OracleOut* o) {
  int n = (int)ev.parts.size();
  if (o->p) {
    for (int s = 0; s < nmax; ++s)
      for (int mu = 0; mu < 4; ++mu)
        o->p[(i * nmax + s) * 4 + mu] = s < n ? ev.parts[s].p[mu] : 0.0;
  }
  for (int s = 0; s < nmax; ++s) {
    bool in = s < n;
    if (o->flav) o->flav[i * nmax + s] = in ? ev.parts[s].fl : 0;
    if (o->col) o->col[i * nmax + s] = in ? ev.parts[s].col : 0;
    if (o->acol) o->acol[i * nmax + s] = in ? ev.parts[s].acol : 0;
    if (o->initial) o->initial[i * nmax + s] = in ? (ev.parts[s].initial ? 1 : 0) : 0;
  }
  if (o->npart) o->npart[i] = n;
  if (o->status) o->status[i] = ev.status;
  if (o->n_emit) o->n_emit[i] = ev.n_emit;
  if (o->weight) o->weight[i] = ev.weight;
  if (o->eta) { o->eta[2 * i] = ev.eta[0]; o->eta[2 * i + 1] = ev.eta[1]; }
  if (o->t_first) o->t_first[i] = ev.t_first;
  if (o->obs) observables(ev, o->obs + i * kNObs);
  if (o->counters) {
    uint64_t* c = o->counters + i * 6;
    c[0] = ev.cnt.steps; c[1] = ev.cnt.trials; c[2] = ev.cnt.isr_trials;
    c[3] = ev.cnt.vetoes; c[4] = ev.cnt.accepts; c[5] = ev.cnt.violations;
  }
}

// Runs hard process + shower + observables for events [first, first + n).
int oracle_run(const OracleConfig* c, uint64_t first, uint64_t n, OracleOut* out) {
  Config k = to_config(c);
  if (k.process != 0 && !k.pdf) return -1;
  Physics ph = make_physics(k);
  Event ev;
  ev.parts.reserve(k.nmax + 1);
  for (uint64_t i = 0; i < n; ++i) {
    run_event(ph, first + i, ev);
    store_event(ev, k.nmax, i, out);
  }
  return 0;
}

// Hard process only (no shower).
int oracle_hard(const OracleConfig* c, uint64_t first, uint64_t n, OracleOut* out) {
  Config k = to_config(c);
  if (k.process != 0 && !k.pdf) return -1;
  Physics ph = make_physics(k);
  Event ev;
  for (uint64_t i = 0; i < n; ++i) {
    generate_hard(ph, ev, first + i);
    store_event(ev, k.nmax, i, out);
  }
  return 0;
}

// Same as oracle_run, split over `threads` std::threads by contiguous event
// ranges (the timing driver for the CPU baseline; results are identical).
int oracle_run_threads(const OracleConfig* c, uint64_t first, uint64_t n, OracleOut* out,
                       int threads) {
  if (threads < 1) threads = 1;
  Config k = to_config(c);
  if (k.process != 0 && !k.pdf) return -1;
  Physics ph = make_physics(k);
  std::vector<std::thread> pool;
  uint64_t chunk = (n + threads - 1) / threads;
  for (int t = 0; t < threads; ++t) {
    uint64_t lo = t * chunk, hi = std::min(n, lo + chunk);
    if (lo >= hi) break;
    pool.emplace_back([&, lo, hi]() {
      Event ev;
      ev.parts.reserve(k.nmax + 1);
      for (uint64_t i = lo; i < hi; ++i) {
        run_event(ph, first + i, ev);
        store_event(ev, k.nmax, i, out);
      }
    });
  }
  for (auto& th : pool) th.join();
  return 0;
}

// Mixed batch: rows[k] are complete configurations (equal seeds), fractions[k]
// their shares; row_out[i] (optional) receives the row of event first + i.
// Runs on `threads` std::threads by contiguous event ranges.
int oracle_run_mix(const OracleConfig* rows, const double* fractions, int n_rows, uint64_t first,
                   uint64_t n, OracleOut* out, int32_t* row_out, int threads) {
  if (n_rows < 1 || n_rows > 8) return -1;
  std::vector<Physics> ph;
  for (int r = 0; r < n_rows; ++r) {
    Config k = to_config(rows + r);
    if (k.process != 0 && !k.pdf) return -1;
    if (k.seed != rows[0].seed || k.nmax != rows[0].nmax) return -1;
    ph.push_back(make_physics(k));
  }
  if (threads < 1) threads = 1;
  const int nmax = rows[0].nmax;
  std::vector<std::thread> pool;
  uint64_t chunk = (n + threads - 1) / threads;
  for (int t = 0; t < threads; ++t) {
    uint64_t lo = t * chunk, hi = std::min(n, lo + chunk);
    if (lo >= hi) break;
    pool.emplace_back([&, lo, hi]() {
      Event ev;
      ev.parts.reserve(nmax + 1);
      for (uint64_t i = lo; i < hi; ++i) {
        const int r = mix_row(rows[0].seed, first + i, fractions, n_rows);
        if (row_out) row_out[i] = r;
        run_event(ph[r], first + i, ev);
        store_event(ev, nmax, i, out);
      }
    });
  }
  for (auto& th : pool) th.join();
  return 0;
}

// Rows of events first .. first + n - 1 of a mixed batch (no showering).
int oracle_mix_rows(uint64_t seed, const double* fractions, int n_rows, uint64_t first, uint64_t n,
                    int32_t* row_out) {
  if (n_rows < 1 || n_rows > 8) return -1;
  for (uint64_t i = 0; i < n; ++i) row_out[i] = mix_row(seed, first + i, fractions, n_rows);
  return 0;
}

// First emission of one isolated dipole (both ends radiate when both are
// coloured partners of each other; flq = 21 makes both partons gluons, joined
// by two colour lines): type 0 FF (final quark + final antiquark,
// s = dipole invariant), 1 FI/IF (final quark + incoming quark of momentum
// fraction eta), 2 II (incoming quark from beam 1 at eta + incoming antiquark
// from beam 2 at eta2 = s/(eta * sqrt_s^2)). The shower runs from t_start
// until its first accepted emission; out_t[i] = its scale or 0 if none.
// Used by the Sudakov pins. With out_rec != NULL the record after the first
// emission is written too: out_rec[i][3][8] = {E, px, py, pz, flavour, colour,
// anticolour, initial} of slots 0..2 (zero past the record), and
// out_eta[i][2] the momentum fractions of slots 0 and 1 (used by the pins of
// the flavour choices and the colour flow).
int oracle_first_emission_record(const OracleConfig* c, int type, int flq, double s, double eta,
                                 uint64_t n, double* out_t, double* out_rec, double* out_eta);
int oracle_first_emission(const OracleConfig* c, int type, int flq, double s, double eta,
                          uint64_t n, double* out_t) {
  return oracle_first_emission_record(c, type, flq, s, eta, n, out_t, nullptr, nullptr);
}
int oracle_first_emission_record(const OracleConfig* c, int type, int flq, double s, double eta,
                                 uint64_t n, double* out_t, double* out_rec, double* out_eta) {
  Config k = to_config(c);
  Physics ph = make_physics(k);
  Event ev;
  double S = k.sqrt_s * k.sqrt_s;
  for (uint64_t e = 0; e < n; ++e) {
    ev.parts.clear();
    ev.rng = Stream{k.seed, e, 0};
    ev.status = kStatusActive;
    ev.n_emit = 0;
    ev.t_first = 0.0;
    ev.cnt = Counters{0, 0, 0, 0, 0, 0};
    ev.t = k.t_start > 0.0 ? k.t_start : S;
    ev.pp = type != 0;
    bool glu = flq == 21;
    if (type == 0) {
      double E = 0.5 * std::sqrt(s);
      if (glu) {
        ev.parts.push_back(Parton{{E, 0.0, 0.0, E}, 21, 1, 2, false});
        ev.parts.push_back(Parton{{E, 0.0, 0.0, -E}, 21, 2, 1, false});
      } else {
        ev.parts.push_back(Parton{{E, 0.0, 0.0, E}, flq, 1, 0, false});
        ev.parts.push_back(Parton{{E, 0.0, 0.0, -E}, -flq, 0, 1, false});
      }
    } else if (type == 1) {
      ev.parts.resize(2);
      ev.parts[0].fl = flq;
      set_beam_parton(ev, 0, eta, k.sqrt_s);
      double Ea = ev.parts[0].p[0];
      double Ek = s / (4.0 * Ea);
      if (glu) {
        ev.parts[0].col = 1; ev.parts[0].acol = 2;
        ev.parts[1] = Parton{{Ek, 0.0, 0.0, -Ek}, 21, 2, 1, false};
      } else {
        set_incoming_quark_colour(ev.parts[0], 1);
        // final parton of the same flavour, colour-connected to the incoming one
        if (flq > 0) ev.parts[1] = Parton{{Ek, 0.0, 0.0, -Ek}, flq, 1, 0, false};
        else ev.parts[1] = Parton{{Ek, 0.0, 0.0, -Ek}, flq, 0, 1, false};
      }
      ev.eta[1] = 0.0;
    } else {
      ev.parts.resize(2);
      ev.parts[0].fl = flq;
      ev.parts[1].fl = glu ? 21 : -flq;
      set_beam_parton(ev, 0, eta, k.sqrt_s);
      set_beam_parton(ev, 1, s / (eta * S), k.sqrt_s);
      if (glu) {
        ev.parts[0].col = 1; ev.parts[0].acol = 2;
        ev.parts[1].col = 2; ev.parts[1].acol = 1;
      } else {
        set_incoming_quark_colour(ev.parts[0], 1);
        set_incoming_quark_colour(ev.parts[1], 1);
      }
    }
    long steps = 0;
    while (ev.status == kStatusActive && ev.n_emit == 0 && steps < kMaxSteps) {
      shower_step(ph, ev);
      ++steps;
    }
    out_t[e] = ev.t_first;
    if (out_rec) {
      for (int q = 0; q < 3; ++q) {
        double* r = out_rec + (e * 3 + q) * 8;
        for (int m = 0; m < 8; ++m) r[m] = 0.0;
        if (q >= (int)ev.parts.size()) continue;
        const Parton& P = ev.parts[q];
        for (int mu = 0; mu < 4; ++mu) r[mu] = P.p[mu];
        r[4] = P.fl; r[5] = P.col; r[6] = P.acol; r[7] = P.initial ? 1.0 : 0.0;
      }
    }
    if (out_eta) { out_eta[2 * e] = ev.eta[0]; out_eta[2 * e + 1] = ev.eta[1]; }
  }
  return 0;
}

int oracle_if_map(double r, double z, double omz, double out[4]) {
  return if_map(r, z, omz, out[0], out[1], out[2], out[3]) ? 1 : 0;
}
int oracle_ii_map(double r, double z, double omz, double out[3]) {
  return ii_map(r, z, omz, out[0], out[1], out[2]) ? 1 : 0;
}

// ---------------------------------------------------------------------------
// Reference of the learned-proposal network: a 4 -> 64 -> 64 -> 1 multilayer
// perceptron with ReLU hidden layers, in FP64. Parameter layout (4545 values):
// W1 [64][4], b1 [64], W2 [64][64], b2 [64], W3 [64], b3 [1]. Loss: the
// asymmetric squared error (expectile) mean_i w_i (y_i - t_i)^2 with
// w_i = tau when the prediction is below the target, 1 - tau otherwise.
// oracle_mlp_loss_grad returns the loss and writes d loss / d params by
// backpropagation written out layer by layer.
// ---------------------------------------------------------------------------
constexpr int kH = 64, kIn = 4;
constexpr int kParams = kH * kIn + kH + kH * kH + kH + kH + 1;

static double mlp_forward_one(const double* P, const double* x, double* h1, double* h2) {
  const double* W1 = P;
  const double* b1 = W1 + kH * kIn;
  const double* W2 = b1 + kH;
  const double* b2 = W2 + kH * kH;
  const double* W3 = b2 + kH;
  const double b3 = W3[kH];
  for (int i = 0; i < kH; ++i) {
    double a = b1[i];
    for (int k = 0; k < kIn; ++k) a += W1[i * kIn + k] * x[k];
    h1[i] = a > 0.0 ? a : 0.0;
  }
  for (int i = 0; i < kH; ++i) {
    double a = b2[i];
    for (int k = 0; k < kH; ++k) a += W2[i * kH + k] * h1[k];
    h2[i] = a > 0.0 ? a : 0.0;
  }
  double y = b3;
  for (int k = 0; k < kH; ++k) y += W3[k] * h2[k];
  return y;
}

void oracle_mlp_forward(const double* P, const double* X, uint64_t n, double* out) {
  double h1[kH], h2[kH];
  for (uint64_t i = 0; i < n; ++i) out[i] = mlp_forward_one(P, X + 4 * i, h1, h2);
}

double oracle_mlp_loss_grad(const double* P, const double* X, const double* T, uint64_t n, double tau,
                            double* grad) {
  for (int q = 0; q < kParams; ++q) grad[q] = 0.0;
  const double* W2 = P + kH * kIn + kH;
  const double* W3 = W2 + kH * kH + kH;
  double* gW1 = grad;
  double* gb1 = gW1 + kH * kIn;
  double* gW2 = gb1 + kH;
  double* gb2 = gW2 + kH * kH;
  double* gW3 = gb2 + kH;
  double* gb3 = gW3 + kH;
  double loss = 0.0;
  double h1[kH], h2[kH], d2[kH], d1[kH];
  for (uint64_t s = 0; s < n; ++s) {
    const double* x = X + 4 * s;
    double y = mlp_forward_one(P, x, h1, h2);
    double r = y - T[s];
    double w = r < 0.0 ? tau : 1.0 - tau;
    loss += w * r * r;
    double dy = 2.0 * w * r / (double)n;  // d loss / d y
    gb3[0] += dy;
    for (int k = 0; k < kH; ++k) {
      gW3[k] += dy * h2[k];
      d2[k] = h2[k] > 0.0 ? dy * W3[k] : 0.0;  // through ReLU
    }
    for (int i = 0; i < kH; ++i) {
      gb2[i] += d2[i];
      for (int k = 0; k < kH; ++k) gW2[i * kH + k] += d2[i] * h1[k];
    }
    for (int k = 0; k < kH; ++k) {
      double a = 0.0;
      for (int i = 0; i < kH; ++i) a += W2[i * kH + k] * d2[i];
      d1[k] = h1[k] > 0.0 ? a : 0.0;
    }
    for (int i = 0; i < kH; ++i) {
      gb1[i] += d1[i];
      for (int k = 0; k < kIn; ++k) gW1[i * kIn + k] += d1[i] * x[k];
    }
  }
  return loss / (double)n;
}

void oracle_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  philox4x32_10(ctr, key, out);
}
double oracle_uniform(uint32_t lo, uint32_t hi) { return uniform_from_words(lo, hi); }

double oracle_pdf_xf(const float* grid, int f, double x, double q2) {
  Pdf p;
  p.init(grid);
  return p.xf(f, x, q2);
}
void oracle_pdf_xf_batch(const float* grid, int f, int n, const double* x, const double* q2,
                         double* out) {
  Pdf p;
  p.init(grid);
  for (int i = 0; i < n; ++i) out[i] = p.xf(f, x[i], q2[i]);
}
double oracle_pdf_bound(const float* grid, int num, int den, double eta) {
  Pdf p;
  p.init(grid);
  return p.ratio_bound(num, den, eta);
}
double oracle_alpha_s(const OracleConfig* c, double t) {
  Physics ph = make_physics(to_config(c));
  return ph.alpha_s(t);
}
double oracle_li2(double x) { return li2(x); }
double oracle_exp(double x) { return ex(x); }
double oracle_log(double x) { return lg(x); }
void oracle_sincos2pi(double R, double out[2]) { sincos2pi(R, out[0], out[1]); }
// collinear pieces with ln(mu_F^2/m^2) = L: which = 0 A, 1 B(x), 2 g(x),
// 3 h_qq(x), 4 h_qg(x)
double oracle_collinear(double as, double L, int which, double x) {
  Collinear C{as, L};
  switch (which) {
    case 0: return C.A();
    case 1: return C.B(x);
    case 2: return C.g(x);
    case 3: return C.hqq(x);
    default: return C.hqg(x);
  }
}
double oracle_born_me2(int f) { return born_me2(f); }
double oracle_born_density(const OracleConfig* c, int k, double ea, double eb) {
  Physics ph = make_physics(to_config(c));
  return born_pair_density(ph, k, ea, eb);
}
double oracle_ee_dsigma(double s, int f, double cth) { return ee_dsigma_dcos(s, f, cth); }
double oracle_ll_dsigma(double s, int f, double cth) { return ll_dsigma_dcos(s, f, cth); }
// overestimate z range: out = {zm, delta}; returns 0 if t is above the limit
int oracle_z_limits(int type, double t, double s, double eta, double out[2]) {
  return z_limits(type, t, s, eta, out[0], out[1]) ? 1 : 0;
}
void oracle_shape_sample(int shape, double zm, double delta, double R, double out[2]) {
  shape_sample((Shape)shape, zm, delta, R, out[0], out[1]);
}
double oracle_shape_integral(int shape, double zm, double delta) {
  return shape_integral((Shape)shape, zm, delta);
}
void oracle_basis(const double P[4], const double K[4], double e1[4], double e2[4]) {
  transverse_basis(P, K, e1, e2);
}
// observables of a given final-state list: out = {1-T, y23, y34}
void oracle_ee_shapes(const double* p, int n, double out[3]) {
  std::vector<std::array<double, 4>> v;
  for (int i = 0; i < n; ++i) v.push_back({p[4 * i], p[4 * i + 1], p[4 * i + 2], p[4 * i + 3]});
  out[0] = 1.0 - thrust(v);
  durham(v, out[1], out[2]);
}
int oracle_antikt(const double* p, int n, double R, double* jets_out) {
  std::vector<std::array<double, 4>> v;
  for (int i = 0; i < n; ++i) v.push_back({p[4 * i], p[4 * i + 1], p[4 * i + 2], p[4 * i + 3]});
  std::vector<Jet> jets;
  antikt(v, R, jets);
  for (size_t j = 0; j < jets.size(); ++j)
    for (int mu = 0; mu < 4; ++mu) jets_out[4 * j + mu] = jets[j].p[mu];
  return (int)jets.size();
}

}  // extern "C"
